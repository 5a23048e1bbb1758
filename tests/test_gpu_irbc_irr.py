"""GPU parity of the non-smooth IRBC model (irreversible investment,
eq. modelkink1; policy (k', mu, lambda), complementarity as Fischer-Burmeister
rows) against the CPU oracle: residuals (FP64 1e-11, F32C 1e-6 of the row
scale), both node modes; the analytic Jacobian against central differences
of the oracle; the semismooth Newton against the oracle's Newton, with the
irreversibility constraint binding in some countries."""
import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_irbc import scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def _model(G, N, const_k=False, level=4):
    I = O.IRBCOracle(N, irreversible=True)
    lam = I.steady_lambda()
    d, m = 2 * N, 2 * N + 1
    pert = synth.irbc_policy_perturbation(synth.BASE_SEED + 700, N)
    base = np.concatenate([np.ones(N), [lam]])

    def fn(dims, X):
        X = np.asarray(X, np.float64)
        if X.ndim == 1:
            X = X.reshape(-1, len(dims))
        full = np.ones((X.shape[0], d))
        if len(dims):
            full[:, list(dims)] = X
        sm = synth.irbc_policy_values(base, pert, dims, X)
        y = np.zeros((X.shape[0], m))
        y[:, :N] = 1.0 if const_k else sm[:, :N]
        y[:, N:2 * N] = 0.0 if const_k else 0.02 * np.maximum(0.0, full[:, N:] - 1.1) ** 2 * 100
        y[:, 2 * N] = sm[:, N]
        return y

    comps = [()] + [(i,) for i in range(d)] + [(j, N + j) for j in range(N)]
    E = O.OracleDDSG(d, m, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    h = G.HDMR(d, m, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in comps:
        E.add_regular(u, level)
        h.add_regular(list(u), level)
    E.fill_values(fn)
    E.hierarchize()
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    M.set_irreversible(True)
    return I, E, h, M, lam


def _guess(N, ns, lam, seed, S):
    g = np.concatenate([S[:, N:] * (1.0 + 0.01 * (synth.uniform_matrix(seed + 1, ns, N) - 0.5)),
                        0.01 * synth.uniform_matrix(seed + 3, ns, N),
                        lam * (1.0 + 0.02 * (synth.uniform_matrix(seed + 2, ns, 1) - 0.5))], 1)
    return np.ascontiguousarray(g)


def _run(M, h, S, g, prec, form, mode, jac=False):
    ns, m = S.shape[0], M.m
    M.set_node_mode(mode)
    sd, gd = torch.from_numpy(S).cuda(), torch.from_numpy(g).cuda()
    r = torch.zeros((ns, m), dtype=torch.float64, device="cuda")
    e = torch.zeros((ns, 2), dtype=torch.float64, device="cuda")
    J = torch.zeros((ns, m, m), dtype=torch.float64, device="cuda") if jac else None
    M.residual(h, sd, gd, r, J, e, prec, form)
    torch.cuda.synchronize()
    return r.cpu().numpy(), e.cpu().numpy(), (J.cpu().numpy() if jac else None)


def _scales(I, S, g, r):
    N = I.N
    k = S[:, N:]
    lhs = np.abs(g[:, 2 * N:] * (1 + I.p["phi"] * (g[:, :N] / k - 1))) + np.abs(g[:, N:2 * N])
    return np.concatenate([2 * lhs + np.abs(r[:, :N]), np.ones((S.shape[0], N)),
                           np.sum(S[:, :N] * I.A * k ** I.p["alpha"], 1, keepdims=True)], 1)


@pytest.mark.parametrize("N,ns", [(4, 100), (40, 6)])
def test_irreversible_residual_matches_oracle(G, N, ns):
    I, E, h, M, lam = _model(G, N)
    S = synth.irbc_states(synth.BASE_SEED + 701, ns, N)
    g = _guess(N, ns, lam, synth.BASE_SEED + 702, S)
    bsum = float(np.sum(np.abs(E.b_coeffs())))
    for form in (1, 0):
        r_ref, e_ref = I.residual(E, S, g, form=form, want_err=True)
        sc = _scales(I, S, g, r_ref)
        for prec, tol in ((0, 1e-11), (1, 1e-6 if form == 1 else 1e-7 * bsum)):
            for mode in (G.NODES_ALL, G.NODES_DELTA):
                r, e, _ = _run(M, h, S, g, prec, form, mode)
                assert np.all(np.abs(r - r_ref) <= tol * sc), (form, prec, mode, np.max(np.abs(r - r_ref) / sc))
                assert np.allclose(e, e_ref, rtol=0, atol=tol if prec else 1e-11)


def test_irreversible_jacobian_matches_central_differences(G):
    N = 3
    I, E, h, M, lam = _model(G, N)
    S = synth.irbc_states(synth.BASE_SEED + 703, 5, N)
    g = _guess(N, 5, lam, synth.BASE_SEED + 704, S)
    for mode in (G.NODES_ALL, G.NODES_DELTA):
        _, _, J = _run(M, h, S, g, 0, 1, mode, jac=True)
        eps = 1e-6
        for s in range(S.shape[0]):
            Jfd = np.zeros((2 * N + 1, 2 * N + 1))
            for c in range(2 * N + 1):
                gp = g[s].copy(); gp[c] += eps
                gm = g[s].copy(); gm[c] -= eps
                Jfd[:, c] = (I.residual(E, S[s:s + 1], gp[None])[0] - I.residual(E, S[s:s + 1], gm[None])[0]) / (2 * eps)
            assert np.all(np.abs(J[s] - Jfd) <= 1e-5 * np.maximum(1.0, np.abs(Jfd))), (mode, s, np.max(np.abs(J[s] - Jfd)))


def test_irreversible_newton_matches_oracle_with_binding_constraints(G):
    N = 3
    I, E, h, M, lam = _model(G, N, const_k=True)
    S = np.array([[1.0, 1.0, 1.0, 1.19, 1.0, 1.05], [0.8, 1.0, 1.1, 1.2, 0.9, 1.0],
                  [1.0, 1.0, 1.0, 1.0, 1.0, 1.0], [0.9, 1.1, 1.0, 0.85, 1.15, 1.0]])
    g0 = np.concatenate([S[:, N:], np.zeros((S.shape[0], N)), np.full((S.shape[0], 1), lam)], 1)
    sol_ref, _, nrm_ref = I.newton(E, S, g0, tol=1e-10)
    assert np.all(nrm_ref <= 1e-10)
    for mode in (G.NODES_ALL, G.NODES_DELTA):
        M.set_node_mode(mode)
        sd = torch.from_numpy(S).cuda()
        z = torch.from_numpy(g0.copy()).cuda()
        st = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
        M.newton(h, sd, z, 40, 1e-10, None, st, None, 0, 1)
        torch.cuda.synchronize()
        z = z.cpu().numpy()
        assert np.all(st.cpu().numpy() == 0)
        assert np.allclose(z, sol_ref, atol=1e-8)
    dl = I.p["delta"]
    inv = sol_ref[:, :N] - (1 - dl) * S[:, N:]
    mu = sol_ref[:, N:2 * N]
    assert (mu > 1e-4).any() and (inv > 1e-4).any()     # some countries bind, some invest
    M.set_node_mode(G.NODES_ALL)
    with pytest.raises(G.DDSGError, match="N\\+1 outputs"):
        I2, E2, h2, M2, _ = _model(G, 2)
        M2.set_irreversible(False)
        M2.residual(h2, torch.ones((1, 4), dtype=torch.float64, device="cuda"),
                    torch.ones((1, 3), dtype=torch.float64, device="cuda"),
                    torch.zeros((1, 3), dtype=torch.float64, device="cuda"))
