"""GPU parity of the node shortcut (irbc_set_node_mode(NODES_DELTA)): the policy
at the 2(N+1) monomial nodes from the no-shock state, the two global-shock
nodes and per-component deltas for the country nodes. Checked against the CPU
oracle's residual (which interpolates every node as written) with the bars of
tests/test_gpu_irbc.py, against the GPU's all-node path (FP64: 1e-13 * scale),
for the Jacobian, for Newton, on a component set with extra (a_i, a_j) and
(a_i, k_j) pairs, and for non-finite states."""
import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_irbc import make_model, states_and_guess, scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def run(G, M, h, S, g, prec, form, mode, jac=False):
    ns, N = S.shape[0], M.N
    M.set_node_mode(mode)
    sd = torch.from_numpy(S).cuda()
    gd = torch.from_numpy(g).cuda()
    r = torch.zeros((ns, N + 1), dtype=torch.float64, device="cuda")
    e = torch.zeros((ns, 2), dtype=torch.float64, device="cuda")
    J = torch.zeros((ns, N + 1, N + 1), dtype=torch.float64, device="cuda") if jac else None
    M.residual(h, sd, gd, r, J, e, prec, form)
    torch.cuda.synchronize()
    M.set_node_mode(G.NODES_ALL)
    return r.cpu().numpy(), e.cpu().numpy(), (J.cpu().numpy() if jac else None)


@pytest.mark.parametrize("N,ns", [(10, 200), (150, 8)])
def test_delta_nodes_match_oracle_and_all_nodes(G, N, ns):
    I, E, h, M, lam = make_model(G, N)
    S, g = states_and_guess(N, ns, lam, synth.BASE_SEED + 411)
    bsum = float(np.sum(np.abs(E.b_coeffs())))
    for form in (1, 0):
        r_ref, e_ref = I.residual(E, S, g, form=form, want_err=True)
        sc = scales(I, S, g, r_ref)
        for prec, tol in ((0, 1e-11), (1, 1e-6 if form == 1 else 1e-7 * bsum)):
            r, e, J = run(G, M, h, S, g, prec, form, G.NODES_DELTA, jac=True)
            assert np.all(np.abs(r - r_ref) <= tol * sc), (form, prec, np.max(np.abs(r - r_ref) / sc))
            assert np.allclose(e, e_ref, rtol=0, atol=tol if prec else 1e-11)
            r_all, _, J_all = run(G, M, h, S, g, prec, form, G.NODES_ALL, jac=True)
            if prec == 0:
                assert np.all(np.abs(r - r_all) <= 1e-13 * sc), (form, np.max(np.abs(r - r_all) / sc))
                assert np.allclose(J, J_all, rtol=1e-12, atol=1e-12)


def test_delta_nodes_general_component_set(G):
    """Extra (a_0, a_1), (a_1, a_3), (a_2, k_3) and (k_0, k_1) pairs with their
    own interactions: the delta for country i sums every component holding
    a_i, and the Jacobian column of k'_i every component holding k_i."""
    N, level = 5, 4
    I = O.IRBCOracle(N, sigma=0.01)
    lam = I.steady_lambda()
    base = np.concatenate([np.ones(N), [lam]])
    pert = synth.irbc_policy_perturbation(synth.BASE_SEED + 412, N)
    extra = [(0, 1), (1, 3), (2, N + 3), (N + 0, N + 1)]

    def fn(dims, X):
        X = np.asarray(X, np.float64)
        if X.ndim == 1:
            X = X.reshape(-1, len(dims))
        y = synth.irbc_policy_values(base, pert, dims, X)
        pos = {dim: a for a, dim in enumerate(dims)}
        for t, (u, v) in enumerate(extra):
            if u in pos and v in pos:
                w = np.sin(7.0 * (X[:, pos[u]] - 1.0)) * np.sin(5.0 * (X[:, pos[v]] - 1.0))
                y += 0.01 * (t + 1) * w[:, None] * np.linspace(1.0, 2.0, N + 1)[None, :]
        return y

    d = 2 * N
    comps = [()] + [(i,) for i in range(d)] + [(j, N + j) for j in range(N)] + extra
    E = O.OracleDDSG(d, N + 1, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    h = G.HDMR(d, N + 1, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in comps:
        E.add_regular(u, level)
        h.add_regular(list(u), level)
    E.fill_values(fn)
    E.hierarchize()
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    S, g = states_and_guess(N, 64, lam, synth.BASE_SEED + 413)
    for form in (1, 0):
        r_ref = I.residual(E, S, g, form=form)
        sc = scales(I, S, g, r_ref)
        for prec in (0, 1):
            r, _, _ = run(G, M, h, S, g, prec, form, G.NODES_DELTA)
            # the bars of the all-node tests: FP64 1e-11; F32C 1e-6 (slice-free),
            # 1e-7 x sum |b| (paper form, whose terms carry the coefficients b)
            tol = 1e-11 if prec == 0 else (1e-6 if form == 1 else 1e-7 * float(np.sum(np.abs(E.b_coeffs()))))
            assert np.all(np.abs(r - r_ref) <= tol * sc), (form, prec, np.max(np.abs(r - r_ref) / sc))
    # the analytic Jacobian on this component set (k_i held by {k_i}, (a_i, k_i),
    # (a_2, k_3) and (k_0, k_1)) against central differences of the oracle
    eps = 1e-6
    for mode in (G.NODES_ALL, G.NODES_DELTA):
        _, _, J = run(G, M, h, S[:4], g[:4], 0, 1, mode, jac=True)
        for s in range(4):
            Jfd = np.zeros((N + 1, N + 1))
            for c in range(N + 1):
                gp = g[s].copy(); gp[c] += eps
                gm = g[s].copy(); gm[c] -= eps
                Jfd[:, c] = (I.residual(E, S[s:s + 1], gp[None])[0] - I.residual(E, S[s:s + 1], gm[None])[0]) / (2 * eps)
            assert np.all(np.abs(J[s] - Jfd) <= 1e-5 * np.maximum(1.0, np.abs(Jfd))), (mode, s, np.max(np.abs(J[s] - Jfd)))


def test_delta_nodes_newton_and_nonfinite_states(G):
    N = 5
    I, E, h, M, lam = make_model(G, N)
    S, g = states_and_guess(N, 6, lam, synth.BASE_SEED + 414)
    sol_ref, _, nrm_ref = I.newton(E, S, g, tol=1e-10)
    M.set_node_mode(G.NODES_DELTA)
    sd = torch.from_numpy(S).cuda()
    z = torch.from_numpy(g.copy()).cuda()
    it = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
    st = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
    M.newton(h, sd, z, 30, 1e-10, it, st, None, 0, 1)
    torch.cuda.synchronize()
    M.set_node_mode(G.NODES_ALL)
    assert np.all(st.cpu().numpy() == 0)
    assert np.allclose(z.cpu().numpy(), sol_ref, atol=1e-7)
    S2 = S.copy()
    S2[2, 1] = np.nan
    g2 = g.copy()
    g2[4, N] = np.inf
    r, _, _ = run(G, M, h, S2, g2, 1, 1, G.NODES_DELTA)
    bad = ~np.isfinite(r).all(1)
    assert bad[2] and bad[4] and not bad[[0, 1, 3, 5]].any()
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        M.set_node_mode(7)


def test_delta_nodes_with_more_terms_than_the_list_holds(G):
    """Every pair at level 7 (N = 3): a_i is held by 6 components with up to
    7 + 5 x 28 tuples, more active terms per a'-value than the delta kernel's
    shared term list holds, so the warp walks those pairs' tuples itself. Same
    results as the all-node path and the oracle."""
    N, level = 3, 7
    I = O.IRBCOracle(N, sigma=0.01)
    lam = I.steady_lambda()
    base = np.concatenate([np.ones(N), [lam]])
    pert = synth.irbc_policy_perturbation(synth.BASE_SEED + 414, N)
    fn = lambda dims, X: synth.irbc_policy_values(base, pert, dims, X)
    d = 2 * N
    comps = O.full_order_components(d, 2)
    E = O.OracleDDSG(d, N + 1, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    h = G.HDMR(d, N + 1, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in comps:
        E.add_regular(u, level)
        h.add_regular(list(u), level)
    E.fill_values(fn)
    E.hierarchize()
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    S, g = states_and_guess(N, 48, lam, synth.BASE_SEED + 415)
    r_ref = I.residual(E, S, g, form=1)
    sc = scales(I, S, g, r_ref)
    for prec in (0, 1):
        r_d, _, _ = run(G, M, h, S, g, prec, 1, G.NODES_DELTA)
        r_a, _, _ = run(G, M, h, S, g, prec, 1, G.NODES_ALL)
        assert np.all(np.abs(r_d - r_a) <= (1e-13 if prec == 0 else 1e-6) * sc), (prec, np.max(np.abs(r_d - r_a) / sc))
        if prec == 0:
            assert np.all(np.abs(r_d - r_ref) <= 1e-11 * sc), np.max(np.abs(r_d - r_ref) / sc)


@pytest.mark.parametrize("N", [80, 170, 200, 300])
def test_delta_nodes_wide_policies(G, N):
    """Policies of N + 1 = 81, 171, 201 and 301 outputs: the delta kernel's
    lanes hold 4, 6 and 8 outputs each (N = 150 takes 5), and at 301 outputs
    it takes two passes. States
    not a multiple of the 32 pairs a warp sums. Delta against the all-node
    path at the bars of the N = 150 case (the all-node path is pinned to the
    oracle there; the F32C bar is twice the oracle one)."""
    I = O.IRBCOracle(N, sigma=0.01)
    lam = I.steady_lambda()
    base = np.concatenate([np.ones(N), [lam]])
    pert = synth.irbc_policy_perturbation(synth.BASE_SEED + 416, N)
    fn = lambda dims, X: synth.irbc_policy_values(base, pert, dims, X)
    d = 2 * N
    h = G.HDMR(d, N + 1, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    comps = [()] + [(i,) for i in range(d)] + [(j, N + j) for j in range(N)]
    for u in comps:
        h.add_regular(list(u), 4)
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    S, g = states_and_guess(N, 3, lam, synth.BASE_SEED + 417)
    for form in (1, 0):
        for prec in (0, 1):
            r_d, _, _ = run(G, M, h, S, g, prec, form, G.NODES_DELTA)
            r_a, _, _ = run(G, M, h, S, g, prec, form, G.NODES_ALL)
            sc = scales(I, S, g, r_a)
            assert np.all(np.isfinite(r_d))
            # F32C: both paths within the oracle bar, so at most twice it apart
            tol = 1e-13 if prec == 0 else 2 * (1e-6 if form == 1 else 1e-7 * float(np.sum(np.abs(h.b_coeffs()))))
            assert np.all(np.abs(r_d - r_a) <= tol * sc), (form, prec, np.max(np.abs(r_d - r_a) / sc))
