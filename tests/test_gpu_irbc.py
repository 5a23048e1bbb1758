"""GPU parity of the IRBC model step (euler_residual, Jacobian, LU, Newton)
against the CPU oracle (Sec. 2.1: eq. model1, model2, law_of_motion).

Bars: residuals FP64 |dr| <= 1e-11 * scale, F32C <= 1e-6 * scale with
scale = |lambda (1 + phi g)| + beta |E| per row (the two sides of eq. model1;
the resource row uses sum_j Y_j); Jacobian vs central differences of the
oracle's residual: |dJ| <= 1e-5 * max(1, |J|) (finite-difference truncation);
Newton: both sides converge to ||r||_inf <= 1e-10 and agree to 1e-7."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def make_model(G, N, level=4, sigma=0.01, seed=synth.BASE_SEED + synth.W_IRBC150, amp=1.0):
    I = O.IRBCOracle(N, sigma=sigma)
    lam = I.steady_lambda()
    base = np.concatenate([np.ones(N), [lam]])
    pert = synth.irbc_policy_perturbation(seed, N)
    pert = tuple(p * amp if i != 1 else p for i, p in enumerate(pert))
    fn = lambda dims, X: synth.irbc_policy_values(base, pert, dims, X)
    E = O.irbc_policy_ddsg(N, level, fn)
    d = 2 * N
    h = G.HDMR(d, N + 1, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    comps = [()] + [(i,) for i in range(d)] + [(j, N + j) for j in range(N)]
    for u in comps:
        h.add_regular(list(u), level)
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    return I, E, h, M, lam


def states_and_guess(N, ns, lam, seed):
    S = synth.irbc_states(seed, ns, N)
    g = np.concatenate([S[:, N:] * (1.0 + 0.01 * (synth.uniform_matrix(seed + 1, ns, N) - 0.5)),
                        lam * (1.0 + 0.02 * (synth.uniform_matrix(seed + 2, ns, 1) - 0.5))], 1)
    return S, np.ascontiguousarray(g)


def gpu_residual(M, h, S, g, prec, form, jac=False):
    ns, N = S.shape[0], M.N
    sd = torch.from_numpy(S).cuda()
    gd = torch.from_numpy(g).cuda()
    r = torch.zeros((ns, N + 1), dtype=torch.float64, device="cuda")
    e = torch.zeros((ns, 2), dtype=torch.float64, device="cuda")
    J = torch.zeros((ns, N + 1, N + 1), dtype=torch.float64, device="cuda") if jac else None
    M.residual(h, sd, gd, r, J, e, prec, form)
    torch.cuda.synchronize()
    return r.cpu().numpy(), e.cpu().numpy(), (J.cpu().numpy() if jac else None)


def scales(I, S, g, r):
    N = I.N
    k = S[:, N:]
    lhs = np.abs(g[:, N:N + 1] * (1 + I.p["phi"] * (g[:, :N] / k - 1)))
    sc = np.concatenate([2 * lhs + np.abs(r[:, :N]),
                         np.sum(S[:, :N] * I.A * k ** I.p["alpha"], 1, keepdims=True)], 1)
    return sc


@pytest.mark.parametrize("N,ns", [(10, 200), (150, 8)])
def test_residual_matches_oracle(G, N, ns):
    I, E, h, M, lam = make_model(G, N)
    S, g = states_and_guess(N, ns, lam, synth.BASE_SEED + 401)
    # The paper form sums b_v-weighted component interpolants (b_empty = 1 - N):
    # FP32 rounding is amplified by sum_v |b_v| (the cancellation the slice-free
    # form removes), so its F32C bar is u_32-sized times that factor.
    bsum = float(np.sum(np.abs(E.b_coeffs())))
    for form in (1, 0):
        r_ref, e_ref = I.residual(E, S, g, form=form, want_err=True)
        sc = scales(I, S, g, r_ref)
        for prec, tol in ((0, 1e-11), (1, 1e-6 if form == 1 else 1e-7 * bsum)):
            r, e, _ = gpu_residual(M, h, S, g, prec, form)
            assert np.all(np.abs(r - r_ref) <= tol * sc), (form, prec, np.max(np.abs(r - r_ref) / sc))
            # Euler error = |beta E / lhs - 1|: compare absolutely (it subtracts numbers near 1)
            assert np.allclose(e, e_ref, rtol=0, atol=tol if prec else 1e-11)


def test_steady_state_residual_is_zero(G):
    N = 6
    I, E, h, M, lam = make_model(G, N, sigma=0.0, amp=0.0)
    S = np.ones((3, 2 * N))
    g = np.tile(np.concatenate([np.ones(N), [lam]]), (3, 1))
    for prec in (0, 1):
        r, e, _ = gpu_residual(M, h, S, g, prec, 1)
        assert np.max(np.abs(r)) < (1e-12 if prec == 0 else 1e-6)


def test_jacobian_matches_central_differences(G):
    N = 4
    I, E, h, M, lam = make_model(G, N)
    S, g = states_and_guess(N, 5, lam, synth.BASE_SEED + 402)
    _, _, J = gpu_residual(M, h, S, g, 0, 1, jac=True)
    eps = 1e-6
    for s in range(S.shape[0]):
        Jfd = np.zeros((N + 1, N + 1))
        for c in range(N + 1):
            gp = g[s].copy(); gp[c] += eps
            gm = g[s].copy(); gm[c] -= eps
            Jfd[:, c] = (I.residual(E, S[s:s + 1], gp[None])[0] - I.residual(E, S[s:s + 1], gm[None])[0]) / (2 * eps)
        assert np.all(np.abs(J[s] - Jfd) <= 1e-5 * np.maximum(1.0, np.abs(Jfd))), (s, np.max(np.abs(J[s] - Jfd)))


def test_lu_solve_batched(G):
    rng = np.random.default_rng(5)
    ns, n = 7, 12
    A = rng.normal(size=(ns, n, n)) + 4 * np.eye(n)
    r = rng.normal(size=(ns, n))
    A[3] = 0.0   # a singular system
    Ad = torch.from_numpy(A).cuda()
    rd = torch.from_numpy(r).cuda()
    dx = torch.zeros((ns, n), dtype=torch.float64, device="cuda")
    st = torch.zeros(ns, dtype=torch.int32, device="cuda")
    G.lu_solve(Ad, rd, dx, st)
    torch.cuda.synchronize()
    dx, st = dx.cpu().numpy(), st.cpu().numpy()
    for s in range(ns):
        if s == 3:
            assert st[s] == 2
        else:
            assert st[s] == 0 and np.allclose(A[s] @ dx[s], -r[s], atol=1e-12)


def test_lu_solve_n151_mixed_precision_and_fallback(G):
    """Systems of the N=150 model's size. The FP32 factors with FP64 refinement
    must reach FP64 backward error. Systems too ill-conditioned for FP32
    (condition numbers 1e9 and 1e12) must come back just as accurate through
    the FP64 re-solve, and an exactly singular one must be flagged."""
    rng = np.random.default_rng(17)
    n = 151
    conds = [1.0, 1e2, 1e4, 1e6, 1e9, 1e12]
    A, R = [], []
    for i in range(24):
        c = conds[i % len(conds)]
        q1, _ = np.linalg.qr(rng.normal(size=(n, n)))
        q2, _ = np.linalg.qr(rng.normal(size=(n, n)))
        A.append(q1 @ np.diag(np.logspace(0, -np.log10(c), n)) @ q2 * rng.uniform(0.1, 10.0))
        R.append(rng.normal(size=n))
    A.append(rng.normal(size=(n, n)))
    A[-1][:, 7] = 0.0                      # singular
    R.append(rng.normal(size=n))
    A, R = np.array(A), np.array(R)
    ns = A.shape[0]
    dx = torch.zeros((ns, n), dtype=torch.float64, device="cuda")
    st = torch.full((ns,), 9, dtype=torch.int32, device="cuda")
    G.lu_solve(torch.from_numpy(A).cuda(), torch.from_numpy(R).cuda(), dx, st)
    torch.cuda.synchronize()
    dx, st = dx.cpu().numpy(), st.cpu().numpy()
    assert st[-1] == 2
    for s in range(ns - 1):
        c = conds[s % len(conds)]
        if c <= 1e2 or c >= 1e9:
            assert st[s] == (1 if c >= 1e9 else 0), (s, c, st[s])   # 1: the FP64 re-solve ran
        else:
            assert st[s] in (0, 1), (s, c, st[s])
        back = np.abs(A[s] @ dx[s] + R[s]).max() / (np.abs(A[s]).sum(1).max() * np.abs(dx[s]).max() + np.abs(R[s]).max())
        assert back <= 1e-14, (s, conds[s % len(conds)], back)
        ref = np.linalg.solve(A[s], -R[s])
        fwd = np.abs(dx[s] - ref).max() / np.abs(ref).max()
        assert fwd <= 1e-15 * conds[s % len(conds)] * n, (s, fwd)


@pytest.mark.parametrize("prec", [0, 1])
def test_newton_matches_oracle(G, prec):
    N = 5
    I, E, h, M, lam = make_model(G, N)
    S, g = states_and_guess(N, 6, lam, synth.BASE_SEED + 403)
    sol_ref, its_ref, nrm_ref = I.newton(E, S, g, tol=1e-10)
    assert np.all(nrm_ref <= 1e-10)
    sd = torch.from_numpy(S).cuda()
    z = torch.from_numpy(g.copy()).cuda()
    it = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
    stt = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
    nr = torch.zeros(S.shape[0], dtype=torch.float64, device="cuda")
    tol = 1e-10 if prec == 0 else 1e-6
    M.newton(h, sd, z, 30, tol, it, stt, nr, prec, 1)
    torch.cuda.synchronize()
    assert np.all(stt.cpu().numpy() == 0) and np.all(nr.cpu().numpy() <= tol)
    assert np.all(it.cpu().numpy() <= 10)
    assert np.allclose(z.cpu().numpy(), sol_ref, atol=1e-7 if prec == 0 else 1e-5)


@pytest.mark.parametrize("mode,prec", [("all", 0), ("delta", 0), ("delta", 1)])
def test_newton_batch_equals_states_solved_apart(G, mode, prec):
    """States that converge after different numbers of iterations leave the
    Newton working set as they converge (the live ones are gathered into
    contiguous slots). Per-state arithmetic does not depend on the slot, so
    the batch must give, bit for bit, the solution, iteration count, status
    and residual norm of each state solved in a batch of its own. Guesses
    from 1x to 8x the base perturbation spread the iteration counts; one state
    gets a non-finite guess (status 1 after the iteration cap, or the
    residual stays NaN)."""
    N = 10
    I, E, h, M, lam = make_model(G, N)
    M.set_node_mode(G.NODES_DELTA if mode == "delta" else G.NODES_ALL)
    S, g = states_and_guess(N, 24, lam, synth.BASE_SEED + 405)
    scale = np.repeat([1.0, 2.0, 4.0, 8.0], 6)[:, None]
    base = np.concatenate([S[:, N:], np.full((24, 1), lam)], 1)
    g = np.ascontiguousarray(base + scale * (g - base))
    g[5, 0] = np.nan

    def solve(idx):
        sd = torch.from_numpy(np.ascontiguousarray(S[idx])).cuda()
        z = torch.from_numpy(np.ascontiguousarray(g[idx])).cuda()
        it = torch.zeros(len(idx), dtype=torch.int32, device="cuda")
        stt = torch.zeros(len(idx), dtype=torch.int32, device="cuda")
        nr = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
        M.newton(h, sd, z, 12, 1e-10 if prec == 0 else 1e-6, it, stt, nr, prec, 1)
        torch.cuda.synchronize()
        return z.cpu().numpy(), it.cpu().numpy(), stt.cpu().numpy(), nr.cpu().numpy()

    try:
        zb, itb, stb, nrb = solve(np.arange(24))
        if prec == 0:
            assert len(set(itb[stb == 0].tolist())) >= 2, itb   # the working set did shrink
        for s in range(24):
            z1, it1, st1, nr1 = solve(np.array([s]))
            assert it1[0] == itb[s] and st1[0] == stb[s], (s, it1, itb[s], st1, stb[s])
            assert np.array_equal(z1[0], zb[s], equal_nan=True), s
            assert np.array_equal(nr1[0], nrb[s], equal_nan=True), s
    finally:
        M.set_node_mode(G.NODES_ALL)
