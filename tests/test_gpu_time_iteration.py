"""GPU adaptive DDSG time iteration (paper_2202_06555_gb300.time_iteration)
against the oracle's (oracle/time_iteration.py): GPU component quadratures
drive eq. 3.18 / 3.19 to the closed-form values; one and two time-iteration
steps give the oracle's component sets and policies (|dy| <= 1e-8 at fresh
states); the iteration lowers the Euler errors."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle.time_iteration import oracle_build_ddsg, oracle_solver, oracle_time_iteration
from test_oracle_time_iteration import _abs_product, _initial_policy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def test_gpu_quadrature_matches_oracle(G):
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + 61, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref = O.OracleDDSG(d, m)
    h = G.HDMR(d, m, 2)
    for u in O.full_order_components(d, 2):
        ref.add_regular(u, 2)
        h.add_regular(list(u), 2)
    ref.build_adaptive(fn, 1e-3, 7)
    G.build_adaptive(h, fn, 1e-3, 7)
    q = h.quadrature().cpu().numpy()
    Q = ref.quadrature()
    assert np.allclose(q, Q, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d,order", [(4, 2), (5, 3)])
def test_expansion_norms_match_oracle(G, d, order):
    """hdmr_expansion_norms (the cut-HDMR component integrals by inclusion-exclusion,
    eta per component, eq. 3.19, and rho, eq. 3.18) against the oracle's
    expansion_rho / active_eta on an adaptive expansion of the kinked family."""
    m = 3
    c = synth.family_coeffs(synth.BASE_SEED + 62 + d, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref = O.OracleDDSG(d, m)
    h = G.HDMR(d, m, order)
    comps = O.full_order_components(d, order)
    for u in comps:
        ref.add_regular(u, 2)
        h.add_regular(list(u), 2)
    ref.build_adaptive(fn, 1e-3, 6)
    G.build_adaptive(h, fn, 1e-3, 6)
    Qf_ref = ref.cut_component_quadratures()
    for k in range(1, order + 1):
        qf, eta, rho_all, rho_kept = h.expansion_norms(k, eps_eta=-1.0)
        assert np.allclose(qf, Qf_ref, rtol=1e-12, atol=1e-15)
        assert abs(rho_all - ref.expansion_rho(k)) <= 1e-12 * max(1.0, ref.expansion_rho(k))
        assert rho_kept == rho_all
        for ci, u in enumerate(comps):
            if len(u) == k:
                assert abs(eta[ci] - ref.active_eta(u)) <= 1e-12 * max(1.0, ref.active_eta(u)), u
            else:
                assert np.isnan(eta[ci])
    # a threshold between the order-2 etas: rho over the components above it only
    qf, eta, _, _ = h.expansion_norms(2)
    thr = float(np.nanmedian(eta))
    _, _, _, rho_kept = h.expansion_norms(2, eps_eta=thr)
    lower = qf[[ci for ci, u in enumerate(comps) if len(u) <= 1]].sum(0)
    kept = qf[[ci for ci, u in enumerate(comps) if len(u) == 2 and eta[ci] > thr]].sum(0)
    assert abs(rho_kept - np.linalg.norm(kept) / np.linalg.norm(lower)) <= 1e-12
    h.close()


def test_eta_rho_closed_forms_on_gpu(G):
    from paper_2202_06555_gb300.time_iteration import build_ddsg
    d, m = 3, 2
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    h, info = build_ddsg(_abs_product, d, m, 2, 3, -1.0, -1.0, 0.0, lo, hi)
    assert len(info["components"]) == 7
    assert abs(info["eta"][(0, 1)] - 0.01 * np.sqrt(1.25) / np.sqrt(5.0)) < 1e-14
    assert info["eta"][(0, 2)] < 1e-15 and info["eta"][(1, 2)] < 1e-15
    assert info["rho"][0] < 1e-15 and abs(info["rho"][1] - info["eta"][(0, 1)]) < 1e-14
    h2, info2 = build_ddsg(_abs_product, d, m, 2, 3, -1.0, 1e-6, 0.0, lo, hi)
    assert info2["components"] == [(), (0,), (1,), (2,), (0, 1)]
    X = synth.uniform_matrix(3, 50, d, 0.8, 1.2)
    y = torch.empty((50, m), dtype=torch.float64, device="cuda")
    h2.eval(torch.from_numpy(X).cuda(), y, G.F64, G.FORM_SLICEFREE)
    torch.cuda.synchronize()
    assert np.allclose(y.cpu().numpy(), _abs_product(X), atol=1e-14)


def _gpu_initial_policy(G, I, N):
    lam = I.steady_lambda()
    d = 2 * N
    h = G.HDMR(d, N + 1, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    comps = [()] + [(i,) for i in range(d)]
    for u in comps:
        h.add_regular(list(u), 2)
    vals = []
    for c, u in enumerate(comps):
        _, _, xs = h.component_points(c)
        y = np.tile(np.concatenate([np.ones(N), [lam]]), (xs.shape[0], 1))
        for a, dim in enumerate(u):
            if dim >= N:
                y[:, dim - N] = xs[:, a]
        vals.append(y)
    h.hierarchize(torch.from_numpy(np.concatenate(vals)).cuda())
    return h


@pytest.mark.parametrize("mode,all_pairs", [(0, False), (1, False), (1, True)])
def test_time_iteration_matches_oracle(G, mode, all_pairs):
    from paper_2202_06555_gb300.time_iteration import time_iteration
    N = 2
    d = 2 * N
    I = O.IRBCOracle(N)
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    pairs = None if all_pairs else (lambda k: [(i,) for i in range(d)] if k == 1 else [(j, N + j) for j in range(N)])
    T = synth.irbc_states(synth.BASE_SEED + 601, 64, N)
    E0 = _initial_policy(I, N)
    Eo, hist_o = oracle_time_iteration(I, E0, 2, 2, 3, -1.0, -1.0, 0.0, lo, hi, T, candidates=pairs)
    h0 = _gpu_initial_policy(G, I, N)
    hg, hist_g = time_iteration(M, h0, 2, 2, 3, -1.0, -1.0, 0.0, lo, hi, T, candidates=pairs,
                                precision=G.F64, node_mode=mode)
    assert [h["components"] for h in hist_g] == [len(h["info"]["components"]) for h in hist_o]
    assert all(h["newton_failed"] == 0 for h in hist_g)
    y = torch.empty((T.shape[0], N + 1), dtype=torch.float64, device="cuda")
    hg.eval(torch.from_numpy(T).cuda(), y, G.F64, G.FORM_SLICEFREE)
    torch.cuda.synchronize()
    assert np.max(np.abs(y.cpu().numpy() - Eo.eval(T, form=1)["y"])) <= 1e-8
    for a, b in zip(hist_g, hist_o):
        assert abs(a["euler_error_mean"] - b["euler_error_mean"]) <= 1e-8
    assert hist_g[1]["euler_error_mean"] < hist_g[0]["euler_error_mean"]


def test_irreversible_time_iteration_matches_oracle(G):
    """Non-smooth model (policy (k', mu, lambda)): two adaptive time-iteration
    steps over the (a_j, k_j) pairs, GPU vs oracle."""
    from paper_2202_06555_gb300.time_iteration import time_iteration
    N = 2
    d, m = 2 * N, 2 * N + 1
    I = O.IRBCOracle(N, irreversible=True)
    lam = I.steady_lambda()
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    M.set_irreversible(True)
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    comps = [()] + [(i,) for i in range(d)]

    def init_vals(u, xs):
        y = np.tile(np.concatenate([np.ones(N), np.zeros(N), [lam]]), (xs.shape[0], 1))
        for a, dim in enumerate(u):
            if dim >= N:
                y[:, dim - N] = xs[:, a]
        return y

    E0 = O.OracleDDSG(d, m, lo=lo, hi=hi)
    h0 = G.HDMR(d, m, 2, lo=lo, hi=hi)
    for u in comps:
        E0.add_regular(u, 2)
        h0.add_regular(list(u), 2)
    E0.fill_values(lambda dims, X: init_vals(dims, np.atleast_2d(X)))
    E0.hierarchize()
    h0.hierarchize(torch.from_numpy(np.concatenate(
        [init_vals(u, h0.component_points(c)[2]) for c, u in enumerate(comps)])).cuda())
    pairs = lambda k: [(i,) for i in range(d)] if k == 1 else [(j, N + j) for j in range(N)]
    T = synth.irbc_states(synth.BASE_SEED + 602, 64, N)
    Eo, hist_o = oracle_time_iteration(I, E0, 2, 2, 3, -1.0, -1.0, 0.0, lo, hi, T, candidates=pairs)
    hg, hist_g = time_iteration(M, h0, 2, 2, 3, -1.0, -1.0, 0.0, lo, hi, T, candidates=pairs, precision=G.F64)
    assert all(h["newton_failed"] == 0 for h in hist_g)
    y = torch.empty((T.shape[0], m), dtype=torch.float64, device="cuda")
    hg.eval(torch.from_numpy(T).cuda(), y, G.F64, G.FORM_SLICEFREE)
    torch.cuda.synchronize()
    assert np.max(np.abs(y.cpu().numpy() - Eo.eval(T, form=1)["y"])) <= 1e-8
    for a, b in zip(hist_g, hist_o):
        assert abs(a["euler_error_mean"] - b["euler_error_mean"]) <= 1e-8


def test_time_iteration_resumes_from_a_checkpoint(G, tmp_path):
    """Two steps in one run equal one step, a save, a load and one more step."""
    from paper_2202_06555_gb300.time_iteration import time_iteration
    N = 2
    d = 2 * N
    I = O.IRBCOracle(N)
    M = G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"], I.p["phi"],
               I.A, I.gamma, I.tau)
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    T = synth.irbc_states(synth.BASE_SEED + 603, 32, N)
    ck = str(tmp_path / "ti.ddsg")
    h2, _ = time_iteration(M, _gpu_initial_policy(G, I, N), 2, 2, 4, 1e-4, 1e-5, 0.0, lo, hi, T)
    h1, _ = time_iteration(M, _gpu_initial_policy(G, I, N), 1, 2, 4, 1e-4, 1e-5, 0.0, lo, hi, T, checkpoint=ck)
    from paper_2202_06555_gb300.time_iteration import resume
    p0, done, hist = resume(ck)
    assert done == 1 and len(hist) == 1 and hist[0]["step"] == 0
    hr, hist2 = time_iteration(M, p0, 1, 2, 4, 1e-4, 1e-5, 0.0, lo, hi, T, start_step=done, history0=hist)
    assert [r["step"] for r in hist2] == [0, 1]
    x = torch.from_numpy(T).cuda()
    ya = torch.empty((T.shape[0], N + 1), dtype=torch.float64, device="cuda")
    yb = torch.empty_like(ya)
    h2.eval(x, ya, G.F64, G.FORM_SLICEFREE)
    hr.eval(x, yb, G.F64, G.FORM_SLICEFREE)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
