"""GPU parity of libddsg against the CPU oracle, through the C ABI.

Bars (from the arithmetic: FP64 rounding over S, FP32 products folded into a
compensated FP32 sum for F32C):
  index work (grid point sets, active-set counts and hashes): bit-exact;
  FP64:  |y_gpu - y_oracle| <= 1e-12 * max(|y|, S), S = sum of |terms| (oracle);
  F32C:  |y_gpu - y_oracle| <= 1e-6  * max(|y|, S);
  surpluses: |alpha_gpu - alpha_oracle| <= 1e-13 * max|values| (cancellation in
  value - coarser interpolant makes a relative bar on alpha meaningless).
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def build_pair(G, d, m, comps, fn, eps=None, level=None, regular_level=2, strict=False,
               lo=None, hi=None, anchor=None):
    ref = O.OracleDDSG(d, m, lo=lo, hi=hi, anchor=anchor)
    h = G.HDMR(d, m, max(len(u) for u in comps), anchor=anchor, lo=lo, hi=hi)
    for u in comps:
        ref.add_regular(u, regular_level)
        h.add_regular(list(u), regular_level)
    if eps is None:
        ref.fill_values(fn)
        ref.hierarchize()
        vals = np.concatenate(ref.values)
        h.hierarchize(torch.from_numpy(vals).cuda())
    else:
        ref.build_adaptive(fn, eps, level, strict)
        G.build_adaptive(h, fn, eps, level, strict)
    return ref, h


def eval_gpu(h, X, prec, form, m, index=True):
    """Values from the configured schedule (no hash/count outputs, which the nodal
    kernel does not produce); with index=True also the active-set hashes and
    counts, from a second call that asks for them."""
    n = X.shape[0]
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.full((n, m), -7.0, dtype=torch.float64, device="cuda")
    h.eval(xd, y, prec, form)
    hs = ct = None
    if index:
        y2 = torch.full((n, m), -7.0, dtype=torch.float64, device="cuda")
        hs = torch.zeros(n, dtype=torch.int64, device="cuda")
        ct = torch.zeros(n, dtype=torch.int32, device="cuda")
        h.eval(xd, y2, prec, form, hs, ct)
        hs, ct = hs.cpu().numpy().view(np.uint64), ct.cpu().numpy()
    torch.cuda.synchronize()
    return y.cpu().numpy(), hs, ct


def oracle_results(ref, X, forms=(0, 1)):
    return {form: ref.eval(X, form=form, want=("y", "S", "hash", "count")) for form in forms}


def check_values(y, r, prec, what=""):
    """|y - y_oracle| <= TOL * max(|y|, S) on finite rows; NaN exactly on the others."""
    scale = np.maximum(np.abs(r["y"]), r["S"])
    fin = np.isfinite(r["y"]).all(1)
    assert np.array_equal(np.isnan(y).any(1), ~fin), what
    rel = np.abs(y[fin] - r["y"][fin]) / np.where(scale[fin] > 0, scale[fin], 1.0)
    assert rel.max(initial=0.0) <= TOL[prec], (what, rel.max())
    return float(rel.max(initial=0.0))


def check_eval(h, ref, X, forms=(0, 1), precs=(0, 1), res=None):
    worst = {}
    res = res or oracle_results(ref, X, forms)
    for form in forms:
        r = res[form]
        for prec in precs:
            y, hs, ct = eval_gpu(h, X, prec, form, ref.m)
            assert np.array_equal(ct, r["count"]), (form, prec)
            assert np.array_equal(hs, r["hash"]), (form, prec)
            worst[(form, prec)] = check_values(y, r, prec, (form, prec))
    return worst


# compiled (kernel, output chunk) pairs per precision: 0 tile, 1 per-tuple, 2-4 the
# level-tuple TMA kernels (chunk per warp group), 5 the nodal-slab kernel (32 = rotated windows)
SCHEDULES = {
    0: [(0, mc) for mc in (2, 4, 6, 8, 12, 16)] + [(1, mc) for mc in (2, 4, 6, 8, 12, 16)] +
       [(2, mc) for mc in (2, 4, 6, 8, 12, 16)] + [(3, mc) for mc in (4, 8, 16)] + [(4, mc) for mc in (4, 8)] +
       [(5, mc) for mc in (4, 8, 16)],
    1: [(0, mc) for mc in (4, 8, 12, 16, 28, 52)] + [(1, mc) for mc in (4, 8, 12, 16, 28, 52)] +
       [(2, mc) for mc in (4, 8, 12, 16, 28, 52)] + [(3, mc) for mc in (8, 16, 28)] + [(4, mc) for mc in (12, 20)] +
       [(5, mc) for mc in (32, 8, 16)] + [(6, 32)],
}


def check_every_schedule(G, h, ref, X, forms=(0, 1), precs=(0, 1), kernels=(0, 1, 2, 3, 4, 5, 6)):
    """Every eligible schedule against the oracle on the same queries, both forms:
    values within the bar, the index work (hash / count) once per form. Returns
    the schedules run and the worst relative error per (form, precision)."""
    res = oracle_results(ref, X, forms)
    ran, worst = [], {}
    saved = {(p, f): h.eval_config(p, f) for p in precs for f in forms}
    for form in forms:
        for prec in precs:
            _, hs, ct = eval_gpu(h, X, prec, form, ref.m)
            assert np.array_equal(ct, res[form]["count"]) and np.array_equal(hs, res[form]["hash"]), (form, prec)
            for kernel, mc in SCHEDULES[prec]:
                if kernel not in kernels:
                    continue
                try:
                    h.set_eval_config(prec, form, kernel, mc)
                except G.DDSGError as e:
                    assert "cannot run" in str(e), e
                    continue
                y, _, _ = eval_gpu(h, X, prec, form, ref.m, index=False)
                e = check_values(y, res[form], prec, (form, prec, kernel, mc))
                worst[(form, prec)] = max(worst.get((form, prec), 0.0), e)
                ran.append((form, prec, kernel, mc))
            h.set_eval_config(prec, form, *saved[(prec, form)])
    return ran, worst


def check_grids(h, ref):
    nc, P = h.sizes()
    assert nc == len(ref.comps)
    for c in range(nc):
        dims, npts, first = h.component_info(c)
        assert dims == ref.comps[c] and npts == ref.npts(c)
        k = len(dims)
        if k:
            lv, ix, _ = h.component_points(c)
            assert np.array_equal(lv, ref.lv[c][:, :k]) and np.array_equal(ix, ref.ix[c][:, :k]), c


def check_surpluses(h, ref):
    a = h.surpluses()
    b = np.concatenate(ref.alpha)
    v = np.concatenate(ref.values)
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(v)))


# ---------------------------------------------------------------------------

def test_regular_4d_single_grid(G):
    """d=4 level-5 regular sparse grid (401 points), m=3 kinked family."""
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + synth.W_SG4, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref, h = build_pair(G, d, m, [(0, 1, 2, 3)], fn, regular_level=5)
    assert h.sizes()[1] == 401
    check_surpluses(h, ref)
    X = synth.uniform_queries(synth.BASE_SEED + synth.W_SG4, 3000, d)
    check_eval(h, ref, X, forms=(0,))
    _, _, ct = eval_gpu(h, X, 0, 0, m)
    assert np.all(ct == 70)
    with pytest.raises(G.DDSGError, match="downward-closed"):
        eval_gpu(h, X, 0, 1, m)


def test_full_expansion_regular_d3(G):
    d, m = 3, 2
    f = lambda X: np.stack([np.exp(-np.sum(X ** 2, 1)), np.prod(np.sin(3 * X + 1), 1)], 1)
    def fn(dims, X):
        P = np.full((X.shape[0], d), 0.5)
        P[:, list(dims)] = X
        return f(P)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 3), fn, regular_level=5)
    assert np.array_equal(h.b_coeffs(), ref.b_coeffs())
    X = synth.uniform_queries(31, 2000, d)
    check_eval(h, ref, X)


@pytest.mark.parametrize("strict", [False, True])
def test_adaptive_d4_order2(G, strict):
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + 99, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=6,
                        strict=strict)
    check_grids(h, ref)
    check_surpluses(h, ref)
    X = np.concatenate([synth.uniform_queries(32, 4000, d), ref.node_coords(5)[:, [0, 0, 0, 0]]])
    check_eval(h, ref, X)
    # node coordinates sit on cell faces of the finer levels: every schedule
    ran, _ = check_every_schedule(G, h, ref, X[-600:])
    assert {k for _, _, k, _ in ran} >= {0, 1, 2, 3, 4, 5}


def test_adaptive_d20_order2_monomial_queries(G):
    """d=20 (N=10) order-2, eps 1e-3, level 10 on the kinked family with m=11;
    queries shaped like the monomial-rule nodes, some leaving [0,1] (clamped)."""
    d, m = 20, 11
    c = synth.family_coeffs(synth.BASE_SEED + synth.W_D20, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=10)
    check_grids(h, ref)
    check_surpluses(h, ref)
    X = synth.monomial_shaped_queries(synth.BASE_SEED + synth.W_D20, 60, 10, s=0.05)
    assert (X < 0).any() or (X > 1).any()
    h.stats(reset=True)
    w = check_eval(h, ref, X)
    st = h.stats()
    assert st["clamped"] > 0 and st["nonfinite_rows"] == 0
    # clamped coordinates at exactly 0 and 1 through every schedule
    ran, _ = check_every_schedule(G, h, ref, X[:400])
    assert {k for _, _, k, _ in ran} >= {0, 1, 2, 3, 4, 5}


def test_edge_queries(G):
    """Nodes, cell faces, domain corners, outside points, NaN/inf rows, n = 0, 1."""
    d, m = 3, 2
    c = synth.family_coeffs(7, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-4, level=8)
    pts = [np.zeros(d), np.ones(d), np.full(d, 0.5), np.array([0.25, 0.75, 0.125]),
           np.array([1 / 3, 2 / 3, 0.7]), np.array([-0.1, 1.3, 0.5]),
           np.array([5e-324, 1 - 2 ** -53, 2 ** -60]), np.array([0.5 + 2 ** -40, 0.5 - 2 ** -40, 0.7]),
           np.array([np.nan, 0.2, 0.3]), np.array([0.2, np.inf, 0.3]), np.array([0.2, 0.3, -np.inf])]
    for l in range(2, 9):
        pts.append(np.array([2.0 ** -(l - 1), 1 - 2.0 ** -(l - 1), 3 * 2.0 ** -(l - 1)]))
    X = np.array(pts)
    check_eval(h, ref, X)
    check_eval(h, ref, X[:1])
    h.stats(reset=True)
    eval_gpu(h, X, 0, 0, m, index=False)        # one evaluation call
    assert h.stats()["nonfinite_rows"] == 3
    y = torch.zeros((0, m), dtype=torch.float64, device="cuda")
    h.eval(torch.zeros((0, d), dtype=torch.float64, device="cuda"), y)
    # the same edge cases (faces, corners, clamps, NaN / inf rows, denormals) through
    # every schedule, including the staged kernels' face flags and bad-row path
    ran, _ = check_every_schedule(G, h, ref, X)
    assert {k for _, _, k, _ in ran} >= {0, 1, 2, 3, 4, 5}
    ran1, _ = check_every_schedule(G, h, ref, X[:1])
    assert len(ran1) == len(ran)


def test_physical_domain_and_anchor(G):
    """IRBC-like box [0.8, 1.2]^4 with the anchor at its centre; a non-central
    anchor is refused by the slice-free form but the paper form still holds."""
    d, m = 4, 2
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    f = lambda P: np.stack([np.log(P).sum(1), (P ** 0.36).prod(1)], 1)
    def fn_at(anchor):
        def fn(dims, X):
            P = np.repeat(anchor[None, :], X.shape[0], 0)
            P[:, list(dims)] = X
            return f(P)
        return fn
    comps = O.full_order_components(d, 2)
    ref, h = build_pair(G, d, m, comps, fn_at(np.full(d, 1.0)), eps=1e-5, level=7, lo=lo, hi=hi)
    X = synth.uniform_matrix(41, 1500, d, 0.75, 1.25)
    check_eval(h, ref, X)
    anc = np.array([0.9, 1.0, 1.1, 1.0])
    ref2, h2 = build_pair(G, d, m, comps, fn_at(anc), regular_level=4, lo=lo, hi=hi, anchor=anc)
    check_eval(h2, ref2, X, forms=(0,))
    with pytest.raises(G.DDSGError, match="slice-free"):
        eval_gpu(h2, X, 0, 1, m)


def test_eval_before_hierarchize_is_an_error(G):
    h = G.HDMR(2, 1, 1)
    h.add_component([])
    h.add_regular([0], 3)
    x = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    y = torch.zeros((4, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(G.DDSGError, match="ERR_STATE"):
        h.eval(x, y)


def test_every_kernel_config_matches_oracle(G):
    """Both evaluation kernels at every compiled output chunk, and the autotuner's
    pick, give the same active sets and values (d=6, order 2, m=11)."""
    d, m = 6, 11
    c = synth.family_coeffs(synth.BASE_SEED + 55, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=9)
    X = synth.uniform_queries(56, 700, d)
    ran, _ = check_every_schedule(G, h, ref, X)
    # every schedule but kernel 6, which needs m > 16 (32-output FP32 windows)
    assert len(ran) == 2 * (len(SCHEDULES[0]) + len(SCHEDULES[1]) - 1)
    xd = torch.from_numpy(X).cuda()
    yd = torch.empty((X.shape[0], m), dtype=torch.float64, device="cuda")
    for prec in (0, 1):
        kernel, mc, ms = h.autotune(xd, yd, prec, 1)
        assert (kernel, mc) in SCHEDULES[prec] and ms > 0
        check_eval(h, ref, X, forms=(1,), precs=(prec,))
    with pytest.raises(G.DDSGError, match="not compiled"):
        h.set_eval_config(0, 0, 0, 5)
    assert h.stats()["wait_timeouts"] == 0


@pytest.mark.parametrize("m", [20, 33, 64, 96, 151])
def test_nodal_kernels_wide_outputs(G, m):
    """The nodal-slab kernels at output counts that fill one window (20, 32 padded),
    spill into a second (33 -> 64), fill two (64), or take 3 and 5 windows (96,
    151 -> 160), on an adaptive d = 5 order-2 expansion, at uniform queries and
    the edge cases (nodes, faces, corners, clamped and non-finite rows), against
    the oracle. Kernel 6 keeps its totals in tensor memory and gives each warp
    group of a block one (query tile, window) item: with 1, 3 or 5 windows a
    block's two groups take different tiles, or one group finds no item. At 151
    outputs the grid stops at level 5 so that a component's node rows fit the
    shared staging buffer."""
    d = 5
    c = synth.family_coeffs(synth.BASE_SEED + 63 + m, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=8 if m <= 96 else 5)
    pts = [np.zeros(d), np.ones(d), np.full(d, 0.5), np.array([0.25, 0.75, 0.125, 0.375, 0.625]),
           np.array([-0.2, 1.4, 0.5, 0.5, 2.0]), np.array([np.nan, 0.2, 0.3, 0.4, 0.5])]
    X = np.concatenate([np.array(pts), ref.node_coords(d + 3)[:, [0, 0, 0, 0, 0]][:60],
                        synth.uniform_queries(64, 700, d)])
    ran, worst = check_every_schedule(G, h, ref, X, kernels=(5, 6))
    assert {(k, mc) for f, p, k, mc in ran if p == 1} == {(5, 32), (5, 8), (5, 16), (6, 32)}
    assert h.stats()["wait_timeouts"] == 0


def test_staged_kernel_refuses_tables_it_cannot_hold(G):
    """The TMA-staged kernels need k <= 2 components; a 3D component makes them ineligible."""
    d, m = 3, 2
    f = lambda X: np.stack([np.exp(-np.sum(X ** 2, 1)), np.prod(np.sin(3 * X + 1), 1)], 1)
    def fn(dims, X):
        P = np.full((X.shape[0], d), 0.5)
        P[:, list(dims)] = X
        return f(P)
    ref, h = build_pair(G, d, m, O.full_order_components(d, 3), fn, regular_level=4)
    with pytest.raises(G.DDSGError, match="cannot run"):
        h.set_eval_config(0, 0, 2, 2)
    with pytest.raises(G.DDSGError, match="cannot run"):
        h.set_eval_config(0, 0, 3, 4)
    with pytest.raises(G.DDSGError, match="cannot run"):
        h.set_eval_config(0, 0, 4, 4)
    with pytest.raises(G.DDSGError, match="cannot run"):
        h.set_eval_config(1, 1, 5, 32)
    with pytest.raises(G.DDSGError, match="cannot run"):
        h.set_eval_config(1, 1, 6, 32)
    check_eval(h, ref, synth.uniform_queries(33, 500, d))
