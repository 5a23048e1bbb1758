"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of the basis (Sec. 3.1), textbook piecewise-linear / bilinear
interpolation and the trapezoid rule, the sparse-grid combination technique
(footnote of Sec. 3.3), exactness of truncated cut-HDMR for additive and
pairwise-additive functions (Sec. 3.3, Fig. 3 discussion), the literal
telescopic sum of eq. 3.16 vs the vectorized a^T b of eq. 4.2, and grid/
component counts printed in the paper (Table 2, Sec. 5.1.3).
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def assemble(anchor, dims, X):
    """Full points: anchor everywhere except coordinates `dims` (cut points)."""
    X = np.asarray(X)
    if X.ndim == 1:
        X = X.reshape(-1, len(dims))
    P = np.repeat(np.asarray(anchor)[None, :], X.shape[0], axis=0)
    for a, j in enumerate(dims):
        P[:, j] = X[:, a]
    return P


def cut_fn(anchor, f_full):
    return lambda dims, X: f_full(assemble(anchor, dims, X))


# ---------------------------------------------------------------------------
# Basis (eq. 3.1 with boundary levels) and its integral (eq. 3.7)
# ---------------------------------------------------------------------------

def test_basis_closed_forms():
    for x in (0.0, 0.3, 0.5, 1.0):
        assert O.phi1d(1, 1, x) == 1.0 and O.active1d(1, 1, x)
    assert O.node1d(1, 1) == 0.5
    # level 2: boundary hats of half-width 1/2
    assert O.phi1d(2, 0, 0.0) == 1.0 and O.phi1d(2, 0, 0.25) == 0.5
    assert O.phi1d(2, 0, 0.5) == 0.0 and not O.active1d(2, 0, 0.5)
    assert O.phi1d(2, 2, 1.0) == 1.0 and O.phi1d(2, 2, 0.75) == 0.5
    assert O.phi1d(2, 2, 0.4) == 0.0
    for l in range(3, 13):
        h = 2.0 ** -(l - 1)
        for i in range(1, 2 ** (l - 1), 2):
            xn = i * h
            assert O.node1d(l, i) == xn
            assert O.phi1d(l, i, xn) == 1.0
            assert O.phi1d(l, i, xn - h) == 0.0 and O.phi1d(l, i, xn + h) == 0.0
            assert not O.active1d(l, i, xn - h) and not O.active1d(l, i, xn + h)
            assert O.phi1d(l, i, xn + h / 2) == 0.5 and O.active1d(l, i, xn - h / 2)
    # integrals: level 1 -> 1, level 2 -> 1/4, level l>=3 -> 2^-(l-1)
    assert O.int1d(1, 1) == 1.0 and O.int1d(2, 0) == 0.25 and O.int1d(2, 2) == 0.25
    for l in range(3, 12):
        xs = np.linspace(0, 1, 2 ** 14 + 1)
        ys = np.array([O.phi1d(l, 1, x) for x in xs])
        assert abs(np.trapezoid(ys, xs) - O.int1d(l, 1)) < 1e-12
        assert O.int1d(l, 1) == 2.0 ** -(l - 1)


# ---------------------------------------------------------------------------
# P8: grid and component counts printed in the paper
# ---------------------------------------------------------------------------

def test_p8_regular_grid_counts_match_table2():
    for d, level, printed in _read_golden("table2_sg_counts.txt"):
        d, level, printed = int(d), int(level), float(printed)
        n = O.sg_point_count(d, level)
        assert float(f"{n:.1e}") == printed, (d, level, n, printed)


def test_p8_enumeration_matches_count():
    for k, level in [(0, 3), (1, 10), (2, 10), (3, 5), (4, 5), (5, 4)]:
        lv, _ = O.regular_grid(k, level)
        assert lv.shape[0] == O.sg_point_count(k, level)
    assert O.sg_point_count(4, 5) == 401          # the d=4, level-5 workload grid
    assert O.sg_point_count(2, 4) == 29           # (k_j, a_j) pair grids at level 4


def test_p8_component_counts():
    for d, order, count in _read_golden("component_counts.txt"):
        comps = O.full_order_components(int(d), int(order))
        assert len(comps) - 1 == int(count)       # minus the empty component


def test_p8_ddsg_d300_level3_saturation():
    for d, level, printed, per in _read_golden("table2_ddsg_d300.txt"):
        d, level, printed, per = int(d), int(level), float(printed), int(per)
        assert O.sg_point_count(1, level) == per
        assert d * per >= printed
    # d=300, level 3: the full grid of every 1D component is exactly the printed count
    assert float(f"{300 * O.sg_point_count(1, 3):.1e}") == 1.5e3


# ---------------------------------------------------------------------------
# P1: node reproduction (interpolant at its nodes = hierarchized values)
# ---------------------------------------------------------------------------

def _adaptive_d4(m=3, eps=1e-3, level=6, strict=False):
    d = 4
    c = synth.family_coeffs(synth.BASE_SEED + 99, m, d)
    E = O.OracleDDSG(d, m)
    for u in O.full_order_components(d, 2):
        E.add_regular(u, 2)
    E.build_adaptive(lambda dims, X: synth.family_cut(c, dims, X), eps, level, strict)
    return E, c


def test_p1_node_reproduction_adaptive_components():
    E, c = _adaptive_d4()
    sizes = [E.npts(i) for i in range(len(E.comps))]
    assert max(sizes) > min(s for s in sizes if s > 1)   # grids are uneven
    for ci, dims in enumerate(E.comps):
        if not dims:
            continue
        single = O.OracleDDSG(len(dims), E.m)
        single.add_component(tuple(range(len(dims))), E.lv[ci], E.ix[ci])
        single.alpha[0] = E.alpha[ci]
        X = E.node_coords(ci)
        y = single.eval(X, want=("y", "S"))
        assert np.all(np.abs(y["y"] - E.values[ci]) <= 8 * EPS * np.maximum(1.0, y["S"]))


def test_p1_node_reproduction_regular_4d():
    f = lambda X: np.stack([np.exp(X.sum(1) * 0.3), np.sin(X @ np.array([1., 2., 3., 4.]))], 1)
    E = O.OracleDDSG(4, 2)
    E.add_regular((0, 1, 2, 3), 5)
    E.fill_values(lambda dims, X: f(X))
    E.hierarchize()
    y = E.eval(E.node_coords(0), want=("y", "S"))
    assert np.all(np.abs(y["y"] - E.values[0]) <= 8 * EPS * np.maximum(1.0, y["S"]))


# ---------------------------------------------------------------------------
# P2: 1D hierarchical interpolant == piecewise-linear interpolation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("level", [1, 2, 3, 5, 10])
def test_p2_1d_equals_piecewise_linear(level):
    fns = lambda x: np.stack([np.sin(3 * x), np.exp(x) * np.cos(7 * x)], 1)
    E = O.OracleDDSG(1, 2)
    E.add_regular((0,), level)
    E.fill_values(lambda dims, X: fns(X[:, 0]))
    E.hierarchize()
    xq = np.concatenate([synth.uniform(11, 10000), [0.0, 0.5, 1.0, 0.25, 0.7]])
    y = E.eval(xq[:, None])["y"]
    if level == 1:
        ref = np.repeat(fns(np.array([0.5])), xq.size, axis=0)
    else:
        nodes = np.linspace(0.0, 1.0, 2 ** (level - 1) + 1)
        fv = fns(nodes)
        ref = np.stack([np.interp(xq, nodes, fv[:, j]) for j in range(2)], 1)
    assert np.max(np.abs(y - ref)) <= 16 * EPS


# ---------------------------------------------------------------------------
# P3: tiny d=2 brute force -- full grid = bilinear; regular SG = combination technique
# ---------------------------------------------------------------------------

def _f2(X):
    return np.stack([np.exp(-X[:, 0] * X[:, 1]) + X[:, 0] ** 3, np.sin(4 * X[:, 0] - 2 * X[:, 1])], 1)


def _nodal_interp(e, X):
    """Anisotropic full-grid (tensor) interpolant with per-dimension excess e_j:
    e_j = 0 -> constant (node 1/2), e_j >= 1 -> linear on 2^e_j + 1 uniform nodes."""
    axes = []
    for ej in e:
        axes.append(np.array([0.5]) if ej == 0 else np.linspace(0, 1, 2 ** ej + 1))
    G = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 2)
    V = _f2(G).reshape(len(axes[0]), len(axes[1]), 2)
    keep = [i for i, ej in enumerate(e) if ej > 0]
    if not keep:
        return np.repeat(V.reshape(1, 2), X.shape[0], axis=0)
    if len(keep) == 1:
        i = keep[0]
        Vi = V[:, 0, :] if i == 0 else V[0, :, :]
        return np.stack([np.interp(X[:, i], axes[i], Vi[:, j]) for j in range(2)], 1)
    out = []
    for j in range(2):
        rgi = RegularGridInterpolator((axes[0], axes[1]), V[:, :, j], method="linear")
        out.append(rgi(X))
    return np.stack(out, 1)


def test_p3_full_grid_is_bilinear():
    L = 4
    lv1, ix1 = O.regular_grid(1, L)
    pts = list(itertools.product(range(lv1.shape[0]), repeat=2))
    lv = np.zeros((len(pts), O.KMAX), np.uint8)
    ix = np.zeros((len(pts), O.KMAX), np.uint32)
    for r, (a, b) in enumerate(pts):
        lv[r, :2] = (lv1[a, 0], lv1[b, 0])
        ix[r, :2] = (ix1[a, 0], ix1[b, 0])
    E = O.OracleDDSG(2, 2)
    E.add_component((0, 1), lv, ix)
    E.fill_values(lambda dims, X: _f2(X))
    E.hierarchize()
    X = synth.uniform_matrix(12, 3000, 2)
    y = E.eval(X)["y"]
    ref = _nodal_interp((L - 1, L - 1), X)
    assert np.max(np.abs(y - ref)) <= 1e-14


@pytest.mark.parametrize("L", [1, 2, 3, 5, 7])
def test_p3_regular_sg_equals_combination_technique(L):
    E = O.OracleDDSG(2, 2)
    E.add_regular((0, 1), L)
    E.fill_values(lambda dims, X: _f2(X))
    E.hierarchize()
    X = synth.uniform_matrix(13, 2000, 2)
    y = E.eval(X)["y"]
    n = L - 1
    ref = sum(_nodal_interp((e1, n - e1), X) for e1 in range(n + 1))
    if n >= 1:
        ref = ref - sum(_nodal_interp((e1, n - 1 - e1), X) for e1 in range(n))
    assert np.max(np.abs(y - ref)) <= 1e-13


# ---------------------------------------------------------------------------
# P4 / P5 / P6: truncated cut-HDMR exactness (Sec. 3.3)
# ---------------------------------------------------------------------------

def test_p4_order1_exact_for_additive_piecewise_linear():
    d, L = 6, 5
    nodes = np.linspace(0, 1, 2 ** (L - 1) + 1)
    H = synth.uniform_matrix(14, d, nodes.size, -1.0, 1.0)
    f = lambda X: np.sum([np.interp(X[:, i], nodes, H[i]) for i in range(d)], axis=0)[:, None]
    anchor = np.full(d, 0.5)
    E = O.OracleDDSG(d, 1)
    for u in O.full_order_components(d, 1):
        E.add_regular(u, L)
    E.fill_values(cut_fn(anchor, f))
    E.hierarchize()
    X = synth.uniform_matrix(15, 3000, d)
    r = E.eval(X, form=0, want=("y", "S"))
    assert np.all(np.abs(r["y"] - f(X)) <= 64 * EPS * np.maximum(1.0, r["S"]))


def test_p4_order1_smooth_additive_equals_sum_of_1d_interpolants():
    d, L = 5, 6
    g = [lambda x, a=a: np.sin((a + 1) * x) for a in range(d)]
    f = lambda X: np.sum([g[i](X[:, i]) for i in range(d)], axis=0)[:, None]
    E = O.OracleDDSG(d, 1)
    for u in O.full_order_components(d, 1):
        E.add_regular(u, L)
    E.fill_values(cut_fn(np.full(d, 0.5), f))
    E.hierarchize()
    X = synth.uniform_matrix(16, 2000, d)
    y = E.eval(X)["y"][:, 0]
    nodes = np.linspace(0, 1, 2 ** (L - 1) + 1)
    ref = np.sum([np.interp(X[:, i], nodes, g[i](nodes)) for i in range(d)], axis=0)
    assert np.max(np.abs(y - ref)) <= 1e-13


def _pairwise_f(d, seed):
    A = synth.uniform_matrix(seed, d, d, 0.5, 2.0)
    def f(X):
        y = np.zeros(X.shape[0])
        for i, j in itertools.combinations(range(d), 2):
            y += np.sin(A[i, j] * X[:, i] - A[j, i] * X[:, j]) * np.exp(-X[:, i] * X[:, j])
        return np.stack([y, y * y], 1)   # second output not pairwise additive
    return f


def test_p5_order2_pairwise_additive_equals_4d_regular_sg():
    d, L = 4, 5
    f = _pairwise_f(d, 17)
    f0 = lambda X: f(X)[:, :1]
    anchor = np.full(d, 0.5)
    E = O.OracleDDSG(d, 1)
    for u in O.full_order_components(d, 2):
        E.add_regular(u, L)
    E.fill_values(cut_fn(anchor, f0))
    E.hierarchize()
    G = O.OracleDDSG(d, 1)
    G.add_regular(tuple(range(d)), L)
    assert G.npts(0) == 401
    G.fill_values(lambda dims, X: f0(X))
    G.hierarchize()
    X = synth.uniform_matrix(18, 2000, d)
    r = E.eval(X, want=("y", "S"))
    yg = G.eval(X)["y"]
    assert np.all(np.abs(r["y"] - yg) <= 1e-12 * np.maximum(np.abs(yg), r["S"]))
    # and the order-1 truncation is NOT exact for it (the pin can fail)
    E1 = O.OracleDDSG(d, 1)
    for u in O.full_order_components(d, 1):
        E1.add_regular(u, L)
    E1.fill_values(cut_fn(anchor, f0))
    E1.hierarchize()
    assert np.max(np.abs(E1.eval(X)["y"] - yg)) > 1e-3


@pytest.mark.parametrize("d", [2, 3])
def test_p6_full_expansion_equals_regular_sg(d):
    L = 5
    f = lambda X: np.stack([np.exp(-np.sum(X ** 2, 1)), np.prod(np.sin(3 * X + 1), 1)], 1)
    E = O.OracleDDSG(d, 2)
    for u in O.full_order_components(d, d):
        E.add_regular(u, L)
    E.fill_values(cut_fn(np.full(d, 0.5), f))
    E.hierarchize()
    G = O.OracleDDSG(d, 2)
    G.add_regular(tuple(range(d)), L)
    G.fill_values(lambda dims, X: f(X))
    G.hierarchize()
    X = synth.uniform_matrix(19, 1500, d)
    yg = G.eval(X)["y"]
    for form in (0, 1):
        r = E.eval(X, form=form, want=("y", "S"))
        assert np.all(np.abs(r["y"] - yg) <= 1e-12 * np.maximum(np.abs(yg), r["S"]))
    assert np.max(np.abs(E.eval_telescopic(X) - yg)) <= 1e-12


# ---------------------------------------------------------------------------
# eq. 4.2 vs eq. 3.16, b coefficients, anchored-slice (slice-free) identity
# ---------------------------------------------------------------------------

def test_b_coefficients_full_order2():
    for d in (4, 20):
        comps = O.full_order_components(d, 2)
        E = O.OracleDDSG(d, 1)
        for u in comps:
            E.add_component(u, np.zeros((1, O.KMAX), np.uint8), np.zeros((1, O.KMAX), np.uint32))
        b = E.b_coeffs()
        # closed form for a full order-2 set: b_0 = 1 - d + C(d,2), b_i = 1 - (d-1), b_ij = 1
        assert b[0] == 1 - d + math.comb(d, 2)
        assert np.all(b[1:d + 1] == 2 - d)
        assert np.all(b[d + 1:] == 1)
    assert 1 - 20 + math.comb(20, 2) == 171 and 1 - 100 + math.comb(100, 2) == 4851


def test_b_coefficients_partial_set():
    # empty + all singles + the pairs (j, N+j): singles get b = 0 (they drop out)
    N = 5
    comps = [()] + [(i,) for i in range(2 * N)] + [(j, N + j) for j in range(N)]
    E = O.OracleDDSG(2 * N, 1)
    for u in comps:
        E.add_component(u, np.zeros((1, O.KMAX), np.uint8), np.zeros((1, O.KMAX), np.uint32))
    b = E.b_coeffs()
    assert b[0] == 1 - 2 * N + N
    assert np.all(b[1:2 * N + 1] == 0)
    assert np.all(b[2 * N + 1:] == 1)


def test_p7_paper_form_telescopic_and_slice_free_agree():
    E, c = _adaptive_d4()
    X = np.concatenate([synth.uniform_queries(20, 1500, 4), np.full((1, 4), 0.5),
                        np.zeros((1, 4)), np.ones((1, 4))])
    p = E.eval(X, form=0, want=("y", "S"))
    s = E.eval(X, form=1, want=("y", "S"))
    t = E.eval_telescopic(X)
    tol = 1e-12 * np.maximum(np.abs(p["y"]), p["S"])
    assert np.all(np.abs(p["y"] - t) <= tol)
    assert np.all(np.abs(p["y"] - s["y"]) <= tol)
    # the slice-free form carries far less cancellation
    assert np.median(s["S"] / np.abs(s["y"])) < np.median(p["S"] / np.abs(p["y"]))


def test_p7_slices_of_pair_grids_equal_lower_grids():
    """Precondition of the slice-free form: the l=1 slice of G_{ab} in dim b is G_a."""
    E, _ = _adaptive_d4()
    index = {u: i for i, u in enumerate(E.comps)}
    for u in E.comps:
        if len(u) != 2:
            continue
        cu = index[u]
        for keep in range(2):
            w = (u[keep],)
            cw = index[w]
            other = 1 - keep
            sel = E.lv[cu][:, other] == 1
            lv_s = E.lv[cu][sel][:, [keep]]
            ix_s = E.ix[cu][sel][:, [keep]]
            assert sorted(zip(lv_s[:, 0], ix_s[:, 0])) == sorted(zip(E.lv[cw][:, 0], E.ix[cw][:, 0]))
            a_s = {(int(l), int(i)): E.alpha[cu][r] for r, (l, i) in
                   zip(np.nonzero(sel)[0], zip(lv_s[:, 0], ix_s[:, 0]))}
            for r in range(E.npts(cw)):
                key = (int(E.lv[cw][r, 0]), int(E.ix[cw][r, 0]))
                assert np.allclose(a_s[key], E.alpha[cw][r], rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# Refinement (eq. 3.8)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("strict", [False, True])
def test_refine_all_significant_gives_regular_grid(strict):
    for k, L in [(1, 8), (2, 6), (3, 4)]:
        E = O.OracleDDSG(k, 1)
        E.add_regular(tuple(range(k)), 2)
        E.build_adaptive(lambda dims, X: np.ones((X.shape[0], 1)) + X.sum(1, keepdims=True) ** 2,
                         -1.0, L, strict)
        lv, ix = O.regular_grid(k, L)
        assert np.array_equal(E.lv[0], lv) and np.array_equal(E.ix[0], ix)


def test_refine_nothing_significant_adds_nothing():
    E = O.OracleDDSG(2, 1)
    E.add_regular((0, 1), 2)
    E.build_adaptive(lambda dims, X: np.sin(X.sum(1, keepdims=True)), 1e9, 10)
    assert E.npts(0) == 5


def test_refine_1d_kink_follows_the_kink():
    """f = max(0, x - 0.7): surpluses vanish wherever f is linear on a hat's
    support, so past level 3 each level holds exactly the two children of the
    one hat whose support contains 0.7."""
    for L in (4, 7, 10):
        E = O.OracleDDSG(1, 1)
        E.add_regular((0,), 2)
        E.build_adaptive(lambda dims, X: np.maximum(0.0, X - 0.7), 1e-10, L)
        assert E.npts(0) == 2 * L - 2
        for l in range(4, L + 1):
            sel = E.lv[0][:, 0] == l
            xs = np.sort(E.ix[0][sel, 0] / 2.0 ** (l - 1))
            assert xs.size == 2 and xs[0] < 0.7 + 2.0 ** -(l - 2)


def test_refine_strict_is_subset_of_any():
    Ea, _ = _adaptive_d4(strict=False)
    Es, _ = _adaptive_d4(strict=True)
    for c in range(len(Ea.comps)):
        A = set(map(tuple, np.concatenate([Ea.lv[c], Ea.ix[c]], 1).tolist()))
        S = set(map(tuple, np.concatenate([Es.lv[c], Es.ix[c]], 1).tolist()))
        assert S <= A


# ---------------------------------------------------------------------------
# P9: quadrature (eq. 3.7) and the adaptivity coefficients (eq. 3.18, 3.19)
# ---------------------------------------------------------------------------

def test_p9_quadrature_is_trapezoid_rule():
    L = 7
    f = lambda x: np.exp(np.sin(3 * x))
    E = O.OracleDDSG(1, 1)
    E.add_regular((0,), L)
    E.fill_values(lambda dims, X: f(X))
    E.hierarchize()
    nodes = np.linspace(0, 1, 2 ** (L - 1) + 1)
    assert abs(E.quadrature()[0, 0] - np.trapezoid(f(nodes), nodes)) <= 1e-14
    # 2D full grid: tensor trapezoid
    lv1, ix1 = O.regular_grid(1, 4)
    pts = list(itertools.product(range(lv1.shape[0]), repeat=2))
    lv = np.zeros((len(pts), O.KMAX), np.uint8)
    ix = np.zeros((len(pts), O.KMAX), np.uint32)
    for r, (a, b) in enumerate(pts):
        lv[r, :2] = (lv1[a, 0], lv1[b, 0])
        ix[r, :2] = (ix1[a, 0], ix1[b, 0])
    G = O.OracleDDSG(2, 2)
    G.add_component((0, 1), lv, ix)
    G.fill_values(lambda dims, X: _f2(X))
    G.hierarchize()
    n1 = np.linspace(0, 1, 9)
    XX = np.stack(np.meshgrid(n1, n1, indexing="ij"), -1).reshape(-1, 2)
    V = _f2(XX).reshape(9, 9, 2)
    ref = np.trapezoid(np.trapezoid(V, n1, axis=1), n1, axis=0)
    assert np.max(np.abs(G.quadrature()[0] - ref)) <= 1e-14


def test_rho_eta_vanish_beyond_the_interaction_order():
    """Fig. 3 protocol on [0,1]^4, anchor (1/2,...): for a pairwise-additive f the
    order-3 cut components vanish, so rho(3) and eta_u (|u| = 3) are ~0 while
    rho(2) is not (eq. 3.18, 3.19)."""
    d = 4
    f = lambda X: (X.sum(1) ** 2)[:, None] + np.sin(X[:, 0] * X[:, 1])[:, None]
    E = O.OracleDDSG(d, 1)
    for u in O.full_order_components(d, 3):
        E.add_regular(u, 5)
    E.fill_values(cut_fn(np.full(d, 0.5), f))
    E.hierarchize()
    assert E.expansion_rho(2) > 1e-4
    assert E.expansion_rho(3) < 1e-13
    assert E.active_eta((0, 1)) > 1e-4
    assert E.active_eta((0, 1, 2)) < 1e-13
    # (x1+..+x4)^1 is additive: order-2 components vanish
    g = lambda X: X.sum(1, keepdims=True)
    E.fill_values(cut_fn(np.full(d, 0.5), g))
    E.hierarchize()
    assert E.expansion_rho(2) < 1e-13


# ---------------------------------------------------------------------------
# P12: active sets -- counts and order-independent hashes
# ---------------------------------------------------------------------------

def test_p12_active_set_count_and_hash_regular_4d():
    E = O.OracleDDSG(4, 1)
    E.add_regular((0, 1, 2, 3), 5)
    E.set_values(0, np.zeros((401, 1)))
    E.hierarchize()
    X = synth.uniform_queries(21, 300, 4)
    r = E.eval(X, want=("hash", "count"))
    # 70 level tuples with sum(l-1) <= 4 in 4 dims: one active point each off the cell faces
    assert math.comb(4 + 4, 4) == 70
    assert np.all(r["count"] == 70)
    for q in range(20):
        h = 0
        n = 0
        for p in range(401):
            if all(O.active1d(E.lv[0][p, j], E.ix[0][p, j], X[q, j]) for j in range(4)):
                h ^= E.point_key(0, p)
                n += 1
        assert n == 70 and h == int(r["hash"][q])
    # a query on a level-5 node lies on faces of finer cells: fewer active points
    xn = np.array([[0.5, 0.25, 0.125, 0.0625]])
    assert E.eval(xn, want=("count",))["count"][0] < 70


def test_p12_pruned_descent_equals_brute_force():
    """The pruned mode (tree descent from each component's root, a child visited
    only from an active parent) finds the same active sets as the brute force,
    which tests every point: C1 (d = 4 regular level-5 grid), the C2 expansion
    (d = 20, order 2, adaptive to level 10, both forms, clamped monomial-shaped
    queries) and an adaptive d = 4 expansion at nodes, faces, corners and
    non-finite rows."""
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + synth.W_SG4, m, d)
    E = O.OracleDDSG(d, m)
    E.add_regular((0, 1, 2, 3), 5)
    E.fill_values(lambda dims, X: synth.family_cut(c, dims, X))
    E.hierarchize()
    X = synth.uniform_queries(5, 2000, d)
    r = E.eval(X, form=0, want=("hash", "count"))
    h, cnt = E.active_pruned(X, 0, threads=4)
    assert np.array_equal(h, r["hash"]) and np.array_equal(cnt, r["count"])

    d, m = 20, 11
    c = synth.family_coeffs(synth.BASE_SEED + synth.W_D20, m, d)
    E = O.OracleDDSG(d, m)
    for u in O.full_order_components(d, 2):
        E.add_regular(u, 2)
    E.build_adaptive(lambda dims, X: synth.family_cut(c, dims, X), 1e-3, 10)
    X = synth.monomial_shaped_queries(synth.BASE_SEED + synth.W_D20, 20, 10, s=0.05)
    for form in (0, 1):
        r = E.eval(X, form=form, want=("hash", "count"))
        h, cnt = E.active_pruned(X, form, threads=3)
        assert np.array_equal(h, r["hash"]) and np.array_equal(cnt, r["count"]), form

    E, _ = _adaptive_d4()
    pts = [np.zeros(4), np.ones(4), np.full(4, 0.5), np.array([0.25, 0.75, 0.125, 0.375]),
           np.array([np.nan, 0.2, 0.3, 0.4]), np.array([0.2, np.inf, 0.3, 0.1])]
    pts += [row for row in E.node_coords(len(E.comps) - 1)[:, [0, 0, 0, 0]][:40]]
    X = np.concatenate([np.array(pts), synth.uniform_queries(6, 300, 4)])
    for form in (0, 1):
        r = E.eval(X, form=form, want=("hash", "count"))
        h, cnt = E.active_pruned(X, form, threads=2)
        assert np.array_equal(h, r["hash"]) and np.array_equal(cnt, r["count"]), form


def test_eval_clamps_to_domain():
    f = lambda X: np.stack([X[:, 0] + 2 * X[:, 1]], 1)
    E = O.OracleDDSG(2, 1, lo=[-1.0, 2.0], hi=[1.0, 4.0])
    E.add_regular((0, 1), 4)
    E.fill_values(lambda dims, X: f(X))
    E.hierarchize()
    y_in = E.eval(np.array([[1.0, 2.0], [-1.0, 4.0]]))["y"]
    y_out = E.eval(np.array([[5.0, -3.0], [-9.0, 40.0]]))["y"]
    assert np.array_equal(y_in, y_out)
    assert abs(y_in[0, 0] - 5.0) < 1e-14 and abs(y_in[1, 0] - 7.0) < 1e-14


def test_eval_non_finite_rows():
    E = O.OracleDDSG(2, 2)
    E.add_regular((0, 1), 3)
    E.fill_values(lambda dims, X: np.stack([X[:, 0], X[:, 1]], 1))
    E.hierarchize()
    X = np.array([[0.3, np.nan], [np.inf, 0.2], [0.3, 0.2]])
    r = E.eval(X, want=("y", "hash", "count"))
    assert np.all(np.isnan(r["y"][:2])) and np.all(np.isfinite(r["y"][2]))
    assert list(r["count"][:2]) == [0, 0] and list(r["hash"][:2]) == [0, 0]
