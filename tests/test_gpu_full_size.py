"""Parity at the full workload sizes, in the launch configurations bench.py
times, on outputs the oracle can compute one by one: d = 100 (2e6 uniform
queries, FP32-compensated, slice-free; the nodal-slab kernel with its rotated
two-window layout and the two-group level-tuple TMA kernel at 28 outputs per
group) and d = 20 (4.4e5 monomial-shaped queries, FP64; the tile kernel and the
nodal-slab kernel). Sampled rows of the timed launch (no hash / count outputs)
are checked against the oracle's brute force; the active-point counts and
hashes of the same rows come from the level-tuple kernels (the nodal form has
no per-point active set); every row is checked for finiteness."""
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


def _pair(G, d, m, wid):
    c = synth.family_coeffs(synth.BASE_SEED + wid, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    ref = O.OracleDDSG(d, m)
    h = G.HDMR(d, m, 2)
    for u in O.full_order_components(d, 2):
        ref.add_regular(u, 2)
        h.add_regular(list(u), 2)
    ref.build_adaptive(fn, 1e-3, 10)
    G.build_adaptive(h, fn, 1e-3, 10)
    return ref, h


def _check(G, ref, h, X, prec, form, kernel, mc, tol, nsample=48):
    n, m = X.shape[0], ref.m
    h.set_eval_config(prec, form, kernel, mc)
    x = torch.from_numpy(X).cuda()
    y = torch.empty((n, m), dtype=torch.float64, device="cuda")
    hs = torch.empty(n, dtype=torch.int64, device="cuda")
    ct = torch.empty(n, dtype=torch.int32, device="cuda")
    h.eval(x, y, prec, form, hs, ct)
    y2 = torch.empty_like(y)
    h.eval(x, y2, prec, form)            # the timed launch (no hash / count outputs)
    torch.cuda.synchronize()
    if kernel not in (5, 6):
        assert torch.equal(y, y2)
    assert bool(torch.isfinite(y2).all())
    idx = np.unique(np.concatenate([[0, 1, n - 2, n - 1],
                                    (synth.uniform(synth.BASE_SEED + 900, nsample) * n).astype(np.int64)]))
    r = ref.eval(X[idx], form=form, want=("y", "S", "hash", "count"))
    ys = y2[torch.from_numpy(idx).cuda()].cpu().numpy()
    scale = np.maximum(np.abs(r["y"]), r["S"])
    assert np.max(np.abs(ys - r["y"]) / scale) <= tol
    assert np.array_equal(ct[torch.from_numpy(idx).cuda()].cpu().numpy(), r["count"])
    assert np.array_equal(hs[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64), r["hash"])
    assert h.stats()["wait_timeouts"] == 0


@pytest.fixture(scope="module")
def d100(G):
    ref, h = _pair(G, 100, 51, synth.W_D100)
    assert h.sizes() == (5051, 1357149)
    X = synth.uniform_queries(synth.BASE_SEED + synth.W_D100, 2_000_000, 100)
    return ref, h, X


@pytest.mark.parametrize("kernel,mc", [(6, 32), (5, 32), (3, 28)])
def test_d100_two_million_queries_f32c(G, d100, kernel, mc):
    ref, h, X = d100
    _check(G, ref, h, X, G.F32C, G.FORM_SLICEFREE, kernel, mc, 1e-6)


def test_d100_active_sets_against_the_pruned_oracle(G, d100):
    """Active-set hashes and counts of all 2e6 queries from the GPU (level-tuple
    kernel with hash / count outputs); every 100th query (20,000 of them) is
    compared with the oracle's pruned tree descent, on all host threads (about
    700 d = 100 queries per second on 16 cores: the whole 2e6 would take most of
    an hour)."""
    import os
    ref, h, X = d100
    n = X.shape[0]
    x = torch.from_numpy(X).cuda()
    y = torch.empty((n, ref.m), dtype=torch.float64, device="cuda")
    hs = torch.empty(n, dtype=torch.int64, device="cuda")
    ct = torch.empty(n, dtype=torch.int32, device="cuda")
    h.eval(x, y, G.F32C, G.FORM_SLICEFREE, hs, ct)
    torch.cuda.synchronize()
    idx = np.arange(0, n, 100)
    ph, pc = ref.active_pruned(X[idx], 1, threads=os.cpu_count() or 1)
    assert np.array_equal(ct.cpu().numpy()[idx], pc)
    assert np.array_equal(hs.cpu().numpy().view(np.uint64)[idx], ph)
    assert int(ct.min().item()) > 0


@pytest.mark.parametrize("kernel,mc", [(0, 12), (5, 8)])
def test_d20_monomial_queries_f64(G, kernel, mc):
    ref, h = _pair(G, 20, 11, synth.W_D20)
    assert h.sizes() == (211, 52981)
    X = synth.monomial_shaped_queries(synth.BASE_SEED + synth.W_D20, 20_000, 10)
    assert X.shape[0] == 440_000
    _check(G, ref, h, X, G.F64, G.FORM_SLICEFREE, kernel, mc, 1e-12, nsample=200)
