"""Failure path of the TMA-staged evaluation kernels, exercised without a fault.

Every mbarrier wait in those kernels is bounded (2^18 polls, about a second). The test switch
hdmr_set_fault_injection withholds the staging copies from one processed
component on, so the waits on them run out. Expected:
  - every query of every block that gave up reads NaN;
  - hdmr_stats counts one timeout per warp that gave up;
  - the copies that were issued land before the block exits, the context stays
    usable and, with the switch off again, the next evaluation (direct or graph
    replay) is bit-identical to one taken before the failure.
"""
import time

import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_eval import build_pair, TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# queries per block and threads per block of the staged kernels 2, 3, 4 and of the
# nodal-slab kernel 5 at a one-window chunk
SHAPE = {2: (256, 256), 3: (192, 384), 4: (160, 480), 5: (256, 256)}


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


@pytest.fixture(scope="module")
def pair_wide(G):
    d, m = 6, 20      # 20 outputs: the 32-output FP32 window of kernel 6
    c = synth.family_coeffs(synth.BASE_SEED + 84, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    return build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=7)


def test_tmem_kernel_withheld_copies_time_out_and_recover(G, pair_wide):
    """Kernel 6 (Kahan totals in tensor memory): waits on withheld copies run out,
    every output is NaN, one timeout per warp, the tensor memory is freed (the
    next launches allocate it again) and the next evaluation is bit-identical."""
    ref, h = pair_wide
    m, form, prec = ref.m, 1, 1
    n = 256 + 41
    X = synth.uniform_queries(95, n, ref.d)
    x = torch.from_numpy(X).cuda()
    saved = h.eval_config(prec, form)
    h.set_eval_config(prec, form, 6, 32)
    h.stats(reset=True)
    want = _eval(h, x, m, prec, form)
    assert h.stats(reset=True)["wait_timeouts"] == 0
    r = ref.eval(X, form=form, want=("y", "S"))
    assert (np.abs(want - r["y"]) / np.maximum(np.abs(r["y"]), r["S"])).max() <= TOL[prec]
    h.set_fault_injection(2)
    y = _eval(h, x, m, prec, form)
    st = h.stats(reset=True)
    assert np.isnan(y).all()
    # 297 queries = 2 tiles of 256 x 1 window of 32 outputs = 2 work items: one
    # block of 16 warps (its two warp groups take one tile each)
    assert st["wait_timeouts"] == 512 // 32
    h.set_fault_injection(-1)
    for _ in range(3):
        assert np.array_equal(_eval(h, x, m, prec, form), want)
    assert h.stats(reset=True)["wait_timeouts"] == 0
    h.set_eval_config(prec, form, *saved)


@pytest.fixture(scope="module")
def pair(G):
    d, m = 6, 5
    c = synth.family_coeffs(synth.BASE_SEED + 83, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    return build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=7)


def _eval(h, x, m, prec, form, graph=False):
    y = torch.full((x.shape[0], m), -1.0, dtype=torch.float64, device="cuda")
    (h.eval_graph if graph else h.eval)(x, y, prec, form)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("kernel,prec,withhold", [(3, 1, 3), (2, 0, 0), (4, 1, 1), (5, 1, 2), (5, 0, 0)])
def test_withheld_copies_time_out_and_context_recovers(G, pair, kernel, prec, withhold):
    ref, h = pair
    m, form = ref.m, 1
    qb, nt = SHAPE[kernel]
    n = qb + 37                                   # two blocks, the second ragged
    X = synth.uniform_queries(97, n, ref.d)
    x = torch.from_numpy(X).cuda()
    mc = {(2, 0): 4, (3, 1): 8, (4, 1): 12, (5, 1): 16, (5, 0): 8}[(kernel, prec)]
    saved = h.eval_config(prec, form)
    h.set_eval_config(prec, form, kernel, mc)
    assert h.eval_config(prec, form) == (kernel, mc)
    h.stats(reset=True)
    want = _eval(h, x, m, prec, form)
    assert h.stats(reset=True)["wait_timeouts"] == 0
    r = ref.eval(X, form=form, want=("y", "S"))
    scale = np.maximum(np.abs(r["y"]), r["S"])
    assert (np.abs(want - r["y"]) / scale).max() <= TOL[prec]

    h.set_fault_injection(withhold)
    t0 = time.perf_counter()
    y = _eval(h, x, m, prec, form)
    dt = time.perf_counter() - t0
    st = h.stats(reset=True)
    assert np.isnan(y).all()
    nblocks = -(-n // qb) * -(-m // (mc * {2: 1, 3: 2, 4: 3, 5: 1}[kernel]))
    assert st["wait_timeouts"] == nblocks * nt // 32, (st, dt)
    print(f"kernel {kernel}: failed evaluation took {dt:.3f} s")

    h.set_fault_injection(-1)
    again = _eval(h, x, m, prec, form)
    assert np.array_equal(again, want)
    assert h.stats(reset=True)["wait_timeouts"] == 0
    h.set_eval_config(prec, form, *saved)


def test_graph_replay_recaptures_around_the_switch(G, pair):
    ref, h = pair
    m, prec, form = ref.m, 1, 1
    X = synth.uniform_queries(98, 300, ref.d)
    x = torch.from_numpy(X).cuda()
    saved = h.eval_config(prec, form)
    h.set_eval_config(prec, form, 3, 8)
    h.stats(reset=True)
    want = _eval(h, x, m, prec, form, graph=True)
    h.set_fault_injection(2)
    assert np.isnan(_eval(h, x, m, prec, form, graph=True)).all()
    assert h.stats(reset=True)["wait_timeouts"] > 0
    h.set_fault_injection(-1)
    assert np.array_equal(_eval(h, x, m, prec, form, graph=True), want)
    assert np.array_equal(_eval(h, x, m, prec, form), want)
    assert h.stats(reset=True)["wait_timeouts"] == 0
    h.set_eval_config(prec, form, *saved)


def test_switch_rejects_bad_argument(G, pair):
    _, h = pair
    with pytest.raises(G.DDSGError, match="hdmr_set_fault_injection"):
        h.set_fault_injection(-2)
