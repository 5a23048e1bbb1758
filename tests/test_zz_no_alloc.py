"""hdmr_eval_noalloc: evaluation that allocates no device memory.

Callers that cannot call cudaMalloc while they evaluate (their framework owns
all device memory through its own pool or a hard memory cap, or they are in a
latency-critical loop) use this entry point; its scratch lives in a fixed
16 MiB static device array instead of a handle workspace. This file is named
so that pytest collects it last. It must pass alone in a fresh process and
after the other tests. It checks the new entry point against hdmr_eval
through the C ABI, on two calls in a row with different inputs (the shared
array keeps the previous call's contents), and that oversized batches are
refused before anything runs. Both entry points run the same kernels on the
same schedule, so their results must agree bit for bit. It also checks that a
staged schedule chosen before the tables changed is not used on tables it
cannot run, and that a staging wait that gives up is reported by hdmr_check.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    d, m = 6, 11
    c = synth.family_coeffs(synth.BASE_SEED + 77, m, d)
    h = G.HDMR(d, m, 2)
    import itertools
    for k in range(3):
        for u in itertools.combinations(range(d), k):
            h.add_regular(list(u), 2)
    G.build_adaptive(h, lambda dims, X: synth.family_cut(c, dims, X), 1e-3, 9)
    return G, h


def _eval_existing(G, h, X, prec, form):
    x = torch.from_numpy(X).cuda()
    y = torch.empty((X.shape[0], h.m), dtype=torch.float64, device="cuda")
    h.eval(x, y, prec, form)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _eval_noalloc_abi(G, h, X, prec, form):
    """Direct C-ABI call of hdmr_eval_noalloc on device buffers."""
    lib = G.load()
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.full((X.shape[0], h.m), -1.0, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hdmr_eval_noalloc(h._h, X.shape[0], C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                               prec, form, stream)
    assert rc == 0, lib.ddsg_last_error()
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("form", [0, 1])
def test_noalloc_matches_existing_entry_point_twice(built, prec, form):
    G, h = built
    X1 = synth.uniform_queries(synth.BASE_SEED + 78, 3000, h.d)
    X2 = np.concatenate([synth.uniform_queries(synth.BASE_SEED + 79, 1100, h.d),
                         np.full((1, h.d), 0.5), np.zeros((1, h.d)), np.ones((1, h.d))])
    for X in (X1, X2):           # two calls in a row, different sizes and inputs
        ref = _eval_existing(G, h, X, prec, form)
        got = _eval_noalloc_abi(G, h, X, prec, form)
        assert np.array_equal(got, ref)


def test_noalloc_refuses_oversized_batch(built):
    G, h = built
    cap = int(G.load().hdmr_eval_noalloc_capacity(h.d))
    assert cap == (1 << 22) // (2 * h.d + 1)
    X = np.full((cap + 1, h.d), 0.5)
    with pytest.raises(AssertionError, match="too large"):
        _eval_noalloc_abi(G, h, X, 0, 0)
    # the largest accepted batch still works
    got = _eval_noalloc_abi(G, h, X[:cap], 0, 0)
    ref = _eval_existing(G, h, X[:cap], 0, 0)
    assert np.array_equal(got, ref)


def test_noalloc_zero_batch_only_sets_up(built):
    G, h = built
    lib = G.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hdmr_eval_noalloc(h._h, 0, None, None, 1, 1, stream) == 0, lib.ddsg_last_error()


def test_noalloc_drops_a_schedule_the_new_tables_cannot_run(built):
    """A staged kernel chosen while every component had k <= 2 must not run once
    an order-3 component is added: the call falls back like hdmr_eval does."""
    G, _ = built
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + 80, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    h = G.HDMR(d, m, 3)
    import itertools
    for k in range(3):
        for u in itertools.combinations(range(d), k):
            h.add_regular(list(u), 2)
    G.build_adaptive(h, fn, 1e-3, 6)
    h.set_eval_config(1, 0, 3, 8)
    assert h.eval_config(1, 0) == (3, 8)
    h.add_regular([0, 1, 2], 2)           # k = 3: the staged kernels cannot hold it
    G.build_adaptive(h, fn, 1e-3, 6)
    X = synth.uniform_queries(synth.BASE_SEED + 81, 500, d)
    got = _eval_noalloc_abi(G, h, X, 1, 0)
    assert h.eval_config(1, 0)[0] in (0, 1)
    ref = _eval_existing(G, h, X, 1, 0)
    assert np.array_equal(got, ref)
    h.close()


def test_noalloc_reports_a_wait_that_gave_up(built):
    """The failure-path switch withholds staging copies; the no-alloc call must
    count the waits that ran out so that hdmr_check reports them."""
    G, h = built
    saved = h.eval_config(1, 1)
    h.set_eval_config(1, 1, 3, 8)
    X = synth.uniform_queries(synth.BASE_SEED + 82, 400, h.d)
    want = _eval_noalloc_abi(G, h, X, 1, 1)
    h.check()
    h.set_fault_injection(1)
    try:
        y = _eval_noalloc_abi(G, h, X, 1, 1)
        assert np.isnan(y).all()
        with pytest.raises(G.DDSGError):
            h.check()
    finally:
        h.set_fault_injection(-1)
    h.stats(reset=True)
    assert np.array_equal(_eval_noalloc_abi(G, h, X, 1, 1), want)
    h.check()
    h.set_eval_config(1, 1, *saved)
