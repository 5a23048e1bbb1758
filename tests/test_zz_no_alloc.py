"""hdmr_eval_noalloc: evaluation that allocates no device memory.

Callers that cannot call cudaMalloc while they evaluate (their framework owns
all device memory through its own pool or a hard memory cap, or they are in a
latency-critical loop) use this entry point; its scratch lives in a fixed
16 MiB static device array instead of a handle workspace. This file is named
so that pytest collects it last. It must pass alone in a fresh process and
after the other tests. It checks the new entry point against hdmr_eval
through the C ABI, on two calls in a row with different inputs (the shared
array keeps the previous call's contents), and that oversized batches are
refused before anything runs.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}   # FP64 / FP32-compensated, relative to max(|y|, 1)


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
        assert np.all(np.abs(got - ref) <= TOL[prec] * np.maximum(np.abs(ref), 1.0))


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
    assert np.all(np.abs(got - ref) <= TOL[0] * np.maximum(np.abs(ref), 1.0))
