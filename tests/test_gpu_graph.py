"""CUDA-graph replay of the evaluation (hdmr_eval_graph) through the C ABI:
bit-identical to hdmr_eval for every precision, form and schedule; reads the
query buffer by address (refilled in place between replays); captures again
when the batch size, buffers, schedule or tables change; ordered against the
caller's stream."""
import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_eval import build_pair, TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


@pytest.fixture(scope="module")
def pair(G):
    d, m = 6, 11
    c = synth.family_coeffs(synth.BASE_SEED + 57, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    return build_pair(G, d, m, O.full_order_components(d, 2), fn, eps=1e-3, level=8)


def _direct(h, x, m, prec, form):
    y = torch.full((x.shape[0], m), -1.0, dtype=torch.float64, device="cuda")
    h.eval(x, y, prec, form)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_graph_replay_is_bit_identical(G, pair):
    ref, h = pair
    m = ref.m
    X = synth.uniform_queries(71, 900, ref.d)
    x = torch.from_numpy(X).cuda()
    for prec in (0, 1):
        for form in (0, 1):
            want = _direct(h, x, m, prec, form)
            y = torch.full((X.shape[0], m), -1.0, dtype=torch.float64, device="cuda")
            for _ in range(3):          # capture, then replays
                y.fill_(-1.0)
                h.eval_graph(x, y, prec, form)
                torch.cuda.synchronize()
                assert np.array_equal(y.cpu().numpy(), want), (prec, form)
    r = ref.eval(X, form=1, want=("y", "S"))
    scale = np.maximum(np.abs(r["y"]), r["S"])
    assert (np.abs(want - r["y"]) / scale).max() <= TOL[1]


def test_graph_reads_inputs_by_address_and_recaptures(G, pair):
    ref, h = pair
    m = ref.m
    n = 700
    x = torch.from_numpy(synth.uniform_queries(72, n, ref.d)).cuda()
    y = torch.empty((n, m), dtype=torch.float64, device="cuda")
    h.eval_graph(x, y, 1, 1)
    # refill the same buffer: the replay sees the new queries
    x.copy_(torch.from_numpy(synth.uniform_queries(73, n, ref.d)))
    h.eval_graph(x, y, 1, 1)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), _direct(h, x, m, 1, 1))
    # another batch size (a view of the same storage) captures again
    ys = torch.empty((n // 2, m), dtype=torch.float64, device="cuda")
    h.eval_graph(x[: n // 2], ys, 1, 1)
    torch.cuda.synchronize()
    assert np.array_equal(ys.cpu().numpy(), _direct(h, x[: n // 2], m, 1, 1))
    # another schedule captures again
    for kernel, mc in ((0, 12), (2, 16), (1, 52), (5, 16)):
        h.set_eval_config(1, 1, kernel, mc)
        h.eval_graph(x, y, 1, 1)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), _direct(h, x, m, 1, 1)), (kernel, mc)
    # new surpluses in the same tables are read by the replay
    vals = np.concatenate(ref.values) * 2.0
    h.hierarchize(torch.from_numpy(vals).cuda())
    h.eval_graph(x, y, 0, 1)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    assert np.array_equal(got, _direct(h, x, m, 0, 1))
    h.hierarchize(torch.from_numpy(np.concatenate(ref.values)).cuda())
    h.eval_graph(x, y, 0, 1)
    torch.cuda.synchronize()
    assert np.allclose(got, 2.0 * y.cpu().numpy(), rtol=1e-13, atol=1e-300)


def test_graph_orders_against_the_callers_stream(G, pair):
    ref, h = pair
    m = ref.m
    n = 2048
    X0 = synth.uniform_queries(74, n, ref.d)
    X1 = synth.uniform_queries(75, n, ref.d)
    x = torch.from_numpy(X0).cuda()
    x1 = torch.from_numpy(X1).cuda()
    y = torch.empty((n, m), dtype=torch.float64, device="cuda")
    h.profile(True)
    h.profile_read(reset=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(4):
            x.copy_(x1)                     # queued on s before the replay
            h.eval_graph(x, y, 1, 1, stream=s)
            out = y.clone()                 # queued on s after the replay
            x.copy_(torch.from_numpy(X0).cuda())
    s.synchronize()
    prof = h.profile_read(reset=True)
    h.profile(False)
    assert np.array_equal(out.cpu().numpy(), _direct(h, x1, m, 1, 1))
    assert prof["graph"][1] == 4 and prof["graph"][0] > 0


def test_eval_host_matches_device_eval(G, pair):
    """hdmr_eval_host with pageable numpy buffers (copied) and with page-locked
    buffers (read by the encoding kernel through their mapped address) gives
    hdmr_eval's result bit for bit, twice in a row."""
    ref, h = pair
    m = ref.m
    X = synth.uniform_queries(76, 1500, ref.d)
    want = _direct(h, torch.from_numpy(X).cuda(), m, 1, 1)
    y = np.zeros((X.shape[0], m))
    for _ in range(2):
        y[:] = -1.0
        h.eval_host(np.ascontiguousarray(X), y, 1, 1)
        assert np.array_equal(y, want)
    xp = torch.from_numpy(X).pin_memory()
    yp = torch.empty((X.shape[0], m), dtype=torch.float64).pin_memory()
    for _ in range(2):
        yp.fill_(-1.0)
        h.eval_host(xp.numpy(), yp.numpy(), 1, 1)
        assert np.array_equal(yp.numpy(), want)
