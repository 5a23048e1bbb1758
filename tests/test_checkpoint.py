"""Checkpoint / resume (hdmr_save / hdmr_load). CPU: missing, foreign,
wrong-version, truncated and corrupt files are refused with DDSG_ERR_ARG before
any device work. GPU: a saved expansion loads into a handle whose evaluations
equal the original's bit for bit, for both precisions and forms."""
import os
import struct

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def G():
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def _fnv(b: bytes) -> int:
    h = 0xcbf29ce484222325
    for x in b:
        h ^= x
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _file(body: bytes, version=1, magic=b"DDSGHDMR", checksum=None):
    head = magic + struct.pack("<II", version, 0)
    return head + body + struct.pack("<Q", _fnv(body) if checksum is None else checksum)


def test_bad_files_are_refused(G, tmp_path):
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        G.HDMR.load(str(tmp_path / "missing.ddsg"))
    # d=1, m=1, order=1, 1 component (the constant), P=1, anchor/lo/hi, k=0 npts=1, alpha
    body = struct.pack("<iiiiq", 1, 1, 1, 1, 1) + struct.pack("<3d", 0.5, 0.0, 1.0) + \
        struct.pack("<iq", 0, 1) + struct.pack("<d", 2.5)
    cases = {"foreign": _file(body, magic=b"NOTDDSG!"), "version": _file(body, version=9),
             "corrupt": _file(body, checksum=12345), "truncated": _file(body)[:-12],
             "short": b"DDSG"}
    for name, blob in cases.items():
        p = tmp_path / f"{name}.ddsg"
        p.write_bytes(blob)
        with pytest.raises(G.DDSGError, match="ERR_ARG"):
            G.HDMR.load(str(p))


@pytest.mark.gpu
def test_save_load_round_trip(G, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    d, m = 6, 5
    c = synth.family_coeffs(synth.BASE_SEED + 63, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    lo, hi = np.full(d, -1.0), np.full(d, 3.0)
    h = G.HDMR(d, m, 2, lo=lo, hi=hi)
    for u in O.full_order_components(d, 2):
        h.add_regular(list(u), 2)
    G.build_adaptive(h, lambda dims, X: fn(dims, (X - lo[list(dims)]) / 4.0), 1e-3, 8)
    path = str(tmp_path / "policy.ddsg")
    h.save(path)
    h2 = G.HDMR.load(path)
    assert (h2.d, h2.m, h2.order) == (d, m, 2)
    assert np.array_equal(h2.lo, lo) and np.array_equal(h2.hi, hi)
    assert h2.sizes() == h.sizes()
    for cc in range(h.sizes()[0]):
        a, b = h.component_points(cc), h2.component_points(cc)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    X = torch.from_numpy(lo + 4.0 * synth.uniform_queries(64, 3000, d)).cuda()
    for prec in (0, 1):
        for form in (0, 1):
            y1 = torch.empty((3000, m), dtype=torch.float64, device="cuda")
            y2 = torch.empty_like(y1)
            h.eval(X, y1, prec, form)
            h2.eval(X, y2, prec, form)
            torch.cuda.synchronize()
            assert torch.equal(y1, y2), (prec, form)
    # the file is stable: saving the loaded handle reproduces it byte for byte
    h2.save(str(tmp_path / "again.ddsg"))
    assert open(path, "rb").read() == open(tmp_path / "again.ddsg", "rb").read()
