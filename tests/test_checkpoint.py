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


# ---------------------------------------------------------------------------
# network checkpoints (mlp_save / mlp_load)
# ---------------------------------------------------------------------------

def _mlp_file(sizes, step, norm, prm, mm, vv, version=1, magic=b"DDSGMLPN", cut=0, checksum=None):
    body = struct.pack("<i", len(sizes) - 1) + struct.pack(f"<{len(sizes)}i", *sizes) + struct.pack("<q", step)
    body += np.asarray(norm, "<f8").tobytes() + np.asarray(prm, "<f4").tobytes()
    body += np.asarray(mm, "<f4").tobytes() + np.asarray(vv, "<f4").tobytes()
    blob = magic + struct.pack("<II", version, 0) + body + struct.pack("<Q", _fnv(body) if checksum is None else checksum)
    return blob[:len(blob) - cut] if cut else blob


def test_mlp_checkpoint_round_trip_without_a_gpu(G, tmp_path):
    sizes = [4, 8, 3]
    norm = (np.arange(4) * 0.1, np.full(4, 2.0), np.linspace(0.9, 1.1, 3), np.full(3, 5.0))
    net = G.MLP(sizes, seed=11, in_shift=norm[0], in_scale=norm[1], out_shift=norm[2], out_scale=norm[3])
    p = tmp_path / "net.ddsg"
    net.save(str(p))
    blob = p.read_bytes()
    assert blob[:8] == b"DDSGMLPN" and struct.unpack("<II", blob[8:16]) == (1, 0)
    npar = 4 * 8 + 8 + 8 * 3 + 3
    L, s0, s1, s2, step = struct.unpack("<iiiiq", blob[16:40])
    assert (L, [s0, s1, s2], step) == (2, sizes, 0)
    nrm = np.frombuffer(blob[40:40 + 8 * 14], "<f8")
    assert np.array_equal(nrm, np.concatenate(norm))
    rest = np.frombuffer(blob[40 + 8 * 14:-8], "<f4")
    assert rest.size == 3 * npar
    assert np.array_equal(rest[:npar], net.flat_params()) and not rest[npar:].any()   # Adam moments start at zero
    assert _fnv(blob[16:-8]) == struct.unpack("<Q", blob[-8:])[0]
    back = G.MLP.load(str(p))
    assert back.sizes == sizes and np.array_equal(back.flat_params(), net.flat_params())
    # refused files
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        G.MLP.load(str(tmp_path / "missing.ddsg"))
    prm = net.flat_params()
    cases = {"foreign": _mlp_file(sizes, 0, np.concatenate(norm), prm, 0 * prm, 0 * prm, magic=b"DDSGHDMR"),
             "version": _mlp_file(sizes, 0, np.concatenate(norm), prm, 0 * prm, 0 * prm, version=2),
             "corrupt": _mlp_file(sizes, 0, np.concatenate(norm), prm, 0 * prm, 0 * prm, checksum=7),
             "truncated": _mlp_file(sizes, 0, np.concatenate(norm), prm, 0 * prm, 0 * prm, cut=20),
             "sizes": _mlp_file([4, 9, 3], 0, np.concatenate(norm), prm, 0 * prm, 0 * prm)}
    for name, b in cases.items():
        q = tmp_path / f"{name}.ddsg"
        q.write_bytes(b)
        with pytest.raises(G.DDSGError, match="ERR_ARG"):
            G.MLP.load(str(q))


@pytest.mark.gpu
def test_mlp_training_resumes_bit_for_bit(G, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sizes = [6, 64, 64, 3]
    norm = (np.full(6, 1.0), np.full(6, 5.0), np.full(3, 1.0), np.full(3, 10.0))
    batches = []
    for b in range(7):
        x = synth.uniform_matrix(500 + b, 512, 6, 0.8, 1.2)
        y = 1.0 + 0.05 * np.sin(x[:, :3] * (b + 1))
        batches.append((torch.from_numpy(x).cuda(), torch.from_numpy(np.ascontiguousarray(y)).cuda()))
    a = G.MLP(sizes, seed=21, in_shift=norm[0], in_scale=norm[1], out_shift=norm[2], out_scale=norm[3])
    for x, y in batches[:4]:
        a.train_step(x, y, 1e-3)
    p = tmp_path / "net.ddsg"
    a.save(str(p))
    b_ = G.MLP.load(str(p))
    assert np.array_equal(b_.flat_params(), a.flat_params())
    for x, y in batches[4:]:
        a.train_step(x, y, 1e-3)
        b_.train_step(x, y, 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(a.flat_params(), b_.flat_params())      # Adam moments and step restored
    xt = batches[0][0]
    ya = torch.zeros((xt.shape[0], 3), dtype=torch.float64, device="cuda")
    yb = torch.zeros_like(ya)
    a.infer(xt, ya)
    b_.infer(xt, yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)


def test_time_iteration_record_must_match_its_policy_file(tmp_path):
    """resume() refuses a step record written for another policy file (a save
    interrupted between the two files). No GPU: the check precedes the load."""
    import json
    from paper_2202_06555_gb300 import time_iteration as TI
    p = tmp_path / "ti.ddsg"
    p.write_bytes(b"DDSGHDMR" + struct.pack("<II", 1, 0) + b"body" + struct.pack("<Q", 0x1122334455667788))
    assert TI._file_checksum(str(p)) == "1122334455667788"
    (tmp_path / "ti.ddsg.json").write_text(json.dumps({"steps_done": 3, "history": [], "policy_checksum": "00"}))
    with pytest.raises(ValueError, match="interrupted save"):
        TI.resume(str(p))
