"""The component partition of a time-iteration step on libddsg, over two ranks.

Two spawned processes join a world-size-2 gloo group and share cuda:0; each
runs two adaptive time-iteration steps of the N = 2 IRBC model with the
library (Alg. 1 around Alg. 2). Inside every refinement sweep the Newton solves
at the new grid points are split over the ranks by component cost
(shard.component_partition) and the value rows all-gathered
(shard.allgather_rows, Alg. 2's synchronize); each rank hierarchizes the whole
table. Expected: both ranks end with the single-process policy bit for bit,
each solved part of the points, and the parts add up to the single-process
count. The ranks' kernels never wait on one another (the exchange runs on the
host), so sharing one GPU is sound."""
import os
import socket

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
pytestmark = pytest.mark.gpu

N = 2
STEPS = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run(group):
    """Two time-iteration steps from the steady-state order-1 policy; returns
    (components, surpluses, history)."""
    import paper_2202_06555_gb300 as G
    from paper_2202_06555_gb300.time_iteration import time_iteration
    G.load()
    d = 2 * N
    t1 = G.irbc_table1(N)
    M = G.IRBC(**t1)
    lam = synth.irbc_steady_lambda(t1["gamma"], t1["tau"], t1["A"], t1["delta"])
    h0 = G.HDMR(d, N + 1, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    comps = [()] + [(i,) for i in range(d)]
    for u in comps:
        h0.add_regular(list(u), 2)
    vals = []
    for c, u in enumerate(comps):
        _, _, xs = h0.component_points(c)
        y = np.tile(np.concatenate([np.ones(N), [lam]]), (xs.shape[0], 1))
        for a, dim in enumerate(u):
            if dim >= N:
                y[:, dim - N] = xs[:, a]
        vals.append(y)
    h0.hierarchize(torch.from_numpy(np.concatenate(vals)).cuda())
    T = synth.irbc_states(synth.BASE_SEED + 611, 32, N)
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    h, hist = time_iteration(M, h0, STEPS, 2, 4, 1e-4, -1.0, 0.0, lo, hi, T, precision=G.F64, group=group)
    nc, _ = h.sizes()
    info = [h.component_info(c)[:2] for c in range(nc)]
    return info, h.surpluses(), hist


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        info, alpha, hist = _run(dist.group.WORLD)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), alpha=alpha,
                 info=np.array([str(x) for x in info]),
                 newton=np.array([h["newton_points"] for h in hist]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_partition_the_node_solves_bit_for_bit(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import multiprocessing as mp
    O.build()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    info, alpha, hist = _run(None)
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(2)]
    single = np.array([h["newton_points"] for h in hist])
    for k in range(2):
        assert r[k]["info"].tolist() == [str(x) for x in info]
        assert np.array_equal(r[k]["alpha"], alpha)
        assert np.all(r[k]["newton"] < single)           # each rank solved a part
    assert np.array_equal(r[0]["newton"] + r[1]["newton"], single)
