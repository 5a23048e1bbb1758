"""Multi-rank host logic on CPU: world-size-2 gloo ranks (spawned processes).

- Query sharding: the ranks' slices cover the batch exactly once, and the
  all-gathered per-rank evaluations equal a single-process evaluation.
- Component partition + all-gather of surplus rows (the one exchange of a
  time-iteration step): the assembled table equals the single-process table.
- The reported step time is the maximum over ranks.
The per-rank compute is the CPU oracle (this file tests the host logic, not
the GPU kernels)."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_2202_06555_gb300 import shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def test_query_slices_cover_once():
    for n in (0, 1, 7, 100, 2_000_001):
        for world in (1, 2, 3, 8):
            sl = [shard.query_slice(n, r, world) for r in range(world)]
            assert sl[0][0] == 0 and sl[-1][1] == n
            assert all(sl[i][1] == sl[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in sl]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.query_slice(5, 2, 2)


def test_component_partition_balances_and_is_deterministic():
    costs = [5, 1, 1, 1, 1, 1, 3, 3, 0]
    parts = shard.component_partition(costs, 2)
    assert sorted(sum(parts, [])) == list(range(len(costs)))
    loads = [sum(costs[c] for c in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(costs)
    assert parts == shard.component_partition(costs, 2)
    assert shard.component_partition(costs, 1) == [list(range(len(costs)))]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, m = 4, 3
        c = synth.family_coeffs(synth.BASE_SEED + 58, m, d)
        fn = lambda dims, X: synth.family_cut(c, dims, X)
        E = O.OracleDDSG(d, m)
        for u in O.full_order_components(d, 2):
            E.add_regular(list(u), 2)
        E.build_adaptive(fn, 1e-3, 6)
        # queries: each rank evaluates its slice, then all ranks gather
        X = synth.uniform_queries(59, 301, d)
        lo, hi = shard.query_slice(X.shape[0], rank, world)
        y = E.eval(X[lo:hi], form=1)["y"]
        Y = shard.allgather_rows(y, np.arange(lo, hi), X.shape[0])
        # components: each rank contributes the surplus rows of its share
        T = E.tables()
        off = T["off"]
        costs = [(off[i + 1] - off[i]) * m for i in range(len(off) - 1)]
        mine = shard.component_partition(costs, world)[rank]
        rows = np.concatenate([np.arange(off[i], off[i + 1]) for i in mine]) if mine else np.zeros(0, np.int64)
        A = shard.allgather_rows(T["alpha"][rows], rows, T["alpha"].shape[0])
        t = shard.max_over_ranks(1.0 + rank)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), Y=Y, A=A, t=t, n_mine=len(mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather(tmp_path):
    import multiprocessing as mp
    import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + 58, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    E = O.OracleDDSG(d, m)
    for u in O.full_order_components(d, 2):
        E.add_regular(list(u), 2)
    E.build_adaptive(fn, 1e-3, 6)
    Y = E.eval(synth.uniform_queries(59, 301, d), form=1)["y"]
    A = E.tables()["alpha"]
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(2)]
    for k in range(2):
        assert np.array_equal(r[k]["Y"], Y)
        assert np.array_equal(r[k]["A"], A)
        assert float(r[k]["t"]) == 2.0
    assert int(r[0]["n_mine"]) > 0 and int(r[1]["n_mine"]) > 0


def _solve_worker(rank, world, port, out_dir):
    from paper_2202_06555_gb300.time_iteration import _solve_partitioned
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = 3
        need = [(c, synth.uniform_matrix(70 + c, n, 5)) for c, n in enumerate([4, 0, 9, 1, 6, 2, 2])]
        calls = []

        def solve(X):
            calls.append(X.shape[0])
            return np.stack([X.sum(1), X[:, 0] * X[:, 1], np.sin(X[:, 2])], 1)
        sol = _solve_partitioned(solve, need, m, dist.group.WORLD)
        np.savez(os.path.join(out_dir, f"s{rank}.npz"), sol=sol, solved=np.array(sum(calls)))
    finally:
        dist.destroy_process_group()


def test_partitioned_node_solves_equal_one_batch(tmp_path):
    """The time iteration's component-partitioned solve: each rank solves the
    new points of its share of the components (by cost), the rows are
    all-gathered, and every rank returns the single-process batch exactly."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    need = [(c, synth.uniform_matrix(70 + c, n, 5)) for c, n in enumerate([4, 0, 9, 1, 6, 2, 2])]
    X = np.concatenate([x for _, x in need])
    want = np.stack([X.sum(1), X[:, 0] * X[:, 1], np.sin(X[:, 2])], 1)
    r = [np.load(tmp_path / f"s{k}.npz") for k in range(2)]
    for k in range(2):
        assert np.array_equal(r[k]["sol"], want)
    assert int(r[0]["solved"]) + int(r[1]["solved"]) == X.shape[0]
    assert int(r[0]["solved"]) > 0 and int(r[1]["solved"]) > 0
