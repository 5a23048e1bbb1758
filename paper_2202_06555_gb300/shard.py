"""Host logic for spreading the DDSG hot path over several ranks.

Evaluation needs no exchange: every rank holds a full replica of the grid
tables and evaluates its own contiguous slice of the queries (or IRBC states).
A time-iteration step has one exchange: after each rank hierarchizes its share
of the components (the paper's component partition over process groups,
Alg. 2 `load_balance` / `synchronize`), the new surplus rows are all-gathered so
that every replica holds the whole table. Both pieces are plain host code over
``torch.distributed`` (any backend; the tests run them on ``gloo``).
"""
from __future__ import annotations

import numpy as np


def query_slice(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of n items owned by `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need n >= 0 and 0 <= rank < world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def component_partition(costs, world: int) -> list[list[int]]:
    """Components per rank, balanced by cost (points x outputs): longest-processing-
    time-first greedy, ties broken by lower rank then lower component id, so that
    every rank computes the same partition without communicating."""
    if world < 1:
        raise ValueError("world >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda c: (-costs[c], c))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for c in order:
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].append(c)
        load[r] += costs[c]
    return [sorted(p) for p in parts]


def allgather_rows(local: np.ndarray, row_ids: np.ndarray, n_rows: int, group=None) -> np.ndarray:
    """Assemble an [n_rows, m] table from each rank's rows (`local[i]` is row
    `row_ids[i]`). Every row must be owned by exactly one rank; raises otherwise."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    local = np.ascontiguousarray(local, dtype=np.float64)
    row_ids = np.ascontiguousarray(row_ids, dtype=np.int64)
    m = local.shape[1] if local.ndim == 2 else 0
    cnt = torch.tensor([row_ids.shape[0]], dtype=torch.int64)
    cnts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(cnts, cnt, group=group)
    cmax = int(max(int(c.item()) for c in cnts))
    ids = torch.full((cmax,), -1, dtype=torch.int64)
    ids[: row_ids.shape[0]] = torch.from_numpy(row_ids)
    vals = torch.zeros((cmax, m), dtype=torch.float64)
    vals[: row_ids.shape[0]] = torch.from_numpy(local.reshape(-1, m))
    all_ids = [torch.empty_like(ids) for _ in range(world)]
    all_vals = [torch.empty_like(vals) for _ in range(world)]
    dist.all_gather(all_ids, ids, group=group)
    dist.all_gather(all_vals, vals, group=group)
    out = np.zeros((n_rows, m))
    seen = np.zeros(n_rows, dtype=np.int64)
    for i_t, v_t in zip(all_ids, all_vals):
        i = i_t.numpy()
        keep = i >= 0
        out[i[keep]] = v_t.numpy()[keep]
        np.add.at(seen, i[keep], 1)
    if not np.all(seen == 1):
        raise RuntimeError("allgather_rows: rows owned by no rank or by several ranks")
    return out


def max_over_ranks(value: float, group=None) -> float:
    """The largest `value` over all ranks (the step time a multi-rank bench reports)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
