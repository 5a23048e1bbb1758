"""Adaptive DDSG time iteration on the GPU (Alg. 1 around Alg. 2 of the paper)
for the smooth IRBC model of Sec. 2.1.

One time-iteration step builds the next policy p' as an adaptive DDSG
expansion (Alg. 2) of the map x -> solve{FOC(. | x, p)}: every new grid point
of every component is a cut state (anchor elsewhere) at which the Euler
equations are solved by the GPU Newton (`irbc_newton`, policy p for the next
period); surpluses, refinement (eq. 3.8) and component quadratures (eq. 3.7)
are GPU calls; the expansion criterion (eq. 3.18) and the active dimension
selection (eq. 3.19) act on the (components x outputs) quadrature table.
The iteration stops when the Euler-equation errors of p' at test states fall
below a threshold (Alg. 1) or after a fixed number of steps.

This module only orchestrates calls into libddsg; all grid, surplus,
interpolation and Newton work runs in its kernels.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from . import F64, FORM_SLICEFREE, HDMR, NODES_DELTA
from .shard import allgather_rows, component_partition


class StateSolver:
    """x -> solve{FOC(. | x, p)} at a batch of states (FP64 Newton on the GPU,
    started from the policy p itself)."""

    def __init__(self, model, policy: HDMR, precision=F64, form=FORM_SLICEFREE, tol=1e-10, max_it=30,
                 node_mode=NODES_DELTA):
        self.model, self.policy = model, policy
        self.precision, self.form, self.tol, self.max_it = precision, form, tol, max_it
        self.node_mode = node_mode
        self.calls = 0
        self.points = 0
        self.failed = 0
        self.iterations = 0

    def __call__(self, X: np.ndarray) -> np.ndarray:
        import torch
        n = X.shape[0]
        m = self.policy.m
        xd = torch.from_numpy(np.ascontiguousarray(X, np.float64)).cuda()
        z = torch.empty((n, m), dtype=torch.float64, device="cuda")
        self.policy.eval(xd, z, self.precision, self.form)
        it = torch.zeros(n, dtype=torch.int32, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.model.set_node_mode(self.node_mode)
        self.model.newton(self.policy, xd, z, self.max_it, self.tol, it, st, None, self.precision, self.form)
        torch.cuda.synchronize()
        self.calls += 1
        self.points += n
        self.failed += int((st != 0).sum().item())
        self.iterations += int(it.sum().item())
        return z.cpu().numpy()


def _rank(group):
    if group is None:
        return 0
    import torch.distributed as dist
    return dist.get_rank(group)


def _solve_partitioned(solve, need, m, group):
    """Values at the new points of every component, the components split over the
    ranks of `group` by cost (new points x outputs; shard.component_partition,
    the same on every rank without communication). Each rank solves its
    components' points, then the value rows are all-gathered (shard.allgather_rows,
    Alg. 2's synchronize), so every rank returns the whole batch."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    sizes = [X.shape[0] for _, X in need]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    parts = component_partition([n * m for n in sizes], world)
    mine = parts[rank]
    if mine:
        sol_mine = solve(np.concatenate([need[i][1] for i in mine]))
        ids = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in mine])
    else:
        sol_mine = np.zeros((0, m))
        ids = np.zeros(0, np.int64)
    return allgather_rows(sol_mine, ids, int(offs[-1]), group)


def _adaptive(h: HDMR, known, solve, anchor, eps_gamma, level, strict=False, max_sweeps=64, group=None):
    """Refine / hierarchize sweeps (eq. 3.8) until no point is added; the values
    of all new points of all components are solved in one batch per sweep (split
    over the ranks of `group` by component when it has more than one rank; each
    rank then hierarchizes the whole, identical table).
    known: values of the leading components (in order), or None."""
    import torch
    ncomp, _ = h.sizes()
    vals = list(known) + [None] * (ncomp - len(known))
    multi = False
    if group is not None:
        import torch.distributed as dist
        multi = dist.get_world_size(group) > 1
    for _ in range(max_sweeps):
        need = []
        for c in range(ncomp):
            dims, npts, _ = h.component_info(c)
            have = 0 if vals[c] is None else vals[c].shape[0]
            if have < npts:
                _, _, xs = h.component_points(c, have, npts - have)
                X = np.tile(anchor, (npts - have, 1))
                if len(dims):
                    X[:, list(dims)] = xs
                need.append((c, X))
        if need:
            if multi:
                sol = _solve_partitioned(solve, need, h.m, group)
            else:
                sol = solve(np.concatenate([X for _, X in need]))
            o = 0
            for c, X in need:
                part = sol[o:o + X.shape[0]]
                o += X.shape[0]
                vals[c] = part if vals[c] is None else np.concatenate([vals[c], part])
        h.hierarchize(torch.from_numpy(np.ascontiguousarray(np.concatenate(vals))).cuda())
        if h.refine(eps_gamma, level, strict) == 0:
            break
    return vals


def build_ddsg(solve, d: int, m: int, order: int, level: int, eps_gamma: float, eps_eta: float,
               eps_rho: float, lo, hi, candidates=None, strict=False, group=None):
    """Alg. 2: the adaptive DDSG expansion of the map `solve` (states -> values).

    Order by order k = 1..order: the candidate components of order k that hold
    no rejected component are refined adaptively together with the accepted
    lower-order ones; for k >= 2 a candidate is kept iff eta_u > eps_eta
    (eq. 3.19), otherwise rejected with all its supersets; after the order,
    rho (eq. 3.18) < eps_rho stops the expansion. candidates(k) optionally
    restricts the order-k index sets (default: all k-subsets of the d dims).
    With a torch.distributed `group` of several ranks, the values at new grid
    points are solved component-partitioned over the ranks and all-gathered
    (every rank builds the same expansion).
    Returns the handle holding the accepted components and an info dict."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    anchor = 0.5 * (lo + hi)
    accepted = [()]
    grids = {}            # u -> (levels, indices, values)
    rejected = []
    info = {"rho": [], "eta": {}, "rejected": [], "points": 0}
    for k in range(1, order + 1):
        pool = candidates(k) if candidates else itertools.combinations(range(d), k)
        cand = [tuple(u) for u in pool if not any(set(z) <= set(u) for z in rejected)]
        if not cand:
            break
        h = HDMR(d, m, order, lo=lo, hi=hi)
        comps, known = [], []
        for u in accepted:
            if u in grids:
                lv, ix, v = grids[u]
                h.add_component(list(u), lv, ix)
                known.append(v)
            else:
                h.add_regular(list(u), 2)   # the empty component, first pass only
                known.append(None)
            comps.append(u)
        for u in cand:
            h.add_regular(list(u), 2)
            comps.append(u)
        vals = _adaptive(h, known, solve, anchor, eps_gamma, level, strict, group=group)
        # eq. 3.19 per order-k component and eq. 3.18 over the kept ones, from the
        # component integrals (eq. 3.7), computed by libddsg
        _, eta_c, _, rho = h.expansion_norms(k, eps_eta)
        keep = []
        for c, u in enumerate(comps):
            if u not in grids:
                lv, ix, _ = h.component_points(c)
                grids[u] = (lv, ix, vals[c])
            if len(u) != k:
                continue
            if k >= 2:
                eta = float(eta_c[c])
                info["eta"][u] = eta
                if not eta > eps_eta:
                    rejected.append(u)
                    info["rejected"].append(u)
                    continue
            keep.append(c)
        accepted += [comps[c] for c in keep]
        info["rho"].append(float(rho))
        h.close()
        if rho < eps_rho:
            break
    import torch
    h = HDMR(d, m, order, lo=lo, hi=hi)
    for u in accepted:
        lv, ix, _ = grids[u]
        h.add_component(list(u), lv, ix)
    h.hierarchize(torch.from_numpy(np.ascontiguousarray(np.concatenate([grids[u][2] for u in accepted]))).cuda())
    info["components"] = list(accepted)
    info["points"] = int(h.sizes()[1])
    return h, info


def euler_errors(model, policy: HDMR, states: np.ndarray, precision=F64, form=FORM_SLICEFREE,
                 node_mode=NODES_DELTA):
    """Unit-free Euler-equation errors of a policy at states (the policy gives
    both today's choice and next period's): per state max over countries of
    |beta E / lhs - 1| and |resource| / output."""
    import torch
    n, m = states.shape[0], policy.m
    sd = torch.from_numpy(np.ascontiguousarray(states, np.float64)).cuda()
    g = torch.empty((n, m), dtype=torch.float64, device="cuda")
    policy.eval(sd, g, precision, form)
    r = torch.empty((n, m), dtype=torch.float64, device="cuda")
    e = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    model.set_node_mode(node_mode)
    model.residual(policy, sd, g, r, None, e, precision, form)
    torch.cuda.synchronize()
    return e.cpu().numpy()


def time_iteration(model, policy0: HDMR, steps: int, order: int, level: int, eps_gamma: float,
                   eps_eta: float, eps_rho: float, lo, hi, test_states: np.ndarray, tol_euler=0.0,
                   candidates=None, precision=F64, form=FORM_SLICEFREE, newton_tol=1e-10, max_it=30,
                   node_mode=NODES_DELTA, tol_change=0.0, checkpoint=None, start_step=0, history0=None,
                   group=None):
    """Alg. 1: p <- build_ddsg(x -> solve{FOC(. | x, p)}) until the mean Euler
    error at test_states is below tol_euler, the largest policy change at the
    test states is below tol_change, or `steps` steps are done. With a
    checkpoint path the policy is saved there after every step (hdmr_save) and
    the step count and history beside it (checkpoint + ".json"); resume() reads
    both back, and passing them as policy0, start_step and history0 continues
    the iteration. Each step ends with hdmr_check on both policies (DDSGError
    on a device wait that gave up). Returns the last policy and one record per
    step (history0's records first)."""
    import torch
    d, m = policy0.d, policy0.m
    policy = policy0
    history = list(history0 or [])
    sd = torch.from_numpy(np.ascontiguousarray(test_states, np.float64)).cuda()
    for step in range(start_step, start_step + steps):
        t_step = time.perf_counter()
        solve = StateSolver(model, policy, precision, form, newton_tol, max_it, node_mode)
        new, info = build_ddsg(solve, d, m, order, level, eps_gamma, eps_eta, eps_rho, lo, hi, candidates,
                               group=group)
        e = euler_errors(model, new, test_states, precision, form, node_mode)
        y0 = torch.empty((sd.shape[0], m), dtype=torch.float64, device="cuda")
        y1 = torch.empty_like(y0)
        policy.eval(sd, y0, precision, form)
        new.eval(sd, y1, precision, form)
        torch.cuda.synchronize()
        policy.check()                 # a staged evaluation that gave up a wait read NaN:
        new.check()                    # stop with DDSG_ERR_TIMEOUT rather than iterate on it
        history.append({"step": step, "points": info["points"], "components": len(info["components"]),
                        "rho": info["rho"], "rejected": len(info["rejected"]),
                        "newton_points": solve.points, "newton_failed": solve.failed,
                        "newton_iters_mean": solve.iterations / max(1, solve.points),
                        "euler_error_mean": float(np.mean(np.max(e, 1))),
                        "euler_error_max": float(np.max(e)),
                        "policy_change_max": float((y1 - y0).abs().max().item()),
                        "seconds": time.perf_counter() - t_step})
        if checkpoint and _rank(group) == 0:     # one writer when the ranks share a file system
            save_checkpoint(checkpoint, new, step + 1, history)
        if policy is not policy0:
            policy.close()
        policy = new
        if history[-1]["euler_error_mean"] < tol_euler or history[-1]["policy_change_max"] < tol_change:
            break
    return policy, history


def _file_checksum(path: str) -> str:
    """The FNV-1a checksum that ends a libddsg checkpoint file, as hex."""
    with open(path, "rb") as f:
        f.seek(-8, os.SEEK_END)
        return f.read(8)[::-1].hex()


def save_checkpoint(path: str, policy: HDMR, steps_done: int, history) -> None:
    """The policy (hdmr_save) at `path` and {steps_done, history, the policy
    file's checksum} at path + ".json"; each written to a temporary name and
    then moved into place."""
    policy.save(path + ".tmp")
    os.replace(path + ".tmp", path)
    rec = {"steps_done": int(steps_done), "history": history, "policy_checksum": _file_checksum(path)}
    with open(path + ".json.tmp", "w") as f:
        json.dump(rec, f)
    os.replace(path + ".json.tmp", path + ".json")


def resume(path: str):
    """(policy, steps_done, history) from a time-iteration checkpoint. Refuses a
    record that does not belong to the policy file next to it (an interrupted
    save): ValueError."""
    with open(path + ".json") as f:
        rec = json.load(f)
    if rec.get("policy_checksum") != _file_checksum(path):
        raise ValueError(f"{path}.json does not match {path} (interrupted save)")
    return HDMR.load(path), int(rec["steps_done"]), rec["history"]
