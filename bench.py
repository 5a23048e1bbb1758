#!/usr/bin/env python
"""Benchmark of batched DDSG (cut-HDMR adaptive sparse grid) interpolation.

Default workload: d = 100 (N = 50), m = 51 outputs, order-2 cut-HDMR with the
anchor at the domain centre (100 1D + 4950 2D components + the empty one),
every component adaptively refined (surplus threshold 1e-3, level 10) on the
seeded kinked test family; 2e6 query points uniform in [0,1]^100. One step is
one evaluation of all 2e6 points (query encoding + interpolation kernels).

  python bench.py [--gpus N --steps K --warmup W] [--workload d100|d20|sg4]
                  [--precision f32c|f64] [--form slicefree|paper]
                  [--impl reference]

Prints one JSON line (rank 0). --impl reference times the CPU oracle (test
infrastructure) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "interp evals/s (points·outputs) at d=100; % HBM roofline; FP32 vs FP64 error"

WORKLOADS = {
    "d100": dict(d=100, m=51, order=2, eps=1e-3, level=10, Q=2_000_000, wid=synth.W_D100,
                 queries="uniform", precision="f32c", form="slicefree"),
    "d20": dict(d=20, m=11, order=2, eps=1e-3, level=10, Q=440_000, wid=synth.W_D20,
                queries="monomial", precision="f64", form="slicefree"),
    "sg4": dict(d=4, m=3, order=4, eps=None, level=5, Q=100_000, wid=synth.W_SG4,
                queries="uniform", precision="f64", form="paper"),
    # IRBC Euler-residual sweep: N = 150 (d = 300, m = 151), policy = empty + 300 singles +
    # 150 (a_j, k_j) pairs on regular level-4 grids; 1e4 states x 302 monomial nodes
    "irbc150": dict(d=300, m=151, N=150, level=4, states=10_000, wid=synth.W_IRBC150,
                    precision="f32c", form="slicefree"),
    # the Newton solve of the same model alone: node shortcut, F32C interpolation, FP64
    # residual and solves, from the initial guess to ||r||_inf <= 1e-6 (1e-10 in FP64)
    "irbc150newton": dict(d=300, m=151, N=150, level=4, states=10_000, wid=synth.W_IRBC150,
                          precision="f32c", form="slicefree"),
    # learned warm start: N = 20 (d = 40, m = 21), 1e6 training pairs, 5e4 test states
    "warmstart20": dict(d=40, m=21, N=20, level=4, states=50_000, train=1_000_000,
                        wid=synth.W_IRBC20, precision="f64", form="slicefree", epochs=10,
                        batch=4096),
    # adaptive DDSG time iteration (Alg. 1 around Alg. 2): N = 10 (d = 20, m = 11), order 2
    # over all pairs with eta / rho pruning, adaptive grids up to level 6
    "ti10": dict(d=20, m=11, N=10, order=2, level=6, eps_gamma=1e-4, eps_eta=1e-5, eps_rho=1e-6,
                 ti_steps=4, test_states=2000, wid=synth.W_IRBC20 + 10, precision="f64",
                 form="slicefree"),
    # Table 2's smooth d = 100 setting: N = 50, order 1, regular level-4 grids (801 points),
    # iterated until the policy stops moving
    "ti50": dict(d=100, m=51, N=50, order=1, level=4, eps_gamma=-1.0, eps_eta=-1.0, eps_rho=0.0,
                 ti_steps=400, tol_change=1e-7, test_states=2000, wid=synth.W_D100 + 50, precision="f64",
                 form="slicefree"),
    # the same on the non-smooth model (irreversible investment): N = 6, policy (k', mu, lambda)
    "ti6irr": dict(d=12, m=13, N=6, order=2, level=6, eps_gamma=1e-4, eps_eta=1e-5, eps_rho=1e-6,
                   ti_steps=4, test_states=2000, wid=synth.W_IRBC20 + 11, precision="f64",
                   form="slicefree", irreversible=True),
}

KERNEL_NAMES = ["tile", "per-tuple", "tma-staged tile", "tma-staged, 2 warp groups", "tma-staged, 3 warp groups",
                "nodal-slab, tma-staged", "nodal-slab, tma-staged, Kahan totals in tensor memory"]

FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (4 schedulers x 32), for the nominal figure only


def device_facts(local):
    """SM count (from the device) and maximum SM clock (nvidia-smi, else the
    device's clock attribute) of the GPU this rank uses."""
    import torch
    props = torch.cuda.get_device_properties(local)
    sms = int(props.multi_processor_count)
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(local), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        mhz = float(out.stdout.strip().splitlines()[0])
    except Exception:
        mhz = None
    if not mhz:
        try:
            mhz = float(getattr(props, "clock_rate", 0)) / 1e3 or None
        except Exception:
            mhz = None
    return sms, mhz


def measure_fma_peaks(G, uuid):
    """FMA throughput measured on this device by the library's probe
    (csrc/ddsg_probe.cu: 8 independent chains per thread, 16 warps per
    scheduler), with the SM clocks sampled while it runs."""
    res = {}
    with ClockSampler(uuid) as clk:
        for name, kind in (("fp64_fma", 0), ("fp32_fma", 1), ("fp32_fma_x2", 2)):
            best = 0.0
            for _ in range(3):
                t, _ = G.probe_fma(kind)
                best = max(best, t)
            res[name] = best
    res["fp32"] = max(res["fp32_fma"], res["fp32_fma_x2"])
    res["source"] = "ddsg_probe_fma (paper_2202_06555_gb300/csrc/ddsg_probe.cu), best of 3 launches"
    res["clocks"] = clk.summary()
    return res


def full_order_components(d, order):
    import itertools
    out = []
    for k in range(order + 1):
        out.extend(itertools.combinations(range(d), k))
    return out


def comp_list(w):
    if w["eps"] is None:
        return [tuple(range(w["d"]))]
    return full_order_components(w["d"], w["order"])


# DRAM traffic of the evaluation kernel from one ncu capture per schedule, per
# query; scaled to a full launch by the query count (the tables stream through
# L2 once per wave of resident blocks, so traffic grows with the queries).
#   (6, 32): profiles/eval_nodal_tmem_d100_ncu_full.md -- the nodal-slab kernel with
#            its Kahan totals in tensor memory, d=100 tables, 38912 queries (one wave
#            of 152 blocks of 256 queries);
#   (5, 32): profiles/eval_nodal_d100_ncu_full.md -- the nodal-slab kernel, d=100
#            tables, 29184 queries (one wave of 152 blocks of 192 queries);
#   (3, 28): profiles/eval_tma_d100_ncu_full.md -- the two-group level-tuple
#            TMA kernel at 28 outputs per group, same tables and queries.
# Valid only for the kernel sources each was taken on (checked by hash).
EVAL_TRAFFIC = [
    {"workload": "d100", "schedule": (6, 32), "dram_bytes_per_query": (365242624 + 4188160) / 38912,
     "sha1": {"ddsg_nodal.cu": "8637d41ca91adbfde6eb48cea990b27088b3dfe8", "ddsg_eval.cuh": "a190d34e3b3fe0a7095a2f5ca6734106056dd7c9", "ddsg_internal.h": "103a72ef0530989e3daa14bf03b10b6c7a671e96", "ddsg_tma.cuh": "3d90c7da8651e19c5d8c36464fa0ee4bdc3e1dbd"}},
    {"workload": "d100", "schedule": (5, 32), "dram_bytes_per_query": (355433472 + 4008448) / 29184,
     "sha1": {"ddsg_nodal.cu": "c3418abccc98544024d6121b90a3260f2c5968df",
              "ddsg_eval.cuh": "a190d34e3b3fe0a7095a2f5ca6734106056dd7c9",
              "ddsg_internal.h": "35e5d984e243926340ad5cc33984726f9818640e",
              "ddsg_tma.cuh": "3d90c7da8651e19c5d8c36464fa0ee4bdc3e1dbd"}},
]


def measured_peaks():
    """MEASURED_PEAKS.json (driver-written per pod), or {} where absent."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def eval_traffic(workload, schedule, n):
    import hashlib
    for t in EVAL_TRAFFIC:
        if workload != t["workload"] or tuple(schedule) != t["schedule"]:
            continue
        for f, h in t["sha1"].items():
            path = os.path.join(ROOT, "paper_2202_06555_gb300", "csrc", f)
            if hashlib.sha1(open(path, "rb").read()).hexdigest() != h:
                return None
        return t["dram_bytes_per_query"] * n
    return None


def make_queries(w, rank=0, world=1):
    """This rank's queries: its contiguous slice (shard.query_slice) of one seeded
    batch of world x Q queries (weak scaling: Q per rank; rank 0 of 1 gets the
    whole single-GPU batch)."""
    from paper_2202_06555_gb300.shard import query_slice
    seed = synth.BASE_SEED + w["wid"]
    if w["queries"] == "monomial":
        N = w["d"] // 2
        per = 2 * (N + 1)
        ns = w["Q"] // per
        lo, hi = query_slice(ns * world, rank, world)
        return synth.monomial_shaped_queries(seed, ns * world, N)[lo * per:hi * per]
    lo, hi = query_slice(w["Q"] * world, rank, world)
    return synth.uniform_queries_rows(seed, lo, hi, w["d"])


def value_fn(w):
    c = synth.family_coeffs(synth.BASE_SEED + w["wid"], w["m"], w["d"])
    return lambda dims, X: synth.family_cut(c, dims, X)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ddsg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def oracle_build(w):
    import oracle as O
    E = O.OracleDDSG(w["d"], w["m"])
    if w["eps"] is None:
        E.add_regular(tuple(range(w["d"])), w["level"])
        E.fill_values(value_fn(w))
        E.hierarchize()
    else:
        for u in comp_list(w):
            E.add_regular(u, 2)
        E.build_adaptive(value_fn(w), w["eps"], w["level"])
    return E


def oracle_rate(E, w, X, budget_s):
    """Oracle evaluation rate (evals/s, points*outputs) on a prefix of X that
    takes about budget_s seconds; returns (rate, n_used)."""
    form = 1 if w["form"] == "slicefree" else 0
    n = 1
    used, t_used = 0, 0.0
    while True:
        t0 = time.perf_counter()
        E.eval(X[used:used + n], form=form)
        dt = time.perf_counter() - t0
        used += n
        t_used += dt
        if t_used >= budget_s or used >= X.shape[0]:
            break
        n = max(1, min(X.shape[0] - used, int(n * 2 if dt < 0.2 * budget_s else n)))
    return used * w["m"] / t_used, used


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, or implementer/part on Arm)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return None
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    impl = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")), None)
    part = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")), None)
    return f"implementer {impl}, part {part}" if impl else None


def oracle_rate_threads(E, w, X, n, threads):
    """Oracle evaluation rate with `threads` host threads, each evaluating a
    contiguous share of X[:n] (the C oracle releases the GIL; its code is the
    same as in the single-thread run); returns evals/s."""
    from concurrent.futures import ThreadPoolExecutor
    form = 1 if w["form"] == "slicefree" else 0
    E.tables()
    E.b_coeffs()
    bounds = [(n * t // threads, n * (t + 1) // threads) for t in range(threads)]
    with ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda b: E.eval(X[b[0]:b[1]], form=form), bounds))
        dt = time.perf_counter() - t0
    return n * w["m"] / dt


def metric_for(w):
    """The headline metric, naming the workload's dimension (d = 100: verbatim)."""
    return METRIC if w["d"] == 100 else METRIC.replace("d=100", "d=%d" % w["d"])


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    E = oracle_build(w)
    X = make_queries(w)
    # each step: a bounded sample sized to ~4 s of single-thread oracle work,
    # never more than the workload's queries
    _, n_probe = oracle_rate(E, w, X, 1.0)
    per_step = max(1, min(int(n_probe * 4), X.shape[0]))
    for s in range(args.warmup):
        E.eval(X[:min(per_step, 2)], form=1 if w["form"] == "slicefree" else 0)
    times = []
    for s in range(args.steps):
        lo = (s * per_step) % max(1, X.shape[0] - per_step)
        t0 = time.perf_counter()
        E.eval(X[lo:lo + per_step], form=1 if w["form"] == "slicefree" else 0)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = per_step * w["m"] / (ms * 1e-3)
    line = {"impl": "reference", "metric": metric_for(w), "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "d": w["d"], "m": w["m"],
                       "queries_per_step": per_step, "form": w["form"]},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} of the {w['Q']} queries per step, single thread"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# IRBC Euler-residual sweep (CUDA arm, and the oracle as the reference arm)
# ---------------------------------------------------------------------------

def irbc_workload(w, G=None):
    """Table 1 model, synthetic policy (steady state + seeded perturbation),
    states and the initial guess (k' = k, lambda = lambda*)."""
    import paper_2202_06555_gb300 as GG
    G = G or GG
    N, level = w["N"], w["level"]
    t1 = G.irbc_table1(N)
    lam = synth.irbc_steady_lambda(t1["gamma"], t1["tau"], t1["A"], t1["delta"])
    base = np.concatenate([np.ones(N), [lam]])
    pert = synth.irbc_policy_perturbation(synth.BASE_SEED + w["wid"], N)
    fn = lambda dims, X: synth.irbc_policy_values(base, pert, dims, X)
    comps = [()] + [(i,) for i in range(2 * N)] + [(j, N + j) for j in range(N)]
    S = synth.irbc_states(synth.BASE_SEED + w["wid"], w["states"], N)
    g = np.ascontiguousarray(np.concatenate([S[:, N:], np.full((S.shape[0], 1), lam)], 1))
    return t1, lam, fn, comps, S, g


def irbc_sweep_flops(G, h, w, t1, comps, fn, S, g, prec, form, sample=1000):
    """Algorithmic flops of one all-node sweep's interpolation: the active points
    of the next-period states at the 2(N+1) monomial nodes of a sample of the
    states (counted by the library's count pass), scaled to all states, each
    point costing 2m + k + 1 (k its component's order). The node queries are
    formed here from the law of motion only to count points."""
    import torch
    N, m, d = w["N"], w["m"], w["d"]
    ns = min(sample, S.shape[0])
    hs = np.sqrt(N + 1.0)
    la = np.log(S[:ns, :N])
    X = np.empty((ns, 2 * (N + 1), d))
    for q in range(2 * (N + 1)):
        e = np.zeros(N)
        if q < 2 * N:
            e[q // 2] = hs if q % 2 == 0 else -hs
        else:
            e[:] = hs if q == 2 * N else -hs
        X[:, q, :N] = np.exp(t1["rho"] * la + t1["sigma"] * e[None, :])
        X[:, q, N:] = g[:ns, :N]
    X = X.reshape(-1, d)
    n = X.shape[0]
    x = torch.from_numpy(X).cuda()
    y = torch.empty((n, m), dtype=torch.float64, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    h.eval(x, y, prec, form, None, cnt)
    torch.cuda.synchronize()
    A = float(cnt.double().sum().item())
    # the order <= 1 part of the same policy, for the k of each point
    h1 = G.HDMR(d, m, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    c1 = [u for u in comps if len(u) <= 1]
    for u in c1:
        h1.add_regular(list(u), w["level"])
    h1.hierarchize(torch.from_numpy(np.concatenate([fn(u, h1.component_points(c)[2]) for c, u in enumerate(c1)])).cuda())
    h1.eval(x, y, prec, form, None, cnt)
    torch.cuda.synchronize()
    A1 = float(cnt.double().sum().item())
    h1.close()
    scale = S.shape[0] / ns
    flops = ((2.0 * m + 1.0) * A + 2.0 * (A - A1) + (A1 - n)) * scale
    return flops, A / n


def run_irbc(args, w):
    N, m, d = w["N"], w["m"], w["d"]
    nq = 2 * (N + 1)
    metric = "Euler-residual policy evals/s (states x monomial nodes x outputs) at N=150"
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return 0
        import oracle as O
        t1, lam, fn, comps, S, g = irbc_workload(w)
        E = O.irbc_policy_ddsg(N, w["level"], fn)
        I = O.IRBCOracle(N)
        for _ in range(args.warmup):
            I.residual(E, S[:1], g[:1])
        per = 4
        times = []
        for s in range(args.steps):
            t0 = time.perf_counter()
            I.residual(E, S[s * per:(s + 1) * per], g[s * per:(s + 1) * per])
            times.append(time.perf_counter() - t0)
        ms = 1e3 * statistics.mean(times)
        value = per * nq * m / (ms * 1e-3)
        print(json.dumps({"impl": "reference", "metric": metric, "value": value, "unit": "evals/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "irbc150_euler_residual", "states_per_step": per},
                          "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1,
                                           "kind": "oracle", "sample": f"{per} states per step"},
                          "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    import torch
    import paper_2202_06555_gb300 as G
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    G.load()
    out = measure_irbc(w, args.steps, args.warmup, fma=measure_fma_peaks(G, None))
    print(json.dumps(out), flush=True)
    return 0


# Newton variants of the N = 150 step: (name, precision, tolerance, node mode)
IRBC_NEWTON_ALL = (("f64", "F64", 1e-6, "NODES_ALL"), ("f32c", "F32C", 1e-6, "NODES_ALL"),
                   ("f64_tight", "F64", 1e-10, "NODES_ALL"),
                   ("f32c_node_shortcut", "F32C", 1e-6, "NODES_DELTA"),
                   ("f64_tight_node_shortcut", "F64", 1e-10, "NODES_DELTA"))


def measure_irbc(w, steps, warmup, newton_variants=IRBC_NEWTON_ALL, fma=None):
    """Euler-residual sweep of the N = 150 model on the GPU (all nodes, then the
    node shortcut) and Newton solves per variant; returns the JSON record."""
    import torch
    import paper_2202_06555_gb300 as G
    G.load()
    N, m, d = w["N"], w["m"], w["d"]
    nq = 2 * (N + 1)
    metric = "Euler-residual policy evals/s (states x monomial nodes x outputs) at N=150"
    t1, lam, fn, comps, S, g = irbc_workload(w, G)
    h = G.HDMR(d, m, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in comps:
        h.add_regular(list(u), w["level"])
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(**t1)
    prec = G.F32C if w["precision"] == "f32c" else G.F64
    form = G.FORM_SLICEFREE if w["form"] == "slicefree" else G.FORM_PAPER
    ns = S.shape[0]
    sd = torch.from_numpy(S).cuda()
    gd = torch.from_numpy(g).cuda()
    r = torch.empty((ns, N + 1), dtype=torch.float64, device="cuda")
    nt = min(ns * nq, 65536)
    xt = torch.from_numpy(np.ascontiguousarray(np.repeat(S[:nt // nq + 1, :], nq, 0)[:nt])).cuda()
    yt = torch.empty((nt, m), dtype=torch.float64, device="cuda")
    tuned = h.autotune(xt, yt, prec, form)
    for _ in range(warmup):
        M.residual(h, sd, gd, r, None, None, prec, form)
    torch.cuda.synchronize()
    M.profile(True)
    M.profile_read(reset=True)
    stream = torch.cuda.current_stream()
    with ClockSampler(None) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            M.residual(h, sd, gd, r, None, None, prec, form)
        e1.record(stream)
        torch.cuda.synchronize()
    prof = M.profile_read(reset=True)
    M.profile(False)
    ms = e0.elapsed_time(e1) / steps
    value = ns * nq * m / (ms * 1e-3)
    # the node shortcut (a separate form: the plain sweep above is the metric)
    M.set_node_mode(G.NODES_DELTA)
    r_d = torch.empty_like(r)
    M.residual(h, sd, gd, r_d, None, None, prec, form)
    torch.cuda.synchronize()
    M.profile(True)
    M.profile_read(reset=True)
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(steps):
        M.residual(h, sd, gd, r_d, None, None, prec, form)
    d1.record(stream)
    torch.cuda.synchronize()
    prof_d = M.profile_read(reset=True)
    M.profile(False)
    M.set_node_mode(G.NODES_ALL)
    ms_d = d0.elapsed_time(d1) / steps
    M.residual(h, sd, gd, r, None, None, prec, form)
    scale = r.abs().clamp_min(1.0)
    shortcut = {"ms_per_step": ms_d, "value": ns * nq * m / (ms_d * 1e-3), "unit": "evals/s",
                "speedup": ms / ms_d,
                "max_abs_diff_vs_all_nodes_scaled": float(((r_d - r).abs() / scale).max().item()),
                "kernels_ms": {k: v[0] / max(1, v[1]) for k, v in prof_d.items()}}
    # Newton from the initial guess, FP64 vs F32C interpolation, same tolerance
    newton = {}
    for name, prn, tol, moden in newton_variants:
        pr, mode = getattr(G, prn), getattr(G, moden)
        M.set_node_mode(mode)
        z = gd.clone()
        it = torch.zeros(ns, dtype=torch.int32, device="cuda")
        st = torch.zeros(ns, dtype=torch.int32, device="cuda")
        nr = torch.zeros(ns, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        M.profile(True)
        M.profile_read(reset=True)
        t0 = time.perf_counter()
        M.newton(h, sd, z, 12, tol, it, st, nr, pr, form)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        prof_n = M.profile_read(reset=True)
        M.profile(False)
        err = torch.zeros((ns, 2), dtype=torch.float64, device="cuda")
        M.set_node_mode(G.NODES_ALL)
        M.residual(h, sd, z, r, None, err, G.F64, form)
        ee = err.cpu().numpy()
        newton[name] = {"seconds": dt, "tol": tol, "iters_mean": float(it.double().mean().item()),
                        "iters_max": int(it.max().item()),
                        "converged": int((st == 0).sum().item()),
                        "euler_error_log10_mean": float(np.log10(np.mean(ee[:, 0]))),
                        "euler_error_log10_max": float(np.log10(np.max(ee[:, 0]))),
                        "kernels_ms_total": {kk: vv[0] for kk, vv in prof_n.items()},
                        "launches": sum(vv[1] for vv in prof_n.values())}
    roof = None
    if fma is not None:
        # the sweep's interpolation (all nodes) against the measured FMA peak
        flops, apq = irbc_sweep_flops(G, h, w, t1, comps, fn, S, g, prec, form)
        ev_tot, ev_n = prof.get("eval", (0.0, 1))
        ev_n = max(1, ev_n) // max(1, steps)   # launches per sweep (chunks of states)
        ev_ms = ev_tot / max(1, steps)        # eval time per sweep
        peak = fma["fp32"] if prec == G.F32C else fma["fp64_fma"]
        achieved = flops / (ev_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "eval (the sweep's interpolation of all 2(N+1) nodes)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel_ms_per_sweep": ev_ms, "launches_per_sweep": ev_n,
                "flops_per_sweep": flops,
                "active_points_per_query": apq,
                "flop_count": "sum over active points of 2m + k + 1, counted on the node queries of "
                              "1,000 of the states and scaled to all",
                "peak_source": "measured (of measured): ddsg_probe_fma %s chains" %
                               ("FP32" if prec == G.F32C else "FP64"),
                "note": "the residual, Jacobian, LU and delta kernels: profiles/irbc150_newton_kernels.md"}
    out = {"metric": metric, "value": value, "unit": "evals/s", "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if prec == G.F32C else "f64", "data": "synthetic",
           "config": {"workload": "irbc150_euler_residual", "N": N, "d": d, "m": m,
                      "states": ns, "nodes": nq, "evals_per_sweep": ns * nq,
                      "policy": "empty + 2N singles + N (a_j,k_j) pairs, regular level 4",
                      "precision": w["precision"], "form": w["form"],
                      "schedule": {"kernel": KERNEL_NAMES[tuned[0]], "outputs_per_pass": tuned[1]}},
           "kernels_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items()},
           "gpu_launches": sum(v[1] for v in prof.values()),
           "node_shortcut": shortcut, "newton": newton, "clocks": clk.summary()}
    if roof is not None:
        out["roofline"] = roof
    h.close()
    M.close()
    return out


def run_irbc_newton(args, w):
    """Newton solves of the N = 150 model at w["states"] states (node shortcut):
    warm-up solves, then timed solves, each from the same initial guess; one more
    traced solve gives the per-kernel split."""
    N, m, d = w["N"], w["m"], w["d"]
    tol = 1e-6 if w["precision"] == "f32c" else 1e-10
    metric = "Newton solve time at N=150 (node shortcut; FP64 residual and solves)"
    t1, lam, fn, comps, S, g = irbc_workload(w)
    ns = S.shape[0]
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return 0
        import oracle as O
        E = O.irbc_policy_ddsg(N, w["level"], fn)
        I = O.IRBCOracle(N)
        per = 1
        for _ in range(args.warmup):
            I.newton(E, S[:per], g[:per], tol=tol)
        times = []
        for s in range(args.steps):
            t0 = time.perf_counter()
            I.newton(E, S[s * per:(s + 1) * per], g[s * per:(s + 1) * per], tol=tol)
            times.append(time.perf_counter() - t0)
        ms = 1e3 * statistics.mean(times) * ns / per   # scaled to the workload's states
        print(json.dumps({"impl": "reference", "metric": metric, "value": ms, "unit": "ms",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "irbc150_newton", "states": ns},
                          "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                                           "sample": f"{per} state per step, scaled to {ns} states"},
                          "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    import torch
    import paper_2202_06555_gb300 as G
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    G.load()
    h = G.HDMR(d, m, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in comps:
        h.add_regular(list(u), w["level"])
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(**t1)
    M.set_node_mode(G.NODES_DELTA)
    prec = G.F32C if w["precision"] == "f32c" else G.F64
    form = G.FORM_SLICEFREE if w["form"] == "slicefree" else G.FORM_PAPER
    # the schedule for the batches this solve interpolates: 3 queries per state
    xt = torch.from_numpy(np.ascontiguousarray(np.repeat(S, 3, 0))).cuda()
    yt = torch.empty((xt.shape[0], m), dtype=torch.float64, device="cuda")
    tuned = h.autotune(xt, yt, prec, form)
    del xt, yt
    sd = torch.from_numpy(S).cuda()
    g0 = torch.from_numpy(g).cuda()
    z = torch.empty_like(g0)
    it = torch.zeros(ns, dtype=torch.int32, device="cuda")
    st = torch.zeros_like(it)
    nr = torch.zeros(ns, dtype=torch.float64, device="cuda")

    def solve():
        z.copy_(g0)
        M.newton(h, sd, z, 12, tol, it, st, nr, prec, form)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    with ClockSampler(None) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solve()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    M.profile(True)
    M.profile_read(reset=True)
    solve()
    torch.cuda.synchronize()
    prof = M.profile_read(reset=True)
    M.profile(False)
    err = torch.zeros((ns, 2), dtype=torch.float64, device="cuda")
    r = torch.zeros((ns, m), dtype=torch.float64, device="cuda")
    M.set_node_mode(G.NODES_ALL)
    M.residual(h, sd, z, r, None, err, G.F64, form)
    ee = err.cpu().numpy()
    print(json.dumps({"metric": metric, "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32" if prec == G.F32C else "f64", "data": "synthetic",
                      "config": {"workload": "irbc150_newton", "N": N, "states": ns, "tol": tol,
                                 "precision": w["precision"], "form": w["form"], "node_mode": "shortcut",
                                 "schedule": {"kernel": tuned[0], "outputs_per_pass": tuned[1]}},
                      "iters_mean": float(it.double().mean().item()), "converged": int((st == 0).sum().item()),
                      "euler_error_log10_mean": float(np.log10(np.mean(ee[:, 0]))),
                      "euler_error_log10_max": float(np.log10(np.max(ee[:, 0]))),
                      "kernels_ms": {kk: vv[0] for kk, vv in prof.items()},
                      "gpu_launches": sum(vv[1] for vv in prof.values()),
                      "clocks": clk.summary()}), flush=True)
    return 0


def run_time_iteration(args, w):
    """Adaptive DDSG time iteration of the smooth IRBC model on the GPU: per step
    the seconds, grid points, Newton solves and the Euler errors at test states."""
    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the time-iteration study has no timed CPU arm (the oracle version is a test pin)"}))
        return 0
    import torch
    import paper_2202_06555_gb300 as G
    from paper_2202_06555_gb300.time_iteration import time_iteration
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    G.load()
    N, d, m = w["N"], w["d"], w["m"]
    t1 = G.irbc_table1(N)
    lam = synth.irbc_steady_lambda(t1["gamma"], t1["tau"], t1["A"], t1["delta"])
    M = G.IRBC(**t1)
    irr = bool(w.get("irreversible"))
    if irr:
        M.set_irreversible(True)
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    # initial policy: k' = k, (mu = 0), lambda = lambda* (exact on level-2 single-dimension grids)
    h0 = G.HDMR(d, m, 2, lo=lo, hi=hi)
    comps = [()] + [(i,) for i in range(d)]
    for u in comps:
        h0.add_regular(list(u), 2)
    vals = []
    for c, u in enumerate(comps):
        _, _, xs = h0.component_points(c)
        y = np.tile(np.concatenate([np.ones(N)] + ([np.zeros(N)] if irr else []) + [[lam]]), (xs.shape[0], 1))
        for a, dim in enumerate(u):
            if dim >= N:
                y[:, dim - N] = xs[:, a]
        vals.append(y)
    h0.hierarchize(torch.from_numpy(np.concatenate(vals)).cuda())
    T = synth.irbc_states(synth.BASE_SEED + w["wid"], w["test_states"], N)
    prec = G.F32C if w["precision"] == "f32c" else G.F64
    # one untimed step first: the first launch of every kernel (libddsg's and the
    # framework's reductions) loads its code; that is not per-step work
    time_iteration(M, h0, 1, w["order"], w["level"], w["eps_gamma"], w["eps_eta"], w["eps_rho"], lo, hi, T,
                   precision=prec, node_mode=G.NODES_DELTA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pol, hist = time_iteration(M, h0, w["ti_steps"], w["order"], w["level"], w["eps_gamma"], w["eps_eta"],
                               w["eps_rho"], lo, hi, T, precision=prec, node_mode=G.NODES_DELTA,
                               tol_change=w.get("tol_change", 0.0))
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    out = {"metric": "adaptive DDSG time-iteration step time (s) and Euler error, %s IRBC N=%d"
                     % ("non-smooth" if irr else "smooth", N),
           "value": total / len(hist), "unit": "s/step", "higher_is_better": False, "n_gpus": 1,
           "data": "synthetic", "dtype": "f64" if prec == G.F64 else "f32",
           "warmup": "one untimed step from the same initial policy",
           "config": {"workload": f"{args.workload}_ddsg_time_iteration", "N": N, "d": d, "m": m,
                      "order": w["order"], "irreversible": irr,
                      "max_level": w["level"], "eps_gamma": w["eps_gamma"], "eps_eta": w["eps_eta"],
                      "eps_rho": w["eps_rho"], "steps": len(hist), "test_states": w["test_states"],
                      "candidates": "all k-subsets", "node_mode": "shortcut"},
           "final": {"steps": len(hist), "points": hist[-1]["points"],
                     "euler_error_log10_mean": float(np.log10(hist[-1]["euler_error_mean"])),
                     "euler_error_log10_max": float(np.log10(hist[-1]["euler_error_max"])),
                     "policy_change_max": hist[-1]["policy_change_max"], "seconds": total},
           "steps": hist if len(hist) <= 10 else hist[:3] + hist[-3:]}
    if args.workload == "ti50":
        # Table 2 of the paper (smooth IRBC, d = 100): context only, other hardware
        out["paper_context"] = {"grid_points": 810, "euler_error_log10_avg_max": [-3.35, -2.21],
                                "hours_per_iteration": 0.5, "nodes": 100,
                                "hardware": "Cray XC50, 12-core CPU nodes, IPOPT per grid point"}
    print(json.dumps(out), flush=True)
    return 0


def run_warmstart(args, w):
    """Time-iteration step at N = 20 with a learned Newton warm start."""
    import torch
    import paper_2202_06555_gb300 as G
    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the warm-start study has no CPU reference arm (GPU-only training)"}))
        return 0
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = measure_warmstart(w)
    print(json.dumps(out), flush=True)
    return 0


def mlp_gemm_flops(sizes, padded, rows):
    """FLOPs of the padded GEMMs one training step (forward, input-gradient and
    weight-gradient GEMMs) and one forward pass run on `rows` batch rows."""
    P = [(v + 63) // 64 * 64 for v in sizes] if padded else list(sizes)
    fwd = sum(2.0 * rows * P[l] * P[l + 1] for l in range(len(P) - 1))
    dgrad = sum(2.0 * rows * P[l] * P[l + 1] for l in range(1, len(P) - 1))
    return fwd, fwd + dgrad + fwd


def measure_warmstart(w):
    """Time-iteration step at N = 20 with a learned Newton warm start: training
    pairs from Newton solves, BF16 tensor-core training, Newton from the
    previous policy vs from the network. Returns the JSON record."""
    import torch
    import paper_2202_06555_gb300 as G
    G.load()
    N, d, m = w["N"], w["d"], w["m"]
    t1, lam, fn, comps, _, _ = irbc_workload(dict(w, states=1), G)
    h = G.HDMR(d, m, 2, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in comps:
        h.add_regular(list(u), w["level"])
    vals = np.concatenate([fn(u, h.component_points(c)[2]) for c, u in enumerate(comps)])
    h.hierarchize(torch.from_numpy(vals).cuda())
    M = G.IRBC(**t1)
    form = G.FORM_SLICEFREE

    def policy_guess(Sd):
        y = torch.empty((Sd.shape[0], m), dtype=torch.float64, device="cuda")
        h.eval(Sd, y, G.F64, form)
        return y

    def solve(Sd, z, prec, tol):
        it = torch.zeros(Sd.shape[0], dtype=torch.int32, device="cuda")
        st = torch.zeros(Sd.shape[0], dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.newton(h, Sd, z, 30, tol, it, st, None, prec, form)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, it, st

    # 1) training pairs: Euler-equation solutions from the previous policy's guesses
    Str = torch.from_numpy(synth.irbc_states(synth.BASE_SEED + w["wid"] + 1, w["train"], N)).cuda()
    ztr = policy_guess(Str)
    t_data, it_tr, st_tr = solve(Str, ztr, G.F32C, 1e-8)
    ok = st_tr == 0
    Str, ztr = Str[ok].contiguous(), ztr[ok].contiguous()
    # 2) train the network (BF16 tensor-core kernels)
    mu = ztr.mean(0).cpu().numpy()
    sd = ztr.std(0).cpu().numpy() + 1e-12
    sizes = [d, 256, 256, 256, m]
    net = G.MLP(sizes, seed=synth.BASE_SEED, in_shift=np.full(d, 1.0), in_scale=np.full(d, 5.0),
                out_shift=mu, out_scale=1.0 / sd)
    ntr, bs = Str.shape[0], w["batch"]
    steps = w["epochs"] * (ntr // bs)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    perm_seed = synth.BASE_SEED + 17
    torch.cuda.synchronize()
    net.profile(True)
    net.profile_read(reset=True)
    t0 = time.perf_counter()
    losses = []
    for s in range(steps):
        ep, k = divmod(s, ntr // bs)
        lr = 1e-3 * 0.5 * (1.0 + math.cos(math.pi * s / steps))   # cosine decay
        net.train_step(Str[k * bs:(k + 1) * bs], ztr[k * bs:(k + 1) * bs], lr, loss)
        if k == 0:
            losses.append(loss)
            loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    tprof = net.profile_read(reset=True)
    net.profile(False)
    # 3) Newton at new states: previous policy vs network guess, same tolerance
    Ste = torch.from_numpy(synth.irbc_states(synth.BASE_SEED + w["wid"] + 2, w["states"], N)).cuda()
    res = {}
    for name in ("previous_policy", "network"):
        if name == "network":
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            z = torch.empty((Ste.shape[0], m), dtype=torch.float64, device="cuda")
            net.infer(Ste, z)
            torch.cuda.synchronize()
            t_guess = time.perf_counter() - t0
        else:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            z = policy_guess(Ste)
            torch.cuda.synchronize()
            t_guess = time.perf_counter() - t0
        g0 = z.clone()
        t_newton, it, st = solve(Ste, z, G.F64, 1e-10)
        r = torch.empty((Ste.shape[0], m), dtype=torch.float64, device="cuda")
        err = torch.empty((Ste.shape[0], 2), dtype=torch.float64, device="cuda")
        M.residual(h, Ste, z, r, None, err, G.F64, form)
        ee = err.cpu().numpy()
        res[name] = {"guess_seconds": t_guess, "newton_seconds": t_newton,
                     "iters_mean": float(it.double().mean().item()), "iters_max": int(it.max().item()),
                     "converged": int((st == 0).sum().item()),
                     "guess_error_max": float((g0 - z).abs().max().item()),
                     "euler_error_log10_mean": float(np.log10(np.mean(ee[:, 0]))),
                     "euler_error_log10_max": float(np.log10(np.max(ee[:, 0])))}
    # per-GEMM throughput: padded GEMM FLOPs of the timed steps over the traced GEMM time
    rows = (bs + 127) // 128 * 128
    f_fwd, f_step = mlp_gemm_flops(sizes, True, rows)
    gemm_ms = tprof.get("gemm_fwd", (0.0, 0))[0] + tprof.get("gemm_bwd", (0.0, 0))[0]
    peaks = measured_peaks()
    bf16_peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1719.5)))
    achieved = steps * f_step / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    out = {"metric": "Newton time at 5e4 states, learned vs previous-policy warm start", "value":
           res["network"]["newton_seconds"] + res["network"]["guess_seconds"], "unit": "s",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "bf16",
           "config": {"workload": "irbc20_warm_start", "N": N, "train_pairs": int(ntr),
                      "mlp": sizes, "epochs": w["epochs"], "batch": bs, "train_steps": steps,
                      "newton_tol": 1e-10},
           "data_generation": {"seconds": t_data, "iters_mean": float(it_tr.double().mean().item())},
           "training": {"seconds": t_train, "samples_per_s": steps * bs / t_train,
                        "loss_first": float(losses[0].item()), "loss_last": float(losses[-1].item()),
                        "kernels_ms": {k: v[0] for k, v in tprof.items()},
                        "launches": sum(v[1] for v in tprof.values())},
           "roofline": {"bound": "tensor", "kernel": "gemm_tc_kernel (tcgen05.mma kind::f16, BF16 in, FP32 accumulate)",
                        "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                        "frac": achieved / bf16_peak if achieved else None, "traffic": None,
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS, of measured)",
                        "flops_per_step": f_step, "gemm_ms_per_step": gemm_ms / max(1, steps),
                        "note": "GEMMs of 4096-row batches over widths <= 256: launch- and latency-bound, "
                                "the traced time includes each launch's event brackets"},
           "newton": res,
           "speedup_newton": res["previous_policy"]["newton_seconds"] / res["network"]["newton_seconds"]}
    h.close()
    M.close()
    net.close()
    return out


def measure_eval_light(w, steps, warmup, uuid, fma):
    """One evaluation workload on the GPU (build, autotune, timed steps with the
    clocks sampled, roofline against the measured FMA peak); returns its record."""
    import torch
    import paper_2202_06555_gb300 as G
    G.load()
    prec = G.F32C if w["precision"] == "f32c" else G.F64
    form = G.FORM_SLICEFREE if w["form"] == "slicefree" else G.FORM_PAPER
    h = G.HDMR(w["d"], w["m"], w["order"])
    fn = value_fn(w)
    for u in comp_list(w):
        h.add_regular(list(u), 2)
    G.build_adaptive(h, fn, w["eps"], w["level"])
    h1 = G.HDMR(w["d"], w["m"], 1)
    for u in full_order_components(w["d"], 1):
        h1.add_regular(list(u), 2)
    G.build_adaptive(h1, fn, w["eps"], w["level"])
    X = make_queries(w)
    n = X.shape[0]
    x = torch.from_numpy(X).cuda()
    y = torch.empty((n, w["m"]), dtype=torch.float64, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    h.eval(x, y, prec, form, None, cnt)
    torch.cuda.synchronize()
    A = float(cnt.double().sum().item())
    h1.eval(x, y, prec, form, None, cnt)
    torch.cuda.synchronize()
    A1 = float(cnt.double().sum().item())
    h1.close()
    flops = (2.0 * w["m"] + 1.0) * A + 2.0 * (A - A1) + (A1 - n)
    ncomp = h.sizes()[0]
    tuned = h.autotune(x[:min(n, 131072)], y[:min(n, 131072)], prec, form)
    for _ in range(warmup):
        h.eval(x, y, prec, form)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    h.profile(True)
    h.profile_read(reset=True)
    with ClockSampler(uuid) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            h.eval(x, y, prec, form)
        e1.record(stream)
        torch.cuda.synchronize()
    prof = h.profile_read(reset=True)
    h.profile(False)
    ms = e0.elapsed_time(e1) / steps
    ev_ms = prof.get("eval", (0.0, 1))[0] / max(1, prof.get("eval", (0.0, 1))[1])
    peak = fma["fp32"] if prec == G.F32C else fma["fp64_fma"]
    achieved = flops / (ev_ms * 1e-3) / 1e12
    h.close()
    return {"metric": metric_for(w), "value": n * w["m"] / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms,
            "steps": steps, "warmup": warmup, "dtype": "f32" if prec == G.F32C else "f64",
            "config": {"workload": "ddsg_d%d" % w["d"], "d": w["d"], "m": w["m"], "queries": n,
                       "components": ncomp, "precision": w["precision"], "form": w["form"],
                       "schedule": {"kernel": KERNEL_NAMES[tuned[0]], "outputs_per_pass": tuned[1]},
                       "active_points_per_query": A / n},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "eval", "kernel_ms": ev_ms,
                         "peak_source": "measured (of measured): ddsg_probe_fma %s chains" %
                                        ("FP32" if prec == G.F32C else "FP64"),
                         "flops_per_launch": flops},
            "kernels_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items()},
            "clocks": clk.summary()}


def run_extra_configs(uuid, fma):
    """The other configurations of the benchmark, each bounded to seconds of GPU
    time: d = 20 FP64 interpolation (4.4e5 monomial-shaped queries), the N = 150
    Euler-residual sweep with Newton solves (node shortcut FP32C vs FP64 at the
    same Euler error, and all nodes in FP32C), and the N = 20 learned warm start."""
    import torch
    out = {}
    t0 = time.perf_counter()
    out["c2_d20_f64"] = measure_eval_light(dict(WORKLOADS["d20"]), 5, 3, uuid, fma)
    out["c2_d20_f64"]["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    rec = measure_irbc(dict(WORKLOADS["irbc150"]), 5, 3,
                       newton_variants=(("f32c_node_shortcut", "F32C", 1e-6, "NODES_DELTA"),
                                        ("f64_tight_node_shortcut", "F64", 1e-10, "NODES_DELTA"),
                                        ("f32c", "F32C", 1e-6, "NODES_ALL")), fma=fma)
    rec["wall_s"] = time.perf_counter() - t0
    out["c4_irbc150"] = rec
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rec = measure_warmstart(dict(WORKLOADS["warmstart20"]))
    rec["wall_s"] = time.perf_counter() - t0
    out["c5_warmstart20"] = rec
    return out


# ---------------------------------------------------------------------------
# CUDA arm
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ddsg", choices=["ddsg", "reference"])
    ap.add_argument("--workload", default="d100", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["f32c", "f64"])
    ap.add_argument("--form", default=None, choices=["slicefree", "paper"])
    ap.add_argument("--queries", type=int, default=None)
    ap.add_argument("--schedule", default=None,
                    help="KERNEL:MC (0 tile, 1 per-tuple, 2 TMA-staged; MC outputs per pass); skips the autotuner")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (d = 20, N = 150 Euler step, N = 20 warm start)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.precision:
        w["precision"] = args.precision
    if args.form:
        w["form"] = args.form
    if args.queries:
        w["Q"] = args.queries
    args.warmup = max(args.warmup, 3) if args.impl == "ddsg" else args.warmup
    if args.workload == "irbc150":
        return run_irbc(args, w)
    if args.workload == "irbc150newton":
        if args.queries:
            w["states"] = args.queries
        return run_irbc_newton(args, w)
    if args.workload == "warmstart20":
        return run_warmstart(args, w)
    if args.workload in ("ti10", "ti6irr", "ti50"):
        return run_time_iteration(args, w)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_2202_06555_gb300 as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (libddsg has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    G.load()
    prec = G.F32C if w["precision"] == "f32c" else G.F64
    form = G.FORM_SLICEFREE if w["form"] == "slicefree" else G.FORM_PAPER

    # -- construction (not timed as a step) ---------------------------------
    t0 = time.perf_counter()
    h = G.HDMR(w["d"], w["m"], w["order"])
    fn = value_fn(w)
    if w["eps"] is None:
        h.add_regular(list(range(w["d"])), w["level"])
        _, _, xs = h.component_points(0)
        h.hierarchize(torch.from_numpy(np.ascontiguousarray(fn(tuple(range(w["d"])), xs))).cuda())
    else:
        for u in comp_list(w):
            h.add_regular(list(u), 2)
        G.build_adaptive(h, fn, w["eps"], w["level"])
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    ncomp, npts = h.sizes()

    X = make_queries(w, rank, world)
    n = X.shape[0]
    x = torch.from_numpy(X).cuda()
    y = torch.empty((n, w["m"]), dtype=torch.float64, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    h.reserve(n)
    stream = torch.cuda.current_stream()

    # algorithmic work of one launch: active points per query (index work is exact)
    h.eval(x, y, prec, form, None, cnt)
    torch.cuda.synchronize()
    active_total = float(cnt.double().sum().item())
    # algorithmic flops: (2m + k + 1) per active point of a k-dimensional component.
    # The order-<=1 part of the expansion (the same 1D grids: refinement is per
    # component) counts the active points of components with k <= 1; the
    # constant component has exactly one per query.
    active_le1 = active_total
    if w["eps"] is not None and w["order"] >= 2:
        h1 = G.HDMR(w["d"], w["m"], 1)
        for u in full_order_components(w["d"], 1):
            h1.add_regular(list(u), 2)
        G.build_adaptive(h1, fn, w["eps"], w["level"])
        h1.eval(x, y, prec, form, None, cnt)
        torch.cuda.synchronize()
        active_le1 = float(cnt.double().sum().item())
        h1.close()
    k_sum = 2.0 * (active_total - active_le1) + (active_le1 - n)
    flops_per_launch = (2.0 * w["m"] + 1.0) * active_total + k_sum

    # batching schedule: autotune kernel / output chunk on a subset of the queries
    nt = min(n, 131072)
    if args.schedule:
        kern, mc = (int(v) for v in args.schedule.split(":"))
        h.set_eval_config(prec, form, kern, mc)
        tuned, nt = (kern, mc), 0
    else:
        tuned = h.autotune(x[:nt], y[:nt], prec, form)
    for _ in range(args.warmup):
        h.eval(x, y, prec, form)
    torch.cuda.synchronize()

    h.profile(True)
    h.profile_read(reset=True)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            h.eval(x, y, prec, form)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    prof = h.profile_read(reset=True)
    h.profile(False)
    ms_total = e0.elapsed_time(e1)
    if dist is not None:
        tt = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_total = float(tt.item())
    ms_step = ms_total / args.steps
    value = world * n * w["m"] / (ms_step * 1e-3)
    launches = sum(v[1] for v in prof.values())
    eval_ms, eval_n = prof.get("eval", (0.0, 0))
    eval_avg_ms = eval_ms / max(1, eval_n)

    # -- roofline of the dominant kernel (interpolation) ----------------------
    # peak: the FMA rate measured on this device by the library's probe
    # (ddsg_probe_fma), beside the nominal figure from the SM count and clock
    n_sm, sm_mhz = device_facts(local)
    fma = measure_fma_peaks(G, uuid)
    nominal_fp32 = n_sm * FP32_LANES_PER_SM * 2 * (sm_mhz or 0.0) * 1e6 / 1e12
    if prec == G.F32C:
        peak = fma["fp32"]
        peak_src = ("measured (of measured): ddsg_probe_fma FP32 chains, %.1f TFLOP/s; nominal %d SMs x %d lanes "
                    "x 2 flop x %.0f MHz = %.1f" % (peak, n_sm, FP32_LANES_PER_SM, sm_mhz or 0.0, nominal_fp32))
    else:
        peak = fma["fp64_fma"]
        peak_src = "measured (of measured): ddsg_probe_fma FP64 chains, %.2f TFLOP/s" % peak
    achieved = flops_per_launch / (eval_avg_ms * 1e-3) / 1e12
    hbm_bytes = n * w["d"] * 8 + n * w["m"] * 8 + npts * w["m"] * (4 if prec == G.F32C else 8)
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_frac = hbm_bytes / (ms_step * 1e-3) / 1e9 / hbm_peak

    # -- register-delivery floor of the gather (F32C on the staged kernels): the
    # L1 returns one 128-byte wavefront per clock per SM. Level-tuple kernels:
    # every level tuple a warp of 32 queries visits moves one padded surplus row
    # per lane (mp floats = mp wavefronts). Nodal-slab kernel: every node row
    # moves rs floats per lane (rs = m rounded up to 32: rs wavefronts), at the
    # node rows per query of its tables.
    l1 = None
    if prec == G.F32C:
        wclk = n_sm * (sm_mhz or 2070.0) * 1e6
        if tuned[0] in (5, 6):
            _, nrows, rows_q = h.nodal_info(form)
            rs = (w["m"] + 31) // 32 * 32 if w["m"] > 16 else (w["m"] + 3) // 4 * 4
            floor_ms = (n / 32.0) * rows_q * rs / wclk * 1e3
            l1 = {"bound": "shared-memory delivery to registers (128 B per clock per SM)",
                  "floor_ms": floor_ms, "kernel_ms": eval_avg_ms, "frac": floor_ms / eval_avg_ms,
                  "node_rows_per_query": rows_q, "node_rows_stored": nrows,
                  "wavefronts_per_32_query_rows": rs,
                  "note": "nodal-slab kernel: each query reads two node rows per slab level; "
                          "lane-rotated 16-byte chunks make every warp load conflict-free"}
        else:
            tuples = 0
            for c in range(ncomp):
                dims, _, _ = h.component_info(c)
                if len(dims) == 0:
                    tuples += 1   # the constant component's single point
                    continue
                lv, _, _ = h.component_points(c)
                inner = lv[np.all(lv >= 2, axis=1)] if w["form"] == "slicefree" else lv
                tuples += len({tuple(r) for r in inner.tolist()})
            mp = (w["m"] + 3) // 4 * 4
            floor_ms = (n / 32.0) * tuples * mp / wclk * 1e3
            l1 = {"bound": "shared-memory delivery to registers (128 B per clock per SM)",
                  "floor_ms": floor_ms, "kernel_ms": eval_avg_ms, "frac": floor_ms / eval_avg_ms,
                  "tuples_per_query": tuples, "wavefronts_per_32_query_tuples": mp,
                  "note": "lower bound for a level-tuple kernel that gives each query thread its own copy of each hit row"}

    # -- end to end: host buffers through the C ABI ---------------------------
    xh = torch.from_numpy(X).pin_memory()
    yh = torch.empty((n, w["m"]), dtype=torch.float64).pin_memory()
    xnp, ynp = xh.numpy(), yh.numpy()
    h.eval_host(xnp, ynp, prec, form)
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        h.eval_host(xnp, ynp, prec, form)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_times)
    if dist is not None:
        tt = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())

    out = {"metric": metric_for(w), "value": value, "unit": "evals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if prec == G.F32C else "f64", "data": "synthetic",
           "config": {"workload": f"ddsg_{args.workload}", "d": w["d"], "m": w["m"],
                      "order": w["order"], "components": ncomp, "grid_points": npts,
                      "eps_gamma": w["eps"], "max_level": w["level"], "queries_per_gpu": n,
                      "precision": w["precision"], "form": w["form"],
                      "active_points_per_query": active_total / n,
                      "schedule": {"kernel": KERNEL_NAMES[tuned[0]], "outputs_per_pass": tuned[1],
                                   "autotune_subset": nt},
                      "l2": "inputs larger than L2 (x %.2f GB, surpluses %.2f GB); no flush"
                            % (n * w["d"] * 8 / 1e9, npts * w["m"] * (4 if prec == G.F32C else 8) / 1e9),
                      "build_s": t_build},
           "gpu_launches": launches,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": eval_traffic(args.workload, tuned[:2], n),
                        "peak_source": peak_src,
                        "kernel": "eval", "kernel_ms": eval_avg_ms,
                        "flops_per_launch": flops_per_launch,
                        "flop_count": "sum over queries and active points of (2m + k + 1), k the component's order",
                        "active_points": active_total, "active_points_order_le1": active_le1},
           "fma_peaks": fma,
           "device": {"sms": n_sm, "sm_max_mhz": sm_mhz},
           "hbm_roofline": {"bytes_per_step": hbm_bytes, "frac": hbm_frac, "peak_gbs": hbm_peak,
                            "note": "compulsory bytes / step time / measured copy bandwidth"},
           "l1_roofline": l1,
           "kernels_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items()},
           "clocks": clk.summary(),
           "e2e": {"value": world * n * w["m"] / e2e_s, "unit": "evals/s",
                   "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(n * w["m"] * 8),
                   "ms_per_step": e2e_s * 1e3}}

    # -- the same step replayed from a CUDA graph (launch overhead removed) -------
    h.eval_graph(x, y, prec, form)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        h.eval_graph(x, y, prec, form)
    g1.record(stream)
    torch.cuda.synchronize()
    g_ms = g0.elapsed_time(g1) / args.steps
    out["graph_replay"] = {"ms_per_step": g_ms, "value": world * n * w["m"] / (g_ms * 1e-3),
                           "unit": "evals/s", "note": "hdmr_eval_graph: encode + fused eval captured once"}

    # -- precision: FP32-compensated vs the plain FP64 GPU form -----------------
    if rank == 0 and not args.no_fp64 and prec == G.F32C:
        ns = min(n, 500_000)
        y64 = torch.empty((ns, w["m"]), dtype=torch.float64, device="cuda")
        y32 = torch.empty((ns, w["m"]), dtype=torch.float64, device="cuda")
        h.eval(x[:ns], y32, G.F32C, form)
        h.eval(x[:ns], y64, G.F64, form)   # warm
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.eval(x[:ns], y64, G.F64, form)
        b.record(stream)
        torch.cuda.synchronize()
        rel = ((y32 - y64).abs() / y64.abs().clamp_min(1e-300))
        out["fp64_gpu"] = {"value": ns * w["m"] / (a.elapsed_time(b) * 1e-3), "unit": "evals/s",
                           "queries": ns}
        out["f32c_vs_f64_gpu"] = {"max_rel": float(rel.max().item()),
                                  "rms_rel": float(rel.pow(2).mean().sqrt().item()),
                                  "per_output_max_rel_max": float(rel.max(0).values.max().item()),
                                  "queries": ns}

    # -- CPU baseline: the oracle on a bounded sample (rank 0, N=1 only) --------
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        E = oracle_build(w)
        rate, used = oracle_rate(E, w, X, 10.0)
        threads = max(1, os.cpu_count() or 1)
        n_par = min(X.shape[0], used * threads)
        rate_par = oracle_rate_threads(E, w, X, n_par, threads) if threads > 1 else rate
        # precision against the FP64 oracle on the sample (scale max(|y|, S))
        r = E.eval(X[:min(used, 400)], form=1 if w["form"] == "slicefree" else 0, want=("y", "S"))
        ys = y[:min(used, 400)].cpu().numpy()   # y holds the last timed step's result
        scale = np.maximum(np.abs(r["y"]), r["S"])
        relo = np.abs(ys - r["y"]) / scale
        out["error_vs_oracle"] = {"queries": int(relo.shape[0]), "max_rel": float(relo.max()),
                                  "rms_rel": float(np.sqrt(np.mean(relo ** 2))),
                                  "per_output_max": [float(v) for v in relo.max(0)],
                                  "scale": "max(|y|, sum of |terms|)"}
        out["cpu_baseline"] = {"value": rate_par, "unit": "evals/s", "cores": threads, "kind": "oracle",
                               "cpu": cpu_model(),
                               "sample": f"first {n_par} of the {n} queries over {threads} host threads "
                                         f"(~10 s of CPU work)",
                               "single_thread": {"value": rate, "sample": f"first {used} queries, "
                                                                          f"~10 s"}}
    # -- the other configurations, each bounded (rank 0, N = 1, default workload) --
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "d100":
        h.close()
        h = None
        t0 = time.perf_counter()
        out["configs"] = run_extra_configs(uuid, fma)
        out["configs"]["wall_s"] = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps(out), flush=True)
    if h is not None:
        h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
