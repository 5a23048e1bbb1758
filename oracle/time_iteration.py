"""Adaptive DDSG time iteration (Alg. 1 around Alg. 2) -- TEST INFRASTRUCTURE ONLY.

Plain restatement with the oracle's own pieces: every component grid is built
on its own (its values are the cut values f(xbar \\ x_u), independent of the
other components), the map being approximated is x -> solve{FOC(. | x, p)}
with the oracle's FP64 Newton (forward-difference Jacobian), and the
expansion criterion (eq. 3.18) and active dimension selection (eq. 3.19) use
the component quadratures of eq. 3.7. It shares no code with the CUDA
library's driver.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import OracleDDSG


def _subsets(u):
    for r in range(len(u) + 1):
        for v in itertools.combinations(u, r):
            yield v


def oracle_solver(I, prev: OracleDDSG, form=1, tol=1e-10, max_it=30):
    """states -> Newton solutions of the Euler equations given policy prev,
    started from prev (memoised per state: the refinement sweeps ask again)."""
    memo = {}

    def solve(states):
        states = np.atleast_2d(np.asarray(states, np.float64))
        out = np.zeros((states.shape[0], prev.m))
        todo = [s for s in range(states.shape[0]) if states[s].tobytes() not in memo]
        if todo:
            X = states[todo]
            guess = prev.eval(X, form=form)["y"]
            sol, _, _ = I.newton(prev, X, guess, form=form, tol=tol, max_it=max_it)
            for t, s in enumerate(todo):
                memo[states[s].tobytes()] = sol[t]
        for s in range(states.shape[0]):
            out[s] = memo[states[s].tobytes()]
        return out

    return solve


def oracle_build_ddsg(solve, d, m, order, level, eps_gamma, eps_eta, eps_rho, lo, hi, candidates=None,
                      strict=False):
    """Alg. 2 over `solve`; returns (OracleDDSG of the accepted components, info)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    anchor = 0.5 * (lo + hi)

    def cut_fn(dims, X):
        S = np.tile(anchor, (X.shape[0], 1))
        if len(dims):
            S[:, list(dims)] = X
        return solve(S)

    built = {}   # u -> (levels, indices, values, Q_u of the component interpolant)

    def build(u):
        E1 = OracleDDSG(d, m, lo=lo, hi=hi)
        E1.add_regular(u, 2)
        E1.build_adaptive(cut_fn, eps_gamma, level, strict)
        built[u] = (E1.lv[0], E1.ix[0], E1.values[0], E1.quadrature()[0])

    def Qf(u):   # integral of the cut-HDMR component function f_u
        acc = np.zeros(m)
        for v in _subsets(u):
            acc += (-1.0) ** (len(u) - len(v)) * built[v][3]
        return acc

    build(())
    accepted = [()]
    rejected = []
    info = {"rho": [], "eta": {}, "rejected": []}
    for k in range(1, order + 1):
        pool = candidates(k) if candidates else itertools.combinations(range(d), k)
        cand = [tuple(u) for u in pool if not any(set(z) <= set(u) for z in rejected)]
        if not cand:
            break
        for u in cand:
            build(u)
        lower = np.zeros(m)
        for u in accepted:
            if len(u) <= k - 1:
                lower += Qf(u)
        keep = []
        for u in cand:
            if k >= 2:
                eta = float(np.linalg.norm(Qf(u)) / np.linalg.norm(lower))
                info["eta"][u] = eta
                if not eta > eps_eta:
                    rejected.append(u)
                    info["rejected"].append(u)
                    continue
            keep.append(u)
        accepted += keep
        top = np.zeros(m)
        for u in keep:
            top += Qf(u)
        rho = float(np.linalg.norm(top) / np.linalg.norm(lower))
        info["rho"].append(rho)
        if rho < eps_rho:
            break
    E = OracleDDSG(d, m, lo=lo, hi=hi)
    for u in accepted:
        c = E.add_component(u, built[u][0], built[u][1])
        E.set_values(c, built[u][2])
    E.hierarchize()
    info["components"] = accepted
    return E, info


def oracle_time_iteration(I, policy0: OracleDDSG, steps, order, level, eps_gamma, eps_eta, eps_rho, lo, hi,
                          test_states, candidates=None, tol=1e-10):
    """Alg. 1 with a fixed number of steps; per step the Euler errors of the new
    policy at test_states (the policy gives today's choice and next period's)."""
    p = policy0
    history = []
    for step in range(steps):
        new, info = oracle_build_ddsg(oracle_solver(I, p, tol=tol), p.d, p.m, order, level, eps_gamma,
                                      eps_eta, eps_rho, lo, hi, candidates)
        g = new.eval(test_states, form=1)["y"]
        _, e = I.residual(new, test_states, g, form=1, want_err=True)
        history.append({"step": step, "info": info, "euler_error_mean": float(np.mean(np.max(e, 1))),
                        "euler_error_max": float(np.max(e)), "policy": new, "previous": p})
        p = new
    return p, history
