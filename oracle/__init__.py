"""CPU oracle for the DDSG interpolant -- TEST INFRASTRUCTURE ONLY.

Plain FP64 restatement of arXiv 2202.06555 (Sec. 3.1-3.3, 4.1) used to check
the CUDA library. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm may import this package. It shares no code with the
CUDA library (paper_2202_06555_gb300) and never imports it.

The heavy loops live in ddsg_oracle.c (and irbc_oracle.c), compiled here with
gcc -O2 -ffp-contract=off into _build/liboracle.so on first use.
"""
from __future__ import annotations

import ctypes as C
import itertools
import os
import subprocess
import threading

import numpy as np

KMAX = 8
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["ddsg_oracle.c", "irbc_oracle.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, gcc)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-pthread", "-o", tmp] + srcs + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_d = C.c_double


def _declare(L):
    L.orc_phi1d.restype = _d
    L.orc_phi1d.argtypes = [C.c_int, C.c_uint32, _d]
    L.orc_active1d.restype = C.c_int
    L.orc_active1d.argtypes = [C.c_int, C.c_uint32, _d]
    L.orc_node1d.restype = _d
    L.orc_node1d.argtypes = [C.c_int, C.c_uint32]
    L.orc_int1d.restype = _d
    L.orc_int1d.argtypes = [C.c_int, C.c_uint32]
    L.orc_regular_grid.restype = _i64
    L.orc_regular_grid.argtypes = [C.c_int, C.c_int, _p, _p]
    L.orc_point_key.restype = C.c_uint64
    L.orc_point_key.argtypes = [_i32, C.c_int, _p, _p]
    L.orc_b_coeffs.restype = None
    L.orc_b_coeffs.argtypes = [C.c_int, _p, _p, _p]
    L.orc_eval.restype = None
    L.orc_eval.argtypes = [C.c_int, C.c_int, C.c_int, _p, _p, _p, _p, _p, _p, _p, _p, _p,
                           C.c_int, _i64, _p, _p, _p, _p, _p]
    L.orc_eval_telescopic.restype = C.c_int
    L.orc_eval_telescopic.argtypes = [C.c_int, C.c_int, C.c_int, _p, _p, _p, _p, _p, _p,
                                      _p, _p, _i64, _p, _p]
    L.orc_hierarchize.restype = None
    L.orc_hierarchize.argtypes = [C.c_int, C.c_int, _p, _p, _p, _p, _p, _p]
    L.orc_nodes.restype = None
    L.orc_nodes.argtypes = [C.c_int, _i64, _i64, _p, _p, _p]
    L.orc_refine.restype = _i64
    L.orc_refine.argtypes = [C.c_int, C.c_int, _i64, _i64, _p, _p, _p, _d, C.c_int, C.c_int,
                             _i64, _p, _p]
    L.orc_active_pruned.restype = C.c_int
    L.orc_active_pruned.argtypes = [C.c_int, C.c_int, _p, _p, _p, _p, _p, _p, _p, _p, C.c_int, _i64,
                                    _p, _p, _p, C.c_int]
    L.orc_quadrature.restype = None
    L.orc_quadrature.argtypes = [C.c_int, C.c_int, _p, _p, _p, _p, _p, _p]
    if hasattr(L, "orc_irbc_residual"):
        _declare_irbc(L)


def _declare_irbc(L):
    L.orc_irbc_params.restype = None
    L.orc_irbc_params.argtypes = [C.c_int, _d, _d, _d, _d, _p, _p, _p]
    L.orc_monomial_nodes.restype = None
    L.orc_monomial_nodes.argtypes = [C.c_int, _p, _p]
    L.orc_irbc_residual.restype = None
    L.orc_irbc_residual.argtypes = [C.c_int, _p, _p, _p, C.c_int, _p, _p, _p, _p, _p, _p, _p, _p,
                                    _p, C.c_int, _i64, _p, _p, _p, _p]
    L.orc_irbc_residual_irr.restype = None
    L.orc_irbc_residual_irr.argtypes = L.orc_irbc_residual.argtypes
    L.orc_lu_solve.restype = C.c_int
    L.orc_lu_solve.argtypes = [C.c_int, _p, _p]


def ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# 1D helpers (thin wrappers, for pins)
# ---------------------------------------------------------------------------

def phi1d(l, i, x):
    return lib().orc_phi1d(int(l), int(i), float(x))


def active1d(l, i, x):
    return bool(lib().orc_active1d(int(l), int(i), float(x)))


def node1d(l, i):
    return lib().orc_node1d(int(l), int(i))


def int1d(l, i):
    return lib().orc_int1d(int(l), int(i))


def regular_grid(k: int, level: int):
    """(levels, indices) of the regular level-`level` grid on k dims,
    arrays of shape (npts, KMAX) in canonical order."""
    n = lib().orc_regular_grid(k, level, None, None)
    if n < 0:
        raise ValueError("grid too large for the oracle enumerator")
    lv = np.zeros((n, KMAX), np.uint8)
    ix = np.zeros((n, KMAX), np.uint32)
    lib().orc_regular_grid(k, level, ptr(lv), ptr(ix))
    return lv, ix


def full_order_components(d: int, order: int):
    """All subsets of {0..d-1} of size <= order, by size then lexicographic."""
    out = []
    for k in range(order + 1):
        out.extend(itertools.combinations(range(d), k))
    return out


# ---------------------------------------------------------------------------
# An HDMR expansion held as flat tables
# ---------------------------------------------------------------------------

class OracleDDSG:
    """Cut-HDMR expansion with one sparse grid per accepted component u.

    Component u's grid interpolates the cut function f(xbar \\ x_u) (eq. ddsg2.2.6,
    eq. 4.2's a_u). Anchor xbar is given in physical units; lo/hi map the
    physical domain to [0,1]^d.
    """

    def __init__(self, d: int, m: int, lo=None, hi=None, anchor=None):
        self.d, self.m = d, m
        self.lo = np.zeros(d) if lo is None else np.asarray(lo, np.float64).copy()
        self.hi = np.ones(d) if hi is None else np.asarray(hi, np.float64).copy()
        self.anchor = (0.5 * (self.lo + self.hi) if anchor is None
                       else np.asarray(anchor, np.float64).copy())
        self.comps = []        # list of dims tuples
        self.lv = []           # per component (npts, KMAX) uint8
        self.ix = []           # per component (npts, KMAX) uint32
        self.alpha = []        # per component (npts, m) float64 or None
        self.values = []       # per component (npts, m) float64 or None

    # -- construction ------------------------------------------------------
    def add_component(self, dims, levels, indices):
        dims = tuple(int(x) for x in dims)
        assert list(dims) == sorted(set(dims))
        self.comps.append(dims)
        self.lv.append(np.ascontiguousarray(levels, np.uint8).reshape(-1, KMAX))
        self.ix.append(np.ascontiguousarray(indices, np.uint32).reshape(-1, KMAX))
        self.alpha.append(None)
        self.values.append(None)
        return len(self.comps) - 1

    def add_regular(self, dims, level):
        lv, ix = regular_grid(len(dims), level)
        return self.add_component(dims, lv, ix)

    def npts(self, c):
        return self.lv[c].shape[0]

    def node_coords(self, c, first=0):
        """Canonical node coordinates of points first.. of component c: (n, k)."""
        k = len(self.comps[c])
        n = self.npts(c) - first
        out = np.zeros((n, max(k, 1)))
        if k:
            lib().orc_nodes(k, first, self.npts(c), ptr(self.lv[c]), ptr(self.ix[c]), ptr(out))
        return out[:, :k]

    def node_coords_phys(self, c, first=0):
        dims = list(self.comps[c])
        xc = self.node_coords(c, first)
        return self.lo[dims] + xc * (self.hi[dims] - self.lo[dims])

    def set_values(self, c, values):
        self.values[c] = np.ascontiguousarray(values, np.float64).reshape(self.npts(c), self.m)

    def fill_values(self, fn, first_only_new=False):
        """fn(dims, phys_coords (n,k)) -> (n, m) cut values. Fills every component."""
        for c, dims in enumerate(self.comps):
            self.set_values(c, fn(dims, self.node_coords_phys(c)))

    def hierarchize(self):
        t = self.tables()
        vals = np.ascontiguousarray(np.concatenate(self.values, axis=0))
        alpha = np.zeros_like(vals)
        lib().orc_hierarchize(self.m, len(self.comps), ptr(t["k"]), ptr(t["off"]),
                              ptr(t["lv"]), ptr(t["ix"]), ptr(vals), ptr(alpha))
        off = t["off"]
        for c in range(len(self.comps)):
            self.alpha[c] = alpha[off[c]:off[c + 1]].copy()
        self._tables = None

    def refine_component(self, c, eps, level, strict=False):
        k = len(self.comps[c])
        P = self.npts(c)
        cap = max(64, 2 * k * P + 16)
        nlv = np.zeros((cap, KMAX), np.uint8)
        nix = np.zeros((cap, KMAX), np.uint32)
        n = lib().orc_refine(self.m, k, 0, P, ptr(self.lv[c]), ptr(self.ix[c]),
                             ptr(self.alpha[c]), float(eps), int(level), int(bool(strict)),
                             cap, ptr(nlv), ptr(nix))
        assert n >= 0
        if n:
            self.lv[c] = np.concatenate([self.lv[c], nlv[:n]])
            self.ix[c] = np.concatenate([self.ix[c], nix[:n]])
            self.alpha[c] = None
        self._tables = None
        return int(n)

    def build_adaptive(self, fn, eps, level, strict=False, max_sweeps=64):
        """Regular level-2 start, then refine/hierarchize sweeps (eq. 3.8) until
        no point is added. fn(dims, phys_coords) -> cut values."""
        for _ in range(max_sweeps):
            self.fill_values(fn)
            self.hierarchize()
            added = sum(self.refine_component(c, eps, level, strict)
                        for c in range(len(self.comps)))
            if added == 0:
                break
        return self

    # -- flat tables -------------------------------------------------------
    _tables = None

    def tables(self):
        if self._tables is not None:
            return self._tables
        C_ = len(self.comps)
        k = np.array([len(u) for u in self.comps], np.int32)
        dims = np.zeros((C_, KMAX), np.int32)
        for c, u in enumerate(self.comps):
            dims[c, :len(u)] = u
        off = np.zeros(C_ + 1, np.int64)
        off[1:] = np.cumsum([self.npts(c) for c in range(C_)])
        lv = np.ascontiguousarray(np.concatenate(self.lv, axis=0))
        ix = np.ascontiguousarray(np.concatenate(self.ix, axis=0))
        t = dict(k=k, dims=dims, off=off, lv=lv, ix=ix)
        if all(a is not None for a in self.alpha):
            t["alpha"] = np.ascontiguousarray(np.concatenate(self.alpha, axis=0))
        self._tables = t
        return t

    def b_coeffs(self):
        t = self.tables()
        b = np.zeros(len(self.comps))
        lib().orc_b_coeffs(len(self.comps), ptr(t["k"]), ptr(t["dims"]), ptr(b))
        return b

    # -- evaluation ----------------------------------------------------------
    def eval(self, x, form=0, want=("y",)):
        """form 0: paper form sum_v b_v s_v (eq. 4.2); form 1: slice-free form.
        Returns dict with any of y (n,m), S (n,m), hash (n,), count (n,)."""
        t = self.tables()
        x = np.ascontiguousarray(x, np.float64).reshape(-1, self.d)
        n = x.shape[0]
        b = self.b_coeffs()
        out = {}
        y = np.zeros((n, self.m)) if "y" in want else None
        S = np.zeros((n, self.m)) if "S" in want else None
        h = np.zeros(n, np.uint64) if "hash" in want else None
        cnt = np.zeros(n, np.int32) if "count" in want else None
        lib().orc_eval(self.d, self.m, len(self.comps), ptr(t["k"]), ptr(t["dims"]),
                       ptr(t["off"]), ptr(t["lv"]), ptr(t["ix"]), ptr(t["alpha"]), ptr(b),
                       ptr(self.lo), ptr(self.hi), int(form), n, ptr(x), ptr(y), ptr(S),
                       ptr(h), ptr(cnt))
        for name, arr in (("y", y), ("S", S), ("hash", h), ("count", cnt)):
            if arr is not None:
                out[name] = arr
        return out

    def active_pruned(self, x, form=0, threads=1):
        """Active-set hashes and counts (as eval's hash / count) by tree descent from
        each component's root (a child is visited only from an active parent);
        `threads` host threads over the queries. Returns (hash, count)."""
        t = self.tables()
        x = np.ascontiguousarray(x, np.float64).reshape(-1, self.d)
        n = x.shape[0]
        b = self.b_coeffs()
        h = np.zeros(n, np.uint64)
        cnt = np.zeros(n, np.int32)
        rc = lib().orc_active_pruned(self.d, len(self.comps), ptr(t["k"]), ptr(t["dims"]), ptr(t["off"]),
                                     ptr(t["lv"]), ptr(t["ix"]), ptr(b), ptr(self.lo), ptr(self.hi),
                                     int(form), n, ptr(x), ptr(h), ptr(cnt), int(threads))
        if rc != 0:
            raise ValueError("a component has no root point (1, ..., 1)")
        return h, cnt

    def eval_telescopic(self, x):
        t = self.tables()
        x = np.ascontiguousarray(x, np.float64).reshape(-1, self.d)
        y = np.zeros((x.shape[0], self.m))
        rc = lib().orc_eval_telescopic(self.d, self.m, len(self.comps), ptr(t["k"]),
                                       ptr(t["dims"]), ptr(t["off"]), ptr(t["lv"]),
                                       ptr(t["ix"]), ptr(t["alpha"]), ptr(self.lo),
                                       ptr(self.hi), x.shape[0], ptr(x), ptr(y))
        if rc != 0:
            raise ValueError("expansion is not downward closed")
        return y

    def quadrature(self):
        """Q_l of every component interpolant (eq. 3.7): (C, m)."""
        t = self.tables()
        Q = np.zeros((len(self.comps), self.m))
        lib().orc_quadrature(self.m, len(self.comps), ptr(t["k"]), ptr(t["off"]),
                             ptr(t["lv"]), ptr(t["ix"]), ptr(t["alpha"]), ptr(Q))
        return Q

    def cut_component_quadratures(self):
        """Q f_u of the cut-HDMR component functions (eq. ddsg2.2.6 applied to
        the interpolants): sum over v subset u of (-1)^{|u|-|v|} Q I f(xbar\\x_v)."""
        Q = self.quadrature()
        index = {u: c for c, u in enumerate(self.comps)}
        out = np.zeros_like(Q)
        for c, u in enumerate(self.comps):
            for r in range(len(u) + 1):
                for v in itertools.combinations(u, r):
                    out[c] += (-1.0) ** (len(u) - r) * Q[index[v]]
        return out

    def expansion_rho(self, k):
        """eq. 3.18: ||sum_{|u|=k} Q f_u||_2 / ||sum_{|u|<=k-1} Q f_u||_2."""
        Qf = self.cut_component_quadratures()
        num = np.zeros(self.m)
        den = np.zeros(self.m)
        for c, u in enumerate(self.comps):
            if len(u) == k:
                num += Qf[c]
            elif len(u) <= k - 1:
                den += Qf[c]
        return float(np.linalg.norm(num) / np.linalg.norm(den))

    def active_eta(self, u):
        """eq. 3.19: ||Q f_u||_2 / ||sum_{|v|<=|u|-1} Q f_v||_2."""
        Qf = self.cut_component_quadratures()
        index = {w: c for c, w in enumerate(self.comps)}
        den = np.zeros(self.m)
        for c, v in enumerate(self.comps):
            if len(v) <= len(u) - 1:
                den += Qf[c]
        return float(np.linalg.norm(Qf[index[tuple(u)]]) / np.linalg.norm(den))

    def point_key(self, c, p):
        k = len(self.comps[c])
        return int(lib().orc_point_key(c, k, ptr(self.lv[c][p]), ptr(self.ix[c][p])))


def sg_point_count(d: int, level: int) -> int:
    """Exact number of points of the regular level-`level` grid on d dims
    (eq. 3.5 constraint sum(l_j - 1) <= level - 1, 1D level sizes 1, 2, 2, 4, 8, ...),
    by expanding prod_j (sum_e n(e+1) z^e) up to z^(level-1) with Python integers."""
    L = level - 1
    per = [1, 2] + [2 ** (e - 1) for e in range(2, L + 1)]
    per = per[:L + 1]
    poly = [1] + [0] * L
    for _ in range(d):
        new = [0] * (L + 1)
        for a, ca in enumerate(poly):
            if ca:
                for e, ne in enumerate(per):
                    if a + e > L:
                        break
                    new[a + e] += ca * ne
        poly = new
    return sum(poly)


# ---------------------------------------------------------------------------
# IRBC model (Sec. 2.1): parameters, monomial rule, residuals, Newton
# ---------------------------------------------------------------------------

IRBC_TABLE1 = dict(beta=0.99, alpha=0.36, delta=0.01, sigma=0.01, rho=0.95, phi=0.5)
IRBC_A_GAMMA = 0.25     # the undefined "a" of Table 1's gamma_j (reading)


class IRBCOracle:
    """IRBC equilibrium conditions at given states, with the policy interpolated
    from an OracleDDSG over x = (a, k). Smooth model (eq. model1, model2; policy
    (k', lambda), m = N+1) or, with irreversible=True, the non-smooth model
    (eq. modelkink1 with the complementarity as a Fischer-Burmeister equation,
    and eq. model2; policy (k', mu, lambda), m = 2N+1)."""

    def __init__(self, N: int, lo=0.8, hi=1.2, irreversible=False, **overrides):
        self.N = N
        self.irreversible = bool(irreversible)
        self.m = 2 * N + 1 if irreversible else N + 1
        p = dict(IRBC_TABLE1)
        p.update(overrides)
        self.p = p
        A = C.c_double()
        self.gamma = np.zeros(N)
        self.tau = np.zeros(N)
        lib().orc_irbc_params(N, IRBC_A_GAMMA, p["beta"], p["alpha"], p["delta"], C.byref(A),
                              ptr(self.gamma), ptr(self.tau))
        self.A = A.value
        self.prm = np.array([p["beta"], p["alpha"], p["delta"], p["sigma"], p["rho"], p["phi"],
                             self.A, 0.0])
        self.lo, self.hi = lo, hi

    def steady_lambda(self):
        """lambda* with sum_j (lambda/tau_j)^(-gamma_j) = N (A - delta), by bisection
        (the deterministic steady state k = k' = 1, a = 1 of eq. model2)."""
        target = self.N * (self.A - self.p["delta"])
        f = lambda lam: np.sum((lam / self.tau) ** (-self.gamma)) - target
        lo, hi = 1e-8, 1e8
        for _ in range(400):
            mid = np.sqrt(lo * hi)
            if f(mid) > 0:
                lo = mid
            else:
                hi = mid
        return np.sqrt(lo * hi)

    def monomial(self, n=None):
        n = self.N + 1 if n is None else n
        nodes = np.zeros((2 * n, n))
        w = np.zeros(2 * n)
        lib().orc_monomial_nodes(n, ptr(nodes), ptr(w))
        return nodes, w

    def residual(self, E: OracleDDSG, states, guess, form=1, want_err=False):
        t = E.tables()
        states = np.ascontiguousarray(states, np.float64).reshape(-1, 2 * self.N)
        guess = np.ascontiguousarray(guess, np.float64).reshape(-1, self.m)
        ns = states.shape[0]
        r = np.zeros((ns, self.m))
        ee = np.zeros((ns, 2)) if want_err else None
        b = E.b_coeffs()
        fn = lib().orc_irbc_residual_irr if self.irreversible else lib().orc_irbc_residual
        fn(self.N, ptr(self.prm), ptr(self.gamma), ptr(self.tau),
                                len(E.comps), ptr(t["k"]), ptr(t["dims"]), ptr(t["off"]),
                                ptr(t["lv"]), ptr(t["ix"]), ptr(t["alpha"]), ptr(b), ptr(E.lo),
                                ptr(E.hi), int(form), ns, ptr(states), ptr(guess), ptr(r), ptr(ee))
        return (r, ee) if want_err else r

    def newton(self, E, states, guess, form=1, tol=1e-10, max_it=30, fd=1e-7):
        """Per-state FP64 Newton: forward-difference Jacobian, dense LU with
        partial pivoting, backtracking on ||r||_2. Returns (solution, iterations,
        final residual norms)."""
        states = np.atleast_2d(states)
        sol = np.array(np.atleast_2d(guess), dtype=np.float64)
        its = np.zeros(states.shape[0], np.int32)
        norms = np.zeros(states.shape[0])
        n = self.m
        for s in range(states.shape[0]):
            z = sol[s].copy()
            r = self.residual(E, states[s:s + 1], z[None], form)[0]
            for it in range(max_it):
                if np.max(np.abs(r)) <= tol:
                    break
                J = np.zeros((n, n))
                for j in range(n):
                    h = fd * max(1.0, abs(z[j]))
                    zp = z.copy()
                    zp[j] += h
                    J[:, j] = (self.residual(E, states[s:s + 1], zp[None], form)[0] - r) / h
                dz = -r.copy()
                Jc = np.ascontiguousarray(J)
                if lib().orc_lu_solve(n, ptr(Jc), ptr(dz)) != 0:
                    break
                step = 1.0
                nr = np.linalg.norm(r)
                while step > 1e-4:
                    zt = z + step * dz
                    rt = self.residual(E, states[s:s + 1], zt[None], form)[0]
                    if np.linalg.norm(rt) < nr:
                        break
                    step *= 0.5
                z, r = zt, rt
                its[s] = it + 1
            sol[s] = z
            norms[s] = np.max(np.abs(r))
        return sol, its, norms


def irbc_policy_ddsg(N: int, level: int, value_fn, lo=0.8, hi=1.2, pairs=True):
    """Policy expansion over x = (a_1..a_N, k_1..k_N): the empty component, all
    2N single dimensions and (optionally) the N pairs (a_j, k_j), each a regular
    level-`level` grid, hierarchized from value_fn(dims, phys_coords)."""
    d = 2 * N
    E = OracleDDSG(d, N + 1, lo=np.full(d, lo), hi=np.full(d, hi))
    comps = [()] + [(i,) for i in range(d)]
    if pairs:
        comps += [(j, N + j) for j in range(N)]
    for u in comps:
        E.add_regular(u, level)
    E.fill_values(value_fn)
    E.hierarchize()
    return E
