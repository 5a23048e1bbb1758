"""Python binding of libddsg (argument marshalling over the C ABI in include/ddsg.h).

Batched evaluation of a cut-HDMR adaptive sparse-grid (DDSG) interpolant on a
GB300 GPU -- Eftekhari & Scheidegger, arXiv 2202.06555, Sec. 3-4. Every step
of the computation runs inside libddsg's CUDA kernels; this module only moves
pointers, sizes and streams across the ABI. PyTorch provides device memory
and streams. There is no CPU fallback: importing works without a GPU (for
the ABI export checks), but every compute call needs the built library and a
CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

F64 = 0
F32C = 1
FORM_PAPER = 0
FORM_SLICEFREE = 1
KMAX = 8

ERRORS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_STATE",
          -5: "ERR_TABLE", -6: "ERR_TIMEOUT", -7: "ERR_NUMERIC"}

# name -> (restype, argtypes); mirrors include/ddsg.h
_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_int = C.c_int
_d = C.c_double
SIGNATURES = {
    "ddsg_last_error": (C.c_char_p, []),
    "ddsg_version": (C.c_char_p, []),
    "hdmr_create": (_int, [_int, _int, _int, _p, _p, _p, C.POINTER(_p)]),
    "hdmr_destroy": (_int, [_p]),
    "hdmr_add_component": (_int, [_p, _int, _p, _i64, _p, _p, C.POINTER(_i32)]),
    "hdmr_add_regular_component": (_int, [_p, _int, _p, _int, C.POINTER(_i32)]),
    "hdmr_num_components": (_int, [_p, C.POINTER(_i32), C.POINTER(_i64)]),
    "hdmr_component_info": (_int, [_p, _i32, C.POINTER(_i32), _p, C.POINTER(_i64), C.POINTER(_i64)]),
    "hdmr_component_points": (_int, [_p, _i32, _i64, _i64, _p, _p, _p]),
    "hdmr_hierarchize": (_int, [_p, _p, _p]),
    "hdmr_refine": (_int, [_p, _d, _int, _int, C.POINTER(_i64), _p]),
    "hdmr_get_surpluses": (_int, [_p, _p, _p]),
    "hdmr_get_b": (_int, [_p, _p]),
    "hdmr_eval": (_int, [_p, _i64, _p, _p, _int, _int, _p, _p, _p]),
    "hdmr_reserve": (_int, [_p, _i64]),
    "hdmr_stats": (_int, [_p, _p, _int, _p]),
    "hdmr_eval_host": (_int, [_p, _i64, _p, _p, _int, _int, _p]),
    "hdmr_profile": (_int, [_p, _int]),
    "hdmr_set_eval_config": (_int, [_p, _int, _int, _int, _int]),
    "hdmr_get_eval_config": (_int, [_p, _int, _int, C.POINTER(_int), C.POINTER(_int)]),
    "hdmr_autotune": (_int, [_p, _i64, _p, _p, _int, _int, _p, C.POINTER(_d)]),
    "hdmr_eval_noalloc": (_int, [_p, _i64, _p, _p, _int, _int, _p]),
    "hdmr_eval_graph": (_int, [_p, _i64, _p, _p, _int, _int, _p]),
    "hdmr_quadrature": (_int, [_p, _p, _p]),
    "hdmr_save": (_int, [_p, C.c_char_p]),
    "hdmr_set_fault_injection": (_int, [_p, _int]),
    "hdmr_check": (_int, [_p, _p]),
    "ddsg_inject_alloc_failure": (_int, [_int, _int]),
    "ddsg_checked_build": (_int, []),
    "mlp_save": (_int, [_p, C.c_char_p]),
    "mlp_load": (_int, [C.c_char_p, _p]),
    "mlp_shape": (_int, [_p, _p, _p]),
    "ddsg_take_check_word": (_int, [_p]),
    "hdmr_load": (_int, [C.c_char_p, _p]),
    "hdmr_shape": (_int, [_p, _p, _p, _p, _p, _p, _p]),
    "hdmr_eval_noalloc_capacity": (_i64, [_int]),
    "irbc_create": (_int, [_p, _p, _p, C.POINTER(_p)]),
    "irbc_create_table1": (_int, [_int, _d, _d, _d, _d, _d, _d, _d, C.POINTER(_p)]),
    "irbc_get_params": (_int, [_p, _p, _p, _p]),
    "hdmr_expansion_norms": (_int, [_p, _int, _d, _p, _p, _p, _p, _p]),
    "irbc_destroy": (_int, [_p]),
    "euler_residual": (_int, [_p, _p, _i64, _p, _p, _p, _p, _p, _int, _int, _p]),
    "irbc_lu_solve": (_int, [_int, _i64, _p, _p, _p, _p, _p]),
    "irbc_newton": (_int, [_p, _p, _i64, _p, _p, _int, _d, _p, _p, _p, _int, _int, _p]),
    "irbc_profile": (_int, [_p, _int]),
    "mlp_create": (_int, [_int, _p, _p, C.c_uint64, C.POINTER(_p)]),
    "mlp_destroy": (_int, [_p]),
    "mlp_set_normalization": (_int, [_p, _p, _p, _p, _p]),
    "mlp_train_step": (_int, [_p, _i64, _p, _p, C.c_float, _p, _p]),
    "mlp_infer": (_int, [_p, _i64, _p, _p, _p]),
    "mlp_num_params": (_i64, [_p]),
    "mlp_get_params": (_int, [_p, _p]),
    "mlp_get_grads": (_int, [_p, _p]),
    "mlp_profile": (_int, [_p, _int]),
    "mlp_profile_read": (_int, [_p, _p, _p, _int]),
    "mlp_check": (_int, [_p]),
    "ddsg_probe_fma": (_int, [_int, _p, _p]),
    "hdmr_nodal_info": (_int, [_p, _int, _p, _p, _p]),
    "irbc_profile_read": (_int, [_p, _p, _p, _int]),
    "irbc_set_node_mode": (_int, [_p, _int]),
    "irbc_set_irreversible": (_int, [_p, _int]),
    "hdmr_profile_read": (_int, [_p, _p, _p, _int]),
}

KERNEL_KINDS = ["encode", "eval", "hierarchize", "convert", "copy", "graph", "k6", "k7"]

_lib = None


class DDSGError(RuntimeError):
    """A libddsg call returned an error; `code` is the DDSG_ERR_* value."""

    def __init__(self, msg: str, code: int | None = None):
        super().__init__(msg)
        self.code = code


def variant() -> str:
    """Library variant this process loads: DDSG_VARIANT, "release" (default) or
    "checked" (kernels with bounds-checked table indices)."""
    return os.environ.get("DDSG_VARIANT", "release")


def library_path() -> str:
    return _build.lib_path(variant())


def load(build_if_missing: bool = True):
    """Load libddsg.so (building it in-tree with nvcc if it is missing/stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing:
        _build.build(variant=variant())
    if not os.path.exists(path):
        raise DDSGError(f"libddsg is not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().ddsg_last_error().decode()
        raise DDSGError(f"{what} failed ({ERRORS.get(rc, rc)}): {msg}", rc)


CHECK_SITES = ["cell", "slot", "row", "stage", "dim", "point", "component"]


def take_check_word() -> list[str]:
    """Checked builds: the table-index test sites that failed since the last
    call (and clear them); always [] in a release build."""
    w = C.c_uint64()
    _check(load().ddsg_take_check_word(C.byref(w)), "ddsg_take_check_word")
    return [s for i, s in enumerate(CHECK_SITES) if w.value >> i & 1] + (["unreadable"] if w.value >> 63 & 1 else [])


def inject_alloc_failure(skip: int = 0, count: int = 1):
    """Test only, process-wide: after `skip` more device allocations by libddsg
    succeed, the next `count` fail with DDSG_ERR_OOM; count=0 turns it off."""
    _check(load().ddsg_inject_alloc_failure(int(skip), int(count)), "ddsg_inject_alloc_failure")


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise DDSGError("libddsg needs CUDA tensors (no CPU path)")
    if not t.is_contiguous():
        raise DDSGError("libddsg needs contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def probe_fma(kind: int):
    """Measured FMA throughput of the current device: kind 0 FP64, 1 FP32, 2 paired
    FP32 (fma.rn.f32x2). Returns (TFLOP/s, ms of the timed launch)."""
    t, ms = C.c_double(), C.c_double()
    _check(load().ddsg_probe_fma(int(kind), C.byref(t), C.byref(ms)), "ddsg_probe_fma")
    return t.value, ms.value


class HDMR:
    """A cut-HDMR expansion with one sparse grid per accepted component.

    Thin wrapper over the hdmr_* calls; see include/ddsg.h for semantics.
    """

    def __init__(self, d: int, m: int, order: int, anchor=None, lo=None, hi=None):
        lib = load()
        self.d, self.m, self.order = int(d), int(m), int(order)
        self.lo = np.zeros(d) if lo is None else np.ascontiguousarray(lo, np.float64)
        self.hi = np.ones(d) if hi is None else np.ascontiguousarray(hi, np.float64)
        self.anchor = (0.5 * (self.lo + self.hi) if anchor is None
                       else np.ascontiguousarray(anchor, np.float64))
        h = C.c_void_p()
        _check(lib.hdmr_create(self.d, self.m, self.order, _np_ptr(self.anchor), _np_ptr(self.lo),
                               _np_ptr(self.hi), C.byref(h)), "hdmr_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().hdmr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- construction ------------------------------------------------------
    def add_component(self, dims, levels=None, indices=None) -> int:
        dims = np.ascontiguousarray(dims, np.int32).reshape(-1)
        k = dims.size
        cid = C.c_int32()
        if k == 0:
            _check(load().hdmr_add_component(self._h, 0, None, 1, None, None, C.byref(cid)),
                   "hdmr_add_component")
            return cid.value
        lv = np.ascontiguousarray(levels, np.uint8).reshape(-1, k)
        ix = np.ascontiguousarray(indices, np.uint32).reshape(-1, k)
        _check(load().hdmr_add_component(self._h, k, _np_ptr(dims), lv.shape[0], _np_ptr(lv),
                                         _np_ptr(ix), C.byref(cid)), "hdmr_add_component")
        return cid.value

    def add_regular(self, dims, level: int) -> int:
        dims = np.ascontiguousarray(dims, np.int32).reshape(-1)
        cid = C.c_int32()
        _check(load().hdmr_add_regular_component(self._h, dims.size, _np_ptr(dims), int(level),
                                                 C.byref(cid)), "hdmr_add_regular_component")
        return cid.value

    def sizes(self):
        nc, npt = C.c_int32(), C.c_int64()
        _check(load().hdmr_num_components(self._h, C.byref(nc), C.byref(npt)), "hdmr_num_components")
        return nc.value, npt.value

    def component_info(self, comp: int):
        k, npts, first = C.c_int32(), C.c_int64(), C.c_int64()
        dims = np.zeros(KMAX, np.int32)
        _check(load().hdmr_component_info(self._h, comp, C.byref(k), _np_ptr(dims), C.byref(npts),
                                          C.byref(first)), "hdmr_component_info")
        return tuple(int(x) for x in dims[:k.value]), npts.value, first.value

    def component_points(self, comp: int, first: int = 0, count=None):
        dims, npts, _ = self.component_info(comp)
        k = len(dims)
        if count is None:
            count = npts - first
        lv = np.zeros((count, max(k, 1)), np.uint8)
        ix = np.zeros((count, max(k, 1)), np.uint32)
        xs = np.zeros((count, max(k, 1)), np.float64)
        _check(load().hdmr_component_points(self._h, comp, first, count, _np_ptr(lv), _np_ptr(ix),
                                            _np_ptr(xs)), "hdmr_component_points")
        return lv[:, :k], ix[:, :k], xs[:, :k]

    def hierarchize(self, values_dev, stream=None):
        _check(load().hdmr_hierarchize(self._h, _dev_ptr(values_dev), _stream_ptr(stream)),
               "hdmr_hierarchize")

    def refine(self, eps_gamma: float, max_level: int, strict: bool = False, stream=None) -> int:
        n = C.c_int64()
        _check(load().hdmr_refine(self._h, float(eps_gamma), int(max_level), int(bool(strict)),
                                  C.byref(n), _stream_ptr(stream)), "hdmr_refine")
        return n.value

    def surpluses(self, stream=None) -> np.ndarray:
        _, P = self.sizes()
        out = np.zeros((P, self.m))
        _check(load().hdmr_get_surpluses(self._h, _np_ptr(out), _stream_ptr(stream)),
               "hdmr_get_surpluses")
        return out

    def b_coeffs(self) -> np.ndarray:
        nc, _ = self.sizes()
        out = np.zeros(nc)
        _check(load().hdmr_get_b(self._h, _np_ptr(out)), "hdmr_get_b")
        return out

    # -- evaluation ----------------------------------------------------------
    def reserve(self, n: int):
        _check(load().hdmr_reserve(self._h, int(n)), "hdmr_reserve")

    def eval(self, x_dev, y_dev, precision: int = F64, form: int = FORM_PAPER, hash_dev=None,
             count_dev=None, stream=None):
        n = x_dev.shape[0]
        _check(load().hdmr_eval(self._h, n, _dev_ptr(x_dev), _dev_ptr(y_dev), int(precision),
                                int(form), _dev_ptr(hash_dev), _dev_ptr(count_dev),
                                _stream_ptr(stream)), "hdmr_eval")

    def eval_noalloc(self, x_dev, y_dev, precision: int = F64, form: int = FORM_PAPER, stream=None):
        """Evaluation that allocates no device memory (scratch in a static device
        array); batches above noalloc_capacity() queries are refused."""
        n = x_dev.shape[0]
        _check(load().hdmr_eval_noalloc(self._h, n, _dev_ptr(x_dev), _dev_ptr(y_dev), int(precision),
                                        int(form), _stream_ptr(stream)), "hdmr_eval_noalloc")

    def eval_graph(self, x_dev, y_dev, precision: int = F64, form: int = FORM_PAPER, stream=None):
        """hdmr_eval replayed from a cached CUDA graph (captured on the first call
        for these buffers, sizes and schedule); same results bit for bit."""
        n = x_dev.shape[0]
        _check(load().hdmr_eval_graph(self._h, n, _dev_ptr(x_dev), _dev_ptr(y_dev), int(precision),
                                      int(form), _stream_ptr(stream)), "hdmr_eval_graph")

    def set_fault_injection(self, withhold_from: int = -1):
        """Test only: withhold the staged kernels' copies from a processed component
        on, so their bounded waits run out (see hdmr_set_fault_injection)."""
        _check(load().hdmr_set_fault_injection(self._h, int(withhold_from)),
               "hdmr_set_fault_injection")

    def check(self, stream=None):
        """Raise DDSGError (DDSG_ERR_TIMEOUT) if a staged evaluation gave up a
        bounded wait since the last check; synchronizes the stream."""
        _check(load().hdmr_check(self._h, _stream_ptr(stream)), "hdmr_check")

    def save(self, path: str):
        """Checkpoint the hierarchized expansion to one file (hdmr_save)."""
        _check(load().hdmr_save(self._h, os.fsencode(path)), "hdmr_save")

    @classmethod
    def load(cls, path: str) -> "HDMR":
        """A hierarchized handle recreated from an hdmr_save file on the current device."""
        lib = load()
        h = C.c_void_p()
        _check(lib.hdmr_load(os.fsencode(path), C.byref(h)), "hdmr_load")
        self = cls.__new__(cls)
        self._h = h
        d, m, order = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib.hdmr_shape(h, C.byref(d), C.byref(m), C.byref(order), None, None, None), "hdmr_shape")
        self.d, self.m, self.order = d.value, m.value, order.value
        self.anchor, self.lo, self.hi = np.zeros(self.d), np.zeros(self.d), np.zeros(self.d)
        _check(lib.hdmr_shape(h, None, None, None, _np_ptr(self.anchor), _np_ptr(self.lo), _np_ptr(self.hi)),
               "hdmr_shape")
        return self

    def quadrature(self, stream=None):
        """Integral of every component interpolant over its unit cube (eq. 3.7):
        a (ncomp, m) FP64 device tensor."""
        import torch
        ncomp, _ = self.sizes()
        q = torch.empty((ncomp, self.m), dtype=torch.float64, device="cuda")
        _check(load().hdmr_quadrature(self._h, _dev_ptr(q), _stream_ptr(stream)), "hdmr_quadrature")
        return q

    def noalloc_capacity(self) -> int:
        return int(load().hdmr_eval_noalloc_capacity(self.d))

    def eval_host(self, x_host: np.ndarray, y_host: np.ndarray, precision: int = F64,
                  form: int = FORM_PAPER, stream=None):
        """End-to-end call with host arrays (copies inside the call)."""
        assert x_host.dtype == np.float64 and y_host.dtype == np.float64
        assert x_host.flags.c_contiguous and y_host.flags.c_contiguous
        n = x_host.shape[0]
        _check(load().hdmr_eval_host(self._h, n, C.c_void_p(x_host.ctypes.data),
                                     C.c_void_p(y_host.ctypes.data), int(precision), int(form),
                                     _stream_ptr(stream)), "hdmr_eval_host")

    def expansion_norms(self, k: int, eps_eta: float = -1.0, stream=None):
        """Alg. 2's criteria for the order-k components (hdmr_expansion_norms): the
        cut-HDMR component integrals Qf (ncomp, m), eta per component (eq. 3.19; NaN
        off order k), rho over all order-k components and over those with
        eta > eps_eta (eq. 3.18)."""
        nc, _ = self.sizes()
        qf = np.zeros((nc, self.m))
        eta = np.zeros(nc)
        ra, rk = C.c_double(), C.c_double()
        _check(load().hdmr_expansion_norms(self._h, int(k), float(eps_eta), _np_ptr(qf), _np_ptr(eta),
                                           C.byref(ra), C.byref(rk), _stream_ptr(stream)), "hdmr_expansion_norms")
        return qf, eta, ra.value, rk.value

    def nodal_info(self, form: int = FORM_SLICEFREE):
        """Tables of the nodal-slab kernel (planned if needed): (eligible, node rows,
        node rows read per uniformly distributed query)."""
        e, r, q = C.c_int32(), C.c_int64(), C.c_double()
        _check(load().hdmr_nodal_info(self._h, int(form), C.byref(e), C.byref(r), C.byref(q)), "hdmr_nodal_info")
        return bool(e.value), r.value, q.value

    def set_eval_config(self, precision: int, form: int, kernel: int, mc: int):
        _check(load().hdmr_set_eval_config(self._h, precision, form, kernel, mc),
               "hdmr_set_eval_config")

    def eval_config(self, precision: int, form: int):
        k, mc = C.c_int(), C.c_int()
        _check(load().hdmr_get_eval_config(self._h, precision, form, C.byref(k), C.byref(mc)),
               "hdmr_get_eval_config")
        return k.value, mc.value

    def autotune(self, x_dev, y_dev, precision: int = F64, form: int = FORM_PAPER, stream=None):
        best = C.c_double()
        _check(load().hdmr_autotune(self._h, x_dev.shape[0], _dev_ptr(x_dev), _dev_ptr(y_dev),
                                    int(precision), int(form), _stream_ptr(stream), C.byref(best)),
               "hdmr_autotune")
        return self.eval_config(precision, form) + (best.value,)

    def profile(self, enable: bool = True):
        _check(load().hdmr_profile(self._h, int(bool(enable))), "hdmr_profile")

    def profile_read(self, reset: bool = True):
        ms = np.zeros(8)
        n = np.zeros(8, np.int64)
        _check(load().hdmr_profile_read(self._h, _np_ptr(ms), _np_ptr(n), int(bool(reset))),
               "hdmr_profile_read")
        return {KERNEL_KINDS[i]: (float(ms[i]), int(n[i])) for i in range(8) if n[i]}

    def stats(self, reset: bool = False, stream=None):
        out = np.zeros(3, np.int64)
        _check(load().hdmr_stats(self._h, _np_ptr(out), int(bool(reset)), _stream_ptr(stream)),
               "hdmr_stats")
        return {"clamped": int(out[0]), "nonfinite_rows": int(out[1]), "wait_timeouts": int(out[2])}


def build_adaptive(h: HDMR, value_fn, eps_gamma: float, max_level: int, strict: bool = False,
                   max_sweeps: int = 64, stream=None):
    """Hierarchize / refine sweeps until no point is added (eq. 3.8).

    value_fn(dims, phys_coords (n, k)) -> (n, m) values of the function at the
    cut points (coordinates outside dims at the anchor). Only the values of new
    points are requested; the library does all grid and surplus work.
    """
    import torch
    ncomp, _ = h.sizes()
    vals = [None] * ncomp
    for _ in range(max_sweeps):
        for c in range(ncomp):
            dims, npts, _ = h.component_info(c)
            have = 0 if vals[c] is None else vals[c].shape[0]
            if have < npts:
                _, _, xs = h.component_points(c, have, npts - have)
                new = np.asarray(value_fn(dims, xs), np.float64).reshape(npts - have, h.m)
                vals[c] = new if vals[c] is None else np.concatenate([vals[c], new])
        allv = torch.from_numpy(np.ascontiguousarray(np.concatenate(vals))).cuda()
        h.hierarchize(allv, stream)
        if h.refine(eps_gamma, max_level, strict, stream) == 0:
            break
    return np.concatenate(vals)


class IrbcParams(C.Structure):
    _fields_ = [("N", C.c_int32), ("beta", C.c_double), ("alpha", C.c_double),
                ("delta", C.c_double), ("sigma", C.c_double), ("rho", C.c_double),
                ("phi", C.c_double), ("A", C.c_double)]


class IRBC:
    """Smooth IRBC model step (Sec. 2.1) over a policy HDMR: residuals,
    Jacobian and batched Newton (see include/ddsg.h)."""

    def __init__(self, N: int, beta: float, alpha: float, delta: float, sigma: float, rho: float,
                 phi: float, A: float, gamma, tau):
        lib = load()
        self.N = int(N)
        self.m = self.N + 1
        self.prm = IrbcParams(self.N, beta, alpha, delta, sigma, rho, phi, A)
        g = np.ascontiguousarray(gamma, np.float64)
        t = np.ascontiguousarray(tau, np.float64)
        h = C.c_void_p()
        _check(lib.irbc_create(C.byref(self.prm), _np_ptr(g), _np_ptr(t), C.byref(h)), "irbc_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().irbc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_irreversible(self, on: bool = True):
        """Non-smooth model (irreversible investment): policy (k', mu, lambda)."""
        _check(load().irbc_set_irreversible(self._h, int(bool(on))), "irbc_set_irreversible")
        self.m = 2 * self.N + 1 if on else self.N + 1

    def set_node_mode(self, mode: int):
        """NODES_ALL: interpolate every monomial node; NODES_DELTA: the no-shock
        state and the two global nodes, country nodes by component deltas."""
        _check(load().irbc_set_node_mode(self._h, int(mode)), "irbc_set_node_mode")

    def residual(self, policy: HDMR, states_dev, guess_dev, resid_dev, jac_dev=None, err_dev=None,
                 precision: int = F64, form: int = FORM_SLICEFREE, stream=None):
        _check(load().euler_residual(self._h, policy._h, states_dev.shape[0], _dev_ptr(states_dev),
                                     _dev_ptr(guess_dev), _dev_ptr(resid_dev), _dev_ptr(jac_dev),
                                     _dev_ptr(err_dev), int(precision), int(form), _stream_ptr(stream)),
               "euler_residual")

    def newton(self, policy: HDMR, states_dev, sol_dev, max_it: int = 30, tol: float = 1e-10,
               iters_dev=None, status_dev=None, resnorm_dev=None, precision: int = F64,
               form: int = FORM_SLICEFREE, stream=None):
        _check(load().irbc_newton(self._h, policy._h, states_dev.shape[0], _dev_ptr(states_dev),
                                  _dev_ptr(sol_dev), int(max_it), float(tol), _dev_ptr(iters_dev),
                                  _dev_ptr(status_dev), _dev_ptr(resnorm_dev), int(precision),
                                  int(form), _stream_ptr(stream)), "irbc_newton")


IRBC_KINDS = ["queries", "eval", "residual", "jacobian", "lu", "newton_aux", "node_delta", "k7"]
NODES_ALL, NODES_DELTA = 0, 1


def _irbc_profile(self, enable=True):
    _check(load().irbc_profile(self._h, int(bool(enable))), "irbc_profile")


def _irbc_profile_read(self, reset=True):
    ms = np.zeros(8)
    n = np.zeros(8, np.int64)
    _check(load().irbc_profile_read(self._h, _np_ptr(ms), _np_ptr(n), int(bool(reset))),
           "irbc_profile_read")
    return {IRBC_KINDS[i]: (float(ms[i]), int(n[i])) for i in range(8) if n[i]}


IRBC.profile = _irbc_profile
IRBC.profile_read = _irbc_profile_read


def lu_solve(A_dev, r_dev, dx_dev, status_dev, stream=None):
    ns, n = r_dev.shape
    _check(load().irbc_lu_solve(n, ns, _dev_ptr(A_dev), _dev_ptr(r_dev), _dev_ptr(dx_dev),
                                _dev_ptr(status_dev), _stream_ptr(stream)), "irbc_lu_solve")


def irbc_table1(N: int, a_gamma: float = 0.25, beta: float = 0.99, alpha: float = 0.36,
                delta: float = 0.01, sigma: float = 0.01, rho: float = 0.95, phi: float = 0.5):
    """Table 1 calibration as libddsg derives it (irbc_create_table1): A, gamma_j
    and tau_j read back from a model the library creates. Returns the keyword
    arguments of IRBC()."""
    lib = load()
    h = _p()
    _check(lib.irbc_create_table1(int(N), float(a_gamma), float(beta), float(alpha), float(delta),
                                  float(sigma), float(rho), float(phi), C.byref(h)), "irbc_create_table1")
    try:
        prm = IrbcParams()
        gamma = np.zeros(int(N))
        tau = np.zeros(int(N))
        _check(lib.irbc_get_params(h, C.byref(prm), _np_ptr(gamma), _np_ptr(tau)), "irbc_get_params")
    finally:
        lib.irbc_destroy(h)
    return dict(N=int(N), beta=prm.beta, alpha=prm.alpha, delta=prm.delta, sigma=prm.sigma, rho=prm.rho,
                phi=prm.phi, A=prm.A, gamma=gamma, tau=tau)


class MLP:
    """Warm-start network (see include/ddsg.h): BF16 tensor-core training and
    inference kernels, FP32 master weights and Adam."""

    def __init__(self, sizes, params=None, seed: int = 0, in_shift=None, in_scale=None,
                 out_shift=None, out_scale=None):
        lib = load()
        self.sizes = [int(s) for s in sizes]
        sz = np.ascontiguousarray(self.sizes, np.int32)
        prm = None if params is None else np.ascontiguousarray(params, np.float32)
        h = C.c_void_p()
        _check(lib.mlp_create(len(self.sizes) - 1, _np_ptr(sz), _np_ptr(prm), int(seed), C.byref(h)),
               "mlp_create")
        self._h = h
        if in_shift is not None:
            arrs = [np.ascontiguousarray(a, np.float64) for a in (in_shift, in_scale, out_shift, out_scale)]
            _check(lib.mlp_set_normalization(self._h, *[_np_ptr(a) for a in arrs]), "mlp_set_normalization")

    def close(self):
        if getattr(self, "_h", None):
            load().mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path: str):
        """Checkpoint: sizes, normalization, weights, Adam moments and step (mlp_save)."""
        _check(load().mlp_save(self._h, os.fsencode(path)), "mlp_save")

    @classmethod
    def load(cls, path: str) -> "MLP":
        """A network recreated from an mlp_save file; training resumes exactly."""
        lib = load()
        h = C.c_void_p()
        _check(lib.mlp_load(os.fsencode(path), C.byref(h)), "mlp_load")
        self = cls.__new__(cls)
        self._h = h
        L = C.c_int32()
        _check(lib.mlp_shape(h, C.byref(L), None), "mlp_shape")
        sz = np.zeros(L.value + 1, np.int32)
        _check(lib.mlp_shape(h, None, _np_ptr(sz)), "mlp_shape")
        self.sizes = [int(s) for s in sz]
        return self

    def train_step(self, x_dev, y_dev, lr: float, loss_dev=None, stream=None):
        _check(load().mlp_train_step(self._h, x_dev.shape[0], _dev_ptr(x_dev), _dev_ptr(y_dev),
                                     float(lr), _dev_ptr(loss_dev), _stream_ptr(stream)), "mlp_train_step")

    def infer(self, x_dev, y_dev, stream=None):
        _check(load().mlp_infer(self._h, x_dev.shape[0], _dev_ptr(x_dev), _dev_ptr(y_dev),
                                _stream_ptr(stream)), "mlp_infer")

    def _unpack(self, flat):
        W, b, off = [], [], 0
        for l in range(len(self.sizes) - 1):
            ni, no = self.sizes[l], self.sizes[l + 1]
            W.append(flat[off:off + ni * no].reshape(no, ni).astype(np.float64))
            off += ni * no
            b.append(flat[off:off + no].astype(np.float64))
            off += no
        return W, b

    def flat_params(self):
        """FP32 parameters in the packed layout of mlp_create / mlp_save."""
        flat = np.zeros(load().mlp_num_params(self._h), np.float32)
        _check(load().mlp_get_params(self._h, _np_ptr(flat)), "mlp_get_params")
        return flat

    def params(self):
        return self._unpack(self.flat_params())

    def grads(self):
        flat = np.zeros(load().mlp_num_params(self._h), np.float32)
        _check(load().mlp_get_grads(self._h, _np_ptr(flat)), "mlp_get_grads")
        return self._unpack(flat)

    def profile(self, enable=True):
        _check(load().mlp_profile(self._h, int(bool(enable))), "mlp_profile")

    def check(self):
        """Raise DDSGError (DDSG_ERR_TIMEOUT) if a tensor-core GEMM of this network gave
        up a bounded wait since the last check; synchronizes the device."""
        _check(load().mlp_check(self._h), "mlp_check")

    def profile_read(self, reset=True):
        ms = np.zeros(8)
        n = np.zeros(8, np.int64)
        _check(load().mlp_profile_read(self._h, _np_ptr(ms), _np_ptr(n), int(bool(reset))),
               "mlp_profile_read")
        names = ["gemm_fwd", "gemm_bwd", "aux", "adam", "k4", "k5", "k6", "k7"]
        return {names[i]: (float(ms[i]), int(n[i])) for i in range(8) if n[i]}
