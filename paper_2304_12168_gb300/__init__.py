"""GB300-native TA / CTA linear-system solvers (Lau & Kalantari, arXiv:2304.12168).

Thin ctypes binding of ``libtacta.so`` (declared in ``include/tacta.h``). The
functions here only marshal arguments: every step of the solvers runs in the
library's CUDA kernels. There is no CPU fallback; if the library is missing,
every call raises.

Matrices are passed as
  * a 2-D float64 array / tensor (dense, row-major), or
  * ``CSR(rowptr, colidx, vals, shape)`` (int32, int32, float64), or
  * any object with ``fmt`` ("dense"/"csr"), ``m``, ``n`` and the arrays
    ``dense`` or ``rowptr``/``colidx``/``vals``.
Arrays may be numpy arrays / CPU tensors (host: the library copies them) or
CUDA tensors (device: all arrays of one call must then be CUDA tensors on the
current device; work runs on torch's current stream).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtacta.so")

# ---------------------------------------------------------------- C structs (include/tacta.h)

TACTA_DENSE, TACTA_CSR = 0, 1
CYCLE_PINGPONG, CYCLE_SAWTOOTH, CYCLE_FIXED = 0, 1, 2
PRECISION_FP64, PRECISION_MIXED = 0, 1
STATUS = {0: "OK", 1: "MAXITER", 2: "BREAKDOWN", 3: "WITNESS", -1: "ERR_INVALID",
          -2: "ERR_NONFINITE", -3: "ERR_CUDA", -4: "ERR_OOM", -5: "ERR_TIMEOUT"}
REASON = {0: "NONE", 1: "RESIDUAL", 2: "NORMAL", 3: "MAXITER", 4: "BREAKDOWN", 5: "WITNESS",
          6: "GAP", 7: "ZERO_RHS", 8: "NONFINITE", 9: "TIMEOUT", 10: "RHO_BOUND", 11: "ENHANCED"}


class tacta_matrix(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("format", ctypes.c_int32), ("on_device", ctypes.c_int32),
                ("vals", ctypes.c_void_p), ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p)]


class tacta_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("tol_normal", ctypes.c_double),
                ("tol_cta", ctypes.c_double), ("pivot_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("t_max", ctypes.c_int32), ("cycle", ctypes.c_int32),
                ("recompute_every", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("poll_every", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("nonneg", ctypes.c_int32), ("enhanced", ctypes.c_int32),
                ("fused_chain", ctypes.c_int32), ("wait_limit_log2", ctypes.c_int32),
                ("rho_max", ctypes.c_double), ("stream", ctypes.c_void_p)]


class tacta_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reason", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("matvecs", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("rel_normal_res", ctypes.c_double), ("rho", ctypes.c_double),
                ("rho_lower", ctypes.c_double), ("trips", ctypes.c_int32),
                ("cta_iters", ctypes.c_int32), ("normal_system", ctypes.c_int32),
                ("hist_len", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("spmv_count", ctypes.c_int32), ("spmv_pad", ctypes.c_int32),
                ("spmv_ms", ctypes.c_double), ("spmv_bytes", ctypes.c_double)]


EXPORTS = ["tacta_default_options", "cta_solve", "ta_solve", "ta_minnorm", "tacta_plan_create",
           "tacta_plan_cta", "tacta_plan_ta", "tacta_plan_minnorm", "tacta_plan_destroy",
           "tacta_plan_transpose", "tacta_plan_matvec", "tacta_plan_residual", "tacta_plan_outer", "tacta_plan_minnorm_bisect",
           "tacta_residual_static", "tacta_last_error", "tacta_version",
           "tacta_batch_create", "tacta_batch_cta", "tacta_batch_destroy", "tacta_batch_tune",
           "tacta_batch_set_config", "tacta_batch_num_configs", "tacta_batch_config_shape",
           "tacta_batch_last_error", "tacta_batch_timeline", "tacta_batch_config_tensor_cores", "tacta_batch_config_stage_bytes", "tacta_batch_set_wide",
           "tacta_batch_wide_plan", "tacta_batch_simulate_makespan", "tacta_batch_plan_search", "tacta_aux_solve", "tacta_dia_tile_plan", "tacta_column_partition"]

_lib_handle = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtacta.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2304_12168_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, dp = ctypes.c_void_p, ctypes.c_void_p
    solve_args = [P(tacta_matrix), dp, dp, P(tacta_options), dp, dp, ctypes.c_int32, P(tacta_info)]
    plan_args = [vp, dp, dp, P(tacta_options), dp, dp, ctypes.c_int32, P(tacta_info)]
    lib.tacta_default_options.argtypes = [P(tacta_options)]
    lib.tacta_default_options.restype = None
    for name in ("cta_solve", "ta_solve", "ta_minnorm"):
        getattr(lib, name).argtypes = solve_args
        getattr(lib, name).restype = ctypes.c_int32
    for name in ("tacta_plan_cta", "tacta_plan_ta", "tacta_plan_minnorm"):
        getattr(lib, name).argtypes = plan_args
        getattr(lib, name).restype = ctypes.c_int32
    lib.tacta_plan_create.argtypes = [P(tacta_matrix), P(tacta_options), P(vp)]
    lib.tacta_plan_create.restype = ctypes.c_int32
    lib.tacta_plan_destroy.argtypes = [vp]
    lib.tacta_plan_destroy.restype = None
    lib.tacta_last_error.argtypes = []
    lib.tacta_last_error.restype = ctypes.c_char_p
    lib.tacta_version.argtypes = []
    lib.tacta_version.restype = ctypes.c_int32
    lib.tacta_residual_static.argtypes = [P(tacta_matrix), dp, dp, dp, dp, vp]
    lib.tacta_residual_static.restype = ctypes.c_int32
    lib.tacta_plan_minnorm_bisect.argtypes = [vp, dp, dp, ctypes.c_int32, P(tacta_options), dp, dp,
                                              ctypes.c_int32, P(tacta_info)]
    lib.tacta_plan_minnorm_bisect.restype = ctypes.c_int32
    lib.tacta_plan_transpose.argtypes = [vp, P(tacta_options), P(vp)]
    lib.tacta_plan_transpose.restype = ctypes.c_int32
    lib.tacta_plan_matvec.argtypes = [vp, ctypes.c_int32, dp, dp, P(tacta_options)]
    lib.tacta_plan_matvec.restype = ctypes.c_int32
    lib.tacta_plan_residual.argtypes = [vp, ctypes.c_int32, dp, dp, dp, P(tacta_options)]
    lib.tacta_plan_residual.restype = ctypes.c_int32
    lib.tacta_plan_outer.argtypes = [vp, ctypes.c_double, dp, dp, dp, P(tacta_options)]
    lib.tacta_plan_outer.restype = ctypes.c_int32
    i32p = P(ctypes.c_int32)
    lib.tacta_batch_create.argtypes = [ctypes.c_int32, i32p, i32p, dp, ctypes.c_int32, ctypes.c_int32,
                                       P(tacta_options), P(vp)]
    lib.tacta_batch_create.restype = ctypes.c_int32
    lib.tacta_batch_cta.argtypes = [vp, dp, dp, vp, vp, vp, P(tacta_options)]
    lib.tacta_batch_cta.restype = ctypes.c_int32
    lib.tacta_batch_destroy.argtypes = [vp]
    lib.tacta_batch_destroy.restype = None
    lib.tacta_batch_tune.argtypes = [vp, dp, P(tacta_options), i32p, P(ctypes.c_double)]
    lib.tacta_batch_config_tensor_cores.argtypes = [ctypes.c_int32]
    lib.tacta_batch_config_tensor_cores.restype = ctypes.c_int32
    lib.tacta_batch_config_stage_bytes.argtypes = [ctypes.c_int32]
    lib.tacta_batch_config_stage_bytes.restype = ctypes.c_int32
    lib.tacta_batch_timeline.argtypes = [vp, vp, vp]
    lib.tacta_batch_timeline.restype = ctypes.c_int32
    lib.tacta_batch_tune.restype = ctypes.c_int32
    lib.tacta_batch_set_config.argtypes = [vp, ctypes.c_int32]
    lib.tacta_batch_set_config.restype = ctypes.c_int32
    lib.tacta_batch_set_wide.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.tacta_batch_set_wide.restype = ctypes.c_int32
    lib.tacta_batch_wide_plan.argtypes = [vp, P(tacta_options), i32p, i32p, i32p, P(ctypes.c_double)]
    lib.tacta_batch_wide_plan.restype = ctypes.c_int32
    lib.tacta_batch_simulate_makespan.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, dp,
                                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.tacta_batch_simulate_makespan.restype = ctypes.c_double
    lib.tacta_batch_plan_search.argtypes = [ctypes.c_int32, dp, vp, vp, vp, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp, vp]
    lib.tacta_batch_plan_search.restype = ctypes.c_double
    lib.tacta_batch_num_configs.argtypes = []
    lib.tacta_batch_num_configs.restype = ctypes.c_int32
    lib.tacta_batch_config_shape.argtypes = [ctypes.c_int32, i32p, i32p]
    lib.tacta_batch_config_shape.restype = ctypes.c_int32
    lib.tacta_batch_last_error.argtypes = []
    lib.tacta_batch_last_error.restype = ctypes.c_char_p
    lib.tacta_column_partition.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, dp, dp,
                                           ctypes.c_int32, dp, dp]
    lib.tacta_column_partition.restype = ctypes.c_int32
    lib.tacta_aux_solve.argtypes = [dp, ctypes.c_int32, ctypes.c_double, dp]
    lib.tacta_aux_solve.restype = ctypes.c_int32
    lib.tacta_dia_tile_plan.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, i32p, ctypes.c_int32,
                                        i32p, i32p]
    lib.tacta_dia_tile_plan.restype = ctypes.c_int32
    _lib_handle = lib
    return lib


# ---------------------------------------------------------------- argument marshalling

@dataclass
class CSR:
    rowptr: object
    colidx: object
    vals: object
    shape: tuple


def _is_cuda(a) -> bool:
    return getattr(a, "is_cuda", False)


def _ptr(a, dtype) -> tuple[int, bool, object]:
    """(address, on_device, keep-alive) of a contiguous array of `dtype`."""
    if a is None:
        return 0, False, None
    if hasattr(a, "data_ptr"):       # torch tensor
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor, got {a.dtype}")
        return a.data_ptr(), bool(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, False, arr


def _matrix(A):
    """tacta_matrix + keep-alive list from a dense array, CSR, or problem-like object."""
    keep = []
    if isinstance(A, CSR) or getattr(A, "fmt", None) == "csr":
        if isinstance(A, CSR):
            rp, ci, va, (m, n) = A.rowptr, A.colidx, A.vals, A.shape
        else:
            rp, ci, va, m, n = A.rowptr, A.colidx, A.vals, A.m, A.n
        pr, d1, k1 = _ptr(rp, np.int32)
        pc, d2, k2 = _ptr(ci, np.int32)
        pv, d3, k3 = _ptr(va, np.float64)
        if not (d1 == d2 == d3):
            raise ValueError("CSR arrays must all be on the host or all on the device")
        nnz = int(k3.numel() if hasattr(k3, "numel") else k3.size)
        keep += [k1, k2, k3]
        return tacta_matrix(int(m), int(n), nnz, TACTA_CSR, int(d1), pv, pr, pc), d1, keep
    D = A.dense if getattr(A, "fmt", None) == "dense" else A
    if len(D.shape) != 2:
        raise ValueError("dense A must be 2-D")
    m, n = int(D.shape[0]), int(D.shape[1])
    pv, dv, kv = _ptr(D, np.float64)
    keep.append(kv)
    return tacta_matrix(m, n, m * n, TACTA_DENSE, int(dv), pv, 0, 0), dv, keep


def _stream_ptr(on_device: bool):
    if not on_device:
        return None
    import torch
    return torch.cuda.current_stream().cuda_stream or None


def make_options(on_device=False, **kw) -> tacta_options:
    o = tacta_options()
    load_library().tacta_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    if "stream" not in kw:
        o.stream = _stream_ptr(on_device)
    return o


def _vec_out(n, on_device, like):
    if on_device:
        import torch
        return torch.empty(n, dtype=torch.float64, device=like.device)
    return np.empty(n, dtype=np.float64)


def _info_dict(st: int, info: tacta_info) -> dict:
    d = {f: getattr(info, f) for f, _ in tacta_info._fields_}
    d["status_name"] = STATUS.get(st, str(st))
    d["reason_name"] = REASON.get(info.reason, str(info.reason))
    return d


class TactaError(RuntimeError):
    pass


def _check(st: int):
    if st < 0:
        msg = load_library().tacta_last_error().decode()
        raise TactaError(f"{STATUS.get(st, st)}: {msg}")


def _solve(name, A, b, x0=None, hist_cap=None, **opts):
    lib = load_library()
    M, on_dev, keep = _matrix(A)
    pb, db_, kb = _ptr(b, np.float64)
    px, dx, kx = _ptr(x0, np.float64)
    if db_ != bool(on_dev) or (x0 is not None and dx != bool(on_dev)):
        raise ValueError("A, b and x0 must all be on the host or all on the device")
    o = make_options(on_dev, **opts)
    if hist_cap is None:
        hist_cap = int(o.max_iter) + 1
    x = _vec_out(int(M.n), on_dev, kb)
    hist = _vec_out(max(hist_cap, 1), on_dev, kb)
    info = tacta_info()
    st = getattr(lib, name)(ctypes.byref(M), pb, px or None, ctypes.byref(o),
                            _ptr(x, np.float64)[0], _ptr(hist, np.float64)[0], int(hist_cap),
                            ctypes.byref(info))
    _check(st)
    del keep, kb, kx
    return x, hist[: info.hist_len], _info_dict(st, info)


def cta_solve(A, b, x0=None, hist_cap=None, **opts):
    """Algorithm 1.1 (CTA, H = A Aᵀ) -> (x, residual history, info dict)."""
    return _solve("cta_solve", A, b, x0, hist_cap, **opts)


def ta_solve(A, b, x0=None, hist_cap=None, **opts):
    """Algorithm 2.2 (TA) -> (x, residual history, info dict)."""
    return _solve("ta_solve", A, b, x0, hist_cap, **opts)


def ta_minnorm(A, b, hist_cap=None, **opts):
    """Hybrid CTA -> Algorithm 2.5 minimum-norm solve -> (x, CTA history, info dict)."""
    return _solve("ta_minnorm", A, b, None, hist_cap, **opts)


def residual_static(A, x, b):
    """tacta_residual_static: r = b - A x, ||r||² and rᵀb with no device allocation by the
    library (for callers that cannot allocate at the point of the call). A, x and b must
    be CUDA tensors; returns (r, ||r||², rᵀb). The output tensor r is allocated here by
    torch, before the call."""
    import torch
    lib = load_library()
    M, on_dev, keep = _matrix(A)
    if not on_dev:
        raise ValueError("residual_static needs CUDA tensors")
    px, dx, kx = _ptr(x, np.float64)
    pb, db, kb = _ptr(b, np.float64)
    if not (dx and db):
        raise ValueError("residual_static needs CUDA tensors")
    devs = {kx.device, kb.device} | {t.device for t in keep if isinstance(t, torch.Tensor)}
    if len(devs) != 1:
        raise ValueError(f"A, x and b must be on one CUDA device (got {sorted(map(str, devs))})")
    # the library works on the current device: make it the tensors' device for the call
    with torch.cuda.device(kb.device):
        r = torch.empty(int(M.m), dtype=torch.float64, device=kb.device)
        norms = np.zeros(2, dtype=np.float64)
        st = lib.tacta_residual_static(ctypes.byref(M), px, pb, r.data_ptr(), norms.ctypes.data,
                                       _stream_ptr(True))
    _check(st)
    del keep, kx, kb
    return r, float(norms[0]), float(norms[1])


class Plan:
    """A on the GPU (plus Aᵀ) reused across right-hand sides (tacta_plan_*)."""

    def __init__(self, A, **opts):
        lib = load_library()
        M, self.on_device, keep = _matrix(A)
        self.m, self.n = int(M.m), int(M.n)
        o = make_options(self.on_device, **opts)
        h = ctypes.c_void_p()
        st = lib.tacta_plan_create(ctypes.byref(M), ctypes.byref(o), ctypes.byref(h))
        _check(st)
        self._h = h
        del keep

    def _call(self, fn, b, x0, hist_cap, opts):
        lib = load_library()
        pb, db_, kb = _ptr(b, np.float64)
        px, _, kx = _ptr(x0, np.float64)
        if db_ != bool(self.on_device):
            raise ValueError("b must be on the same side as the plan's matrix")
        o = make_options(self.on_device, **opts)
        if hist_cap is None:
            hist_cap = int(o.max_iter) + 1
        x = _vec_out(self.n, self.on_device, kb)
        hist = _vec_out(max(hist_cap, 1), self.on_device, kb)
        info = tacta_info()
        st = getattr(lib, fn)(self._h, pb, px or None, ctypes.byref(o), _ptr(x, np.float64)[0],
                              _ptr(hist, np.float64)[0], int(hist_cap), ctypes.byref(info))
        _check(st)
        del kb, kx
        return x, hist[: info.hist_len], _info_dict(st, info)

    def cta(self, b, x0=None, hist_cap=None, **opts):
        return self._call("tacta_plan_cta", b, x0, hist_cap, opts)

    def ta(self, b, x0=None, hist_cap=None, **opts):
        return self._call("tacta_plan_ta", b, x0, hist_cap, opts)

    def minnorm(self, b, hist_cap=None, **opts):
        return self._call("tacta_plan_minnorm", b, None, hist_cap, opts)

    def minnorm_bisect(self, b, x_eps, normal=False, log_cap=256, **opts):
        """tacta_plan_minnorm_bisect: Algorithm 2.5 alone from x_eps ->
        (x, trip log as a (trips, 6) array: rho, reason, rho_hi, rho_lo, iters, 0; info dict)."""
        lib = load_library()
        pb, db_, kb = _ptr(b, np.float64)
        pe, de, ke = _ptr(x_eps, np.float64)
        if db_ != bool(self.on_device) or de != bool(self.on_device):
            raise ValueError("b and x_eps must be on the same side as the plan's matrix")
        o = make_options(self.on_device, **opts)
        x = _vec_out(self.n, self.on_device, kb)
        log = np.zeros((max(int(log_cap), 1), 6), dtype=np.float64)
        info = tacta_info()
        st = lib.tacta_plan_minnorm_bisect(self._h, pb, pe, int(bool(normal)), ctypes.byref(o),
                                           _ptr(x, np.float64)[0], log.ctypes.data, int(log_cap),
                                           ctypes.byref(info))
        _check(st)
        del kb, ke
        return x, log[: min(info.trips, int(log_cap))].copy(), _info_dict(st, info)

    def transpose(self, **opts):
        """tacta_plan_transpose: a plan for Aᵀ from this plan's device copy."""
        lib = load_library()
        o = make_options(self.on_device, **opts)
        h = ctypes.c_void_p()
        _check(lib.tacta_plan_transpose(self._h, ctypes.byref(o), ctypes.byref(h)))
        q = Plan.__new__(Plan)
        q._h, q.on_device, q.m, q.n = h, self.on_device, self.n, self.m
        return q

    def matvec(self, x, transpose=False, **opts):
        """tacta_plan_matvec: A x, or Aᵀ x with transpose=True."""
        lib = load_library()
        px, _, kx = _ptr(x, np.float64)
        y = _vec_out(self.n if transpose else self.m, self.on_device, kx)
        o = make_options(self.on_device, **opts)
        _check(lib.tacta_plan_matvec(self._h, int(bool(transpose)), px, _ptr(y, np.float64)[0],
                                     ctypes.byref(o)))
        return y

    def residual(self, x, b, transpose=False, **opts):
        """tacta_plan_residual: b - A x, or b - Aᵀ x with transpose=True."""
        lib = load_library()
        px, _, kx = _ptr(x, np.float64)
        pb, _, kb = _ptr(b, np.float64)
        r = _vec_out(self.n if transpose else self.m, self.on_device, kx)
        o = make_options(self.on_device, **opts)
        _check(lib.tacta_plan_residual(self._h, int(bool(transpose)), px, pb, _ptr(r, np.float64)[0],
                                       ctypes.byref(o)))
        del kb
        return r

    def outer(self, alpha, u, v, out, **opts):
        """tacta_plan_outer: out[k] += alpha u[row(k)] v[col(k)] over A's stored entries."""
        lib = load_library()
        pu, _, ku = _ptr(u, np.float64)
        pv, _, kv = _ptr(v, np.float64)
        po, _, ko = _ptr(out, np.float64)
        o = make_options(self.on_device, **opts)
        _check(lib.tacta_plan_outer(self._h, float(alpha), pu, pv, po, ctypes.byref(o)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load_library().tacta_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BATCH_FP64, BATCH_FP32, BATCH_BF16 = 0, 1, 2


def column_partition(rowptr, colidx, m, n, nparts):
    """tacta_column_partition: (col_begin (nparts + 1), shard_nnz (nparts)) for host CSR arrays."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    cb = np.zeros(nparts + 1, dtype=np.int64)
    sn = np.zeros(nparts, dtype=np.int64)
    _check(load_library().tacta_column_partition(int(m), int(n), int(ci.size), rp.ctypes.data, ci.ctypes.data,
                                                 int(nparts), cb.ctypes.data, sn.ctypes.data))
    return cb, sn


def aux_solve(phi, t, pivot_tol=1e-12):
    """tacta_aux_solve: alpha (t values) and the order of the block solved; phi[1..2t] used."""
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    if ph.size < 2 * t + 1:
        raise ValueError("phi needs 2t + 1 entries")
    al = np.zeros(max(int(t), 1), dtype=np.float64)
    rank = load_library().tacta_aux_solve(ph.ctypes.data, int(t), float(pivot_tol), al.ctypes.data)
    if rank < 0:
        raise ValueError("t must be in 1..8")
    return al[: int(t)], int(rank)


def dia_tile_plan(rows, cols, offsets, tile):
    """tacta_dia_tile_plan: (fits, runs as 4 (first, length) pairs, 8 slot bases) of one
    256-row tile of the diagonal form; fits is None on invalid arguments."""
    off = (ctypes.c_int32 * max(1, len(offsets)))(*[int(o) for o in offsets])
    runs = (ctypes.c_int32 * 8)()
    sb = (ctypes.c_int32 * 8)()
    st = load_library().tacta_dia_tile_plan(int(rows), int(cols), len(offsets), off, int(tile), runs, sb)
    if st < 0:
        return None, None, None
    return bool(st), [(runs[2 * i], runs[2 * i + 1]) for i in range(4)], list(sb)


def _check_batch(st: int):
    if st < 0:
        msg = load_library().tacta_batch_last_error().decode()
        raise TactaError(f"{STATUS.get(st, st)}: {msg}")


class Batch:
    """Many independent dense systems solved by CTA in one persistent launch (tacta_batch_*).

    mats: a list of 2-D float64 arrays (numpy or torch, all on the host or all on one
    CUDA device). storage: BATCH_FP64, BATCH_FP32 or BATCH_BF16.
    """

    def __init__(self, mats, storage=BATCH_FP32, **opts):
        lib = load_library()
        self.m = np.array([int(a.shape[0]) for a in mats], dtype=np.int32)
        self.n = np.array([int(a.shape[1]) for a in mats], dtype=np.int32)
        self.count = len(mats)
        self.on_device = bool(mats) and _is_cuda(mats[0])
        if self.on_device:
            import torch
            flat = torch.cat([a.reshape(-1) for a in mats]) if mats else None
        else:
            flat = np.concatenate([np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in mats]) \
                if mats else np.zeros(1)
        pv, _, keep = _ptr(flat, np.float64)
        o = make_options(self.on_device, **opts)
        h = ctypes.c_void_p()
        _check_batch(lib.tacta_batch_create(self.count, self.m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            self.n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), pv,
                                            int(self.on_device), int(storage), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.b_offsets = np.concatenate([[0], np.cumsum(self.m, dtype=np.int64)])
        self.x_offsets = np.concatenate([[0], np.cumsum(self.n, dtype=np.int64)])
        del keep

    def cta(self, b, **opts):
        """Solve all systems; b packed (sum m values). Returns (x packed, iters, rel_res, reason)."""
        lib = load_library()
        pb, db_, kb = _ptr(b, np.float64)
        o = make_options(db_, **opts)
        x = _vec_out(int(self.x_offsets[-1]), db_, kb)
        iters = np.zeros(self.count, dtype=np.int32)
        rel = np.zeros(self.count, dtype=np.float64)
        reason = np.zeros(self.count, dtype=np.int32)
        _check_batch(lib.tacta_batch_cta(self._h, pb, _ptr(x, np.float64)[0], iters.ctypes.data,
                                         rel.ctypes.data, reason.ctypes.data, ctypes.byref(o)))
        del kb
        return x, iters, rel, reason

    def tune(self, b, **opts):
        """Autotune the launch configuration on (self, b); returns (config, ms)."""
        lib = load_library()
        pb, db_, kb = _ptr(b, np.float64)
        o = make_options(db_, **opts)
        cfg = ctypes.c_int32()
        ms = ctypes.c_double()
        _check_batch(lib.tacta_batch_tune(self._h, pb, ctypes.byref(o), ctypes.byref(cfg), ctypes.byref(ms)))
        del kb
        return int(cfg.value), float(ms.value)

    def set_config(self, config: int):
        _check_batch(load_library().tacta_batch_set_config(self._h, int(config)))

    def set_wide(self, systems: int = -1, cluster: int = 0, clusters: int = 0):
        """Thread-block clusters for the longest systems (tacta_batch_set_wide): systems -1
        planned from the earlier solves' measured times, 0 off, > 0 that many systems from
        the head of the queue order on `clusters` clusters of `cluster` blocks (0: chosen)."""
        _check_batch(load_library().tacta_batch_set_wide(self._h, int(systems), int(cluster), int(clusters)))

    def wide_plan(self, **opts):
        """(systems, cluster, clusters, predicted_ms) the next solve with these options would
        use (tacta_batch_wide_plan)."""
        o = make_options(False, **opts)
        v = [ctypes.c_int32() for _ in range(3)]
        ms = ctypes.c_double()
        _check_batch(load_library().tacta_batch_wide_plan(self._h, ctypes.byref(o), *[ctypes.byref(a) for a in v],
                                                          ctypes.byref(ms)))
        return v[0].value, v[1].value, v[2].value, float(ms.value)

    @staticmethod
    def simulate_makespan(w, clusters, cluster, d, sms, per_sm):
        """The planner's schedule model (tacta_batch_simulate_makespan; host only)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        return float(load_library().tacta_batch_simulate_makespan(
            w.ctypes.data if w.size else None, int(w.size), int(clusters), int(cluster),
            d.ctypes.data if d.size else None, int(d.size), int(sms), int(per_sm)))

    @staticmethod
    def plan_search(dur, steps, m, n, storage, t_max, cycle, sms, per_sm, max_clusters, a_cap, wide_mode=-1,
                    wide_cluster=0, wide_clusters=0, h0=12000.0):
        """The planner (tacta_batch_plan_search; host only): (makespan ms, (systems,
        cluster, clusters), queue order). max_clusters and a_cap: five entries each, for
        cluster sizes 16, 8, 4, 2, 1."""
        dur = np.ascontiguousarray(dur, dtype=np.float64)
        count = dur.size
        st = None if steps is None else np.ascontiguousarray(steps, dtype=np.int32)
        m = np.ascontiguousarray(m, dtype=np.int32)
        n = np.ascontiguousarray(n, dtype=np.int32)
        mc = np.ascontiguousarray(max_clusters, dtype=np.int32)
        ac = np.ascontiguousarray(a_cap, dtype=np.int64)
        plan = np.zeros(3, dtype=np.int32)
        order = np.zeros(max(count, 1), dtype=np.int32)
        ms = load_library().tacta_batch_plan_search(
            count, dur.ctypes.data if count else None, st.ctypes.data if st is not None else None,
            m.ctypes.data if count else None, n.ctypes.data if count else None, int(storage), int(t_max),
            int(cycle), int(sms), int(per_sm), mc.ctypes.data, ac.ctypes.data, int(wide_mode), int(wide_cluster),
            int(wide_clusters), float(h0), plan.ctypes.data, order.ctypes.data)
        return float(ms), tuple(int(v) for v in plan), order[:count]

    def timeline(self):
        """(t_begin, t_end): int64 device-clock nanoseconds at which each system of the last
        solve was taken by a block (or cluster) and finished (tacta_batch_timeline)."""
        tb = np.zeros(self.count, dtype=np.int64)
        te = np.zeros(self.count, dtype=np.int64)
        _check_batch(load_library().tacta_batch_timeline(self._h, tb.ctypes.data, te.ctypes.data))
        return tb, te

    @staticmethod
    def configs():
        """[(threads per block, blocks per SM, ring stage bytes)] of the launch configurations
        (the stage is 0 for the configurations without the bulk-copy ring)."""
        lib = load_library()
        out = []
        for c in range(lib.tacta_batch_num_configs()):
            t, p = ctypes.c_int32(), ctypes.c_int32()
            _check_batch(lib.tacta_batch_config_shape(c, ctypes.byref(t), ctypes.byref(p)))
            out.append((t.value, p.value, int(lib.tacta_batch_config_stage_bytes(c))))
        return out

    @staticmethod
    def tensor_core_configs():
        """Indices of the launch configurations whose products run on the tensor cores
        (BF16 storage only)."""
        lib = load_library()
        return [c for c in range(lib.tacta_batch_num_configs()) if lib.tacta_batch_config_tensor_cores(c)]

    def split(self, v, which="x"):
        """Per-system views of a packed vector."""
        off = self.x_offsets if which == "x" else self.b_offsets
        return [v[int(off[i]):int(off[i + 1])] for i in range(self.count)]

    def close(self):
        if getattr(self, "_h", None):
            load_library().tacta_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["cta_solve", "ta_solve", "ta_minnorm", "residual_static", "aux_solve", "Plan", "CSR", "Batch",
           "load_library",
           "make_options", "TactaError", "EXPORTS", "LIB_PATH", "BATCH_FP64", "BATCH_FP32", "BATCH_BF16"]
