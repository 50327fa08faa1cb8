"""Python binding of libfapath: f(A) b by multi-shift BiCGstab(l) on a GB300.

Argument marshalling only.  Every step of the computation runs in the CUDA
kernels of `libfapath.so` behind the C-ABI declared in `include/fapath.h`;
PyTorch provides device memory and the current CUDA stream.  There is no CPU
fallback: importing works without a GPU, but every call needs the built
library and a CUDA device, and raises otherwise.

Fields are complex128 tensors in the canonical layouts
    spinor (T, Z, Y, X, 4, 3)        gauge (T, Z, Y, X, 4, 3, 3)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfapath.so")

FA_OK, FA_EINVAL, FA_ENOMEM, FA_ECUDA, FA_EBREAKDOWN, FA_ENOCONV, FA_ENONFINITE, FA_ETIMEOUT, \
    FA_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
SINGLE, DOUBLE, PSEUDO = 0, 1, 2
F64, F32, MIXED, DF, MIXED_DF = 0, 1, 2, 3, 4
_PREC = {"f64": F64, "f32": F32, "mixed": MIXED, "df": DF, "mixed_df": MIXED_DF,
         F64: F64, F32: F32, MIXED: MIXED, DF: DF, MIXED_DF: MIXED_DF}
_MODE = {"single": SINGLE, "double": DOUBLE, "pseudo": PSEUDO, SINGLE: SINGLE, DOUBLE: DOUBLE,
         PSEUDO: PSEUDO}

EXPORTS = (
    "fa_create", "fa_destroy", "fa_set_gauge", "fa_set_params", "fa_estimate_scale",
    "fa_set_poles", "fa_neuberger_poles", "fa_zolotarev_poles", "fa_apply_dw", "fa_apply_A", "fa_solve_multishift",
    "fa_apply_f", "fa_apply_sign", "fa_apply_overlap", "fa_apply_sign_deflated", "fa_apply_f_host", "fa_sync", "fa_launch_count", "fa_hop_timing",
    "fa_hop_timing_split", "fa_hop_timing_reset", "fa_device_bytes", "fa_status_string", "fa_last_error", "fa_version",
    "fa_apply_A_noalloc", "fa_grad", "fa_apply_f_batched", "fa_share_gauge",
    "fa_set_hop_shape", "fa_get_hop_shape", "fa_autotune", "fa_autotune_batched",
    "fa_eigs_smallest", "fa_trace_start", "fa_trace_stop", "fa_fp32_issue_rate",
)

# FP32 sweep launch shapes (fa_hop_shape)
SHAPE_AUTO, SHAPE_WIDE, SHAPE_NARROW = 0, 1, 2
_SHAPE = {"auto": SHAPE_AUTO, "wide": SHAPE_WIDE, "narrow": SHAPE_NARROW,
          SHAPE_AUTO: SHAPE_AUTO, SHAPE_WIDE: SHAPE_WIDE, SHAPE_NARROW: SHAPE_NARROW}


class FAError(RuntimeError):
    def __init__(self, status, where):
        lib = load_library()
        msg = lib.fa_status_string(status).decode()
        detail = lib.fa_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


class SolverParams(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int), ("tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("switch_resid", ctypes.c_double), ("flags", ctypes.c_int),
                ("store_gb", ctypes.c_double), ("reliable_every", ctypes.c_int),
                ("shift_chunk", ctypes.c_int)]


class SolverStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("switch_outer", ctypes.c_int), ("ns", ctypes.c_int),
                ("iters_per_shift", ctypes.c_int * 64), ("resid_recurrence", ctypes.c_double),
                ("n_mv", ctypes.c_longlong), ("n_dot", ctypes.c_longlong),
                ("n_launch", ctypes.c_longlong), ("stored_outer", ctypes.c_int),
                ("t_pass1_ms", ctypes.c_double),
                ("t_sweep_ms", ctypes.c_double), ("t_pass2_ms", ctypes.c_double)]

    def as_dict(self):
        return dict(status=self.status, outer_iters=self.outer_iters,
                    switch_outer=self.switch_outer,
                    iters_per_shift=list(self.iters_per_shift[:self.ns]),
                    resid_recurrence=self.resid_recurrence, n_mv=self.n_mv, n_dot=self.n_dot,
                    n_launch=self.n_launch, stored_outer=self.stored_outer,
                    t_pass1_ms=self.t_pass1_ms,
                    t_sweep_ms=self.t_sweep_ms, t_pass2_ms=self.t_pass2_ms)


_lib = None


def load_library(path=LIB_PATH):
    """Load libfapath.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libfapath.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "fa_create": (I, [ctypes.POINTER(P), ctypes.POINTER(I), P]),
        "fa_destroy": (I, [P]),
        "fa_set_gauge": (I, [P, P, I]),
        "fa_share_gauge": (I, [P, P]),
        "fa_set_params": (I, [P, D, D, I, D]),
        "fa_estimate_scale": (I, [P, P, I, ctypes.POINTER(D)]),
        "fa_set_poles": (I, [P, I, P, P]),
        "fa_neuberger_poles": (I, [I, P, P]),
        "fa_zolotarev_poles": (I, [I, D, P, P, ctypes.POINTER(D)]),
        "fa_apply_dw": (I, [P, P, P, I, I]),
        "fa_apply_A": (I, [P, P, P, I, I]),
        "fa_apply_A_noalloc": (I, [P, P, P, I]),
        "fa_solve_multishift": (I, [P, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_apply_f": (I, [P, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_apply_sign": (I, [P, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_apply_overlap": (I, [P, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_apply_sign_deflated": (I, [P, P, P, I, P, P, P, I, ctypes.POINTER(SolverParams),
                                       ctypes.POINTER(SolverStats)]),
        "fa_apply_f_host": (I, [P, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_apply_f_batched": (I, [P, I, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_grad": (I, [P, P, P, P, ctypes.POINTER(D), ctypes.POINTER(D), P,
                        ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
        "fa_sync": (I, [P]),
        "fa_launch_count": (LL, [P]),
        "fa_fp32_issue_rate": (I, [I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "fa_hop_timing": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(LL)]),
        "fa_hop_timing_split": (I, [P, I, I, ctypes.POINTER(D), ctypes.POINTER(LL)]),
        "fa_hop_timing_reset": (I, [P]),
        "fa_device_bytes": (I, [P, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]),
        "fa_set_hop_shape": (I, [P, I]),
        "fa_get_hop_shape": (I, [P]),
        "fa_autotune": (I, [P, I, ctypes.POINTER(D)]),
        "fa_autotune_batched": (I, [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), I]),
        "fa_eigs_smallest": (I, [P, I, I, D, I, ctypes.POINTER(SolverParams), ctypes.c_ulonglong, P, P, P,
                                 ctypes.POINTER(I), ctypes.POINTER(I)]),
        "fa_trace_start": (I, [LL]),
        "fa_trace_stop": (I, [P, LL, ctypes.POINTER(LL), ctypes.POINTER(LL)]),
        "fa_status_string": (ctypes.c_char_p, [I]),
        "fa_last_error": (ctypes.c_char_p, []),
        "fa_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def _check(status, where):
    if status != FA_OK:
        raise FAError(status, where)


def neuberger_poles(ns):
    """(omega, sigma) of Neuberger's expansion, computed by the library."""
    lib = load_library()
    om = np.empty(ns, dtype=np.float64)
    sg = np.empty(ns, dtype=np.float64)
    _check(lib.fa_neuberger_poles(ns, om.ctypes.data, sg.ctypes.data), "fa_neuberger_poles")
    return om, sg


def zolotarev_poles(ns, eps):
    """(omega, sigma, delta) of Zolotarev's expansion on [eps^2, 1], computed by the library."""
    lib = load_library()
    om = np.empty(ns, dtype=np.float64)
    sg = np.empty(ns, dtype=np.float64)
    d = ctypes.c_double()
    _check(lib.fa_zolotarev_poles(ns, float(eps), om.ctypes.data, sg.ctypes.data, ctypes.byref(d)),
           "fa_zolotarev_poles")
    return om, sg, d.value


def apply_f_batched(contexts, sources, check=True, **kw):
    """y_i = f(A_i) b_i for a list of contexts (systems of equal lattice shape
    share every kernel launch).  Returns (list of y, list of stats dicts)."""
    lib = load_library()
    n = len(contexts)
    for c, b in zip(contexts, sources):
        _spinor_check(b, c.spinor_shape, "b")
    ys = [c.empty_spinor() for c in contexts]
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in contexts])
    bs = (ctypes.c_void_p * n)(*[b.data_ptr() for b in sources])
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    p = Context.params(**kw)
    st = (SolverStats * n)()
    rc = lib.fa_apply_f_batched(hs, n, bs, yp, ctypes.byref(p), st)
    if check:
        _check(rc, "fa_apply_f_batched")
    return ys, [s.as_dict() for s in st]


def autotune_batched(contexts, reps=10):
    """Pick the launch shape of the batched multi-RHS FP32 sweep for this batch
    (fa_autotune_batched): right-hand sides per block and blocks per SM, kept in
    contexts[0].  Returns {"rhs_per_block", "min_blocks", "times_ms"}."""
    lib = load_library()
    n = len(contexts)
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in contexts])
    rpb, mb = ctypes.c_int(), ctypes.c_int()
    times = (ctypes.c_double * 14)()
    _check(lib.fa_autotune_batched(hs, n, int(reps), ctypes.byref(rpb), ctypes.byref(mb), times, 14),
           "fa_autotune_batched")
    grid = [(r, m) for r in (1, 2, 3, 4, 6, 12, 16) for m in (7, 4)]
    return {"rhs_per_block": rpb.value, "min_blocks": mb.value,
            "times_ms": {f"{r}x{m}": float(t) for (r, m), t in zip(grid, times)}}


# kernel timeline tracing (fa_trace_start / fa_trace_stop)
TRACE_KERNELS = {1: "k_update_u", 2: "k_update_r", 3: "k_gram", 4: "k_mr", 5: "k_hop_sys", 6: "k_hop_mrhs",
                 7: "k_hop_sys_rows", 8: "k_hop1_rows", 9: "k_hop1", 10: "k_hop_gram", 11: "k_reliable",
                 12: "k_gather", 13: "k_sweep", 14: "k_coef_reduce", 15: "k_advance"}
TRACE_PRECISION = {0: "f64", 1: "f32", 2: "df"}
TRACE_DTYPE = [("t_start_ns", "<u8"), ("t_end_ns", "<u8"), ("kernel", "<i4"), ("block", "<i4"), ("sm", "<i4"),
               ("grid", "<i4")]


def fp32_issue_rate(reps=5):
    """Measured FP32 instruction issue rate of the current device (fa_fp32_issue_rate):
    (thread instructions per second, ms of the best probe launch)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().fa_fp32_issue_rate(int(reps), ctypes.byref(rate), ctypes.byref(ms)), "fa_fp32_issue_rate")
    return rate.value, ms.value


def trace_start(capacity=1 << 21):
    """Turn kernel timeline tracing on for the current device (fa_trace_start)."""
    _check(load_library().fa_trace_start(int(capacity)), "fa_trace_start")


def trace_stop(capacity=1 << 21):
    """Turn tracing off; returns (records, dropped): a numpy structured array
    with the fields of fa_trace_record, and the number of records lost."""
    import numpy as np
    rec = np.zeros(int(capacity), dtype=TRACE_DTYPE)
    n, dropped = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load_library().fa_trace_stop(rec.ctypes.data, int(capacity), ctypes.byref(n), ctypes.byref(dropped)),
           "fa_trace_stop")
    return rec[: n.value], dropped.value


def trace_kernel_name(kernel):
    """'k_hop1<f32, dot>' style name of a record's kernel field."""
    base = TRACE_KERNELS.get(kernel & 0xff, str(kernel & 0xff))
    tags = [TRACE_PRECISION.get((kernel >> 8) & 3, "?")]
    if (kernel >> 10) & 1:
        tags.append("dot" if base.startswith("k_hop") else "shifts")
    return f"{base}<{', '.join(tags)}>"


def trace_launches(records):
    """Group block records into launches of one stream: sorted by entry time, a
    launch ends where a block enters after every block so far has left.
    Returns a list of dicts: kernel, name, start_ns, end_ns, blocks, grid,
    tail_ns (latest exit minus the second latest: the last block's own tail)."""
    import numpy as np
    if len(records) == 0:
        return []
    r = records[np.argsort(records["t_start_ns"], kind="stable")]
    out = []
    cur = None
    ends = []
    for x in r:
        t0, t1 = int(x["t_start_ns"]), int(x["t_end_ns"])
        if cur is None or t0 > cur["end_ns"]:
            if cur is not None:
                ends.sort()
                cur["tail_ns"] = ends[-1] - ends[-2] if len(ends) > 1 else 0
            cur = {"kernel": int(x["kernel"]), "name": trace_kernel_name(int(x["kernel"])), "start_ns": t0,
                   "end_ns": t1, "blocks": 0, "grid": int(x["grid"])}
            out.append(cur)
            ends = []
        cur["end_ns"] = max(cur["end_ns"], t1)
        cur["blocks"] += 1
        ends.append(t1)
    ends.sort()
    cur["tail_ns"] = ends[-1] - ends[-2] if len(ends) > 1 else 0
    return out


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the fapath path runs on the GPU only")
    return torch


def _spinor_check(t, shape, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128
            and t.is_contiguous() and tuple(t.shape) == shape):
        raise ValueError(f"{name}: expected a contiguous complex128 CUDA tensor of shape {shape}")
    return t


@dataclass
class Result:
    y: object
    stats: dict


class Context:
    """One lattice, gauge field and operator, bound to a CUDA stream."""

    def __init__(self, dims, stream=None):
        torch = _torch()
        self.lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        X, Y, Z, T = self.dims
        self.spinor_shape = (T, Z, Y, X, 4, 3)
        self.gauge_shape = (T, Z, Y, X, 4, 3, 3)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        _check(self.lib.fa_create(ctypes.byref(h), arr, ctypes.c_void_p(self.stream.cuda_stream)),
               "fa_create")
        self.h = h
        self.ns = 0

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.fa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_spinor(self):
        torch = _torch()
        return torch.empty(self.spinor_shape, dtype=torch.complex128, device="cuda")

    # -- setup
    def set_gauge(self, U):
        torch = _torch()
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            assert U.shape == self.gauge_shape
            _check(self.lib.fa_set_gauge(self.h, U.ctypes.data, 0), "fa_set_gauge")
        else:
            if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous()
                    and tuple(U.shape) == self.gauge_shape):
                raise ValueError("gauge field: contiguous complex128 CUDA tensor expected")
            _check(self.lib.fa_set_gauge(self.h, U.data_ptr(), 1), "fa_set_gauge")

    def share_gauge(self, owner):
        """Use owner's packed gauge field (same lattice) instead of a copy."""
        _check(self.lib.fa_share_gauge(self.h, owner.h), "fa_share_gauge")
        self._gauge_owner = owner      # keep the owner alive

    def set_params(self, mass, mu, t_bc=-1, scale=1.0):
        _check(self.lib.fa_set_params(self.h, float(mass), float(mu), int(t_bc), float(scale)),
               "fa_set_params")

    def set_poles(self, omega, sigma):
        om = np.ascontiguousarray(omega, dtype=np.float64)
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        _check(self.lib.fa_set_poles(self.h, len(om), om.ctypes.data, sg.ctypes.data), "fa_set_poles")
        self.ns = len(om)

    def estimate_scale(self, v0, iters=100):
        v0 = _spinor_check(v0, self.spinor_shape, "v0")
        out = ctypes.c_double()
        _check(self.lib.fa_estimate_scale(self.h, v0.data_ptr(), int(iters), ctypes.byref(out)),
               "fa_estimate_scale")
        return out.value

    # -- operators
    def apply_dw(self, x, dagger=False, precision="f64", out=None):
        x = _spinor_check(x, self.spinor_shape, "x")
        out = self.empty_spinor() if out is None else _spinor_check(out, self.spinor_shape, "out")
        _check(self.lib.fa_apply_dw(self.h, x.data_ptr(), out.data_ptr(), int(bool(dagger)),
                                    _PREC[precision]), "fa_apply_dw")
        return out

    def apply_A(self, x, dagger=False, precision="f64", out=None):
        x = _spinor_check(x, self.spinor_shape, "x")
        out = self.empty_spinor() if out is None else _spinor_check(out, self.spinor_shape, "out")
        _check(self.lib.fa_apply_A(self.h, x.data_ptr(), out.data_ptr(), int(bool(dagger)),
                                   _PREC[precision]), "fa_apply_A")
        return out

    # -- solvers
    @staticmethod
    def params(ell=2, tol=1e-10, max_outer=2000, mode="double", precision="f64",
               switch_resid=0.0, timing=False, hop_timing=False, store_gb=0.0, graph=False,
               reliable_every=0, fixed_iters=False, overlap=True, gram_epilogue=True, shift_chunk=0):
        return SolverParams(int(ell), float(tol), int(max_outer), _MODE[mode], _PREC[precision],
                            float(switch_resid),
                            (1 if timing else 0) | (2 if hop_timing else 0) | (4 if graph else 0)
                            | (8 if fixed_iters else 0) | (0 if overlap else 16) | (0 if gram_epilogue else 32),
                            float(store_gb), int(reliable_every), int(shift_chunk))

    def apply_f(self, b, out=None, check=True, **kw):
        b = _spinor_check(b, self.spinor_shape, "b")
        y = self.empty_spinor() if out is None else _spinor_check(out, self.spinor_shape, "out")
        p = self.params(**kw)
        st = SolverStats()
        rc = self.lib.fa_apply_f(self.h, b.data_ptr(), y.data_ptr(), ctypes.byref(p), ctypes.byref(st))
        if check:
            _check(rc, "fa_apply_f")
        return Result(y, st.as_dict())

    def apply_sign(self, b, out=None, check=True, **kw):
        """sign(g5 D_w(mu)) b = sqrt(c) g5 D_w f(A) b (Sec. 1); keywords as apply_f."""
        return self._sign_call(self.lib.fa_apply_sign, "fa_apply_sign", b, out, check, kw)

    def apply_overlap(self, b, out=None, check=True, **kw):
        """D_ov(mu) b = b + g5 sign(g5 D_w(mu)) b (Sec. 1); keywords as apply_f."""
        return self._sign_call(self.lib.fa_apply_overlap, "fa_apply_overlap", b, out, check, kw)

    def apply_sign_deflated(self, b, lam, R, Lv, overlap=False, out=None, check=True, **kw):
        """sign(H) b (or D_ov b) with k eigenpairs of H = g5 D_w treated exactly:
        lam (k complex), R and Lv (complex128 CUDA tensors of shape (k,) + the
        spinor shape: right and left eigenvectors, Lv_i^H R_j = delta_ij)."""
        b = _spinor_check(b, self.spinor_shape, "b")
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128))
        k = lam.size
        shape = (k,) + tuple(self.spinor_shape)
        for t, nm in ((R, "R"), (Lv, "Lv")):
            torch = _torch()
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128
                    and t.is_contiguous() and tuple(t.shape) == shape):
                raise ValueError(f"{nm}: expected a contiguous complex128 CUDA tensor of shape {shape}")
        y = self.empty_spinor() if out is None else _spinor_check(out, self.spinor_shape, "out")
        p = self.params(**kw)
        st = SolverStats()
        rc = self.lib.fa_apply_sign_deflated(self.h, b.data_ptr(), y.data_ptr(), k, lam.ctypes.data,
                                             R.data_ptr(), Lv.data_ptr(), int(bool(overlap)), ctypes.byref(p),
                                             ctypes.byref(st))
        if check:
            _check(rc, "fa_apply_sign_deflated")
        return Result(y, st.as_dict())

    def _sign_call(self, fn, name, b, out, check, kw):
        b = _spinor_check(b, self.spinor_shape, "b")
        y = self.empty_spinor() if out is None else _spinor_check(out, self.spinor_shape, "out")
        p = self.params(**kw)
        st = SolverStats()
        rc = fn(self.h, b.data_ptr(), y.data_ptr(), ctypes.byref(p), ctypes.byref(st))
        if check:
            _check(rc, name)
        return Result(y, st.as_dict())

    def apply_f_host(self, b, check=True, **kw):
        """b, y in host memory (numpy complex128, canonical shape)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        assert b.shape == self.spinor_shape
        y = np.empty_like(b)
        p = self.params(**kw)
        st = SolverStats()
        rc = self.lib.fa_apply_f_host(self.h, b.ctypes.data, y.ctypes.data, ctypes.byref(p),
                                      ctypes.byref(st))
        if check:
            _check(rc, "fa_apply_f_host")
        return Result(y, st.as_dict())

    def solve_multishift(self, b, **kw):
        b = _spinor_check(b, self.spinor_shape, "b")
        xs = [self.empty_spinor() for _ in range(self.ns)]
        ptrs = (ctypes.c_void_p * self.ns)(*[x.data_ptr() for x in xs])
        kw.setdefault("mode", "single")
        p = self.params(**kw)
        st = SolverStats()
        _check(self.lib.fa_solve_multishift(self.h, b.data_ptr(), ptrs, ctypes.byref(p),
                                            ctypes.byref(st)), "fa_solve_multishift")
        return Result(xs, st.as_dict())

    def grad(self, b, eta, ell=2, tol=1e-12, max_outer=4000, want_db=True, shift_chunk=0):
        """(L, dL/dU, dL/dmu, dL/db, stats) for L = Re <eta, f(A) b> (single-pass FP64
        solves; shift_chunk > 0: that many poles at a time)."""
        torch = _torch()
        b = _spinor_check(b, self.spinor_shape, "b")
        eta = _spinor_check(eta, self.spinor_shape, "eta")
        gU = torch.empty(self.gauge_shape, dtype=torch.complex128, device="cuda")
        gb = self.empty_spinor() if want_db else None
        dmu, L = ctypes.c_double(), ctypes.c_double()
        p = self.params(ell=ell, tol=tol, max_outer=max_outer, mode="single", precision="f64",
                        shift_chunk=shift_chunk)
        st = SolverStats()
        _check(self.lib.fa_grad(self.h, b.data_ptr(), eta.data_ptr(), gU.data_ptr(), ctypes.byref(dmu),
                                ctypes.byref(L), gb.data_ptr() if want_db else None, ctypes.byref(p),
                                ctypes.byref(st)), "fa_grad")
        return L.value, gU, dmu.value, gb, st.as_dict()

    def eigs_smallest(self, k, m=None, tol=1e-10, max_restarts=50, seed=1, solve_tol=1e-12, check=True, **kw):
        """The k eigenpairs of H = g5 D_w(mu) smallest in magnitude (fa_eigs_smallest):
        (lambda (k complex), R, Lv (complex128 CUDA tensors (k,) + spinor shape,
        Lv_i^H R_j = delta_ij), info dict).  tol: Ritz-pair convergence; solve_tol
        and kw: the inner solves' settings (apply_f's)."""
        torch = _torch()
        m = 2 * k + 8 if m is None else m
        shape = (k,) + tuple(self.spinor_shape)
        R = torch.empty(shape, dtype=torch.complex128, device="cuda")
        Lv = torch.empty(shape, dtype=torch.complex128, device="cuda")
        lam = np.empty(2 * k, dtype=np.float64)
        nconv, nsolve = ctypes.c_int(), ctypes.c_int()
        kw["tol"] = solve_tol
        kw.setdefault("mode", "double")
        p = self.params(**kw)
        rc = self.lib.fa_eigs_smallest(self.h, int(k), int(m), float(tol), int(max_restarts), ctypes.byref(p),
                                       int(seed), lam.ctypes.data, R.data_ptr(), Lv.data_ptr(), ctypes.byref(nconv),
                                       ctypes.byref(nsolve))
        if check:
            _check(rc, "fa_eigs_smallest")
        return lam[0::2] + 1j * lam[1::2], R, Lv, {"status": rc, "converged": nconv.value, "solves": nsolve.value}

    def sync(self):
        _check(self.lib.fa_sync(self.h), "fa_sync")

    def launch_count(self):
        return int(self.lib.fa_launch_count(self.h))

    def hop_timing(self, precision="f32", dot=None):
        """Mean event-timed ms per sweep and the count; dot: None (all sweeps),
        False (plain sweeps), True (sweeps that also form an inner product),
        "gram" (the FP32 sweep with the Gram-matrix epilogue)."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        with_dot = -1 if dot is None else (2 if dot == "gram" else int(bool(dot)))
        _check(self.lib.fa_hop_timing_split(self.h, _PREC[precision], with_dot, ctypes.byref(ms),
                                            ctypes.byref(n)), "fa_hop_timing_split")
        return ms.value, n.value

    def device_bytes(self):
        """(lattice-sized bytes, scalar bytes) of device memory the context owns."""
        f, sc = ctypes.c_ulonglong(), ctypes.c_ulonglong()
        _check(self.lib.fa_device_bytes(self.h, ctypes.byref(f), ctypes.byref(sc)), "fa_device_bytes")
        return f.value, sc.value

    def hop_timing_reset(self):
        _check(self.lib.fa_hop_timing_reset(self.h), "fa_hop_timing_reset")

    def set_hop_shape(self, shape):
        """FP32 sweep launch shape: "auto", "wide" or "narrow" (fa_set_hop_shape)."""
        _check(self.lib.fa_set_hop_shape(self.h, _SHAPE[shape]), "fa_set_hop_shape")

    def hop_shape(self):
        return int(self.lib.fa_get_hop_shape(self.h))

    def autotune(self, reps=20, cache=None):
        """Pick the fastest FP32 sweep launch shape for this lattice (fa_autotune).

        With `cache` (a JSON file path), a choice stored for the same lattice
        dimensions and GPU is applied without timing, and a new timing is stored.
        Returns {"shape": k, "times_ms": [wide, narrow] or None, "cached": bool}."""
        key = tune_key(self.dims, _device_name())
        if cache is not None:
            entry = load_tune_cache(cache).get(key)
            if entry is not None:
                self.set_hop_shape(int(entry["shape"]))
                return {"shape": int(entry["shape"]), "times_ms": entry.get("times_ms"), "cached": True}
        times = (ctypes.c_double * SHAPE_NARROW)()
        rc = self.lib.fa_autotune(self.h, int(reps), times)
        if rc < 0:
            _check(rc, "fa_autotune")
        result = {"shape": int(rc), "times_ms": [float(t) for t in times], "cached": False}
        if cache is not None:
            store_tune_cache(cache, key, {"shape": result["shape"], "times_ms": result["times_ms"]})
        return result


# ------------------------------------------------------------------ autotuner cache
def _device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "none"


def tune_key(dims, device_name, precision="f32"):
    """Cache key of an autotuned launch shape: lattice dimensions, precision, GPU."""
    return f"{'x'.join(str(int(d)) for d in dims)}|{precision}|{device_name}"


def load_tune_cache(path):
    """The autotuner cache (a JSON object), or {} when the file is absent or unreadable."""
    import json
    import os
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_tune_cache(path, key, entry):
    """Add one entry to the autotuner cache (written to a temporary file, then renamed)."""
    import json
    import os
    data = load_tune_cache(path)
    data[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
