"""Python binding of the C ABI in include/dm.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: arrays are passed by pointer to libdm_gb300.so.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA); they
must be float64 and C-contiguous with the layouts of include/dm.h:
A, B, C as [N, m, m], b and x as [N, m, nrhs].

The library must have been built (``paper_1505_06864_gb300.build.build()`` or
``__graft_entry__.build()``); loading raises if it is missing, there is no
other code path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

DM_OK, DM_PENDING = 0, 1
DM_EINVAL, DM_ENOMEM, DM_ESINGULAR, DM_ENOTCONV = -1, -2, -3, -4
DM_EAGAIN, DM_ECUDA, DM_ESTATE, DM_ETIMEOUT = -5, -6, -7, -8
DM_FP64, DM_FP32, DM_TF32, DM_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": DM_FP64, "fp32": DM_FP32, "tf32": DM_TF32, "bf16x3": DM_BF16X3}
_NAMES = {0: "DM_OK", 1: "DM_PENDING", -1: "DM_EINVAL", -2: "DM_ENOMEM", -3: "DM_ESINGULAR",
          -4: "DM_ENOTCONV", -5: "DM_EAGAIN", -6: "DM_ECUDA", -7: "DM_ESTATE", -8: "DM_ETIMEOUT"}


class DMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class dm_plan_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("m", ctypes.c_int), ("nrhs", ctypes.c_int), ("P", ctypes.c_int),
                ("levels", ctypes.c_int), ("P2", ctypes.c_int), ("precision", ctypes.c_int),
                ("count", ctypes.c_int), ("last_iters", ctypes.c_int), ("max_rows", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("last_relres", ctypes.c_double),
                ("last_correction", ctypes.c_double), ("factor_flops", ctypes.c_double),
                ("solve_flops", ctypes.c_double), ("residual_mode", ctypes.c_int),
                ("residual_tc_systems", ctypes.c_int), ("J", ctypes.c_int)]


class dm_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} not found: build it first (paper_1505_06864_gb300.build.build())")
        L = ctypes.CDLL(LIB)
        P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
        sig = {
            "dm_plan": (I, [ctypes.POINTER(P), I, I, I, I, I, I]),
            "dm_plan_batch": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), ctypes.POINTER(I),
                                  ctypes.POINTER(I), I]),
            "dm_plan_tune": (I, [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "dm_plan_ex": (I, [ctypes.POINTER(P), I, I, I, I, I, I, I]),
            "dm_plan_inside": (I, [ctypes.POINTER(P), I, I, I, I, I, I, I]),
            "dm_plan_complex": (I, [ctypes.POINTER(P), I, I, I, I, I, I]),
            "dm_factor_complex": (I, [P, P, P, P]),
            "dm_solve_complex": (I, [P, P, P, ctypes.POINTER(D)]),
            "dm_partition_sizes": (I, [I, I, I, I, I, ctypes.POINTER(I)]),
            "dm_autotune": (I, [I, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
            "dm_autotune_ex": (I, [I, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                   ctypes.POINTER(D)]),
            "dm_tuned": (I, [I, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "dm_factor": (I, [P, P, P, P]),
            "dm_solve": (I, [P, P, P, ctypes.POINTER(D)]),
            "dm_solve_last": (I, [P, P, P]),
            "dm_set_stream": (I, [P, P]),
            "dm_set_refinement": (I, [P, D, I]),
            "dm_set_residual": (I, [P, I]),
            "dm_residual": (I, [P, P, P, P, ctypes.POINTER(D)]),
            "dm_set_borrow_inputs": (I, [P, I]),
            "dm_set_side_stream": (I, [P, I]),
            "dm_plan_query": (I, [P, ctypes.POINTER(dm_plan_info)]),
            "dm_profile": (I, [P, I, ctypes.POINTER(dm_profile_entry), I, ctypes.POINTER(I)]),
            "dm_launch_count": (ctypes.c_longlong, [P]),
            "dm_solve_noalloc": (I, [I, I, I, I, P, P, P, P, P, P]),
            "dm_submit": (I, [P, P, P, ctypes.POINTER(ctypes.c_uint64)]),
            "dm_submit_system": (I, [P, P, P, P, P, P, ctypes.POINTER(ctypes.c_uint64)]),
            "dm_submit_cols": (I, [P, P, P, I, ctypes.POINTER(ctypes.c_uint64)]),
            "dm_serve_budget": (I, [D]),
            "dm_serve_stats": (I, [ctypes.POINTER(ctypes.c_longlong)]),
            "dm_poll": (I, [ctypes.c_uint64, ctypes.POINTER(I), ctypes.POINTER(D)]),
            "dm_poll_times": (I, [ctypes.c_uint64, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D)]),
            "dm_serve_slots": (I, [I]),
            "dm_peak_probe": (I, [I, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
            "dm_destroy": (V, [P]),
            "dm_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def dm_last_error() -> str:
    return lib().dm_last_error().decode()


def _check(rc, allow=(DM_OK,)):
    if rc not in allow:
        raise DMError(rc, dm_last_error())
    return rc


def _ptr(a, writable=False):
    """Raw pointer of a float64 C-contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be float64 and C-contiguous")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("output array is read-only")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be float64 and contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _ptrc(a, writable=False):
    """Raw pointer of a complex128 C-contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("complex arrays must be complex128 and C-contiguous")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("output array is read-only")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.complex128 or not a.is_contiguous():
            raise ValueError("complex tensors must be complex128 and contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def dm_plan_complex(N, m, nrhs, P=0, levels=0, precision=DM_FP64):
    """Plan a complex system (solved through its real embedding of block size 2m)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = ctypes.c_void_p()
    _check(lib().dm_plan_complex(ctypes.byref(h), int(N), int(m), int(nrhs), int(P), int(levels), int(precision)))
    return h


def dm_factor_complex(plan, A, B, C):
    return _check(lib().dm_factor_complex(plan, _ptrc(A), _ptrc(B), _ptrc(C)))


def dm_solve_complex(plan, b, x, allow_notconv=False):
    rel = ctypes.c_double(0.0)
    rc = lib().dm_solve_complex(plan, _ptrc(b), _ptrc(x, True), ctypes.byref(rel))
    _check(rc, (DM_OK, DM_ENOTCONV) if allow_notconv else (DM_OK,))
    return rel.value


def dm_plan(N, m, nrhs, P=0, levels=0, precision=DM_FP64):
    """Create a plan; returns an opaque handle (free with dm_destroy)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = ctypes.c_void_p()
    _check(lib().dm_plan(ctypes.byref(h), int(N), int(m), int(nrhs), int(P), int(levels), int(precision)))
    return h


DM_PLAN_EQUAL_TIME = 1
DM_PLAN_FP64_FMA = 2
DM_PLAN_FP64_INV_COLUMN = 4


def dm_plan_ex(N, m, nrhs, P=0, levels=0, precision=DM_FP64, flags=0):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = ctypes.c_void_p()
    _check(lib().dm_plan_ex(ctypes.byref(h), int(N), int(m), int(nrhs), int(P), int(levels), int(precision),
                            int(flags)))
    return h


def dm_plan_inside(N, m, nrhs, M, J, outer_levels=1, precision=DM_FP64):
    """DM with M subsystems, each solved by DM with J sub-subsystems (Section 4.2.2)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = ctypes.c_void_p()
    _check(lib().dm_plan_inside(ctypes.byref(h), int(N), int(m), int(nrhs), int(M), int(J), int(outer_levels),
                                int(precision)))
    return h


def dm_partition_sizes(N, m, nrhs, P, flags=0):
    """Subsystem sizes the planner uses (host only)."""
    Pe = dm_plan_tune(N, m, nrhs, P, 1)[0]
    out = (ctypes.c_int * Pe)()
    _check(lib().dm_partition_sizes(int(N), int(m), int(nrhs), int(P), int(flags), out))
    return list(out)


def dm_plan_batch(Ns, ms, rs, precision=DM_FP64):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    n = len(Ns)
    arr = lambda v: (ctypes.c_int * n)(*[int(x) for x in v])
    h = ctypes.c_void_p()
    _check(lib().dm_plan_batch(ctypes.byref(h), n, arr(Ns), arr(ms), arr(rs), int(precision)))
    return h


def dm_plan_tune(N, m, nrhs, P=0, levels=0):
    """(P, levels, P2) that dm_plan would use; host only, no GPU needed."""
    p, lv, p2 = ctypes.c_int(P), ctypes.c_int(levels), ctypes.c_int(0)
    _check(lib().dm_plan_tune(int(N), int(m), int(nrhs), ctypes.byref(p), ctypes.byref(lv), ctypes.byref(p2)))
    return p.value, lv.value, p2.value


def dm_autotune(N, m, nrhs, precision=DM_FP64):
    """(P, levels, ms) of the fastest measured decomposition for this shape."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    p, lv, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib().dm_autotune(int(N), int(m), int(nrhs), int(precision), ctypes.byref(p), ctypes.byref(lv),
                             ctypes.byref(ms)))
    return p.value, lv.value, ms.value


def dm_autotune_ex(N, m, nrhs, precision=DM_FP64):
    """(P, levels, flags, ms): dm_autotune, then the kernel variants timed at
    that choice; flags are the fastest variant's plan flags."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    p, lv, fl, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib().dm_autotune_ex(int(N), int(m), int(nrhs), int(precision), ctypes.byref(p), ctypes.byref(lv),
                                ctypes.byref(fl), ctypes.byref(ms)))
    return p.value, lv.value, fl.value, ms.value


def dm_tuned(N, m, nrhs, precision=DM_FP64):
    """(P, levels, flags) stored by the tuner for this shape; raises DMError if none."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    p, lv, fl = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().dm_tuned(int(N), int(m), int(nrhs), int(precision), ctypes.byref(p), ctypes.byref(lv),
                          ctypes.byref(fl)))
    return p.value, lv.value, fl.value


def dm_factor(plan, A, B, C):
    return _check(lib().dm_factor(plan, _ptr(A), _ptr(B), _ptr(C)))


def dm_solve(plan, b, x, count=1, allow_notconv=False):
    """Solve into x (preallocated, same shape as b); returns the relative
    residual(s) max_c ||b - T x||/||b|| (a float, or a list for batch plans)."""
    rel = (ctypes.c_double * max(1, count))()
    rc = lib().dm_solve(plan, _ptr(b), _ptr(x, True), rel)
    _check(rc, (DM_OK, DM_ENOTCONV) if allow_notconv else (DM_OK,))
    return rel[0] if count == 1 else list(rel)


DM_RESIDUAL_FP64 = 0
DM_RESIDUAL_SLICED = 1
DM_RESIDUAL_AUTO = 2
RESIDUAL_MODES = {"fp64": DM_RESIDUAL_FP64, "sliced": DM_RESIDUAL_SLICED, "auto": DM_RESIDUAL_AUTO}


def dm_set_residual(plan, mode):
    """Residual method: "fp64" (CUDA-core float64), "sliced" (exact digit
    products on the tensor cores, float64-accurate) or "auto" (sliced where
    faster)."""
    if isinstance(mode, str):
        mode = RESIDUAL_MODES[mode]
    return _check(lib().dm_set_residual(plan, int(mode)))


def dm_residual(plan, x, b, r):
    """r = b - T x with the plan's blocks (after dm_factor); returns max over
    columns of ||r|| / ||b||."""
    rel = ctypes.c_double(0.0)
    _check(lib().dm_residual(plan, _ptr(x), _ptr(b), _ptr(r, True), ctypes.byref(rel)))
    return rel.value


def dm_solve_last(plan, b_last, x_last):
    """x_N for a right-hand side that is zero except its last block row b_last."""
    return _check(lib().dm_solve_last(plan, _ptr(b_last), _ptr(x_last, True)))


def dm_set_stream(plan, stream):
    """stream: a torch.cuda.Stream, an int handle, or None for the plan's own."""
    h = getattr(stream, "cuda_stream", stream)
    return _check(lib().dm_set_stream(plan, ctypes.c_void_p(h) if h else None))


def dm_set_borrow_inputs(plan, enable=True):
    return _check(lib().dm_set_borrow_inputs(plan, 1 if enable else 0))


def dm_set_side_stream(plan, enable=True):
    return _check(lib().dm_set_side_stream(plan, 1 if enable else 0))


def dm_set_refinement(plan, tol, max_iters):
    return _check(lib().dm_set_refinement(plan, float(tol), int(max_iters)))


def dm_plan_query(plan) -> dict:
    info = dm_plan_info()
    _check(lib().dm_plan_query(plan, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in dm_plan_info._fields_}


def dm_profile(plan, enable=True):
    """Per-kernel-class sums since the last call (launches, ms, flops, bytes),
    keyed by class name ("fwd_factor") for the top level and "name@d" for the
    supplementary system at recursion depth d; then clears them and switches
    event timing on or off."""
    buf = (dm_profile_entry * 64)()
    n = ctypes.c_int(0)
    _check(lib().dm_profile(plan, 1 if enable else 0, buf, 64, ctypes.byref(n)))
    return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, flops=buf[i].flops,
                                       bytes=buf[i].bytes) for i in range(n.value)}


def dm_launch_count(plan) -> int:
    return int(lib().dm_launch_count(plan))


def dm_solve_noalloc(N, m, nrhs, P, A, B, C, b, x, stream=None):
    """Factor + solve one system in the library's static device workspace
    (no allocation).  All arrays must be CUDA tensors of the current device;
    x must not overlap b.  Host arrays are refused here, before the call."""
    for name, a in (("A", A), ("B", B), ("C", C), ("b", b), ("x", x)):
        if not (hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)):
            raise DMError(DM_EINVAL, f"dm_solve_noalloc: {name} must be a CUDA tensor, not {type(a).__name__}")
    h = getattr(stream, "cuda_stream", stream)
    return _check(lib().dm_solve_noalloc(int(N), int(m), int(nrhs), int(P), _ptr(A), _ptr(B), _ptr(C),
                                         _ptr(b), _ptr(x, True), ctypes.c_void_p(h) if h else None))


def dm_submit(plan, b, x):
    """Queue a solve of b on the plan's resident factors; returns a ticket."""
    t = ctypes.c_uint64(0)
    _check(lib().dm_submit(plan, _ptr(b), _ptr(x, True), ctypes.byref(t)))
    return t.value


def dm_submit_system(plan, A, B, C, b, x):
    """Queue a factor of (A, B, C) and a solve of b; returns a ticket."""
    t = ctypes.c_uint64(0)
    _check(lib().dm_submit_system(plan, _ptr(A), _ptr(B), _ptr(C), _ptr(b), _ptr(x, True), ctypes.byref(t)))
    return t.value


def dm_poll(ticket):
    """(status, relres): status DM_PENDING while the request runs."""
    st, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib().dm_poll(ctypes.c_uint64(ticket), ctypes.byref(st), ctypes.byref(rel)))
    return st.value, rel.value


def dm_poll_times(ticket):
    """(status, relres, (t_submit, t_start, t_done)) -- times in seconds on the
    library's monotonic clock, None while DM_PENDING."""
    st, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    t = (ctypes.c_double * 3)()
    _check(lib().dm_poll_times(ctypes.c_uint64(ticket), ctypes.byref(st), ctypes.byref(rel), t))
    return st.value, rel.value, (None if st.value == DM_PENDING else (t[0], t[1], t[2]))


def dm_serve_slots(slots):
    return _check(lib().dm_serve_slots(int(slots)))


def dm_submit_cols(plan, b, x, ncols):
    """Queue a solve of ncols columns ([N][m][ncols]) on the plan's resident
    factors; narrow requests queued on one plan share one solve."""
    t = ctypes.c_uint64(0)
    _check(lib().dm_submit_cols(plan, _ptr(b), _ptr(x, True), int(ncols), ctypes.byref(t)))
    return t.value


def dm_serve_budget(seconds):
    """Latency budget for admission (0: none); refused submits raise DMError(DM_EAGAIN)."""
    return _check(lib().dm_serve_budget(float(seconds)))


def dm_serve_stats():
    """dict(admitted, refused, runs, merged) since the process started."""
    out = (ctypes.c_longlong * 4)()
    _check(lib().dm_serve_stats(out))
    return dict(admitted=out[0], refused=out[1], runs=out[2], merged=out[3])


DM_PROBE_FP64, DM_PROBE_FP32, DM_PROBE_TF32, DM_PROBE_BF16 = 0, 1, 2, 3


def dm_peak_probe(kind, repeat=3):
    """(TFLOP/s, ms) of the best of `repeat` timed launches of the probe kernel."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().dm_peak_probe(int(kind), int(repeat), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def dm_destroy(plan):
    if plan:
        lib().dm_destroy(plan)
