"""Python binding of the C ABI in ``include/ata.h`` (argument marshalling only).

Every step of C = A^t A runs in the CUDA library ``_lib/libata.so``; this
module only converts torch tensors / numpy arrays into pointers, sizes and a
stream handle.  PyTorch supplies device memory and streams.  If the library
is missing the import fails: there is no other code path.

Functions keep the C names (``ata_plan_create``, ``ata_execute``, ...); the
:class:`Plan` and :class:`Server` classes wrap the handles.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "ATA_F64", "ATA_F32_BF16X3", "ATA_F32_TF32", "ATA_F64_OZAKI", "ATA_STRASSEN", "ATA_WINOGRAD",
    "AtaError", "Plan", "Server", "ata_plan_query", "ata_plan_create", "ata_execute", "ata_execute_host",
    "ata_execute_host_async", "ata_plan_wait", "ata_batched_graph_kernels",
    "ata_execute_batched", "Batch", "packed_layout", "ata_plan_destroy", "ata_server_create", "ata_submit", "ata_poll", "load",
    "packed_size", "lib_path", "ata_device_bytes_held", "ata_tune",
]

ATA_F64, ATA_F32_BF16X3, ATA_F32_TF32, ATA_F64_OZAKI = 0, 1, 2, 3
ATA_STRASSEN, ATA_WINOGRAD = 0, 1
ATA_OK, ATA_EINVAL, ATA_ENOMEM, ATA_EUNSUPPORTED, ATA_ECUDA, ATA_PENDING, ATA_ETIMEOUT, ATA_EBUSY = range(8)
_STATUS = ["ATA_OK", "ATA_EINVAL", "ATA_ENOMEM", "ATA_EUNSUPPORTED", "ATA_ECUDA", "ATA_PENDING",
           "ATA_ETIMEOUT", "ATA_EBUSY"]
DTYPE_NAMES = {"f64": ATA_F64, "bf16x3": ATA_F32_BF16X3, "tf32": ATA_F32_TF32, "ozaki": ATA_F64_OZAKI}


class AtaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{_STATUS[status] if 0 <= status < len(_STATUS) else status}: {msg}")


class PlanInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("cutoff", ctypes.c_int32), ("depth", ctypes.c_int32), ("n_diag_leaves", ctypes.c_int32),
                ("n_nodes", ctypes.c_int32), ("max_strassen_levels", ctypes.c_int32),
                ("n_leaf_products", ctypes.c_int32), ("n_leaf_tiles", ctypes.c_int32),
                ("n_sum_tasks", ctypes.c_int32), ("n_combine_tasks", ctypes.c_int32),
                ("n_launches", ctypes.c_int32), ("mults", ctypes.c_int64), ("classical_mults", ctypes.c_int64),
                ("adds", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("leaf_tile_rows", ctypes.c_int32), ("leaf_tile_cols", ctypes.c_int32), ("r", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanOptions(ctypes.Structure):
    _fields_ = [("cutoff", ctypes.c_int32), ("variant", ctypes.c_int32), ("fuse_levels", ctypes.c_int32),
                ("max_strassen_levels", ctypes.c_int32), ("cta_pair", ctypes.c_int32),
                ("wait_limit_us", ctypes.c_int32)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load ``libata.so`` (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or os.environ.get("ATA_AUTOBUILD", "1") == "1":
        path = _build.build()
    lib = ctypes.CDLL(path)
    i64, i32, vp, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    sig = {
        "ata_status_string": ([i32], ctypes.c_char_p),
        "ata_last_error_message": ([], ctypes.c_char_p),
        "ata_device_bytes_held": ([], i64),
        "ata_plan_query": ([i64, i64, i32, i32, ctypes.POINTER(PlanInfo)], i32),
        "ata_plan_query_opts": ([i64, i64, i32, ctypes.POINTER(PlanOptions), ctypes.POINTER(PlanInfo)], i32),
        "ata_plan_create": ([ctypes.POINTER(vp), i64, i64, i32, i32], i32),
        "ata_plan_create_opts": ([ctypes.POINTER(vp), i64, i64, i32, ctypes.POINTER(PlanOptions)], i32),
        "ata_plan_check": ([i64, i64, i32, ctypes.POINTER(PlanOptions)], i32),
        "ata_gemm_query": ([i64, i64, i64, i32, ctypes.POINTER(PlanOptions), ctypes.POINTER(PlanInfo)], i32),
        "ata_gemm_plan_check": ([i64, i64, i64, i32, ctypes.POINTER(PlanOptions)], i32),
        "ata_gemm_plan_create": ([ctypes.POINTER(vp), i64, i64, i64, i32, ctypes.POINTER(PlanOptions)], i32),
        "ata_gemm_tn": ([vp, vp, i64, vp, i64, dp, i64, vp], i32),
        "ata_plan_get_info": ([vp, ctypes.POINTER(PlanInfo)], i32),
        "ata_tune": ([i64, i64, i32, ctypes.POINTER(PlanOptions), i32, ctypes.POINTER(PlanOptions),
                      ctypes.POINTER(ctypes.c_float)], i32),
        "ata_plan_workspace_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], i32),
        "ata_execute": ([vp, vp, i64, dp, vp], i32),
        "ata_execute_host": ([vp, vp, i64, dp, vp], i32),
        "ata_execute_host_async": ([vp, vp, i64, dp], i32),
        "ata_plan_wait": ([vp], i32),
        "ata_execute_batched": ([ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                 ctypes.POINTER(vp), vp], i32),
        "ata_plan_destroy": ([vp], None),
        "ata_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                              ctypes.POINTER(i64)], i32),
        "ata_batch_execute": ([vp, vp, dp, vp], i32),
        "ata_batch_graph_kernels": ([vp, ctypes.POINTER(ctypes.c_int32)], i32),
        "ata_batch_destroy": ([vp], None),
        "ata_execute_static_scratch": ([i64, i64, vp, i64, dp, i32, vp], i32),
        "ata_plan_device_status": ([vp, ctypes.POINTER(ctypes.c_int)], i32),
        "ata_plan_graph_kernels": ([vp, ctypes.POINTER(ctypes.c_int32)], i32),
        "ata_batched_graph_kernels": ([ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32)],
                                      i32),
        "ata_plan_enable_stage_timing": ([vp, i32], i32),
        "ata_plan_stage_times": ([vp, ctypes.POINTER(ctypes.c_float)], i32),
        "ata_server_create": ([ctypes.POINTER(vp), ctypes.c_size_t, i32, i32], i32),
        "ata_submit": ([vp, i64, i64, vp, i64, dp, ctypes.POINTER(ctypes.c_uint64)], i32),
        "ata_poll": ([vp, ctypes.c_uint64, i32], i32),
        "ata_server_stats": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(i64)], i32),
        "ata_server_destroy": ([vp], None),
        "ata_server_reset_stats": ([vp], i32),
        "ata_server_kernels": ([vp, ctypes.POINTER(i64)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(st: int):
    if st != ATA_OK:
        raise AtaError(st, load().ata_last_error_message().decode(errors="replace"))


def ata_device_bytes_held() -> int:
    """Device bytes the library holds for plans, batches and servers."""
    return int(load().ata_device_bytes_held())


def packed_size(n: int) -> int:
    return n * (n + 1) // 2


def _dtype_code(dtype) -> int:
    if isinstance(dtype, str):
        return DTYPE_NAMES[dtype]
    return int(dtype)


def _opts(cutoff=0, variant=-1, fuse_levels=-1, max_strassen_levels=-1, cta_pair=-1,
          wait_limit_us=-1) -> PlanOptions:
    return PlanOptions(int(cutoff), int(variant), int(fuse_levels), int(max_strassen_levels), int(cta_pair),
                       int(wait_limit_us))


def ata_plan_query(m: int, n: int, dtype=ATA_F64, cutoff: int = 0, **opts) -> dict:
    """Planner statistics for (m, n, dtype, cutoff) without touching a GPU."""
    info = PlanInfo()
    o = _opts(cutoff, **opts)
    _check(load().ata_plan_query_opts(m, n, _dtype_code(dtype), ctypes.byref(o), ctypes.byref(info)))
    return info.as_dict()


def ata_tune(m: int, n: int, dtype=ATA_F64, candidates: int = 3, **opts) -> dict:
    """Measured tuning on the current device (``ata_tune``): returns the
    winning plan options as keyword arguments for :class:`Plan` (``cutoff``,
    ``cta_pair`` and the given ones) and ``best_ms``."""
    base = _opts(0, **opts)
    out = PlanOptions()
    ms = ctypes.c_float()
    _check(load().ata_tune(int(m), int(n), _dtype_code(dtype), ctypes.byref(base), int(candidates),
                           ctypes.byref(out), ctypes.byref(ms)))
    res = {k: getattr(out, k) for k, _ in PlanOptions._fields_}
    res["best_ms"] = ms.value
    return res


def ata_plan_check(m: int, n: int, dtype=ATA_F64, cutoff: int = 0, **opts):
    """Host-side bounds and coverage check of the plan (raises AtaError)."""
    o = _opts(cutoff, **opts)
    _check(load().ata_plan_check(m, n, _dtype_code(dtype), ctypes.byref(o)))


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A plan handle: ``Plan(m, n, dtype, cutoff)`` then ``plan(A, C)``."""

    def __init__(self, m: int, n: int, dtype=ATA_F64, cutoff: int = 0, **opts):
        self.m, self.n, self.dtype = int(m), int(n), _dtype_code(dtype)
        h = ctypes.c_void_p()
        o = _opts(cutoff, **opts)
        _check(load().ata_plan_create_opts(ctypes.byref(h), self.m, self.n, self.dtype, ctypes.byref(o)))
        self.handle = h

    @property
    def info(self) -> dict:
        info = PlanInfo()
        _check(load().ata_plan_get_info(self.handle, ctypes.byref(info)))
        return info.as_dict()

    @property
    def in_dtype(self):
        import torch
        return torch.float64 if self.dtype in (ATA_F64, ATA_F64_OZAKI) else torch.float32

    def device_status(self) -> int:
        """Error word of the plan's tensor-core kernels (0 = none); synchronises."""
        c = ctypes.c_int()
        _check(load().ata_plan_device_status(self.handle, ctypes.byref(c)))
        return c.value

    def graph_kernels(self) -> int:
        """Kernel launches one execution makes (nodes of the captured graph)."""
        k = ctypes.c_int32()
        _check(load().ata_plan_graph_kernels(self.handle, ctypes.byref(k)))
        return k.value

    def enable_stage_timing(self, enable: bool = True):
        _check(load().ata_plan_enable_stage_timing(self.handle, int(enable)))

    def stage_times(self) -> dict:
        """Milliseconds of the split, prep, leaf and combine stages of the
        last (completed) execution; needs enable_stage_timing()."""
        ms = (ctypes.c_float * 4)()
        _check(load().ata_plan_stage_times(self.handle, ms))
        return {"split_ms": ms[0], "prep_ms": ms[1], "leaf_ms": ms[2], "combine_ms": ms[3]}

    def __call__(self, A, C=None, stream=None):
        return ata_execute(self, A, C, stream)

    def close(self):
        if getattr(self, "handle", None):
            load().ata_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ata_plan_create(m: int, n: int, dtype=ATA_F64, cutoff: int = 0, **opts) -> Plan:
    return Plan(m, n, dtype, cutoff, **opts)


class GemmPlan(Plan):
    """A general-product plan: ``GemmPlan(m, p, r, dtype, cutoff)`` then
    ``plan(X, Y, C)`` for C = X^t Y (X: m x p, Y: m x r, C: p x r FP64)."""

    def __init__(self, m: int, p: int, r: int, dtype=ATA_F64, cutoff: int = 0, **opts):
        self.m, self.n, self.r, self.dtype = int(m), int(p), int(r), _dtype_code(dtype)
        h = ctypes.c_void_p()
        o = _opts(cutoff, **opts)
        _check(load().ata_gemm_plan_create(ctypes.byref(h), self.m, self.n, self.r, self.dtype, ctypes.byref(o)))
        self.handle = h

    def __call__(self, X, Y, C=None, stream=None):
        return ata_gemm_tn(self, X, Y, C, stream)


def ata_gemm_plan_create(m: int, p: int, r: int, dtype=ATA_F64, cutoff: int = 0, **opts) -> GemmPlan:
    return GemmPlan(m, p, r, dtype, cutoff, **opts)


def ata_gemm_query(m: int, p: int, r: int, dtype=ATA_F64, cutoff: int = 0, **opts) -> dict:
    info = PlanInfo()
    o = _opts(cutoff, **opts)
    _check(load().ata_gemm_query(m, p, r, _dtype_code(dtype), ctypes.byref(o), ctypes.byref(info)))
    return info.as_dict()


def ata_gemm_plan_check(m: int, p: int, r: int, dtype=ATA_F64, cutoff: int = 0, **opts):
    """Host-side bounds and coverage check of a general-product plan (raises AtaError)."""
    o = _opts(cutoff, **opts)
    _check(load().ata_gemm_plan_check(m, p, r, _dtype_code(dtype), ctypes.byref(o)))


def _operand_ld(T, rows, cols, name, in_dtype):
    if not T.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if T.dtype != in_dtype:
        raise TypeError(f"{name} must be {in_dtype} for this plan")
    if T.dim() != 2 or tuple(T.shape) != (rows, cols):
        raise ValueError(f"{name} must be {rows} x {cols}")
    if rows > 0 and cols > 0 and T.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    return max(T.stride(0), cols, 1) if rows > 1 else max(cols, 1)


def ata_gemm_tn(plan: GemmPlan, X, Y, C=None, stream=None):
    """C = X^t Y on the GPU (X: m x p, Y: m x r row-major CUDA tensors; C a
    p x r float64 CUDA tensor, allocated when None).  Asynchronous on `stream`."""
    import torch
    ldx = _operand_ld(X, plan.m, plan.n, "X", plan.in_dtype)
    ldy = _operand_ld(Y, plan.m, plan.r, "Y", plan.in_dtype)
    if C is None:
        C = torch.empty((plan.n, plan.r), dtype=torch.float64, device=X.device)
    if C.dtype != torch.float64 or tuple(C.shape) != (plan.n, plan.r) or (plan.n > 0 and plan.r > 0 and C.stride(1) != 1):
        raise ValueError("C must be a row-major float64 tensor of p x r")
    ldc = max(C.stride(0), plan.r, 1) if plan.n > 1 else max(plan.r, 1)
    _check(load().ata_gemm_tn(plan.handle, ctypes.c_void_p(X.data_ptr()), ldx, ctypes.c_void_p(Y.data_ptr()), ldy,
                              ctypes.c_void_p(C.data_ptr()), ldc, _stream_handle(stream)))
    return C


def ata_plan_destroy(plan: Plan):
    plan.close()


def _check_A(plan: Plan, A):
    import torch
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.dtype != plan.in_dtype:
        raise TypeError(f"A must be {plan.in_dtype} for this plan")
    if A.dim() != 2 or tuple(A.shape) != (plan.m, plan.n):
        raise ValueError(f"A must be {plan.m} x {plan.n}")
    if plan.m > 0 and plan.n > 0 and A.stride(1) != 1:
        raise ValueError("A must be row-major (unit column stride)")
    return max(A.stride(0), plan.n, 1) if plan.m > 1 else max(plan.n, 1)


def ata_execute(plan: Plan, A, C=None, stream=None):
    """C_packed = A^t A on the GPU; A (m x n, row-major CUDA tensor) and the
    packed FP64 output C (allocated when None).  Asynchronous on `stream`."""
    import torch
    lda = _check_A(plan, A)
    if C is None:
        C = torch.empty(packed_size(plan.n), dtype=torch.float64, device=A.device)
    if C.dtype != torch.float64 or C.numel() != packed_size(plan.n) or not C.is_contiguous():
        raise ValueError("C must be a contiguous float64 tensor of n(n+1)/2 entries")
    _check(load().ata_execute(plan.handle, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(C.data_ptr()),
                              _stream_handle(stream)))
    return C


def ata_execute_host(plan: Plan, A, C=None, stream=None):
    """End to end from host memory (numpy array or CPU tensor, pinned or not)."""
    import numpy as np
    A_np = A.numpy() if hasattr(A, "numpy") and not isinstance(A, np.ndarray) else A
    want = np.float64 if plan.dtype in (ATA_F64, ATA_F64_OZAKI) else np.float32
    if A_np.dtype != want or A_np.shape != (plan.m, plan.n) or not A_np.flags.c_contiguous:
        raise ValueError(f"A must be a C-contiguous {want.__name__} array of shape ({plan.m}, {plan.n})")
    if C is None:
        C = np.empty(packed_size(plan.n), dtype=np.float64)
    C_np = C.numpy() if hasattr(C, "numpy") and not isinstance(C, np.ndarray) else C
    if C_np.dtype != np.float64 or C_np.size != packed_size(plan.n) or not C_np.flags.c_contiguous:
        raise ValueError("C must be a contiguous float64 array of n(n+1)/2 entries")
    _check(load().ata_execute_host(plan.handle, ctypes.c_void_p(A_np.ctypes.data), max(plan.n, 1),
                                   ctypes.c_void_p(C_np.ctypes.data), _stream_handle(stream)))
    return C


def ata_batched_graph_kernels(plans, As) -> int:
    """Kernel launches one ata_execute_batched(plans, As) makes (after it has run)."""
    count = len(plans)
    ph = (ctypes.c_void_p * count)(*[p.handle for p in plans])
    ld = (ctypes.c_int64 * count)(*[_check_A(p, A) for p, A in zip(plans, As)])
    k = ctypes.c_int32()
    _check(load().ata_batched_graph_kernels(ph, count, ld, ctypes.byref(k)))
    return k.value


def ata_execute_host_async(plan: Plan, A, C=None):
    """Pipelined end to end from host memory: queues the copy-in, execution
    and copy-out and returns C at once.  A must stay unmodified, and C
    unread, until ata_plan_wait(plan); both should be pinned."""
    import numpy as np
    A_np = A.numpy() if hasattr(A, "numpy") and not isinstance(A, np.ndarray) else A
    want = np.float64 if plan.dtype in (ATA_F64, ATA_F64_OZAKI) else np.float32
    if A_np.dtype != want or A_np.shape != (plan.m, plan.n) or not A_np.flags.c_contiguous:
        raise ValueError(f"A must be a C-contiguous {want.__name__} array of shape ({plan.m}, {plan.n})")
    if C is None:
        C = np.empty(packed_size(plan.n), dtype=np.float64)
    C_np = C.numpy() if hasattr(C, "numpy") and not isinstance(C, np.ndarray) else C
    if C_np.dtype != np.float64 or C_np.size != packed_size(plan.n) or not C_np.flags.c_contiguous:
        raise ValueError("C must be a contiguous float64 array of n(n+1)/2 entries")
    _check(load().ata_execute_host_async(plan.handle, ctypes.c_void_p(A_np.ctypes.data), max(plan.n, 1),
                                         ctypes.c_void_p(C_np.ctypes.data)))
    return C


def ata_plan_wait(plan: Plan):
    """Wait for every call queued by ata_execute_host_async on plan."""
    _check(load().ata_plan_wait(plan.handle))


def ata_execute_batched(plans, As, Cs=None, stream=None):
    """Run many plans in one queued batch (one persistent leaf launch)."""
    import torch
    count = len(plans)
    if Cs is None:
        Cs = [torch.empty(packed_size(p.n), dtype=torch.float64, device=A.device) for p, A in zip(plans, As)]
    ph = (ctypes.c_void_p * count)(*[p.handle for p in plans])
    ap = (ctypes.c_void_p * count)(*[A.data_ptr() for A in As])
    ld = (ctypes.c_int64 * count)(*[_check_A(p, A) for p, A in zip(plans, As)])
    cp = (ctypes.c_void_p * count)(*[C.data_ptr() for C in Cs])
    _check(load().ata_execute_batched(ph, count, ap, ld, cp, _stream_handle(stream)))
    return Cs


def _round_up(x: int, q: int) -> int:
    return -(-x // q) * q


def packed_layout(shapes, lda=None, elem: int = 8, align_bytes: int = 256):
    """Back-to-back layout of a batch's instances (m_i, n_i): element offsets
    of each A_i (row-major, leading dimension lda[i], default n_i) in one
    input buffer of `elem`-byte elements and of each packed C_i in one FP64
    output buffer, every instance starting on an `align_bytes` boundary.
    Returns (lda, a_offsets, c_offsets, a_numel, c_numel)."""
    shapes = [(int(m), int(n)) for m, n in shapes]
    lda = [max(n, 1) for _, n in shapes] if lda is None else [int(x) for x in lda]
    a_sizes = [(m - 1) * l + n if m > 0 and n > 0 else 0 for (m, n), l in zip(shapes, lda)]
    c_sizes = [packed_size(n) for _, n in shapes]

    def offsets(sizes, e):
        offs, off = [], 0
        for sz in sizes:
            offs.append(off)
            off += _round_up(sz, max(1, align_bytes // e))
        return offs

    a_off, c_off = offsets(a_sizes, elem), offsets(c_sizes, 8)
    a_numel = max([o + sz for o, sz in zip(a_off, a_sizes)], default=0)
    c_numel = max([o + sz for o, sz in zip(c_off, c_sizes)], default=0)
    return lda, a_off, c_off, a_numel, c_numel


class Batch:
    """A prepared batch (``ata_batch_create``): the plans bound once to one
    packed input buffer and one packed FP64 output buffer, so that
    ``batch(A, C)`` (``ata_batch_execute``) marshals two pointers.  Without
    offsets the instances are laid out back to back, each starting on an
    ``align_bytes`` boundary, A_i row-major with leading dimension n_i."""

    def __init__(self, plans, a_offsets=None, c_offsets=None, lda=None, align_bytes: int = 256):
        self.plans = list(plans)  # the plans must outlive the batch
        count = len(self.plans)
        self.elem = 8 if count == 0 or self.plans[0].dtype in (ATA_F64, ATA_F64_OZAKI) else 4
        shapes = [(p.m, p.n) for p in self.plans]
        self.lda, a_off, c_off, _, _ = packed_layout(shapes, lda, self.elem, align_bytes)
        self.a_offsets = a_off if a_offsets is None else [int(x) for x in a_offsets]
        self.c_offsets = c_off if c_offsets is None else [int(x) for x in c_offsets]
        if len(self.lda) != count or len(self.a_offsets) != count or len(self.c_offsets) != count:
            raise ValueError("plans, lda and offsets must have the same length")
        a_sizes = [(m - 1) * l + n if m > 0 and n > 0 else 0 for (m, n), l in zip(shapes, self.lda)]
        self.a_numel = max([o + sz for o, sz in zip(self.a_offsets, a_sizes)], default=0)
        self.c_numel = max([o + packed_size(n) for o, (_, n) in zip(self.c_offsets, shapes)], default=0)
        ph = (ctypes.c_void_p * max(count, 1))(*[p.handle for p in self.plans])
        ld = (ctypes.c_int64 * max(count, 1))(*self.lda)
        ao = (ctypes.c_int64 * max(count, 1))(*self.a_offsets)
        co = (ctypes.c_int64 * max(count, 1))(*self.c_offsets)
        h = ctypes.c_void_p()
        _check(load().ata_batch_create(ctypes.byref(h), ph, count, ld, ao, co))
        self.handle = h

    @property
    def in_dtype(self):
        import torch
        return torch.float64 if self.elem == 8 else torch.float32

    def input_views(self, A):
        """Instance i's m_i x n_i view (leading dimension lda[i]) of the packed input A."""
        return [A.as_strided((p.m, p.n), (l, 1), o) for p, l, o in zip(self.plans, self.lda, self.a_offsets)]

    def output_views(self, C):
        """Instance i's packed n_i(n_i+1)/2 result inside the packed output C."""
        return [C[o:o + packed_size(p.n)] for p, o in zip(self.plans, self.c_offsets)]

    def execute(self, A, C=None, stream=None):
        import torch
        if not A.is_cuda or A.dtype != self.in_dtype or not A.is_contiguous() or A.numel() < self.a_numel:
            raise ValueError(f"A must be a contiguous {self.in_dtype} CUDA tensor of >= {self.a_numel} elements")
        if C is None:
            C = torch.empty(self.c_numel, dtype=torch.float64, device=A.device)
        if not C.is_cuda or C.dtype != torch.float64 or not C.is_contiguous() or C.numel() < self.c_numel:
            raise ValueError(f"C must be a contiguous float64 CUDA tensor of >= {self.c_numel} elements")
        _check(load().ata_batch_execute(self.handle, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                                        _stream_handle(stream)))
        return C

    __call__ = execute

    def graph_kernels(self) -> int:
        """Kernel launches one execution makes (nodes of the captured graphs)."""
        k = ctypes.c_int32()
        _check(load().ata_batch_graph_kernels(self.handle, ctypes.byref(k)))
        return k.value

    def close(self):
        if getattr(self, "handle", None):
            load().ata_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ata_execute_static_scratch(A, C=None, cutoff: int = 64, stream=None):
    """FP64 C_packed = A^t A with no device allocation: scratch comes from a
    64 MiB array inside the library, shared by every call (calls that overlap
    on the GPU race).  A is an m x n float64 CUDA tensor, row-major."""
    import torch
    if not A.is_cuda or A.dtype != torch.float64 or A.dim() != 2:
        raise ValueError("A must be a 2-D float64 CUDA tensor")
    m, n = A.shape
    if m > 0 and n > 0 and A.stride(1) != 1:
        raise ValueError("A must be row-major (unit column stride)")
    lda = max(A.stride(0), n, 1) if m > 1 else max(n, 1)
    if C is None:
        C = torch.empty(packed_size(n), dtype=torch.float64, device=A.device)
    _check(load().ata_execute_static_scratch(m, n, ctypes.c_void_p(A.data_ptr()), lda,
                                             ctypes.c_void_p(C.data_ptr()), int(cutoff), _stream_handle(stream)))
    return C


class Server:
    """Continuous-batching server (``ata_server_create`` / ``ata_submit`` / ``ata_poll``)."""

    def __init__(self, budget_bytes: int, dtype=ATA_F32_BF16X3, max_inflight: int = 8):
        h = ctypes.c_void_p()
        _check(load().ata_server_create(ctypes.byref(h), int(budget_bytes), _dtype_code(dtype), int(max_inflight)))
        self.handle = h
        self.dtype = _dtype_code(dtype)
        self._keep = {}

    def submit(self, A, C) -> int:
        t = ctypes.c_uint64()
        m, n = A.shape
        _check(load().ata_submit(self.handle, m, n, ctypes.c_void_p(A.data_ptr()), max(A.stride(0), n, 1),
                                 ctypes.c_void_p(C.data_ptr()), ctypes.byref(t)))
        self._keep[t.value] = (A, C)
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0) -> int:
        st = load().ata_poll(self.handle, ticket, int(timeout_us))
        if st == ATA_OK:
            self._keep.pop(ticket, None)
        elif st not in (ATA_PENDING, ATA_ETIMEOUT):
            self._keep.pop(ticket, None)
            _check(st)
        return st

    def stats(self) -> dict:
        p50, p99, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(load().ata_server_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n)))
        return {"p50_us": p50.value, "p99_us": p99.value, "completed": n.value}

    def reset_stats(self):
        _check(load().ata_server_reset_stats(self.handle))

    def kernels(self) -> int:
        """Kernel launches of the executions queued since creation or the last reset."""
        k = ctypes.c_int64()
        _check(load().ata_server_kernels(self.handle, ctypes.byref(k)))
        return k.value

    def close(self):
        if getattr(self, "handle", None):
            load().ata_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ata_server_create(budget_bytes: int, dtype=ATA_F32_BF16X3, max_inflight: int = 8) -> Server:
    return Server(budget_bytes, dtype, max_inflight)


def ata_submit(server: Server, A, C) -> int:
    return server.submit(A, C)


def ata_poll(server: Server, ticket: int, timeout_us: int = 0) -> int:
    return server.poll(ticket, timeout_us)
