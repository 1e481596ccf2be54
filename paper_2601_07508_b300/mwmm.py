"""Thin Python binding over libmwmm (include/mwmm.h): argument marshalling only.

Every step of the product runs in the library's CUDA kernels; this module
only turns torch tensors / numpy arrays into pointers, sizes and streams.
PyTorch supplies device memory and streams.  If the library has not been
built, or cannot be loaded, every call raises: there is no CPU fallback.

The functions carry the C names (mwmm_plan, mwmm_matmul, ...); ``Plan`` is a
small owner object around a plan handle.  Before any call that hands
matrices to the library, the binding checks their shapes against the
product and that they share the current device (ValueError otherwise): the
C entry points receive pointers and leading dimensions only.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmwmm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "mwmm.h")

MWMM_OK = 0
STATUS = {0: "MWMM_OK", 1: "MWMM_ERR_ARG", 2: "MWMM_ERR_PRIME", 3: "MWMM_ERR_BOUND", 4: "MWMM_ERR_RANGE",
          5: "MWMM_ERR_NOMEM", 6: "MWMM_ERR_BUDGET", 7: "MWMM_ERR_CUDA", 8: "MWMM_ERR_TIMEOUT",
          9: "MWMM_ERR_BUSY", 10: "MWMM_ERR_UNSUPPORTED"}
FORM_AUTO, FORM_FP64, FORM_INT8, FORM_CRT8 = 0, 1, 2, 3
FORMS = {"auto": FORM_AUTO, "fp64": FORM_FP64, "int8": FORM_INT8, "crt8": FORM_CRT8}


class MwmmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s%s (%d: %s)" % (what + ": " if what else "", STATUS.get(status, "?"), status,
                                            _status_str(status)))


class PlanOpts(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_int64), ("validate", ctypes.c_int32), ("tc_chunk", ctypes.c_int32),
                ("kc", ctypes.c_int64), ("tc_pair", ctypes.c_int32),
                ("f64_concat", ctypes.c_int32), ("ksplit", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("tc_fused", ctypes.c_int32), ("tc_seg", ctypes.c_int32), ("tc_digit_bits", ctypes.c_int32),
                ("tc_fill", ctypes.c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [("split_a_ms", ctypes.c_double), ("split_b_ms", ctypes.c_double), ("gemm_ms", ctypes.c_double),
                ("recombine_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("calls", ctypes.c_int64),
                ("launches", ctypes.c_int64)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64), ("p", ctypes.c_uint64),
                ("form", ctypes.c_int32), ("u", ctypes.c_int32), ("v", ctypes.c_int32),
                ("alpha", ctypes.c_uint64), ("beta", ctypes.c_uint64),
                ("lambda_", ctypes.c_int64), ("lambda_max", ctypes.c_int64), ("tc_chunk", ctypes.c_int64),
                ("kc", ctypes.c_int64), ("tc_pair", ctypes.c_int32), ("nkc", ctypes.c_int32), ("nsums", ctypes.c_int32),
                ("q", ctypes.c_double),
                ("kb_elems", ctypes.c_int64), ("nkb", ctypes.c_int64), ("A_rows", ctypes.c_int64),
                ("B_rows", ctypes.c_int64), ("B_wpad", ctypes.c_int32), ("tc_fused", ctypes.c_int32),
                ("A_off", ctypes.c_uint64), ("B_off", ctypes.c_uint64),
                ("S_off", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64),
                ("f64_concat", ctypes.c_int32), ("ksplit", ctypes.c_int32),
                ("tuned_ms", ctypes.c_double), ("tuned_tried", ctypes.c_int32), ("tc_seg", ctypes.c_int32),
                ("crt_m", ctypes.c_uint32 * 24), ("tc_digit_bits", ctypes.c_int32), ("tc_cert_chunk", ctypes.c_int32)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            val = getattr(self, name)
            d[name.rstrip("_")] = list(val) if isinstance(val, ctypes.Array) else val
        return d


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64), ("p", ctypes.c_uint64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("form", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("items", ctypes.c_int64), ("launches", ctypes.c_int64), ("workspace_bytes", ctypes.c_uint64),
                ("table_bytes", ctypes.c_uint64), ("flops_2mnk", ctypes.c_double), ("word_flops", ctypes.c_double),
                ("tuned_groups", ctypes.c_int32), ("pad0", ctypes.c_int32), ("tuned_ms", ctypes.c_double)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("form", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8)]


class ServeReport(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("mean_batch", ctypes.c_double), ("peak_queue", ctypes.c_int64),
                ("peak_inflight", ctypes.c_int64), ("peak_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("flops_2mnk", ctypes.c_double), ("busy_s", ctypes.c_double), ("gops", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


_lib: Optional[ctypes.CDLL] = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64


def lib() -> ctypes.CDLL:
    """Load libmwmm.so (raises if it is missing: no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmwmm.so is not built (run python -m paper_2601_07508_b300.build); "
                          "the mwmm product has no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    L.mwmm_plan.argtypes = [ctypes.POINTER(_vp), _i64, _i64, _i64, _u64, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int, ctypes.POINTER(PlanOpts)]
    L.mwmm_plan_info.argtypes = [_vp, ctypes.POINTER(PlanDesc)]
    L.mwmm_workspace_size.argtypes = [_vp]
    L.mwmm_workspace_size.restype = ctypes.c_size_t
    L.mwmm_matmul.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp, ctypes.c_size_t, _vp]
    L.mwmm_matmul_host.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp]
    L.mwmm_matmul_host_async.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp]
    L.mwmm_matmul_reuse_a.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, ctypes.c_size_t, _vp]
    L.mwmm_plan_check.argtypes = [_vp, _vp]
    L.mwmm_plan_destroy.argtypes = [_vp]
    L.mwmm_plan_destroy.restype = None
    L.mwmm_split.argtypes = [_vp, ctypes.c_int, _vp, _i64, _vp, _vp]
    L.mwmm_fmod.argtypes = [_vp, _i64, _u64, _vp, _vp]
    L.mwmm_selftest_wait_timeout.argtypes = [_i64, _vp]
    L.mwmm_measure_fp64_rate.argtypes = [_i64, ctypes.POINTER(ctypes.c_double), _vp]
    L.mwmm_tc_residency.argtypes = [ctypes.POINTER(ctypes.c_int32)] * 3
    L.mwmm_plan_autotuned.argtypes = [ctypes.POINTER(_vp), _i64, _i64, _i64, _u64, ctypes.c_int, _vp, _i64, _vp,
                                      _i64, _vp]
    L.mwmm_autotune_cache_entries.restype = ctypes.c_int64
    L.mwmm_autotune_cache_clear.restype = None
    L.mwmm_autotune_cache_save.argtypes = [ctypes.c_char_p]
    L.mwmm_autotune_cache_load.argtypes = [ctypes.c_char_p]
    L.mwmm_mulmod.argtypes = [_vp, _vp, _i64, _u64, _vp, _vp]
    L.mwmm_matmul_noalloc.argtypes = [_i64, _i64, _i64, _u64, _vp, _i64, _vp, _i64, _vp, _i64, _vp]
    L.mwmm_tensor_form.argtypes = [_i64, _i64, _i64, _u64]
    L.mwmm_tensor_form.restype = ctypes.c_int
    L.mwmm_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(PlanOpts)]
    L.mwmm_batch_run.argtypes = [_vp, _vp]
    L.mwmm_batch_check.argtypes = [_vp, _vp]
    L.mwmm_batch_info.argtypes = [_vp, ctypes.POINTER(BatchDesc)]
    L.mwmm_batch_problem_info.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(PlanDesc)]
    L.mwmm_batch_destroy.argtypes = [_vp]
    L.mwmm_batch_destroy.restype = None
    L.mwmm_matmul_batched.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp), _vp]
    L.mwmm_serve_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ServeOpts)]
    L.mwmm_serve_now.argtypes = [_vp]
    L.mwmm_serve_now.restype = ctypes.c_double
    L.mwmm_serve_submit.argtypes = [_vp, ctypes.POINTER(Problem), ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]
    L.mwmm_serve_poll.argtypes = [_vp, ctypes.c_uint64]
    L.mwmm_serve_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int]
    L.mwmm_serve_latency.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    L.mwmm_serve_stats.argtypes = [_vp, ctypes.POINTER(ServeReport)]
    L.mwmm_serve_reset_stats.argtypes = [_vp]
    L.mwmm_serve_destroy.argtypes = [_vp]
    L.mwmm_serve_destroy.restype = None
    L.mwmm_plan_set_timing.argtypes = [_vp, ctypes.c_int]
    L.mwmm_plan_timing.argtypes = [_vp, ctypes.POINTER(Timing)]
    L.mwmm_status_str.argtypes = [ctypes.c_int]
    L.mwmm_status_str.restype = ctypes.c_char_p
    L.mwmm_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _status_str(s: int) -> str:
    try:
        return lib().mwmm_status_str(s).decode()
    except Exception:
        return "?"


def _check(st: int, what: str):
    if st != MWMM_OK:
        raise MwmmError(st, what)


def declared_symbols():
    """Names of the functions include/mwmm.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mwmm_\w+)\s*\(", text)))


# --------------------------------------------------------------------------- marshalling
def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtypes=None) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtypes is not None and t.dtype not in dtypes:
        raise TypeError("unexpected dtype %s" % t.dtype)
    return t.data_ptr()


def _u64_dtypes():
    import torch
    return (torch.int64, torch.uint64)


def _ld(t) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a row-major 2-D matrix")
    return max(t.stride(0), 1)


# The C entry points see a pointer and a leading dimension per matrix, not
# its extent: a matrix smaller than the plan's product, or one on another
# device, would be read or written out of bounds by the kernels.  The binding
# checks both before any call.
def _shape(t, rows: int, cols: int, what: str, k: int = -1):
    """rows x cols exactly; where the extent is the product's k and k = 0
    (an empty sum: nothing is read), any extent."""
    ok = len(t.shape) == 2 and all(int(t.shape[i]) == want or (k == 0 and want == 0)
                                   for i, want in enumerate((rows, cols)))
    if not ok:
        raise ValueError("%s is %s; the product needs %d x %d" % (what, tuple(t.shape), rows, cols))


def _one_device(*ts):
    """One device for all operands, and for CUDA tensors the current one (the
    kernels run on the current device)."""
    devs = {t.device for t in ts if t is not None}
    if len(devs) > 1:
        raise ValueError("operands on different devices: %s" % sorted(str(d) for d in devs))
    d = next(iter(devs), None)
    if d is not None and d.type == "cuda":
        import torch
        if d.index is not None and d.index != torch.cuda.current_device():
            raise ValueError("operands on %s while cuda:%d is current" % (d, torch.cuda.current_device()))


def _plan_mnk(h: int, info: Optional[dict] = None):
    d = info if info is not None else mwmm_plan_info(h)
    return int(d["m"]), int(d["n"]), int(d["k"])


# --------------------------------------------------------------------------- C-named calls
def mwmm_plan(m: int, n: int, k: int, p: int, u: int = 0, v: int = 0, form="auto", lam: int = 0,
              validate: bool = False, tc_chunk: int = 0, kc: int = 0, tc_pair: Optional[bool] = None,
              f64_concat: int = 0, ksplit: int = 0, tc_fused: int = 0, tc_seg: int = 0,
              tc_digit_bits: int = 0, tc_fill: int = 0) -> int:
    if isinstance(form, str):
        form = FORMS[form]
    h = _vp()
    o = PlanOpts()
    o.lambda_ = lam
    o.validate = 1 if validate else 0
    o.tc_chunk = tc_chunk
    o.kc = kc
    # None: the planner's choice; True / False: the two-CTA / one-CTA kernel; an int is passed as is
    o.tc_pair = 0 if tc_pair is None else ((1 if tc_pair else -1) if isinstance(tc_pair, bool) else int(tc_pair))
    o.f64_concat = f64_concat
    o.ksplit = ksplit
    o.tc_fused = tc_fused
    o.tc_seg = tc_seg
    o.tc_digit_bits = tc_digit_bits
    o.tc_fill = tc_fill
    _check(lib().mwmm_plan(ctypes.byref(h), m, n, k, p, u, v, form, ctypes.byref(o)), "mwmm_plan")
    return h.value


def mwmm_tensor_form(m: int, n: int, k: int, p: int) -> str:
    """The tensor form ("int8" or "crt8") batches and the serving loop use
    for this product under form "auto" (host only; "auto" if none plans)."""
    f = lib().mwmm_tensor_form(m, n, k, p)
    return {v: name for name, v in FORMS.items()}[f]


def mwmm_plan_autotuned(m: int, n: int, k: int, p: int, form="auto", A=None, B=None, stream=None) -> int:
    """Plan whose configuration was timed on the device (A, B: optional
    device tensors of the product; zeros are used when omitted)."""
    if isinstance(form, str):
        form = FORMS[form]
    dt = _u64_dtypes()
    a = _dev_ptr(A, dt) if A is not None else None
    b = _dev_ptr(B, dt) if B is not None else None
    if A is not None:
        _shape(A, m, k, "A", k)
    if B is not None:
        _shape(B, k, n, "B", k)
    _one_device(A, B)
    h = _vp()
    _check(lib().mwmm_plan_autotuned(ctypes.byref(h), m, n, k, p, form, a, _ld(A) if A is not None else 0, b,
                                     _ld(B) if B is not None else 0, _stream_ptr(stream)), "mwmm_plan_autotuned")
    return h.value


def mwmm_autotune_cache_entries() -> int:
    return int(lib().mwmm_autotune_cache_entries())


def mwmm_autotune_cache_clear():
    lib().mwmm_autotune_cache_clear()


def mwmm_autotune_cache_save(path: str):
    _check(lib().mwmm_autotune_cache_save(path.encode()), "mwmm_autotune_cache_save")


def mwmm_autotune_cache_load(path: str):
    _check(lib().mwmm_autotune_cache_load(path.encode()), "mwmm_autotune_cache_load")


def mwmm_plan_info(h: int) -> dict:
    d = PlanDesc()
    _check(lib().mwmm_plan_info(h, ctypes.byref(d)), "mwmm_plan_info")
    return d.as_dict()


def mwmm_workspace_size(h: int) -> int:
    return int(lib().mwmm_workspace_size(h))


def mwmm_matmul(h: int, A, B, C, workspace=None, stream=None, info: Optional[dict] = None):
    """C = A B mod p on device tensors (int64 or uint64 holding entries < p).
    A must be m x k, B k x n and C m x n for the plan's m, n, k, all on one
    device (ValueError otherwise)."""
    dt = _u64_dtypes()
    m, n, k = _plan_mnk(h, info)
    _shape(A, m, k, "A", k)
    _shape(B, k, n, "B", k)
    _shape(C, m, n, "C")
    _one_device(A, B, C, workspace)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = _dev_ptr(workspace), workspace.numel() * workspace.element_size()
    _check(lib().mwmm_matmul(h, _dev_ptr(A, dt), _ld(A), _dev_ptr(B, dt), _ld(B), _dev_ptr(C, dt), _ld(C),
                             ws_ptr, ws_bytes, _stream_ptr(stream)), "mwmm_matmul")


def mwmm_matmul_reuse_a(h: int, B, C, workspace=None, stream=None, info: Optional[dict] = None):
    """C = A B mod p with the A words left in the workspace by the last product."""
    dt = _u64_dtypes()
    m, n, k = _plan_mnk(h, info)
    _shape(B, k, n, "B", k)
    _shape(C, m, n, "C")
    _one_device(B, C, workspace)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = _dev_ptr(workspace), workspace.numel() * workspace.element_size()
    _check(lib().mwmm_matmul_reuse_a(h, _dev_ptr(B, dt), _ld(B), _dev_ptr(C, dt), _ld(C), ws_ptr, ws_bytes,
                                     _stream_ptr(stream)), "mwmm_matmul_reuse_a")


def mwmm_matmul_host(h: int, A: np.ndarray, B: np.ndarray, C: np.ndarray, stream=None):
    """Same product with host arrays (uint64/int64, row-major)."""
    for x in (A, B, C):
        if x.dtype not in (np.uint64, np.int64) or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("host matrices must be C-contiguous uint64/int64")
    m, n, k = _plan_mnk(h)
    _shape(A, m, k, "A", k)
    _shape(B, k, n, "B", k)
    _shape(C, m, n, "C")
    _check(lib().mwmm_matmul_host(h, A.ctypes.data, max(A.shape[1], 1), B.ctypes.data, max(B.shape[1], 1),
                                  C.ctypes.data, max(C.shape[1], 1), _stream_ptr(stream)), "mwmm_matmul_host")


def mwmm_matmul_host_ptr(h: int, a_ptr: int, lda: int, b_ptr: int, ldb: int, c_ptr: int, ldc: int, stream=None):
    _check(lib().mwmm_matmul_host(h, a_ptr, lda, b_ptr, ldb, c_ptr, ldc, _stream_ptr(stream)), "mwmm_matmul_host")


def mwmm_matmul_host_async_ptr(h: int, a_ptr: int, lda: int, b_ptr: int, ldb: int, c_ptr: int, ldc: int,
                               stream=None):
    """Enqueue a host-buffer product (page-locked buffers) without waiting."""
    _check(lib().mwmm_matmul_host_async(h, a_ptr, lda, b_ptr, ldb, c_ptr, ldc, _stream_ptr(stream)),
           "mwmm_matmul_host_async")


def mwmm_matmul_noalloc(A, B, C, p: int, stream=None) -> int:
    """INT8-form product with the library's static scratch (no device
    allocation); synchronous.  Returns the status (0 = ok).

    The C entry point sees only pointers and sizes, so the shapes and the
    device are checked here: B must be k x n for A of shape m x k, C must be
    m x n, and all three must sit on one CUDA device, which is made current
    for the call (the scratch array used is that device's)."""
    import torch
    dt = _u64_dtypes()
    if A.dim() != 2 or B.dim() != 2 or C.dim() != 2:
        raise ValueError("A, B and C must be 2-D matrices")
    m, k = A.shape
    if B.shape[0] != k:
        raise ValueError("B has %d rows; A (%d x %d) needs %d" % (B.shape[0], m, k, k))
    n = B.shape[1]
    if tuple(C.shape) != (m, n):
        raise ValueError("C is %s; the product is %d x %d" % (tuple(C.shape), m, n))
    if not (A.is_cuda and B.is_cuda and C.is_cuda) or not (A.device == B.device == C.device):
        raise ValueError("A, B and C must be on one CUDA device")
    with torch.cuda.device(A.device):
        return int(lib().mwmm_matmul_noalloc(m, n, k, p, _dev_ptr(A, dt), _ld(A), _dev_ptr(B, dt), _ld(B),
                                             _dev_ptr(C, dt), _ld(C), _stream_ptr(stream)))


def mwmm_plan_check(h: int, stream=None) -> int:
    """Synchronise and return the device-side status (0 = ok)."""
    return int(lib().mwmm_plan_check(h, _stream_ptr(stream)))


def mwmm_plan_destroy(h: int):
    lib().mwmm_plan_destroy(h)


def mwmm_split(h: int, side: int, M, words, stream=None):
    """Words of A (side 0, M is m x k) or of B (side 1, M is k x n) into the
    byte tensor `words`, which must hold the side's whole word region."""
    d = mwmm_plan_info(h)
    m, n, k = _plan_mnk(h, d)
    if side == 0:
        _shape(M, m, k, "A", k)
        need = d["u"] * d["nkb"] * d["A_rows"] * 128
    elif side == 1:
        _shape(M, k, n, "B", k)
        need = (d["v"] + 2 * d["B_wpad"]) * d["nkb"] * d["B_rows"] * 128
    else:
        raise ValueError("side is 0 (A) or 1 (B)")
    if words.numel() * words.element_size() < need:
        raise ValueError("words holds %d bytes; the side's words take %d" % (words.numel() * words.element_size(),
                                                                            need))
    _one_device(M, words)
    _check(lib().mwmm_split(h, side, _dev_ptr(M, _u64_dtypes()), _ld(M), _dev_ptr(words), _stream_ptr(stream)),
           "mwmm_split")


def mwmm_fmod(x, p: int, out, stream=None):
    import torch
    _check(lib().mwmm_fmod(_dev_ptr(x, (torch.float64,)), x.numel(), p, _dev_ptr(out, (torch.float64,)),
                           _stream_ptr(stream)), "mwmm_fmod")


def mwmm_mulmod(x, y, p: int, out, stream=None):
    import torch
    f = (torch.float64,)
    _check(lib().mwmm_mulmod(_dev_ptr(x, f), _dev_ptr(y, f), x.numel(), p, _dev_ptr(out, f), _stream_ptr(stream)),
           "mwmm_mulmod")


def mwmm_measure_fp64_rate(iters: int = 1 << 16, stream=None) -> float:
    """The device's FP64 fused multiply-add rate in GFLOP/s (a DFMA loop
    timed with CUDA events)."""
    g = ctypes.c_double(0)
    _check(lib().mwmm_measure_fp64_rate(iters, ctypes.byref(g), _stream_ptr(stream)), "mwmm_measure_fp64_rate")
    return g.value


def mwmm_tc_residency() -> dict:
    """SM count, resident CTAs of the one-CTA word-product kernel and
    co-resident clusters of the pair kernel on the current device."""
    v = [ctypes.c_int32(0) for _ in range(3)]
    _check(lib().mwmm_tc_residency(*[ctypes.byref(x) for x in v]), "mwmm_tc_residency")
    return {"sms": v[0].value, "ctas": v[1].value, "pair_clusters": v[2].value}


def mwmm_selftest_wait_timeout(cycles: int, stream=None) -> int:
    """Run the bounded-wait routine on a barrier nothing completes; returns the
    status code (MWMM_ERR_TIMEOUT = 8 is the expected outcome)."""
    return int(lib().mwmm_selftest_wait_timeout(cycles, _stream_ptr(stream)))


def mwmm_plan_set_timing(h: int, on: bool = True):
    _check(lib().mwmm_plan_set_timing(h, 1 if on else 0), "mwmm_plan_set_timing")


def mwmm_plan_timing(h: int) -> dict:
    t = Timing()
    _check(lib().mwmm_plan_timing(h, ctypes.byref(t)), "mwmm_plan_timing")
    return {name: getattr(t, name) for name, _ in t._fields_}


def mwmm_status_str(s: int) -> str:
    return _status_str(s)


def mwmm_version() -> str:
    return lib().mwmm_version().decode()


def _problems(items):
    """items: sequence of (A, B, C, p) device tensors (row-major)."""
    arr = (Problem * len(items))()
    for i, (A, B, C, p) in enumerate(items):  # every problem checked before any pointer is taken
        if len(A.shape) != 2 or len(B.shape) != 2:
            raise ValueError("problem %d: A and B must be 2-D matrices" % i)
        _shape(B, int(A.shape[1]), int(B.shape[1]), "B of problem %d" % i)
        _shape(C, int(A.shape[0]), int(B.shape[1]), "C of problem %d" % i)
        _one_device(A, B, C)
    for i, (A, B, C, p) in enumerate(items):
        dt = _u64_dtypes()
        arr[i].m, arr[i].k = int(A.shape[0]), int(A.shape[1])
        arr[i].n = int(B.shape[1])
        arr[i].p = p
        arr[i].A, arr[i].lda = _dev_ptr(A, dt), _ld(A)
        arr[i].B, arr[i].ldb = _dev_ptr(B, dt), _ld(B)
        arr[i].C, arr[i].ldc = _dev_ptr(C, dt), _ld(C)
    return arr


def mwmm_batch_create(items, form="auto", tc_chunk: int = 0, kc: int = 0, autotune: bool = False) -> int:
    if isinstance(form, str):
        form = FORMS[form]
    probs = _problems(items)
    o = PlanOpts()
    o.tc_chunk = tc_chunk
    o.kc = kc
    o.autotune = 1 if autotune else 0
    h = _vp()
    _check(lib().mwmm_batch_create(ctypes.byref(h), probs, len(items), form, ctypes.byref(o)), "mwmm_batch_create")
    return h.value


def mwmm_batch_run(h: int, stream=None):
    _check(lib().mwmm_batch_run(h, _stream_ptr(stream)), "mwmm_batch_run")


def mwmm_batch_check(h: int, stream=None) -> int:
    return int(lib().mwmm_batch_check(h, _stream_ptr(stream)))


def mwmm_batch_info(h: int) -> dict:
    d = BatchDesc()
    _check(lib().mwmm_batch_info(h, ctypes.byref(d)), "mwmm_batch_info")
    return {name: getattr(d, name) for name, _ in d._fields_}


def mwmm_batch_problem_info(h: int, index: int) -> dict:
    d = PlanDesc()
    _check(lib().mwmm_batch_problem_info(h, index, ctypes.byref(d)), "mwmm_batch_problem_info")
    return d.as_dict()


def mwmm_batch_destroy(h: int):
    lib().mwmm_batch_destroy(h)


def mwmm_matmul_batched(items, form="auto", stream=None):
    """Create, run, synchronise and destroy a batch in one call."""
    if isinstance(form, str):
        form = FORMS[form]
    probs = _problems(items)
    _check(lib().mwmm_matmul_batched(probs, len(items), form, None, _stream_ptr(stream)), "mwmm_matmul_batched")


class Batch:
    """Owns a batch handle over device tensors [(A, B, C, p), ...]."""

    def __init__(self, items, form="auto", tc_chunk: int = 0, kc: int = 0, autotune: bool = False):
        self.items = list(items)  # keep the tensors alive
        self.handle = mwmm_batch_create(self.items, form, tc_chunk, kc, autotune)
        self.info = mwmm_batch_info(self.handle)

    def run(self, stream=None):
        mwmm_batch_run(self.handle, stream)

    def check(self, stream=None) -> int:
        return mwmm_batch_check(self.handle, stream)

    def problem_info(self, i: int) -> dict:
        return mwmm_batch_problem_info(self.handle, i)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                import torch
                torch.cuda.synchronize()
                mwmm_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


def mwmm_serve_create(budget_bytes: int, max_inflight: int = 2, max_batch: int = 0, form="auto") -> int:
    o = ServeOpts()
    o.max_batch = max_batch
    o.form = FORMS[form] if isinstance(form, str) else form
    h = _vp()
    _check(lib().mwmm_serve_create(ctypes.byref(h), budget_bytes, max_inflight, ctypes.byref(o)), "mwmm_serve_create")
    return h.value


def mwmm_serve_now(h: int) -> float:
    return float(lib().mwmm_serve_now(h))


def mwmm_serve_submit(h: int, A, B, C, p: int, t_arrival: float = -1.0):
    """Returns (status, ticket)."""
    prob = _problems([(A, B, C, p)])
    t = ctypes.c_uint64(0)
    st = lib().mwmm_serve_submit(h, prob, t_arrival, ctypes.byref(t))
    return int(st), int(t.value)


def mwmm_serve_submit_ptr(h: int, prob: Problem, t_arrival: float = -1.0):
    t = ctypes.c_uint64(0)
    st = lib().mwmm_serve_submit(h, ctypes.byref(prob), t_arrival, ctypes.byref(t))
    return int(st), int(t.value)


def mwmm_serve_poll(h: int, ticket: int) -> int:
    return int(lib().mwmm_serve_poll(h, ticket))


def mwmm_serve_wait(h: int, ticket: int, timeout_ms: int = -1) -> int:
    return int(lib().mwmm_serve_wait(h, ticket, timeout_ms))


def mwmm_serve_latency(h: int, ticket: int) -> float:
    s = ctypes.c_double(0)
    _check(lib().mwmm_serve_latency(h, ticket, ctypes.byref(s)), "mwmm_serve_latency")
    return s.value


def mwmm_serve_stats(h: int) -> dict:
    r = ServeReport()
    st = lib().mwmm_serve_stats(h, ctypes.byref(r))
    d = {name: getattr(r, name) for name, _ in r._fields_}
    d["status"] = int(st)
    return d


def mwmm_serve_reset_stats(h: int):
    _check(lib().mwmm_serve_reset_stats(h), "mwmm_serve_reset_stats")


def mwmm_serve_destroy(h: int):
    lib().mwmm_serve_destroy(h)


class Server:
    """Owns a serving loop: ``Server(budget_bytes)``, then ``submit`` / ``wait``."""

    def __init__(self, budget_bytes: int, max_inflight: int = 2, max_batch: int = 0, form="auto"):
        self.handle = mwmm_serve_create(budget_bytes, max_inflight, max_batch, form)

    def now(self) -> float:
        return mwmm_serve_now(self.handle)

    def submit(self, A, B, C, p: int, t_arrival: float = -1.0):
        return mwmm_serve_submit(self.handle, A, B, C, p, t_arrival)

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        return mwmm_serve_wait(self.handle, ticket, timeout_ms)

    def poll(self, ticket: int) -> int:
        return mwmm_serve_poll(self.handle, ticket)

    def latency(self, ticket: int) -> float:
        return mwmm_serve_latency(self.handle, ticket)

    def stats(self) -> dict:
        return mwmm_serve_stats(self.handle)

    def reset_stats(self):
        mwmm_serve_reset_stats(self.handle)

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            mwmm_serve_destroy(h)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- owner object
class Plan:
    """Owns a plan handle: ``Plan(m, n, k, p, form="int8")``, then ``.matmul(A, B)``."""

    def __init__(self, m: int, n: int, k: int, p: int, u: int = 0, v: int = 0, form="auto", lam: int = 0,
                 validate: bool = False, tc_chunk: int = 0, kc: int = 0, tc_pair: Optional[bool] = None,
                 f64_concat: int = 0, ksplit: int = 0, tc_fused: int = 0, tc_seg: int = 0,
                 tc_digit_bits: int = 0, tc_fill: int = 0):
        self.handle = mwmm_plan(m, n, k, p, u, v, form, lam, validate, tc_chunk, kc, tc_pair, f64_concat, ksplit,
                                tc_fused, tc_seg, tc_digit_bits, tc_fill)
        self.info = mwmm_plan_info(self.handle)
        self.workspace = None

    @classmethod
    def autotuned(cls, m: int, n: int, k: int, p: int, form="auto", A=None, B=None, stream=None):
        """Plan with the configuration the autotuner measured fastest."""
        self = cls.__new__(cls)
        self.handle = mwmm_plan_autotuned(m, n, k, p, form, A, B, stream)
        self.info = mwmm_plan_info(self.handle)
        self.workspace = None
        return self

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                mwmm_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def workspace_bytes(self) -> int:
        return int(self.info["workspace_bytes"])

    def alloc_workspace(self, device="cuda"):
        """Allocate the workspace through PyTorch (256-byte aligned by the caching allocator)."""
        import torch
        if self.workspace is None and self.workspace_bytes > 0:
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)
        return self.workspace

    def matmul(self, A, B, C=None, stream=None):
        import torch
        if C is None:
            C = torch.empty((self.info["m"], self.info["n"]), dtype=A.dtype, device=A.device)
        mwmm_matmul(self.handle, A, B, C, self.alloc_workspace(A.device), stream, self.info)
        return C

    def matmul_reuse_a(self, B, C=None, stream=None):
        """Product with the A words of the previous matmul (only B is split)."""
        import torch
        if C is None:
            C = torch.empty((self.info["m"], self.info["n"]), dtype=B.dtype, device=B.device)
        mwmm_matmul_reuse_a(self.handle, B, C, self.alloc_workspace(B.device), stream, self.info)
        return C

    def matmul_host(self, A: np.ndarray, B: np.ndarray) -> np.ndarray:
        C = np.empty((self.info["m"], self.info["n"]), dtype=np.uint64)
        mwmm_matmul_host(self.handle, np.ascontiguousarray(A), np.ascontiguousarray(B), C)
        return C

    def check(self, stream=None) -> int:
        return mwmm_plan_check(self.handle, stream)
