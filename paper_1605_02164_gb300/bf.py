"""Python binding of libbf (include/bf.h): the same entry points, argument
marshalling only.  Every step of the filter runs in the library's CUDA
kernels; there is no Python or CPU fallback, and loading fails loudly when the
compiled library is missing.

Device buffers are passed as integers (``tensor.data_ptr()``) and streams as
integers (``torch.cuda.current_stream().cuda_stream``); helpers at the bottom
accept torch tensors directly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

BF_OK = 0
BF_ERR_ARG = -1
BF_ERR_NOT_SPD = -2
BF_ERR_D_RANGE = -3
BF_ERR_ALIGN = -4
BF_ERR_NOMEM = -5
BF_ERR_BUDGET = -6
BF_ERR_TIMEOUT = -7
BF_ERR_CUDA = -8
BF_ERR_UNSUPPORTED = -9
BF_ERR_BOUNDS = -10

BF_FAULT_ALLOC = 1      # bf_debug_inject: the next library allocation request fails
BF_FAULT_TC_WAIT = 2    # bf_debug_inject: the next tensor-core launch's bounded wait runs out

BF_MAX_D = 8
BF_MAX_RADIUS = 32
BF_MAX_PLAN_RADIUS = 4096
BF_MAX_N = 4096
BF_MAX_K = 65536
BF_NOALLOC_MAX_ITEMS = 256

BF_FP32 = 0
BF_FP16TC = 1
BF_BF16TC = 2
BF_FP32_RECURSIVE = 3
VARIANTS = {"fp32": BF_FP32, "fp16tc": BF_FP16TC, "bf16tc": BF_BF16TC, "fp32rec": BF_FP32_RECURSIVE}

BF_WHITEN_CHOLESKY = 0
BF_WHITEN_EIGEN = 1

_lock = threading.Lock()
_lib = None


class BFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _load().bf_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


class bf_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int)]


def library_path() -> str:
    return os.environ.get("BF_LIBRARY") or _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("BF_LIBRARY") or _build.LIB  # e.g. the checked build
        if not os.path.exists(path):
            raise ImportError(f"libbf is not built ({path} missing); run paper_1605_02164_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.bf_plan.argtypes = [i, dp, d, i, i, u64, ctypes.POINTER(vp)]
        lib.bf_plan_ex.argtypes = [i, dp, d, i, i, u64, i, i, ctypes.POINTER(vp)]
        lib.bf_plan_get_freqs.argtypes = [vp, dp, ip]
        lib.bf_plan_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                     ctypes.POINTER(i), dp]
        lib.bf_plan_destroy.argtypes = [vp]
        lib.bf_filter.argtypes = [vp, vp, vp, i, i, i, i, vp]
        lib.bf_filter_batch.argtypes = [ctypes.POINTER(bf_item), i, i, vp]
        lib.bf_filter_batch_noalloc.argtypes = [ctypes.POINTER(bf_item), i, i, vp]
        lib.bf_filter_host.argtypes = [vp, vp, vp, i, i, i, vp]
        lib.bf_filter_host_async.argtypes = [vp, vp, vp, i, i, i, vp]
        lib.bf_rgb_to_lab.argtypes = [vp, vp, i, i, i, vp]
        lib.bf_lab_to_rgb.argtypes = [vp, vp, i, i, i, vp]
        lib.bf_last_status.argtypes = [vp]
        lib.bf_debug_inject.argtypes = [i]
        lib.bf_error_string.argtypes = [i]
        lib.bf_error_string.restype = ctypes.c_char_p
        lib.bf_version.restype = i
        lib.bf_tune_size_class.argtypes = [i, i]
        lib.bf_tune_set.argtypes = [i, i, i, i, i, i]
        lib.bf_tune_get.argtypes = [i, i, i, i, i, ctypes.POINTER(i)]
        _lib = lib
        return lib


def lib():
    return _load()


def _check(rc: int, where: str):
    if rc != BF_OK:
        raise BFError(rc, where)


class Plan:
    """Owning handle of a bf_plan_t; destroyed on close() or garbage collection."""

    def __init__(self, handle: int, d: int, K: int, N: int, r: int, sigma_s: float):
        self.handle = handle
        self.d, self.K, self.N, self.r, self.sigma_s = d, K, N, r, sigma_s

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)

    def close(self):
        if self.handle:
            _load().bf_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __repr__(self):
        return f"Plan(d={self.d}, K={self.K}, N={self.N}, r={self.r}, sigma_s={self.sigma_s})"


def bf_plan(d: int, C, sigma_s: float, N: int = 0, K: int = 64, seed: int = 0, whiten: int = BF_WHITEN_CHOLESKY,
            radius: int = -1) -> Plan:
    """bf_plan / bf_plan_ex: whitened, seeded frequency list on the device."""
    C = np.ascontiguousarray(C, np.float64)
    h = ctypes.c_void_p()
    rc = _load().bf_plan_ex(int(d), C.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(sigma_s), int(N),
                            int(K), ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(whiten), int(radius),
                            ctypes.byref(h))
    _check(rc, "bf_plan")
    return bf_plan_info(Plan(h.value, d, K, 0, 0, sigma_s))


def bf_plan_info(plan: Plan) -> Plan:
    d, K, N, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    s = ctypes.c_double()
    _check(_load().bf_plan_info(plan, ctypes.byref(d), ctypes.byref(K), ctypes.byref(N), ctypes.byref(r),
                                ctypes.byref(s)), "bf_plan_info")
    plan.d, plan.K, plan.N, plan.r, plan.sigma_s = d.value, K.value, N.value, r.value, s.value
    return plan


def bf_plan_get_freqs(plan: Plan):
    """(nu, Y): nu_t in turns (K, d) float64 and Y_t (K, d) int32."""
    nu = np.zeros((plan.K, plan.d), np.float64)
    Y = np.zeros((plan.K, plan.d), np.int32)
    _check(_load().bf_plan_get_freqs(plan, nu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     Y.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "bf_plan_get_freqs")
    return nu, Y


def bf_plan_destroy(plan: Plan):
    plan.close()


def bf_filter(plan: Plan, in_ptr: int, out_ptr: int, H: int, W: int, pitch: int, variant: int = BF_FP32,
              stream: int = 0):
    _check(_load().bf_filter(plan, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(H), int(W), int(pitch),
                             int(variant), ctypes.c_void_p(stream)), "bf_filter")


def bf_filter_batch(items, variant: int = BF_FP32, stream: int = 0):
    """items: sequence of (plan, in_ptr, out_ptr, H, W, pitch)."""
    arr = (bf_item * max(1, len(items)))()
    keep = []
    for k, (plan, ip, op, H, W, pitch) in enumerate(items):
        arr[k] = bf_item(plan.handle, ip, op, H, W, pitch)
        keep.append(plan)
    _check(_load().bf_filter_batch(arr, len(items), int(variant), ctypes.c_void_p(stream)), "bf_filter_batch")


def bf_filter_batch_noalloc(items, variant: int = BF_FP16TC, stream: int = 0):
    """As bf_filter_batch for the tensor-core variants, without any allocation
    (scratch in a static device array; at most BF_NOALLOC_MAX_ITEMS images)."""
    arr = (bf_item * max(1, len(items)))()
    for k, (plan, ip, op, H, W, pitch) in enumerate(items):
        arr[k] = bf_item(plan.handle, ip, op, H, W, pitch)
    _check(_load().bf_filter_batch_noalloc(arr, len(items), int(variant), ctypes.c_void_p(stream)),
           "bf_filter_batch_noalloc")


def bf_filter_host(plan: Plan, in_host: np.ndarray, out_host: np.ndarray | None = None, variant: int = BF_FP32,
                   stream: int = 0) -> np.ndarray:
    """Host (d, H, W) float32 in, host (d, H, W) float32 out; synchronous."""
    x = np.ascontiguousarray(in_host, np.float32)
    d, H, W = x.shape
    if out_host is None:
        out_host = np.empty_like(x)
    assert out_host.flags["C_CONTIGUOUS"] and out_host.dtype == np.float32 and out_host.shape == x.shape
    _check(_load().bf_filter_host(plan, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(out_host.ctypes.data),
                                  H, W, int(variant), ctypes.c_void_p(stream)), "bf_filter_host")
    return out_host


def bf_rgb_to_lab(in_ptr: int, out_ptr: int, H: int, W: int, pitch: int, stream: int = 0):
    """sRGB (0..255) -> CIE 1976 L*a*b*, planar [3][H][pitch] device buffers (in place allowed)."""
    _check(_load().bf_rgb_to_lab(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(H), int(W), int(pitch),
                                 ctypes.c_void_p(stream)), "bf_rgb_to_lab")


def bf_lab_to_rgb(in_ptr: int, out_ptr: int, H: int, W: int, pitch: int, stream: int = 0):
    """CIE 1976 L*a*b* -> sRGB (0..255), planar [3][H][pitch] device buffers (in place allowed)."""
    _check(_load().bf_lab_to_rgb(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(H), int(W), int(pitch),
                                 ctypes.c_void_p(stream)), "bf_lab_to_rgb")


def bf_filter_host_async(plan: Plan, in_host: np.ndarray, out_host: np.ndarray, variant: int = BF_FP32,
                         stream: int = 0) -> np.ndarray:
    """Queues copy in, filter and copy out on `stream` and returns (host arrays
    (d, H, W) float32, C-contiguous, pinned for asynchronous copies; out_host is
    valid once the stream has reached this work)."""
    for a in (in_host, out_host):
        assert a.flags["C_CONTIGUOUS"] and a.dtype == np.float32 and a.shape == in_host.shape
    d, H, W = in_host.shape
    _check(_load().bf_filter_host_async(plan, ctypes.c_void_p(in_host.ctypes.data),
                                        ctypes.c_void_p(out_host.ctypes.data), H, W, int(variant),
                                        ctypes.c_void_p(stream)), "bf_filter_host_async")
    return out_host


def bf_last_status(stream: int = 0) -> int:
    return int(_load().bf_last_status(ctypes.c_void_p(stream)))


def bf_version() -> int:
    return int(_load().bf_version())


BF_TUNE_ALONE = 0
BF_TUNE_BATCH = 1


def bf_tune_size_class(H: int, W: int) -> int:
    c = int(_load().bf_tune_size_class(int(H), int(W)))
    if c < 0:
        raise BFError(c, "bf_tune_size_class")
    return c


def bf_tune_set(variant: int, d: int, r: int, size_class: int, context: int, tile_rows: int) -> None:
    _check(_load().bf_tune_set(variant, d, r, size_class, context, tile_rows), "bf_tune_set")


def bf_tune_get(variant: int, d: int, r: int, size_class: int, context: int) -> int:
    out = ctypes.c_int(0)
    _check(_load().bf_tune_get(variant, d, r, size_class, context, ctypes.byref(out)), "bf_tune_get")
    return int(out.value)


def bf_tune_clear() -> None:
    _check(_load().bf_tune_clear(), "bf_tune_clear")


def bf_tune_count() -> int:
    return int(_load().bf_tune_count())


def bf_debug_inject(faults: int) -> None:
    """Arm one-shot faults for tests of the error paths (0 disarms)."""
    _check(_load().bf_debug_inject(int(faults)), "bf_debug_inject")


# ---------------------------------------------------------------------------
# torch conveniences (marshalling only)
# ---------------------------------------------------------------------------

def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def filter_tensor(plan: Plan, x, variant: int = BF_FP32, out=None, stream=None):
    """Filter a CUDA float32 tensor of shape (d, H, W) whose last-dim stride is
    1 and row stride a multiple of 4 (pitch); returns ``out``."""
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.dim() == 3 and x.stride(2) == 1
    d, H, W = x.shape
    pitch = x.stride(1)
    assert x.stride(0) == H * pitch, "planes must be contiguous [d][H][pitch]"
    if out is None:
        out = torch.empty_strided(x.shape, x.stride(), dtype=x.dtype, device=x.device)
    bf_filter(plan, x.data_ptr(), out.data_ptr(), H, W, pitch, variant, _stream_ptr(stream))
    return out


def convert_tensor(x, to_lab: bool, out=None, stream=None):
    """bf_rgb_to_lab / bf_lab_to_rgb on a CUDA float32 (3, H, W) pitched tensor."""
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.dim() == 3 and x.shape[0] == 3 and x.stride(2) == 1
    _, H, W = x.shape
    assert x.stride(0) == H * x.stride(1), "planes must be contiguous [3][H][pitch]"
    if out is None:
        out = torch.empty_strided(x.shape, x.stride(), dtype=x.dtype, device=x.device)
    fn = bf_rgb_to_lab if to_lab else bf_lab_to_rgb
    fn(x.data_ptr(), out.data_ptr(), H, W, x.stride(1), _stream_ptr(stream))
    return out


def filter_lab_tensor(plan: Plan, x, variant: int = BF_FP32, out=None, stream=None):
    """Filter an sRGB image in CIE-Lab (Section 4, Fig. 4): convert, filter
    with `plan` (its C in Lab units), convert back.  Returns ``out`` (RGB)."""
    lab = convert_tensor(x, True, stream=stream)
    lab_out = filter_tensor(plan, lab, variant, stream=stream)
    return convert_tensor(lab_out, False, out=out, stream=stream)


def pitched_empty(d: int, H: int, W: int, device="cuda"):
    """(d, H, W) float32 view over a [d][H][pitch] buffer with pitch % 4 == 0."""
    import torch
    pitch = (W + 3) // 4 * 4
    buf = torch.empty((d, H, pitch), dtype=torch.float32, device=device)
    return buf[:, :, :W]


def to_pitched(x_np: np.ndarray, device="cuda"):
    import torch
    d, H, W = x_np.shape
    t = pitched_empty(d, H, W, device)
    t.copy_(torch.from_numpy(np.ascontiguousarray(x_np, np.float32)))
    return t
