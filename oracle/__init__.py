"""FP64 CPU oracle for the Monte Carlo shiftable bilateral filter of
vector-valued images (Ghosh & Chaudhury, arXiv 1605.02164).

TEST INFRASTRUCTURE ONLY.  This package is imported by the test suite, by the
package smoke check and by the CPU-baseline leg of the benchmark.  The CUDA
library and its Python binding never import it, and it imports nothing from
them.  The arithmetic lives in ``mcsf_oracle.c`` (plain C, FP64); this module
compiles it with gcc, loads it with ctypes and adds the few steps that are
plain bookkeeping (the exhaustive expectation of Prop. 2, Eq. MSE).

Every function names the passage it follows.  Pins (tests that tie each
function to something other than itself) are in ``tests/test_oracle_*.py``.
Function with no numeric pin: none of the filter functions; the Fig. 5
accuracy claim (sub-pixel MSE at N=10, T>300) is checked qualitatively only
and is "parity unpinned" as a number.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from itertools import product

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcsf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmcsf_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_ERR_NOT_SPD = -2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, IEEE semantics: no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp, ip = P(ctypes.c_double), P(ctypes.c_int32)
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_splitmix64.restype = ctypes.c_uint64
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_sample_Y.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ip]
        lib.orc_cholesky.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_whiten.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.orc_freqs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip, dp]
        lib.orc_freqs.restype = None
        lib.orc_direct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                   ctypes.c_int, dp, dp, dp]
        lib.orc_mcsf.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
                                 dp, ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp, dp, dp]
        lib.orc_mcsf_pairwise.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                          ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ip, dp,
                                          ctypes.c_int, ip, dp, dp, dp]
        lib.orc_rc_direct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                      ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.orc_deriche_blur.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp]
        lib.orc_mcsf_deriche.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp,
                                         ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp]
        lib.orc_mcsf_deriche_pairwise.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                                  dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ip, dp]
        lib.orc_rgb_to_lab.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_lab_to_rgb.argtypes = [ctypes.c_int, dp, dp]
        _lib = lib
        return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    """Threads the OpenMP loops of the oracle use."""
    return int(_load().orc_num_threads())


def radius(sigma_s: float) -> int:
    """Half-width of the window [-3 sigma_s, 3 sigma_s]^2 on the integer grid
    (Section 1): offsets with |j| <= 3 sigma_s, i.e. floor(3 sigma_s).  The
    1e-9 guards against 3*sigma_s landing a hair below an integer."""
    return int(math.floor(3.0 * sigma_s + 1e-9))


# ----------------------------------------------------------------------------
# Sampling and whitening (Prop. 2, Eq. COB)
# ----------------------------------------------------------------------------

def splitmix64(seed: int, i: int) -> int:
    return int(_load().orc_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, i))


def sample_Y(d: int, N: int, K: int, seed: int) -> np.ndarray:
    """Y^(1..K) = N - 2 X^(t), X^(t) ~ B(N, 1/2)^d (Prop. 2, Eq. finalApproxY). (K, d) int32."""
    Y = np.zeros((K, d), np.int32)
    rc = _load().orc_sample_Y(d, N, K, seed & 0xFFFFFFFFFFFFFFFF, _ip(Y))
    if rc:
        raise ValueError(f"orc_sample_Y failed: {rc}")
    return Y


def cholesky(C) -> np.ndarray:
    C = _f64(C)
    d = C.shape[0]
    L = np.zeros((d, d))
    rc = _load().orc_cholesky(d, _dp(C), _dp(L))
    if rc == ORC_ERR_NOT_SPD:
        raise np.linalg.LinAlgError("C is not positive definite")
    if rc:
        raise ValueError(rc)
    return L


def whiten(C, mode: int = 0) -> np.ndarray:
    """W with W C W^T = I: mode 0 = L^{-1} (Cholesky), mode 1 = diag(alpha) Q^T (Eq. COB)."""
    C = _f64(C)
    d = C.shape[0]
    Wm = np.zeros((d, d))
    rc = _load().orc_whiten(d, _dp(C), mode, _dp(Wm))
    if rc == ORC_ERR_NOT_SPD:
        raise np.linalg.LinAlgError("C is not positive definite")
    if rc:
        raise ValueError(rc)
    return Wm


def freqs(Wm, Y, N: int) -> np.ndarray:
    """omega_t = W^T Y_t / sqrt(N), radians per intensity unit (K, d)."""
    Wm = _f64(Wm)
    Y = np.ascontiguousarray(Y, np.int32)
    K, d = Y.shape
    om = np.zeros((K, d))
    _load().orc_freqs(d, K, N, _dp(Wm), _ip(Y), _dp(om))
    return om


def plan(d: int, C, sigma_s: float, N: int, K: int, seed: int, whiten_mode: int = 0) -> dict:
    """The oracle's own plan for (d, C, sigma_s, N, K, seed): sampled Y, the
    whitening W, frequencies omega and nu = omega / (2 pi) in turns."""
    N = 10 if N == 0 else N
    Y = sample_Y(d, N, K, seed)
    Wm = whiten(C, whiten_mode)
    om = freqs(Wm, Y, N)
    return {"Y": Y, "W": Wm, "omega": om, "nu": om / (2.0 * math.pi), "N": N, "K": K,
            "r": radius(sigma_s), "sigma_s": float(sigma_s), "C": _f64(C)}


def exhaustive_Y(d: int, N: int):
    """All Y in {-N, -N+2, ..., N}^d with the probabilities of Prop. 2:
    prod_k binom(N, n_k) / 2^N, n_k = (N - Y_k)/2 (Eq. expansion)."""
    vals = [(N - 2 * n, math.comb(N, n) / 2.0 ** N) for n in range(N + 1)]
    Ys, ws = [], []
    for combo in product(vals, repeat=d):
        Ys.append([v for v, _ in combo])
        ws.append(math.prod(p for _, p in combo))
    return np.asarray(Ys, np.int32), np.asarray(ws, np.float64)


# ----------------------------------------------------------------------------
# Filters
# ----------------------------------------------------------------------------

def _img(f):
    f = _f64(f)
    if f.ndim == 2:
        f = f[None]
    return f


def direct(f, sigma_s: float, C, r: int | None = None, return_Z: bool = False):
    """Part A: the direct filter of Eqs. (BF), (normal)."""
    f = _img(f)
    d, H, W = f.shape
    r = radius(sigma_s) if r is None else r
    out = np.zeros_like(f)
    Z = np.zeros((H, W))
    rc = _load().orc_direct(d, H, W, _dp(f), float(sigma_s), r, _dp(_f64(C)), _dp(out), _dp(Z))
    if rc:
        raise ValueError(f"orc_direct failed: {rc}")
    return (out, Z) if return_Z else out


def mcsf(f, sigma_s: float, Wm, N: int, Y, weights=None, r: int | None = None) -> dict:
    """Part B1: Algorithm 1 (shiftable form); returns S = Re P / Re Z and the
    real and imaginary parts of P and Z (Eqs. numerator, denom)."""
    f = _img(f)
    d, H, W = f.shape
    Y = np.ascontiguousarray(Y, np.int32)
    K = Y.shape[0]
    r = radius(sigma_s) if r is None else r
    w = None if weights is None else _f64(weights)
    out = np.zeros_like(f)
    Pre, Pim = np.zeros_like(f), np.zeros_like(f)
    Zre, Zim = np.zeros((H, W)), np.zeros((H, W))
    rc = _load().orc_mcsf(d, H, W, _dp(f), float(sigma_s), r, _dp(_f64(Wm)), N, K, _ip(Y), _dp(w),
                          _dp(out), _dp(Pre), _dp(Zre), _dp(Pim), _dp(Zim))
    if rc:
        raise ValueError(f"orc_mcsf failed: {rc}")
    return {"S": out, "Pre": Pre, "Zre": Zre, "Pim": Pim, "Zim": Zim}


def mcsf_pairwise(f, sigma_s: float, Wm, N: int, Y, pix, weights=None, r: int | None = None) -> dict:
    """Part B2: the estimator in pairwise form at the listed (y, x) pixels."""
    f = _img(f)
    d, H, W = f.shape
    Y = np.ascontiguousarray(Y, np.int32)
    K = Y.shape[0]
    r = radius(sigma_s) if r is None else r
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    n = pix.shape[0]
    w = None if weights is None else _f64(weights)
    out = np.zeros((n, d))
    Pre = np.zeros((n, d))
    Zre = np.zeros(n)
    rc = _load().orc_mcsf_pairwise(d, H, W, _dp(f), float(sigma_s), r, _dp(_f64(Wm)), N, K, _ip(Y), _dp(w),
                                   n, _ip(pix), _dp(out), _dp(Pre), _dp(Zre))
    if rc:
        raise ValueError(f"orc_mcsf_pairwise failed: {rc}")
    return {"S": out, "Pre": Pre, "Zre": Zre}


def rc_direct(f, sigma_s: float, Wm, N: int, r: int | None = None, return_Z: bool = False):
    """Part C1: direct filter with the raised-cosine kernel of Eq. (approx)."""
    f = _img(f)
    d, H, W = f.shape
    r = radius(sigma_s) if r is None else r
    out = np.zeros_like(f)
    Z = np.zeros((H, W))
    rc = _load().orc_rc_direct(d, H, W, _dp(f), float(sigma_s), r, _dp(_f64(Wm)), N, _dp(out), _dp(Z))
    if rc:
        raise ValueError(f"orc_rc_direct failed: {rc}")
    return (out, Z) if return_Z else out


def mcsf_exhaustive(f, sigma_s: float, Wm, N: int, r: int | None = None) -> dict:
    """Part C2: the expectation of Prop. 2 taken exactly, i.e. Algorithm 1 run
    over every Y with its binomial probability as weight."""
    d = _img(f).shape[0]
    Y, w = exhaustive_Y(d, N)
    return mcsf(f, sigma_s, Wm, N, Y, weights=w, r=r)


def deriche_blur(img, sigma: float):
    """Recursive (Deriche) Gaussian blur of a real (H, W) image, zero outside:
    the O(1)-in-sigma convolution of Section 3."""
    img = _f64(img)
    assert img.ndim == 2
    out = np.zeros_like(img)
    if _load().orc_deriche_blur(img.shape[0], img.shape[1], _dp(img), float(sigma), _dp(out)):
        raise ValueError("orc_deriche_blur failed")
    return out


def mcsf_deriche(f, sigma_s: float, Wm, N: int, Y, weights=None) -> dict:
    """Algorithm 1 with the recursive blur: S = Re P / Re Z (dict S, Pre, Zre)."""
    f = _img(f)
    d, H, W = f.shape
    Y = np.ascontiguousarray(Y, np.int32)
    K = Y.shape[0]
    S, P, Z = np.zeros_like(f), np.zeros_like(f), np.zeros((H, W))
    wts = None if weights is None else _f64(weights)
    rc = _load().orc_mcsf_deriche(d, H, W, _dp(f), float(sigma_s), _dp(_f64(Wm)), N, K, _ip(Y), _dp(wts),
                                  _dp(S), _dp(P), _dp(Z))
    if rc:
        raise ValueError(f"orc_mcsf_deriche failed: {rc}")
    return {"S": S, "Pre": P, "Zre": Z}


def mcsf_deriche_pairwise(f, sigma_s: float, Wm, N: int, Y, pix) -> np.ndarray:
    """Pairwise form with the closed-form recursive kernel at pixels pix (n, 2) -> (n, d)."""
    f = _img(f)
    d, H, W = f.shape
    Y = np.ascontiguousarray(Y, np.int32)
    pix = np.ascontiguousarray(pix, np.int32)
    out = np.zeros((pix.shape[0], d))
    rc = _load().orc_mcsf_deriche_pairwise(d, H, W, _dp(f), float(sigma_s), _dp(_f64(Wm)), N, Y.shape[0], _ip(Y),
                                           pix.shape[0], _ip(pix), _dp(out))
    if rc:
        raise ValueError(f"orc_mcsf_deriche_pairwise failed: {rc}")
    return out


def rgb_to_lab(f):
    """sRGB on the 0..255 scale (3, H, W) -> CIE 1976 (L*, a*, b*), the colour
    transform of Section 4's Lab experiment (Fig. 4); D65 white, no clipping."""
    f = _img(f)
    assert f.shape[0] == 3
    out = np.zeros_like(f)
    if _load().orc_rgb_to_lab(f[0].size, _dp(f), _dp(out)):
        raise ValueError("orc_rgb_to_lab failed")
    return out


def lab_to_rgb(lab):
    """Inverse of rgb_to_lab (no clipping)."""
    lab = _img(lab)
    assert lab.shape[0] == 3
    out = np.zeros_like(lab)
    if _load().orc_lab_to_rgb(lab[0].size, _dp(lab), _dp(out)):
        raise ValueError("orc_lab_to_rgb failed")
    return out


# ----------------------------------------------------------------------------
# Accuracy measures (Eq. MSE)
# ----------------------------------------------------------------------------

def mse(B, S) -> float:
    """Eq. (MSE) generalised to d channels: mean over d|Omega| of squared differences."""
    B = np.asarray(B, np.float64)
    S = np.asarray(S, np.float64)
    return float(np.mean((B - S) ** 2))


def mse_db(B, S) -> float:
    """10 log10(MSE), the paper's 'dB' figure (Section 4)."""
    return 10.0 * math.log10(mse(B, S))


def psnr(B, S, peak: float = 255.0) -> float:
    m = mse(B, S)
    return float("inf") if m == 0 else 10.0 * math.log10(peak * peak / m)
