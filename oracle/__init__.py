"""FP64 CPU oracle for (Fast) Iterative Filtering -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1802_01359_gb300``)
never imports it and shares no code with it.

The arithmetic lives in ``fif_oracle.c`` (plain C, binary64), which this module
compiles with gcc on first use and calls through ctypes.  Two tiers:

* :func:`iterative` -- tier A, Algorithm 2 of the paper (Sec. 3): repeated
  periodic convolution with the sampled triangle window, stopping rule eq. SD.
* :func:`direct` -- tier B, the FIF direct method of Sec. 4 (eq. One
  step_algo), with m chosen by evaluating eq. SD for successively larger m
  through Parseval (Theorem 2 proof, Theorem 5).

Building blocks exported for the pins: :func:`dft` (definition, O(n^2)),
:func:`fft` (hand-written mixed-radix recursion), :func:`window_spectrum`
(closed form of the circulant's eigenvalues, eq. Lambdas / eq. eig2),
:func:`taps`, :func:`count_extrema`, :func:`count_zero_crossings`,
:func:`mask_length`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fif_oracle.c")
_HDR = os.path.join(_HERE, "fif_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfif_oracle.so")

STOP_EXTREMA = 1
STOP_MASK = 2
STOP_MAX_IMFS = 3
STOP_FORCED_END = 4
STOP_NONFINITE = 5
FLAG_NEAR_DELTA_TIE = 1 << 8
FLAG_MASK_TIE = 1 << 9
FLAG_MAX_INNER_HIT = 1 << 10
FLAG_L_CLAMPED = 1 << 12

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fif_oracle.c into a shared library (gcc, -O2, strict IEEE)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("mask_scale", ctypes.c_int), ("delta", ctypes.c_double),
                ("max_inner", ctypes.c_int), ("max_imfs", ctypes.c_int),
                ("L_in", ctypes.POINTER(ctypes.c_int)), ("absolute", ctypes.c_int),
                ("apriori", ctypes.c_int), ("gamma", ctypes.c_double), ("peak_mask", ctypes.c_int),
                ("shape", ctypes.POINTER(ctypes.c_double)), ("shape_len", ctypes.c_int)]


class _Outputs(ctypes.Structure):
    _fields_ = [("imfs", ctypes.POINTER(ctypes.c_double)), ("m", ctypes.POINTER(ctypes.c_int)),
                ("L", ctypes.POINTER(ctypes.c_int)), ("kext", ctypes.POINTER(ctypes.c_int)),
                ("n_imfs", ctypes.POINTER(ctypes.c_int)), ("status", ctypes.POINTER(ctypes.c_int)),
                ("sd_m", ctypes.POINTER(ctypes.c_double)), ("sd_prev", ctypes.POINTER(ctypes.c_double)),
                ("sd_trace", ctypes.POINTER(ctypes.c_double)),
                ("imf_flags", ctypes.POINTER(ctypes.c_int))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.fifo_iterative.argtypes = [dp, ctypes.c_long, ctypes.POINTER(_Params), ctypes.POINTER(_Outputs)]
            lib.fifo_direct.argtypes = lib.fifo_iterative.argtypes
            lib.fifo_dft_bruteforce.argtypes = [dp, dp, ctypes.c_long, ctypes.c_int, dp, dp]
            lib.fifo_fft.argtypes = [dp, dp, ctypes.c_long, ctypes.c_int]
            lib.fifo_triangle_taps.argtypes = [ctypes.c_long, ctypes.c_int, dp]
            lib.fifo_window_spectrum.argtypes = [ctypes.c_long, ctypes.c_int, dp]
            lib.fifo_count_extrema.argtypes = [dp, ctypes.c_long]
            lib.fifo_count_extrema.restype = ctypes.c_long
            lib.fifo_count_zero_crossings.argtypes = [dp, ctypes.c_long]
            lib.fifo_count_zero_crossings.restype = ctypes.c_long
            lib.fifo_mask_length.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_int]
            lib.fifo_mask_length.restype = ctypes.c_int
            lib.fifo_apriori_n0.argtypes = [ctypes.c_double, ctypes.c_long, ctypes.c_long,
                                            ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]
            lib.fifo_apriori_n0.restype = ctypes.c_int
            lib.fifo_spectral_peak.argtypes = [dp, dp, ctypes.c_long, ctypes.POINTER(ctypes.c_int)]
            lib.fifo_spectral_peak.restype = ctypes.c_long
            for f in ("fifo_shape_taps", "fifo_shape_spectrum"):
                getattr(lib, f).argtypes = [ctypes.c_long, ctypes.c_int, dp, ctypes.c_int, dp]
                getattr(lib, f).restype = ctypes.c_int
            lib.fifo_shape_filter.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.fifo_shape_filter.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _as_f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def dft(re, im=None, sign: int = -1):
    """Brute-force DFT, the definition (O(n^2)); returns complex128."""
    re = _as_f64(re)
    n = re.size
    im = np.zeros(n) if im is None else _as_f64(im)
    ore, oim = np.empty(n), np.empty(n)
    _load().fifo_dft_bruteforce(_dptr(re), _dptr(im), n, sign, _dptr(ore), _dptr(oim))
    return ore + 1j * oim


def fft(x, sign: int = -1):
    """The oracle's own mixed-radix FFT (unnormalised); returns complex128."""
    x = np.asarray(x)
    re = _as_f64(np.real(x)).copy()
    im = _as_f64(np.imag(x)).copy() if np.iscomplexobj(x) else np.zeros(re.size)
    if _load().fifo_fft(_dptr(re), _dptr(im), re.size, sign) != 0:
        raise RuntimeError("fifo_fft failed")
    return re + 1j * im


def taps(n: int, L: int) -> np.ndarray:
    c = np.empty(n)
    _load().fifo_triangle_taps(n, L, _dptr(c))
    return c


def window_spectrum(n: int, L: int) -> np.ndarray:
    w = np.empty(n)
    _load().fifo_window_spectrum(n, L, _dptr(w))
    return w


def _shape_call(fn, n, L, g):
    g = _as_f64(g)
    out = np.empty(n)
    rc = getattr(_load(), fn)(n, L, _dptr(g), g.size, _dptr(out))
    if rc != 0:
        raise ValueError(f"{fn}: invalid shape or length (rc={rc})")
    return out


def shape_filter(L: int, g) -> np.ndarray:
    """The generating filter h_i = g((i + 1/2)/L), i < L, of a shape window."""
    g = _as_f64(g)
    h = np.empty(L)
    if _load().fifo_shape_filter(_dptr(g), g.size, L, _dptr(h)) != 0:
        raise ValueError("fifo_shape_filter: invalid shape or length")
    return h


def shape_taps(n: int, L: int, g) -> np.ndarray:
    """Taps (h * h normalised, at d mod n) of the window generated by shape g."""
    return _shape_call("fifo_shape_taps", n, L, g)


def shape_spectrum(n: int, L: int, g) -> np.ndarray:
    """w_hat_k, k < n, of the window generated by shape g (DFT of its taps)."""
    return _shape_call("fifo_shape_spectrum", n, L, g)


def count_extrema(r) -> int:
    r = _as_f64(r)
    return int(_load().fifo_count_extrema(_dptr(r), r.size))


def count_zero_crossings(r) -> int:
    r = _as_f64(r)
    return int(_load().fifo_count_zero_crossings(_dptr(r), r.size))


def apriori_n0(snorm: float, n: int, kzero: int, delta: float, max_inner: int):
    """(N0, near_tie) of eq. N0_discrete (Theorem 5); N0 = max_inner + 1 if none <= max_inner."""
    tie = ctypes.c_int()
    N0 = _load().fifo_apriori_n0(float(snorm), int(n), int(kzero), float(delta), int(max_inner),
                                 ctypes.byref(tie))
    return int(N0), bool(tie.value)


def spectral_peak(x):
    """(k*, tie) of fifo_spectral_peak for the real signal x (spectrum by the oracle's FFT)."""
    x = _as_f64(x)
    re, im = x.copy(), np.zeros_like(x)
    _load().fifo_fft(_dptr(re), _dptr(im), x.size, -1)
    tie = ctypes.c_int()
    k = _load().fifo_spectral_peak(_dptr(re), _dptr(im), x.size, ctypes.byref(tie))
    return int(k), bool(tie.value)


def mask_length(n: int, k: int, nu: float = 1.6, mask_scale: int = 1) -> int:
    return int(_load().fifo_mask_length(n, k, nu, mask_scale))


def _run(fn_name, s, *, nu=1.6, mask_scale=1, delta=1e-3, max_inner=200, max_imfs=10,
         force_L=None, absolute=False, apriori=False, gamma=0.0, peak_mask=False, shape=None,
         trace=False):
    lib = _load()
    s = _as_f64(s)
    n = s.size
    keep = []
    p = _Params(nu=nu, mask_scale=mask_scale, delta=delta, max_inner=max_inner, max_imfs=max_imfs,
                L_in=None, absolute=1 if absolute else 0, apriori=1 if apriori else 0,
                gamma=float(gamma), peak_mask=1 if peak_mask else 0, shape=None, shape_len=0)
    if shape is not None:
        g = _as_f64(shape).copy()
        keep.append(g)
        p.shape = _dptr(g)
        p.shape_len = g.size
    if force_L is not None:
        Lin = np.zeros(max(max_imfs, 1), dtype=np.int32)
        fl = np.asarray(force_L, dtype=np.int32)[:max_imfs]
        Lin[:fl.size] = fl
        keep.append(Lin)
        p.L_in = _iptr(Lin)
    imfs = np.zeros((max_imfs + 1, n))
    m = np.zeros(max(max_imfs, 1), dtype=np.int32)
    L = np.zeros(max(max_imfs, 1), dtype=np.int32)
    kext = np.zeros(max_imfs + 1, dtype=np.int32)
    n_imfs = np.zeros(1, dtype=np.int32)
    status = np.zeros(1, dtype=np.int32)
    sd_m = np.zeros(max(max_imfs, 1))
    sd_prev = np.zeros(max(max_imfs, 1))
    sd_trace = np.full((max(max_imfs, 1), max_inner), np.nan) if trace else None
    imf_flags = np.zeros(max_imfs + 1, dtype=np.int32)
    o = _Outputs(_dptr(imfs), _iptr(m), _iptr(L), _iptr(kext), _iptr(n_imfs), _iptr(status),
                 _dptr(sd_m), _dptr(sd_prev), _dptr(sd_trace) if trace else None,
                 _iptr(imf_flags))
    rc = getattr(lib, fn_name)(_dptr(s), n, ctypes.byref(p), ctypes.byref(o))
    if rc != 0:
        raise ValueError(f"{fn_name}: invalid arguments (rc={rc})")
    K = int(n_imfs[0])
    out = {
        "imfs": imfs[:K].copy(), "remainder": imfs[K].copy(), "n_imfs": K,
        "m": m[:K].copy(), "L": L[:K].copy(), "kext": kext[:K + 1].copy(),
        "status": int(status[0]), "stop": int(status[0]) & 0xFF, "sd_m": sd_m[:K].copy(),
        "sd_prev": sd_prev[:K].copy(), "imf_flags": imf_flags[:K + 1].copy(),
    }
    if trace:
        out["sd_trace"] = sd_trace[:K].copy()
    return out


def iterative(s, **kw):
    """Tier A: Algorithm 2 (time-domain iteration).  Returns a dict with
    imfs [K, n], remainder [n], m [K], L [K], kext [K+1], status, stop,
    sd_m, sd_prev, imf_flags [K+1] (the flags raised at each outer step; entry K
    is the final stop test) and optionally sd_trace [K, max_inner]."""
    return _run("fifo_iterative", s, **kw)


def direct(s, **kw):
    """Tier B: the FIF direct method (Sec. 4).  Same outputs as iterative()."""
    return _run("fifo_direct", s, **kw)
