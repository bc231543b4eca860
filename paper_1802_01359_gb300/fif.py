"""ctypes binding of libfif.so (the C ABI declared in include/fif.h).

Argument marshalling only: every step of the decomposition runs in the CUDA
kernels behind the C ABI.  PyTorch provides device memory and the stream.
There is no CPU fallback: without the built library every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfif.so")

FIF_OK = 0
FIF_EINVAL = 1
FIF_ENOMEM = 2
FIF_ECUDA = 3
FIF_ETIMEOUT = 4
FIF_EUNSUPPORTED = 5

STOP_EXTREMA = 1
STOP_MASK = 2
STOP_MAX_IMFS = 3
STOP_FORCED_END = 4
STOP_NONFINITE = 5
FLAG_NEAR_DELTA_TIE = 1 << 8
FLAG_EXTREMA_TIE = 1 << 9
FLAG_MAX_INNER_HIT = 1 << 10
FLAG_FP64_TIEBREAK = 1 << 11
FLAG_L_CLAMPED = 1 << 12
FORCE_L = 1
FORCE_MULTIPASS = 2
APRIORI_N0 = 4
PEAK_MASK = 8
WIN_TRIANGLE = 0
WIN_SHAPE = 1
PREC_FP32 = 0
PREC_SPLIT_BF16 = 1

# every symbol include/fif.h declares
EXPORTS = ("fif_plan_create", "fif_plan_destroy", "fif_plan_set_stream", "fif_plan_prepare",
           "fif_decompose", "fif_decompose_batch", "fif_decompose_batch_host", "fif_fused_max_n",
           "fif_status_string", "fif_decompose_noalloc", "fif_plan_tune", "fif_plan_get_schedule",
           "fif_plan_save_tuning", "fif_plan_load_tuning", "fif_plan_batch_launches",
           "fif_plan_get_multipass_schedule")
NOALLOC_MAX_N = 16384


class FifError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


class PlanDesc(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("nu", ctypes.c_double), ("mask_scale", ctypes.c_int32),
                ("delta", ctypes.c_double), ("max_inner", ctypes.c_int32),
                ("max_imfs", ctypes.c_int32), ("precision", ctypes.c_int),
                ("max_n", ctypes.c_int64), ("flags", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("window_shape", ctypes.POINTER(ctypes.c_double)),
                ("window_shape_len", ctypes.c_int32)]


class ImfDiag(ctypes.Structure):
    _fields_ = [("k_extrema", ctypes.c_int32), ("zero_crossings", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("inf_norm", ctypes.c_float)]


DIAG_DTYPE = np.dtype([("k_extrema", np.int32), ("zero_crossings", np.int32), ("flags", np.int32),
                       ("inf_norm", np.float32)])

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfif.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1802_01359_gb300.build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32p, i64p, fp = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    lib.fif_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PlanDesc), vp]
    lib.fif_plan_destroy.argtypes = [vp]
    lib.fif_plan_set_stream.argtypes = [vp, vp]
    lib.fif_plan_prepare.argtypes = [vp, i64p, ctypes.c_int64]
    lib.fif_decompose.argtypes = [vp, fp, ctypes.c_int64, fp, i32p, i32p, i32p, i32p, vp]
    lib.fif_decompose_batch.argtypes = [vp, fp, i64p, ctypes.c_int64, fp, i64p, i32p, i32p, i32p,
                                        i32p, vp]
    lib.fif_decompose_batch_host.argtypes = lib.fif_decompose_batch.argtypes
    lib.fif_decompose_noalloc.argtypes = [ctypes.POINTER(PlanDesc), fp, ctypes.c_int64, fp, i32p,
                                          i32p, i32p, i32p, vp, vp]
    lib.fif_decompose_noalloc.restype = ctypes.c_int
    lib.fif_fused_max_n.argtypes = []
    lib.fif_fused_max_n.restype = ctypes.c_int64
    lib.fif_status_string.argtypes = [ctypes.c_int]
    lib.fif_status_string.restype = ctypes.c_char_p
    lib.fif_plan_tune.argtypes = [vp, fp, i64p, ctypes.c_int64, fp, i64p, i32p, i32p, i32p, i32p]
    lib.fif_plan_get_schedule.argtypes = [vp, ctypes.c_int64, i32p, i32p, i32p]
    lib.fif_plan_get_multipass_schedule.argtypes = [vp, ctypes.c_int64] + [i32p] * 7
    lib.fif_plan_batch_launches.argtypes = [vp, ctypes.c_void_p]
    lib.fif_plan_save_tuning.argtypes = [vp, ctypes.c_char_p]
    lib.fif_plan_load_tuning.argtypes = [vp, ctypes.c_char_p]
    for name in ("fif_plan_create", "fif_plan_destroy", "fif_plan_set_stream", "fif_plan_prepare",
                 "fif_decompose", "fif_decompose_batch", "fif_decompose_batch_host",
                 "fif_plan_tune", "fif_plan_get_schedule", "fif_plan_save_tuning",
                 "fif_plan_load_tuning", "fif_plan_get_multipass_schedule"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load_library().fif_status_string(code).decode()


def _check(code: int, where: str):
    if code != FIF_OK:
        raise FifError(code, where)


def fused_max_n() -> int:
    return int(load_library().fif_fused_max_n())


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Decomposition:
    """Outputs of one decomposed signal (views on the batch outputs for batches)."""
    imfs: object          # [(max_imfs+1), n]; rows >= n_imfs+1 are not written
    m: object             # [max_imfs]
    mask_len: object      # [max_imfs]
    n_imfs: int
    status: int
    diag: Optional[np.ndarray] = None

    @property
    def stop(self) -> int:
        return self.status & 0xFF


@dataclass
class BatchResult:
    imfs: object          # packed, signal i at out_offsets[i], shape ((max_imfs+1) * n_i,)
    out_offsets: np.ndarray
    lengths: np.ndarray
    m: object             # [batch, max_imfs]
    mask_len: object      # [batch, max_imfs]
    n_imfs: object        # [batch]
    status: object        # [batch]
    diag: object = None   # [batch, max_imfs+1, 4] int32 view or None
    max_imfs: int = 0

    def signal(self, i: int) -> Decomposition:
        n = int(self.lengths[i])
        o = int(self.out_offsets[i])
        imfs = self.imfs[o:o + (self.max_imfs + 1) * n].reshape(self.max_imfs + 1, n)
        dg = None
        if self.diag is not None:
            d = self.diag[i]
            d = d.cpu().numpy() if hasattr(d, "cpu") else np.asarray(d)
            dg = np.ascontiguousarray(d).view(DIAG_DTYPE).reshape(-1)
        return Decomposition(imfs, self.m[i], self.mask_len[i], int(self.n_imfs[i]),
                             int(self.status[i]), dg)


def out_layout(lengths: Sequence[int], max_imfs: int) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.int64)
    out = np.zeros(lengths.size, dtype=np.int64)
    if lengths.size > 1:
        out[1:] = np.cumsum(lengths[:-1] * (max_imfs + 1))
    return out


class Plan:
    """A decomposition plan (fif_plan_create).  Parameters follow include/fif.h."""

    def __init__(self, *, nu: float = 1.6, mask_scale: int = 1, delta: float = 1e-3,
                 max_inner: int = 200, max_imfs: int = 10, max_n: int = 16384,
                 force_L: bool = False, multipass: bool = False, apriori_n0: bool = False,
                 gamma: float = 0.0, peak_mask: bool = False, window_shape=None, stream=None,
                 precision: int = 0):
        """window_shape: None for the triangle, else the samples of the generating
        shape g on [0, 1] (FIF_WIN_SHAPE; copied by the plan).  precision: PREC_FP32 or
        PREC_SPLIT_BF16 (tensor-core radix-16 passes of the fused inverse FFT)."""
        import torch
        lib = load_library()
        self.max_imfs = max_imfs
        self.max_n = max_n
        self.force_L = force_L
        self.desc = PlanDesc(0, nu, mask_scale, delta, max_inner, max_imfs, int(precision), max_n,
                             (FORCE_L if force_L else 0) | (FORCE_MULTIPASS if multipass else 0)
                             | (APRIORI_N0 if apriori_n0 else 0) | (PEAK_MASK if peak_mask else 0),
                             float(gamma))
        shape = None
        if window_shape is not None:
            shape = np.ascontiguousarray(np.asarray(window_shape, dtype=np.float64))
            self.desc.window = WIN_SHAPE
            self.desc.window_shape = shape.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self.desc.window_shape_len = shape.size
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.fif_plan_create(ctypes.byref(h), ctypes.byref(self.desc),
                                   ctypes.c_void_p(stream.cuda_stream)), "fif_plan_create")
        self._h = h
        self.desc.window_shape = None  # the plan holds its own copy
        del shape

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().fif_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self._stream = stream
        _check(load_library().fif_plan_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)),
               "fif_plan_set_stream")

    def prepare(self, lengths: Sequence[int]):
        arr = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
        _check(load_library().fif_plan_prepare(self._h, _np_ptr(arr), arr.size), "fif_plan_prepare")

    # ---------------------------------------------------------- one signal
    def decompose(self, signal, mask_len=None, diag: bool = False) -> Decomposition:
        """Plain staged path (one launch per step) on one float32 CUDA tensor."""
        import torch
        assert signal.is_cuda and signal.dtype == torch.float32 and signal.dim() == 1
        signal = signal.contiguous()
        n = signal.numel()
        dev = signal.device
        K = self.max_imfs
        imfs = torch.zeros((K + 1, n), dtype=torch.float32, device=dev)
        m = torch.zeros(max(K, 1), dtype=torch.int32, device=dev)
        L = torch.zeros(max(K, 1), dtype=torch.int32, device=dev)
        if mask_len is not None:
            L[:len(mask_len)] = torch.as_tensor(np.asarray(mask_len, dtype=np.int32), device=dev)
        nim = torch.zeros(1, dtype=torch.int32, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        dg = torch.zeros((K + 1, 4), dtype=torch.int32, device=dev) if diag else None
        _check(load_library().fif_decompose(self._h, _ptr(signal), n, _ptr(imfs), _ptr(m), _ptr(L),
                                            _ptr(nim), _ptr(st), _ptr(dg)), "fif_decompose")
        torch.cuda.current_stream().synchronize() if self._stream is None else self._stream.synchronize()
        d = None
        if dg is not None:
            d = np.ascontiguousarray(dg.cpu().numpy()).view(DIAG_DTYPE).reshape(-1)
        return Decomposition(imfs, m[:K], L[:K], int(nim.item()), int(st.item()), d)

    # ---------------------------------------------------------- batches
    def alloc_batch_outputs(self, lengths: Sequence[int], device, diag: bool = False) -> BatchResult:
        import torch
        lengths = np.asarray(lengths, dtype=np.int64)
        K = self.max_imfs
        out_off = out_layout(lengths, K)
        total = int(out_off[-1] + lengths[-1] * (K + 1)) if lengths.size else 0
        B = lengths.size
        return BatchResult(
            imfs=torch.empty(total, dtype=torch.float32, device=device), out_offsets=out_off,
            lengths=lengths,
            m=torch.zeros((B, max(K, 1)), dtype=torch.int32, device=device),
            mask_len=torch.zeros((B, max(K, 1)), dtype=torch.int32, device=device),
            n_imfs=torch.zeros(B, dtype=torch.int32, device=device),
            status=torch.zeros(B, dtype=torch.int32, device=device),
            diag=torch.zeros((B, K + 1, 4), dtype=torch.int32, device=device) if diag else None,
            max_imfs=K)

    def decompose_batch(self, signals, offsets, out: Optional[BatchResult] = None,
                        diag: bool = False) -> BatchResult:
        """Fused batch path.  signals: packed float32 CUDA tensor; offsets: host int64[batch+1]."""
        import torch
        assert signals.is_cuda and signals.dtype == torch.float32
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        lengths = np.diff(offsets)
        if out is None:
            out = self.alloc_batch_outputs(lengths, signals.device, diag)
        oo = np.ascontiguousarray(out.out_offsets)
        _check(load_library().fif_decompose_batch(
            self._h, _ptr(signals), _np_ptr(offsets), lengths.size, _ptr(out.imfs), _np_ptr(oo),
            _ptr(out.m), _ptr(out.mask_len), _ptr(out.n_imfs), _ptr(out.status), _ptr(out.diag)),
            "fif_decompose_batch")
        return out

    def tune(self, signals, offsets, out: Optional[BatchResult] = None) -> BatchResult:
        """Autotune the fused schedule of every fused length class of this batch (see
        fif_plan_tune); returns the outputs of the final run with the chosen schedules."""
        import torch
        assert signals.is_cuda and signals.dtype == torch.float32
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        lengths = np.diff(offsets)
        if out is None:
            out = self.alloc_batch_outputs(lengths, signals.device)
        oo = np.ascontiguousarray(out.out_offsets)
        _check(load_library().fif_plan_tune(
            self._h, _ptr(signals), _np_ptr(offsets), lengths.size, _ptr(out.imfs), _np_ptr(oo),
            _ptr(out.m), _ptr(out.mask_len), _ptr(out.n_imfs), _ptr(out.status)), "fif_plan_tune")
        return out

    def schedule(self, n: int) -> tuple:
        """(E, threads, tuned) of the fused schedule for length n."""
        E, T, tuned = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load_library().fif_plan_get_schedule(self._h, int(n), ctypes.byref(E),
                                                    ctypes.byref(T), ctypes.byref(tuned)),
               "fif_plan_get_schedule")
        return E.value, T.value, bool(tuned.value)

    def multipass_schedule(self, n: int) -> dict:
        """The multi-pass schedule of length n (fif_plan_get_multipass_schedule)."""
        v = [ctypes.c_int32() for _ in range(7)]
        _check(load_library().fif_plan_get_multipass_schedule(self._h, int(n),
                                                              *[ctypes.byref(x) for x in v]),
               "fif_plan_get_multipass_schedule")
        R1, R2, E1, TJ1, E2, TJ2, tuned = (x.value for x in v)
        return dict(R1=R1, R2=R2, E1=E1, TJ1=TJ1, E2=E2, TJ2=TJ2, tuned=bool(tuned))

    def batch_launches(self) -> int:
        """Kernel launches one decompose_batch call enqueues for the last prepared layout."""
        v = ctypes.c_int64()
        _check(load_library().fif_plan_batch_launches(self._h, ctypes.byref(v)),
               "fif_plan_batch_launches")
        return int(v.value)

    def save_tuning(self, path: str):
        _check(load_library().fif_plan_save_tuning(self._h, os.fsencode(path)),
               "fif_plan_save_tuning")

    def load_tuning(self, path: str):
        _check(load_library().fif_plan_load_tuning(self._h, os.fsencode(path)),
               "fif_plan_load_tuning")

    def decompose_batch_host(self, signals: np.ndarray, offsets, mask_len=None,
                             diag: bool = False, out: Optional[dict] = None) -> BatchResult:
        """Host-buffer entry point: copies in, decomposes, copies out (blocking)."""
        signals = np.ascontiguousarray(signals, dtype=np.float32)
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        lengths = np.diff(offsets)
        K = self.max_imfs
        B = lengths.size
        oo = out_layout(lengths, K)
        if out is None:
            total = int(oo[-1] + lengths[-1] * (K + 1)) if B else 0
            out = dict(imfs=np.empty(total, np.float32), m=np.zeros((B, max(K, 1)), np.int32),
                       mask_len=np.zeros((B, max(K, 1)), np.int32), n_imfs=np.zeros(B, np.int32),
                       status=np.zeros(B, np.int32),
                       diag=np.zeros((B, K + 1, 4), np.int32) if diag else None)
        if mask_len is not None:
            out["mask_len"][...] = mask_len
        _check(load_library().fif_decompose_batch_host(
            self._h, _np_ptr(signals), _np_ptr(offsets), B, _np_ptr(out["imfs"]), _np_ptr(oo),
            _np_ptr(out["m"]), _np_ptr(out["mask_len"]), _np_ptr(out["n_imfs"]),
            _np_ptr(out["status"]), _np_ptr(out["diag"])), "fif_decompose_batch_host")
        return BatchResult(out["imfs"], oo, lengths, out["m"], out["mask_len"], out["n_imfs"],
                           out["status"], out["diag"], K)


def decompose_noalloc(signal, *, nu: float = 1.6, mask_scale: int = 1, delta: float = 1e-3,
                      max_inner: int = 200, max_imfs: int = 10, mask_len=None, diag: bool = False,
                      apriori_n0: bool = False, gamma: float = 0.0, peak_mask: bool = False,
                      stream=None) -> Decomposition:
    """fif_decompose_noalloc on one float32 CUDA tensor (no plan, no device allocation
    inside the library; the output tensors are allocated here by PyTorch)."""
    import torch
    assert signal.is_cuda and signal.dtype == torch.float32 and signal.dim() == 1
    signal = signal.contiguous()
    n = signal.numel()
    dev = signal.device
    K = max_imfs
    desc = PlanDesc(0, nu, mask_scale, delta, max_inner, max_imfs, 0, n,
                    (FORCE_L if mask_len is not None else 0) | (APRIORI_N0 if apriori_n0 else 0)
                    | (PEAK_MASK if peak_mask else 0), float(gamma))
    imfs = torch.zeros((K + 1, n), dtype=torch.float32, device=dev)
    m = torch.zeros(max(K, 1), dtype=torch.int32, device=dev)
    L = torch.zeros(max(K, 1), dtype=torch.int32, device=dev)
    if mask_len is not None:
        L[:len(mask_len)] = torch.as_tensor(np.asarray(mask_len, dtype=np.int32), device=dev)
    nim = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    dg = torch.zeros((K + 1, 4), dtype=torch.int32, device=dev) if diag else None
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    _check(load_library().fif_decompose_noalloc(
        ctypes.byref(desc), _ptr(signal), n, _ptr(imfs), _ptr(m), _ptr(L), _ptr(nim), _ptr(st),
        _ptr(dg), ctypes.c_void_p(stream.cuda_stream)), "fif_decompose_noalloc")
    stream.synchronize()
    d = None
    if dg is not None:
        d = np.ascontiguousarray(dg.cpu().numpy()).view(DIAG_DTYPE).reshape(-1)
    return Decomposition(imfs, m[:K], L[:K], int(nim.item()), int(st.item()), d)
