"""FFT-based Iterative Filtering (FIF) for GB300 (sm_103a).

The decomposition runs in hand-written CUDA kernels behind the C ABI declared in
``include/fif.h`` (``libfif.so``); :mod:`paper_1802_01359_gb300.fif` is the thin
ctypes binding.  :mod:`paper_1802_01359_gb300.signals` draws seeded synthetic inputs.
"""
__all__ = ["fif", "signals"]
