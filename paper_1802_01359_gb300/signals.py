"""Seeded synthetic input signals shaped like the paper's workloads.

This module holds no part of the decomposition method: it only draws signals.
It is the one module that both the CUDA path's callers (bench, tests) and the
FP64 oracle's tests use, so that both sides see identical inputs.

Signals live on the periodic grid x_j = j/n, j = 0..n-1.  A "component" is a
chirped, amplitude-modulated sinusoid

    A * (1 + d*cos(2*pi*f_am*x + psi)) * sin(2*pi*(f0*x + c*x^2) + phi)

with f0 log-uniform in [2, min(2000, n/8)] cycles, chirp rate c ~ U[0, 0.5*f0],
modulation depth d ~ U[0, 0.5], integer modulation frequency f_am ~ U{1..4},
amplitude A ~ U[0.1, 1] and phases ~ U[0, 2*pi).  Capping f0 at n/8 keeps the
peak instantaneous frequency f0 + 2c below n/4 (no aliasing).  Gaussian noise
is added last.  Signals are generated in float64 and rounded to float32; the
oracle consumes the float32 values widened back to float64.

Seeds: signal i of workload ``wid`` uses ``numpy.random.SeedSequence([wid, i])``.
"""
from __future__ import annotations

import math

import numpy as np

# Workload ids (the seed stream of each synthetic workload).
W_SINGLE_4096 = 0      # one n=4096 three-component test signal, numpy default_rng(0) noise
W_BATCH_16384 = 1      # 1024 signals, n=16384, 2-5 components
W_UNEVEN = 2           # 4096 signals, n log-uniform in [256, 2^20] rounded to 2^a 3^b
W_LONG_2P24 = 3        # one n=2^24 signal, 6 components spanning 1..1e6 cycles
W_BATCH_4096 = 4       # 65536 signals, n=4096


def single_4096(n: int = 4096) -> np.ndarray:
    """The three-component signal on x in [0,1): sin(2 pi 8x) + 0.5 sin(2 pi (60x + 40x^2))
    + 0.3 (1 + 0.5 cos(2 pi 2x)) sin(2 pi 300x) + N(0, 0.01^2) noise from default_rng(0).
    Returned as float32."""
    x = np.arange(n, dtype=np.float64) / n
    rng = np.random.default_rng(0)
    s = (np.sin(2 * np.pi * 8 * x) + 0.5 * np.sin(2 * np.pi * (60 * x + 40 * x ** 2))
         + 0.3 * (1 + 0.5 * np.cos(2 * np.pi * 2 * x)) * np.sin(2 * np.pi * 300 * x)
         + rng.normal(0.0, 0.01, n))
    return s.astype(np.float32)


def _component_params(rng: np.random.Generator, n: int, n_comp: int, f0_fixed=None):
    fmax = min(2000.0, n / 8.0)
    out = []
    for c in range(n_comp):
        if f0_fixed is not None:
            f0 = float(f0_fixed[c])
        else:
            f0 = math.exp(rng.uniform(math.log(2.0), math.log(max(fmax, 2.0))))
        out.append(dict(f0=f0, c=rng.uniform(0.0, 0.5 * f0), phi=rng.uniform(0, 2 * np.pi),
                        d=rng.uniform(0.0, 0.5), f_am=int(rng.integers(1, 5)),
                        psi=rng.uniform(0, 2 * np.pi), A=rng.uniform(0.1, 1.0)))
    return out


def component_signal(wid: int, idx: int, n: int, *, sigma: float = 0.01, n_comp=None,
                     f0_fixed=None) -> np.ndarray:
    """Signal ``idx`` of workload ``wid``: 2-5 random components (or ``n_comp``), plus
    N(0, sigma^2) noise, float32."""
    rng = np.random.default_rng(np.random.SeedSequence([wid, idx]))
    if n_comp is None:
        n_comp = int(rng.integers(2, 6))
    x = np.arange(n, dtype=np.float64) / n
    s = np.zeros(n)
    for p in _component_params(rng, n, n_comp, f0_fixed):
        s += (p["A"] * (1 + p["d"] * np.cos(2 * np.pi * p["f_am"] * x + p["psi"]))
              * np.sin(2 * np.pi * (p["f0"] * x + p["c"] * x * x) + p["phi"]))
    s += rng.normal(0.0, sigma, n)
    return s.astype(np.float32)


def smooth_lengths_between(lo: int, hi: int) -> np.ndarray:
    """All n = 2^a 3^b with lo <= n <= hi, sorted."""
    vals = []
    p3 = 1
    while p3 <= hi:
        v = p3
        while v <= hi:
            if v >= lo:
                vals.append(v)
            v *= 2
        p3 *= 3
    return np.array(sorted(vals), dtype=np.int64)


def uneven_lengths(count: int, lo: int = 256, hi: int = 1 << 20, wid: int = W_UNEVEN) -> np.ndarray:
    """Lengths log-uniform in [lo, hi], each rounded (in log) to the nearest 2^a 3^b."""
    rng = np.random.default_rng(np.random.SeedSequence([wid, 1 << 30]))
    cand = smooth_lengths_between(lo, hi)
    logc = np.log(cand.astype(np.float64))
    u = rng.uniform(math.log(lo), math.log(hi), count)
    idx = np.abs(u[:, None] - logc[None, :]).argmin(axis=1)
    return cand[idx]


def batch(wid: int, count: int, n, *, first: int = 0, sigma: float = 0.01) -> tuple[np.ndarray, np.ndarray]:
    """Signals first..first+count-1 of workload ``wid`` packed end to end.

    ``n`` is one length for all signals or an array of per-signal lengths.
    Returns (float32 samples, int64 offsets[count+1])."""
    lens = np.full(count, int(n), dtype=np.int64) if np.isscalar(n) else np.asarray(n, dtype=np.int64)
    offsets = np.zeros(count + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    data = np.empty(int(offsets[-1]), dtype=np.float32)
    for i in range(count):
        data[offsets[i]:offsets[i + 1]] = component_signal(wid, first + i, int(lens[i]), sigma=sigma)
    return data, offsets


def long_signal(n: int = 1 << 24, wid: int = W_LONG_2P24) -> np.ndarray:
    """Six components with f0 = 10^{0, 1.2, 2.4, 3.6, 4.8, 6} cycles, chirp and AM drawn as
    for the batch workloads, noise sigma = 1e-3."""
    f0 = [10.0 ** e for e in (0.0, 1.2, 2.4, 3.6, 4.8, 6.0)]
    return component_signal(wid, 0, n, sigma=1e-3, n_comp=6, f0_fixed=f0)
