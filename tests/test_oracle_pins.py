"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the DFT
definition (brute force), closed forms derived from the paper's theorems,
invariants the paper proves, exact symmetries, and the agreement of the two
independent tiers (time-domain Algorithm 2 vs. the spectral direct method of
Sec. 4).
"""
import math

import numpy as np
import pytest

from paper_1802_01359_gb300 import signals

SMOOTH_SMALL = [n for n in signals.smooth_lengths_between(1, 2048)]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# ----------------------------------------------------------------- FFT

@pytest.mark.parametrize("n", list(range(1, 65)) + [96, 243, 256, 729, 1024, 1536, 2048])
def test_fft_matches_bruteforce_dft(oracle_mod, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, +1):
        X = oracle_mod.fft(x, sign)
        D = oracle_mod.dft(x.real, x.imag, sign)
        assert rel(X, D) < 1e-13
    # the definition itself, on an impulse and a constant (exact closed forms)
    e = np.zeros(n); e[min(1, n - 1)] = 1.0
    k = np.arange(n)
    assert np.allclose(oracle_mod.dft(e), np.exp(-2j * np.pi * k * min(1, n - 1) / n), atol=1e-13)
    assert np.allclose(oracle_mod.dft(np.ones(n)), np.where(k == 0, n, 0), atol=1e-12 * n)


def test_fft_against_numpy_pocketfft(oracle_mod):
    for n in SMOOTH_SMALL:
        x = np.random.default_rng(n + 7).standard_normal(n)
        assert rel(oracle_mod.fft(x), np.fft.fft(x)) < 1e-13


# --------------------------------------------------------- window spectrum

@pytest.mark.parametrize("n,L", [(64, 8), (64, 5), (65, 7), (243, 40), (256, 2), (1000, 333),
                                 (2048, 409), (729, 364), (4096, 409)])
def test_window_spectrum_is_dft_of_taps(oracle_mod, n, L):
    """eq. Lambdas: the circulant's eigenvalues are the DFT of its first row; the
    closed form must equal the brute-force DFT of the sampled, normalised taps."""
    c = oracle_mod.taps(n, L)
    assert abs(c.sum() - 1.0) < 1e-15 and (c >= 0).all()            # row stochastic (eq. W_m)
    assert np.allclose(c[1:], c[1:][::-1], atol=0)                  # symmetric: c_{n-j} = c_j
    lam = oracle_mod.dft(c)
    assert np.abs(lam.imag).max() < 1e-13                           # real spectrum (Theorem 4)
    w = oracle_mod.window_spectrum(n, L)
    assert np.abs(w - lam.real).max() < 1e-13


@pytest.mark.parametrize("n,L", [(64, 8), (243, 40), (4096, 409), (16384, 7), (16384, 8191)])
def test_window_spectrum_range(oracle_mod, n, L):
    """Theorem 4 / Corollary 2: lambda_0 = 1, every other eigenvalue in [0, 1)."""
    w = oracle_mod.window_spectrum(n, L)
    assert w[0] == 1.0
    assert w[1:].min() >= 0.0 and w[1:].max() < 1.0
    # zeros exactly where k*L is a multiple of n (sin(pi k L / n) = 0)
    k = np.arange(1, n)
    assert np.array_equal(w[1:] == 0.0, (k * L) % n == 0)


# ------------------------------------------------------------ mask length

def test_mask_length_rule(oracle_mod):
    # eq. Unif_Mask_length with leading factor 1 and 2
    assert oracle_mod.mask_length(4096, 16) == 409          # floor(409.6)
    assert oracle_mod.mask_length(4096, 16, mask_scale=2) == 818
    assert oracle_mod.mask_length(1000, 16) == 100          # exact integer quotient
    assert oracle_mod.mask_length(4096, 606) == 10
    assert oracle_mod.mask_length(10, 9) == 1               # clamped later to 2


def test_extrema_and_zero_crossings_small(oracle_mod):
    assert oracle_mod.count_extrema([0, 1, 0, 1]) == 4       # periodic alternation
    assert oracle_mod.count_extrema([0, 1, 2, 3]) == 2       # ramp: max at 3, min at 0 (wrap)
    assert oracle_mod.count_extrema([1, 1, 1, 1]) == 0
    assert oracle_mod.count_extrema([0, 1, 1, 0]) == 0       # flat tops count no strict extremum
    assert oracle_mod.count_extrema([0, 2, 1, 2]) == 4
    n = 4096
    j = np.arange(n)
    assert oracle_mod.count_extrema(np.cos(2 * np.pi * 8 * j / n + 0.3)) == 16
    assert oracle_mod.count_zero_crossings(np.cos(2 * np.pi * 8 * j / n + 0.3)) == 16
    assert oracle_mod.count_zero_crossings([1, -1, 1, -1]) == 4


# -------------------------------------------------------- Theorem 2 / 5

def test_pure_tone_scaled_by_multiplier(oracle_mod):
    """A tone at bin k0 is an eigenvector of W: Algorithm 2 returns it scaled by
    (1 - lambda_k0)^m (eq. IMF_IF_stop, eq. IMF1_direct), and SD_j = lambda_k0
    for every j (eq. SD with Parseval), so m is 1 or max_inner."""
    n, k0, phi = 4096, 8, 0.3
    j = np.arange(n)
    s = np.cos(2 * np.pi * k0 * j / n + phi)
    a = oracle_mod.iterative(s, max_imfs=1, trace=True)
    # 16 extrema, L = floor(1.6*4096/16) = 409
    assert a["kext"][0] == 16 and a["L"][0] == 409
    lam = oracle_mod.dft(oracle_mod.taps(n, 409)).real[k0]      # eigenvalue by the definition
    assert abs(lam - 0.05541415768287662) < 1e-14
    assert lam > 1e-3 and a["m"][0] == 200                         # SD never drops below delta
    assert a["status"] & oracle_mod.FLAG_MAX_INNER_HIT
    assert np.allclose(a["sd_trace"][0], lam, rtol=1e-11, atol=0)
    scale = (1 - lam) ** 200
    assert abs(scale - 1.1176000063634996e-05) < 1e-15
    # 200 steps of round-off stay at ~1e-15 of ||s|| (the IMF itself is 1e-5 ||s||)
    assert np.linalg.norm(a["imfs"][0] - scale * s) < 1e-13 * np.linalg.norm(s)
    b = oracle_mod.direct(s, max_imfs=1)
    assert b["m"][0] == 200
    assert np.linalg.norm(b["imfs"][0] - scale * s) < 1e-13 * np.linalg.norm(s)
    # a tone at a zero of the window spectrum passes unchanged after one step
    s2 = np.cos(2 * np.pi * 16 * j / 256)
    a2 = oracle_mod.iterative(s2, force_L=[16], max_imfs=1)          # 16*16 = 256: lambda_16 = 0
    assert a2["m"][0] == 1 and rel(a2["imfs"][0], s2) < 1e-13


def _two_tone_sd(lam4, j):
    a = (1 - lam4) ** 2
    return math.sqrt(lam4 ** 2 * a ** (j - 1) / (a ** (j - 1) + 1))


def test_interior_m_closed_form(oracle_mod):
    """Two equal tones, one on a zero of the window spectrum (bin 8, L = 8, n = 64)
    and one at lambda_4: SD_j^2 = lambda_4^2 a^{j-1} / (a^{j-1} + 1), a =
    (1-lambda_4)^2, first below delta = 1e-3 at j = 13 (interior m)."""
    n = 64
    j = np.arange(n)
    s = np.cos(2 * np.pi * 8 * j / n) + np.cos(2 * np.pi * 4 * j / n)
    lam = oracle_mod.dft(oracle_mod.taps(n, 8)).real
    assert abs(lam[8]) < 1e-15
    lam4 = lam[4]
    assert abs(lam4 - 1 / (64 * math.sin(math.pi / 16) ** 2)) < 1e-14
    sd = [_two_tone_sd(lam4, jj) for jj in range(1, 40)]
    m_expected = next(jj for jj in range(1, 40) if sd[jj - 1] < 1e-3)
    assert m_expected == 13
    for tier in (oracle_mod.iterative, oracle_mod.direct):
        r = tier(s, force_L=[8], max_imfs=1, delta=1e-3, trace=True)
        assert r["m"][0] == 13
        assert np.allclose(r["sd_trace"][0][:13], sd[:13], rtol=1e-10, atol=0)
        g = (1 - lam) ** 13
        expected = np.real(np.fft.ifft(g * np.fft.fft(s)))           # eq. One step_algo
        assert rel(r["imfs"][0], expected) < 1e-12


def test_absolute_criterion_bound(oracle_mod):
    """Theorem 5: under the absolute rule (eq. Discrete_Abs_StopCond) the
    iteration stops no later than the a-priori N0 of eq. N0_discrete.  With m
    counting applications of (I-W), the rule is met for m - 1 >= N0."""
    for seed, n in [(1, 256), (2, 384), (3, 512)]:
        s = signals.component_signal(99, seed, n).astype(np.float64)
        s /= np.linalg.norm(s)                                        # Sec. 3: WLOG ||s||_2 = 1
        delta = 1e-3
        r = oracle_mod.iterative(s, max_imfs=1, delta=delta, absolute=True, max_inner=100000)
        L = int(r["L"][0])
        lam = oracle_mod.window_spectrum(n, L)
        kz = int((lam[1:] == 0).sum())
        st = np.abs(oracle_mod.fft(s)) / math.sqrt(n)                # unitary DFT (U^T s)
        bound = delta / (st.max() * math.sqrt(n - 1 - kz))
        # smallest N0 with N0^N0 / (N0+1)^(N0+1) < bound, in logs
        N0 = next(N for N in range(1, 10 ** 8)
                  if N * math.log(N) - (N + 1) * math.log(N + 1) < math.log(bound))
        m_abs = int(r["m"][0])
        assert m_abs - 1 <= N0, (m_abs, N0)
        d = oracle_mod.direct(s, max_imfs=1, delta=delta, absolute=True, max_inner=100000)
        assert d["m"][0] == m_abs


# ----------------------------------------------- direct = iterative (Thm 5)

CASES = [(0, 128, 1e-3), (1, 256, 1e-2), (2, 384, 1e-3), (3, 729, 1e-2), (4, 1024, 1e-2),
         (5, 243, 5e-2), (6, 512, 3e-2)]


@pytest.mark.parametrize("seed,n,delta", CASES)
def test_direct_equals_iterative(oracle_mod, seed, n, delta):
    s = signals.component_signal(98, seed, n).astype(np.float64)
    kw = dict(max_imfs=5, max_inner=80, delta=delta, trace=True)
    a = oracle_mod.iterative(s, **kw)
    b = oracle_mod.direct(s, **kw)
    assert a["n_imfs"] == b["n_imfs"] and a["status"] == b["status"]
    assert np.array_equal(a["m"], b["m"]) and np.array_equal(a["L"], b["L"])
    assert np.array_equal(a["kext"], b["kext"])
    for i in range(a["n_imfs"]):
        assert rel(a["imfs"][i], b["imfs"][i]) < 1e-11
        mm = a["m"][i]
        # Parseval: the time-domain SD sequence equals the spectral one
        assert np.allclose(a["sd_trace"][i][:mm], b["sd_trace"][i][:mm], rtol=1e-10, atol=0)
    assert rel(a["remainder"], b["remainder"]) < 1e-11


def test_interior_m_occurs_in_random_cases(oracle_mod):
    """At least some of the parametrised cases above exercise 1 < m < max_inner."""
    ms = []
    for seed, n, delta in CASES:
        s = signals.component_signal(98, seed, n).astype(np.float64)
        ms += list(oracle_mod.direct(s, max_imfs=5, max_inner=80, delta=delta)["m"])
    assert any(1 < m < 80 for m in ms)


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("tier", ["iterative", "direct"])
def test_reconstruction_and_zero_mean(oracle_mod, tier):
    """Algorithm 1/2 telescopes: s = sum of IMFs + remainder.  Every IMF has zero
    mean (lambda_0 = 1 removes the DC bin)."""
    s = signals.single_4096().astype(np.float64)[:1024]
    r = getattr(oracle_mod, tier)(s, max_imfs=6)
    assert r["n_imfs"] == 6
    assert np.abs(r["imfs"].sum(0) + r["remainder"] - s).max() < 1e-13
    assert np.abs(r["imfs"].mean(axis=1)).max() < 1e-14


def test_sd_monotone_nonincreasing(oracle_mod):
    """SD_j^2 is the mean of lambda^2 under weights |r_k|^2 (1-lambda_k)^{2(j-1)};
    raising j reweights towards small lambda, so SD_j never increases."""
    for seed in range(6):
        s = signals.component_signal(97, seed, 512).astype(np.float64)
        r = oracle_mod.direct(s, max_imfs=3, max_inner=200, delta=1e-9, trace=True)
        for i in range(r["n_imfs"]):
            t = r["sd_trace"][i]
            assert (np.diff(t) <= 1e-15 * t[:-1]).all()


def test_linearity_with_fixed_schedule(oracle_mod):
    """With L and m fixed, each IMF is a fixed linear map of s (eq. MatrixForm),
    so the decomposition superposes (the nonlinearity of Sec. 2 comes only from
    choosing L from the data)."""
    n = 512
    x = signals.component_signal(96, 0, n).astype(np.float64)
    y = signals.component_signal(96, 1, n).astype(np.float64)
    kw = dict(force_L=[4, 12, 40], max_imfs=3, max_inner=30, delta=1e-300)
    for tier in (oracle_mod.iterative, oracle_mod.direct):
        rx, ry = tier(x, **kw), tier(y, **kw)
        rz = tier(2.5 * x - 0.75 * y, **kw)
        assert (rz["m"] == 30).all() and rz["n_imfs"] == 3
        assert rel(rz["imfs"], 2.5 * rx["imfs"] - 0.75 * ry["imfs"]) < 1e-12
        assert rel(rz["remainder"], 2.5 * rx["remainder"] - 0.75 * ry["remainder"]) < 1e-12


def test_exact_symmetries(oracle_mod):
    """Negation and power-of-two scaling are exact in binary64: identical integers and
    exactly transformed outputs.  A circular shift leaves the integers unchanged and
    shifts every IMF."""
    s = signals.component_signal(95, 3, 768).astype(np.float64)
    kw = dict(max_imfs=4, max_inner=60, delta=1e-2)
    b = oracle_mod.direct(s, **kw)
    for f in (-1.0, 4.0, 0.125):
        t = oracle_mod.direct(f * s, **kw)
        assert np.array_equal(t["m"], b["m"]) and np.array_equal(t["L"], b["L"])
        assert np.array_equal(t["imfs"], f * b["imfs"])
    a = oracle_mod.iterative(s, **kw)
    for f in (-1.0, 4.0):
        t = oracle_mod.iterative(f * s, **kw)
        assert np.array_equal(t["m"], a["m"]) and np.array_equal(t["imfs"], f * a["imfs"])
    sh = oracle_mod.direct(np.roll(s, 37), **kw)
    assert np.array_equal(sh["m"], b["m"]) and np.array_equal(sh["L"], b["L"])
    assert rel(sh["imfs"], np.roll(b["imfs"], 37, axis=1)) < 1e-12


def test_trivial_and_degenerate_inputs(oracle_mod):
    for tier in (oracle_mod.iterative, oracle_mod.direct):
        z = tier(np.zeros(64))
        assert z["n_imfs"] == 0 and z["stop"] == oracle_mod.STOP_EXTREMA
        assert (z["remainder"] == 0).all()
        c = tier(np.full(100, 3.25))
        assert c["n_imfs"] == 0 and (c["remainder"] == 3.25).all()
        one = tier(np.array([1.0]))
        assert one["n_imfs"] == 0
        # a single period of a cosine has k = 2: L = floor(1.6 n/2) makes 2L-1 > n
        n = 128
        cos1 = np.cos(2 * np.pi * np.arange(n) / n)
        t = tier(cos1)
        assert t["n_imfs"] == 0 and t["stop"] == oracle_mod.STOP_MASK
        nan = np.ones(16); nan[3] = np.nan
        t = tier(nan)
        assert t["stop"] == oracle_mod.STOP_NONFINITE and t["n_imfs"] == 0
        # max_imfs = 0: no IMF, the signal is the remainder
        t = tier(signals.component_signal(94, 0, 256).astype(np.float64), max_imfs=0)
        assert t["n_imfs"] == 0 and t["stop"] == oracle_mod.STOP_MAX_IMFS
        # a tiny L is clamped to 2 and flagged (alternating signal: k = n)
        alt = np.tile([1.0, -1.0], 32)
        t = tier(alt, max_imfs=1)
        assert t["L"][0] == 2 and t["status"] & oracle_mod.FLAG_L_CLAMPED


def test_config_single_4096_saturates_max_inner(oracle_mod):
    """The three-component n=4096 signal at delta=1e-3: SD_200 stays above delta for
    every IMF (m = max_inner), the outer loop stops on max_imfs = 10."""
    s = signals.single_4096().astype(np.float64)
    b = oracle_mod.direct(s)
    assert b["n_imfs"] == 10 and b["stop"] == oracle_mod.STOP_MAX_IMFS
    assert (b["m"] == 200).all()
    assert b["status"] & oracle_mod.FLAG_MAX_INNER_HIT
    assert set(b["L"].tolist()) <= {10, 11}


def test_golden_single_4096_regression(oracle_mod):
    """Regression fixture written by tests/golden/make_golden.py (oracle only): both tiers
    still produce the stored integers on the n=4096 three-component signal, and so do the
    direct tier's options (a-priori N0, threshold, peak mask, shape window)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "single_4096_oracle.json")) as f:
        g = json.load(f)
    s = signals.single_4096().astype(np.float64)
    b = oracle_mod.direct(s)
    assert b["m"].tolist() == g["direct"]["m"] and b["L"].tolist() == g["direct"]["L"]
    assert b["kext"].tolist() == g["direct"]["kext"] and b["status"] == g["direct"]["status"]
    assert g["iterative"]["m"] == g["direct"]["m"] and g["iterative"]["L"] == g["direct"]["L"]
    assert np.allclose([np.linalg.norm(x) for x in b["imfs"]], g["direct"]["imf_l2"], rtol=1e-12)
    modes = {"apriori_delta2": dict(apriori=True, delta=2.0, max_inner=1 << 16),
             "threshold_gamma0.05": dict(gamma=0.05),
             "peak_mask": dict(peak_mask=True),
             "shape_sine33": dict(shape=np.sin(np.pi * np.linspace(0.0, 1.0, 33)))}
    for name, kw in modes.items():
        r, ref = oracle_mod.direct(s, **kw), g["direct_" + name]
        assert r["m"].tolist() == ref["m"] and r["L"].tolist() == ref["L"], name
        assert r["kext"].tolist() == ref["kext"] and r["status"] == ref["status"], name
        assert np.allclose([np.linalg.norm(x) for x in r["imfs"]], ref["imf_l2"], rtol=1e-12), name


def _algorithm2_high_precision(s, *, max_imfs, max_inner, delta, nu=1.6, dps=60):
    """Algorithm 2 (time-domain iteration, eq. s_m+1 and eq. SD) in 60-digit arithmetic,
    written independently of the C oracle, for tiny n."""
    import mpmath as mp
    mp.mp.dps = dps
    n = len(s)
    r = [mp.mpf(float(x)) for x in s]
    out = {"m": [], "L": [], "kext": []}

    def extrema(v):
        c = 0
        for i in range(n):
            a, b = v[i] - v[i - 1], v[(i + 1) % n] - v[i]
            c += (a > 0 and b < 0) or (a < 0 and b > 0)
        return c

    K = 0
    while True:
        k = extrema(r)
        out["kext"].append(k)
        if k < 2:
            out["stop"] = 1
            break
        L = int(math.floor((nu * n) / k))
        L = max(L, 2)
        if 2 * L - 1 > n:
            out["stop"] = 2
            break
        if K == max_imfs:
            out["stop"] = 3
            break
        taps = {d: mp.mpf(L - abs(d)) / (L * L) for d in range(-(L - 1), L)}
        tot = sum(taps.values())
        taps = {d: c / tot for d, c in taps.items()}
        u = r[:]
        for j in range(1, max_inner + 1):
            v = [sum(c * u[(i - d) % n] for d, c in taps.items()) for i in range(n)]
            num = sum(x * x for x in v)
            den = sum(x * x for x in u)
            u = [a - b for a, b in zip(u, v)]
            if mp.sqrt(num / den) < delta:
                break
        out["m"].append(j)
        out["L"].append(L)
        r = [a - b for a, b in zip(r, u)]
        K += 1
    return out


@pytest.mark.parametrize("seed,n,delta", [(1, 6, 2e-2), (0, 8, 1e-3), (2, 12, 2e-2), (3, 16, 1e-2),
                                          (4, 16, 1e-3), (5, 12, 1e-3)])
def test_direct_matches_high_precision_algorithm2(oracle_mod, seed, n, delta):
    """Tier B against Algorithm 2 carried out in 60-digit arithmetic: same extrema counts,
    L, m and number of IMFs.  The (seed 1, n 6) case uses L = 2 twice: the window
    eigenvalue at n/2 is exactly 0, exact arithmetic empties that bin of the
    remainder, and m of the second IMF is max_inner; a binary64 time-domain iteration
    keeps round-off there that ends the second inner loop early."""
    s = signals.component_signal(50, seed, n).astype(np.float64)
    hp = _algorithm2_high_precision(s, max_imfs=4, max_inner=200, delta=delta)
    b = oracle_mod.direct(s, max_imfs=4, max_inner=200, delta=delta)
    assert b["m"].tolist() == hp["m"]
    assert b["L"].tolist() == hp["L"]
    assert b["kext"].tolist() == hp["kext"]
    assert b["stop"] == hp["stop"]


def test_exactly_zero_window_bins_stay_empty(oracle_mod):
    """Where w_hat_k = 0 the multiplier (1 - w_hat_k)^m is 1: the IMF takes the whole bin
    and the remainder spectrum is exactly 0 there (tier B)."""
    n = 64
    s = signals.component_signal(49, 0, n).astype(np.float64)
    b = oracle_mod.direct(s, force_L=[8], max_imfs=1, max_inner=20, delta=1e-300)
    w = oracle_mod.window_spectrum(n, 8)
    zero = np.nonzero(w == 0.0)[0]
    assert zero.size > 0
    R = np.fft.fft(b["remainder"])
    assert np.abs(R[zero]).max() < 1e-13 * np.abs(R).max()
    I = np.fft.fft(b["imfs"][0])
    S = np.fft.fft(s)
    assert np.allclose(I[zero], S[zero], rtol=1e-12, atol=1e-12 * np.abs(S).max())


# ---------------------------------------------------------------- a-priori N0 mode
# Theorem 5, eq. N0_discrete: m = the least natural N0 with
# N0^N0 / (N0+1)^(N0+1) < delta / (||U^T r||_inf sqrt(n - 1 - k)).

def _n0_exact(snorm, n, kzero, delta, cap):
    """Least N >= 1 (or cap + 1) with f(N) < delta / (snorm sqrt(dof)), decided in exact
    rational arithmetic on the squared inequality f(N)^2 snorm^2 dof < delta^2."""
    from fractions import Fraction
    dof = n - 1 - kzero
    sn, de = Fraction(snorm), Fraction(delta)
    for N in range(1, cap + 1):
        f = Fraction(N ** N, (N + 1) ** (N + 1))
        if f * f * sn * sn * dof < de * de:
            return N
    return cap + 1


@pytest.mark.parametrize("seed", range(12))
def test_apriori_n0_is_the_least_solution(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.choice([16, 64, 100, 256, 1024]))
    kzero = int(rng.integers(0, 4))
    snorm = float(10.0 ** rng.uniform(-1, 1.5))
    delta = float(10.0 ** rng.uniform(-2, 0))
    N0, tie = oracle_mod.apriori_n0(snorm, n, kzero, delta, 250)
    if tie:
        pytest.skip("boundary within 1e-6: either integer is admissible")
    assert N0 == _n0_exact(snorm, n, kzero, delta, 250)


def test_apriori_n0_degenerate_right_sides(oracle_mod):
    assert oracle_mod.apriori_n0(0.0, 64, 0, 1e-3, 200) == (1, False)   # zero remainder
    assert oracle_mod.apriori_n0(5.0, 8, 7, 1e-3, 200) == (1, False)    # n - 1 - k = 0
    assert oracle_mod.apriori_n0(1e9, 64, 0, 1e-9, 200)[0] == 201       # beyond the cap


@pytest.mark.parametrize("n,L", [(64, 8), (64, 6), (96, 12), (243, 27), (100, 10), (128, 7)])
def test_zero_eigenvalue_count_is_gcd_minus_one(oracle_mod, n, L):
    """w_hat_k = 0 exactly for k in [1, n-1] with kL = 0 mod n: gcd(n, L) - 1 of them."""
    import math
    w = oracle_mod.window_spectrum(n, L)
    assert int(np.sum(w[1:] == 0.0)) == math.gcd(n, L) - 1


def _apply_i_minus_w(u, L):
    """u - W u with W the periodic convolution by the sampled triangle c_d = (L-|d|)/L^2."""
    n = u.size
    out = u.copy()
    for d in range(-(L - 1), L):
        out -= (L - abs(d)) / L ** 2 * np.roll(u, d)
    return out


@pytest.mark.parametrize("seed,n", [(0, 64), (1, 96), (2, 128)])
def test_apriori_mode_meets_theorem5(oracle_mod, seed, n):
    """With m = N0 every IMF satisfies the absolute criterion of Theorem 5 at the next step:
    ||(I-W)^(N0+1) r - (I-W)^N0 r||_2 < delta, r the remainder it was taken from."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    s = np.sin(2 * np.pi * 3 * x) + 0.4 * np.sin(2 * np.pi * 11 * x) + 0.05 * rng.standard_normal(n)
    delta = 0.05
    res = oracle_mod.iterative(s, apriori=True, delta=delta, max_inner=2000, max_imfs=3)
    K = int(res["n_imfs"])
    assert K >= 1
    import math
    r = s.copy()
    for k in range(K):
        imf = res["imfs"][k]
        L = int(res["L"][k])
        nxt = _apply_i_minus_w(imf, L)
        assert np.linalg.norm(nxt - imf) < delta
        # and m is the least N0 for this remainder: ||U^T r||_inf from numpy's FFT
        # (unitary: / sqrt(n)), k = gcd(n, L) - 1 zero eigenvalues, exact comparison
        snorm = np.abs(np.fft.fft(r)).max() / math.sqrt(n)
        if not res["status"] & oracle_mod.FLAG_NEAR_DELTA_TIE:
            assert int(res["m"][k]) == _n0_exact(snorm, n, math.gcd(n, L) - 1, delta, 2000)
        r = r - imf


@pytest.mark.parametrize("seed,n", [(3, 64), (4, 72), (5, 81), (6, 128)])
def test_apriori_direct_equals_iterative(oracle_mod, seed, n):
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    s = np.sin(2 * np.pi * 2 * x) + 0.5 * np.sin(2 * np.pi * 9 * x) + 0.02 * rng.standard_normal(n)
    kw = dict(apriori=True, delta=0.02, max_inner=5000, max_imfs=4)
    a, b = oracle_mod.iterative(s, **kw), oracle_mod.direct(s, **kw)
    K = int(a["n_imfs"])
    assert K == int(b["n_imfs"]) and a["status"] == b["status"]
    assert np.array_equal(a["m"][:K], b["m"][:K]) and np.array_equal(a["L"][:K], b["L"][:K])
    assert np.abs(a["imfs"][:K + 1] - b["imfs"][:K + 1]).max() < 1e-10 * np.abs(s).max()


def test_apriori_caps_at_max_inner(oracle_mod):
    n = 64
    s = np.cos(2 * np.pi * 5 * np.arange(n) / n) * 100.0
    r = oracle_mod.direct(s, apriori=True, delta=1e-9, max_inner=50, max_imfs=1)
    assert r["m"][0] == 50 and r["status"] & oracle_mod.FLAG_MAX_INNER_HIT


# ---------------------------------------------------------------- thresholded IMF
# eq. I_gamma / eq. IMF_cont_stop_threshold: with m fixed by the stopping rule, every bin
# with (1 - w_hat_k)^m >= 1 - gamma passes whole into the IMF (w_hat_k taken as 0).

def _what_closed_form(n, L):
    k = np.arange(n)
    with np.errstate(invalid="ignore", divide="ignore"):
        w = (np.sin(np.pi * k * L / n) / (L * np.sin(np.pi * k / n))) ** 2
    w[0] = 1.0
    w[(k * L) % n == 0] = np.where(k[(k * L) % n == 0] == 0, 1.0, 0.0)
    return w


@pytest.mark.parametrize("k0,L,m", [(3, 8, 5), (6, 10, 40)])
def test_threshold_pure_tone_passes_whole_or_scales(oracle_mod, k0, L, m):
    n = 128
    x = np.arange(n) / n
    s = np.cos(2 * np.pi * k0 * x + 0.4)
    w = _what_closed_form(n, L)[k0]
    g = (1.0 - w) ** m
    for gamma, expect_whole in ((1.0 - g + 1e-3, True), (max(1.0 - g - 1e-3, 1e-9), False)):
        # force L and m: a tone's SD is w_hat for every j, so delta above it stops at j = 1;
        # take m through the a-priori mode's cap instead
        r = oracle_mod.direct(s, force_L=[L], max_imfs=1, apriori=True, delta=1e-300,
                              max_inner=m, gamma=gamma)
        assert r["m"][0] == m
        ref = s if expect_whole else g * s
        assert np.abs(r["imfs"][0] - ref).max() < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_threshold_bins_follow_the_definition(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n, L, m, gamma = 96, 7, 9, 0.2
    s = rng.standard_normal(n)
    r = oracle_mod.direct(s, force_L=[L], max_imfs=1, apriori=True, delta=1e-300, max_inner=m,
                          gamma=gamma)
    assert r["m"][0] == m
    S = np.fft.fft(s)
    G = (1.0 - _what_closed_form(n, L)) ** m
    passing = G >= 1.0 - gamma
    assert passing.any() and (~passing).any()
    want = np.where(passing, S, G * S)
    got = np.fft.fft(r["imfs"][0])
    assert np.abs(got - want).max() < 1e-10 * np.abs(S).max()
    # the remainder keeps the rest; IMF + remainder = s
    assert np.abs(r["imfs"][0] + r["remainder"] - s).max() < 1e-12


def test_threshold_reconstruction_and_zero_gamma(oracle_mod):
    n = 256
    x = np.arange(n) / n
    s = np.sin(2 * np.pi * 3 * x) + 0.5 * np.sin(2 * np.pi * 17 * x) + 0.2 * np.cos(2 * np.pi * 41 * x)
    r = oracle_mod.direct(s, gamma=0.05, max_imfs=5)
    assert np.abs(r["imfs"].sum(0) + r["remainder"] - s).max() < 1e-12
    a = oracle_mod.direct(s, max_imfs=5)
    b = oracle_mod.direct(s, gamma=0.0, max_imfs=5)
    assert np.array_equal(a["imfs"], b["imfs"])


def test_threshold_rejected_by_the_time_domain_tier(oracle_mod):
    with pytest.raises(Exception):
        oracle_mod.iterative(np.ones(16), gamma=0.1)


# ---------------------------------------------------------------- Fourier-peak mask length
# End of Sec. 2: L from the spectrum's peak instead of the extrema count.  Reading: the
# largest |r_hat_k|, 1 <= k <= n/2 (smallest k on ties), with the extrema rule at the
# count a tone of k* cycles has (2 k*).

@pytest.mark.parametrize("n,k0", [(256, 7), (243, 11), (1024, 100)])
def test_peak_mask_pure_tone_matches_the_extrema_rule(oracle_mod, n, k0):
    x = np.arange(n) / n
    s = np.cos(2 * np.pi * k0 * x + 0.3)
    assert oracle_mod.spectral_peak(s) == (k0, False)
    a = oracle_mod.direct(s, peak_mask=True, max_imfs=1)
    b = oracle_mod.direct(s, max_imfs=1)
    assert oracle_mod.count_extrema(s) == 2 * k0
    assert a["L"][0] == b["L"][0] == oracle_mod.mask_length(n, 2 * k0)


@pytest.mark.parametrize("seed", range(6))
def test_spectral_peak_is_the_argmax_of_numpys_spectrum(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.choice([64, 100, 243, 512]))
    s = rng.standard_normal(n)
    mag = np.abs(np.fft.fft(s))[1:n // 2 + 1]
    k, tie = oracle_mod.spectral_peak(s)
    order = np.sort(mag)[::-1]
    if order[1] >= order[0] * (1 - 1e-5):
        assert tie
    else:
        assert k == 1 + int(np.argmax(mag)) and not tie


def test_spectral_peak_tie_flag(oracle_mod):
    n = 128
    x = np.arange(n) / n
    s = np.cos(2 * np.pi * 5 * x) + np.cos(2 * np.pi * 9 * x)
    k, tie = oracle_mod.spectral_peak(s)
    assert tie and k in (5, 9)               # equal up to round-off: either, flagged
    r = oracle_mod.direct(s, peak_mask=True, max_imfs=1)
    assert r["status"] & oracle_mod.FLAG_MASK_TIE


@pytest.mark.parametrize("seed,n", [(7, 64), (8, 96), (9, 81)])
def test_peak_mask_direct_equals_iterative(oracle_mod, seed, n):
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    s = np.sin(2 * np.pi * 2 * x) + 0.6 * np.sin(2 * np.pi * 13 * x) + 0.05 * rng.standard_normal(n)
    kw = dict(peak_mask=True, delta=1e-3, max_inner=300, max_imfs=3)
    a, b = oracle_mod.iterative(s, **kw), oracle_mod.direct(s, **kw)
    K = int(a["n_imfs"])
    assert K == int(b["n_imfs"]) and np.array_equal(a["L"], b["L"]) and np.array_equal(a["m"], b["m"])
    assert np.abs(a["imfs"] - b["imfs"]).max() < 1e-10 * np.abs(s).max()


# ------------------------------------------- shape-generated windows (f4)

SHAPES = {
    "sine": np.sin(np.pi * np.linspace(0.0, 1.0, 33)),          # zero ends, positive inside
    "ramp": np.array([0.2, 1.0]),                               # skewed: h is not symmetric
    "hat": np.array([0.0, 1.0, 0.0]),
    "rough": np.random.default_rng(11).uniform(0.1, 1.0, 7),
}


@pytest.mark.parametrize("g", [[1.0], [2.5], [1.0, 1.0], [3.0, 3.0, 3.0]])
@pytest.mark.parametrize("n,L", [(64, 5), (65, 9), (128, 30), (243, 121)])
def test_constant_shape_gives_the_triangle(oracle_mod, g, n, L):
    """A constant shape generates a box, and box * box is the triangle
    (Theorem 4's construction): taps and spectrum equal the triangle's closed
    form (eq. triangular, eq. eig2)."""
    assert np.abs(oracle_mod.shape_taps(n, L, g) - oracle_mod.taps(n, L)).max() < 1e-16
    assert np.abs(oracle_mod.shape_spectrum(n, L, g) - _what_closed_form(n, L)).max() < 2e-14


def test_constant_shape_decomposition_is_the_triangles(oracle_mod):
    s = signals.component_signal(98, 2, 384).astype(np.float64)
    for tier in ("direct", "iterative"):
        a = getattr(oracle_mod, tier)(s, max_imfs=4, max_inner=80)
        b = getattr(oracle_mod, tier)(s, max_imfs=4, max_inner=80, shape=[1.0])
        assert a["status"] == b["status"] and np.array_equal(a["m"], b["m"])
        assert np.array_equal(a["L"], b["L"])
        assert np.abs(a["imfs"] - b["imfs"]).max() < 1e-12 * np.abs(s).max()


@pytest.mark.parametrize("L", [1, 2, 7, 40])
def test_shape_filter_samples_cell_midpoints(oracle_mod, L):
    x = (np.arange(L) + 0.5) / L
    assert np.array_equal(oracle_mod.shape_filter(L, [0.7]), np.full(L, 0.7))
    assert np.allclose(oracle_mod.shape_filter(L, [0.2, 1.0]), 0.2 + 0.8 * x, rtol=0, atol=1e-15)
    assert np.allclose(oracle_mod.shape_filter(L, [0.0, 1.0, 0.0]), 1.0 - np.abs(2 * x - 1),
                       rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", sorted(SHAPES))
@pytest.mark.parametrize("n,L", [(96, 11), (97, 30), (256, 100), (60, 1)])
def test_shape_spectrum_is_the_squared_filter_spectrum(oracle_mod, name, n, L):
    """The window is h * h, so w_hat = |DFT(h)|^2 / (sum h)^2 (the
    autocorrelation theorem; numpy's FFT of h, an independent route), in
    [0, 1] with w_hat_0 = 1.  The taps are even, sum to 1 and vanish for
    |d| >= L."""
    g = SHAPES[name]
    h = oracle_mod.shape_filter(L, g)
    assert (h > 0).all()
    ref = np.abs(np.fft.fft(h, n)) ** 2 / h.sum() ** 2
    w = oracle_mod.shape_spectrum(n, L, g)
    assert np.abs(w - ref).max() < 1e-13
    assert w[0] == 1.0 and (w >= 0).all() and (w <= 1).all()
    c = oracle_mod.shape_taps(n, L, g)
    assert abs(c.sum() - 1) < 1e-14
    d = np.arange(n)
    assert np.allclose(c, c[(-d) % n], rtol=0, atol=1e-17)
    support = (d < L) | (d > n - L)
    assert (c[~support] == 0).all() and (c[support] > 0).all()


def test_shape_pure_tone_scaled_by_multiplier(oracle_mod):
    """A tone at bin k0 is an eigenvector of the circulant W: with SD_j =
    w_hat_k0 for every j (eq. SD), m = max_inner here and the IMF is
    (1 - w_hat_k0)^m times the tone, w_hat from numpy's FFT of h."""
    n, k0, L = 512, 6, 25
    g = SHAPES["sine"]
    s = np.cos(2 * np.pi * k0 * np.arange(n) / n + 0.4)
    h = oracle_mod.shape_filter(L, g)
    lam = np.abs(np.fft.fft(h, n)[k0]) ** 2 / h.sum() ** 2
    assert 1e-3 < lam < 0.9
    for tier in ("direct", "iterative"):
        r = getattr(oracle_mod, tier)(s, force_L=[L], max_imfs=1, max_inner=120, shape=g)
        assert r["m"][0] == 120 and r["L"][0] == L
        assert np.abs(r["imfs"][0] - (1 - lam) ** 120 * s).max() < 1e-13


@pytest.mark.parametrize("name", ["sine", "ramp", "rough"])
@pytest.mark.parametrize("seed,n,delta", [(0, 128, 1e-3), (3, 729, 1e-2), (6, 512, 3e-2)])
def test_shape_direct_equals_iterative(oracle_mod, name, seed, n, delta):
    s = signals.component_signal(98, seed, n).astype(np.float64)
    kw = dict(max_imfs=5, max_inner=80, delta=delta, shape=SHAPES[name], trace=True)
    a, b = oracle_mod.iterative(s, **kw), oracle_mod.direct(s, **kw)
    assert a["n_imfs"] == b["n_imfs"] and a["status"] == b["status"]
    assert np.array_equal(a["m"], b["m"]) and np.array_equal(a["L"], b["L"])
    for i in range(a["n_imfs"]):
        assert rel(a["imfs"][i], b["imfs"][i]) < 1e-11
        mm = a["m"][i]
        assert np.allclose(a["sd_trace"][i][:mm], b["sd_trace"][i][:mm], rtol=1e-10, atol=0)
    assert rel(a["remainder"], b["remainder"]) < 1e-11


def test_shape_windows_change_the_decomposition(oracle_mod):
    """The shape reaches the result: a non-constant shape gives other m and IMFs."""
    s = signals.component_signal(98, 6, 512).astype(np.float64)
    a = oracle_mod.direct(s, max_imfs=4, max_inner=80, delta=3e-2)
    b = oracle_mod.direct(s, max_imfs=4, max_inner=80, delta=3e-2, shape=SHAPES["sine"])
    assert not np.array_equal(a["m"], b["m"])
    assert rel(a["imfs"][0], b["imfs"][0]) > 1e-2


@pytest.mark.parametrize("g", [[], [-1.0, 1.0], [1.0, np.nan], [1.0, 0.0, 1.0], [0.0], [0.0, 0.0]])
def test_invalid_shapes_are_rejected(oracle_mod, g):
    s = signals.component_signal(98, 0, 64).astype(np.float64)
    with pytest.raises(ValueError):
        oracle_mod.direct(s, shape=np.asarray(g, dtype=np.float64))


def test_shape_with_apriori_is_rejected(oracle_mod):
    s = signals.component_signal(98, 0, 64).astype(np.float64)
    with pytest.raises(ValueError):
        oracle_mod.direct(s, shape=[1.0], apriori=True)


def test_per_step_flags_are_the_status_flags_by_step(oracle_mod):
    """The oracle's per-step flag records OR to its status flags, and a near tie of SD_m
    with delta is recorded at the IMF where it occurs (eq. SD, the 1e-6 delta band)."""
    from paper_1802_01359_gb300 import signals
    for kw in ({}, {"peak_mask": True}, {"max_inner": 30, "delta": 3e-2}):
        s = signals.component_signal(90, 0, 1024).astype(np.float64)
        for fn in (oracle_mod.direct, oracle_mod.iterative):
            r = fn(s, **kw)
            acc = 0
            for f in r["imf_flags"]:
                acc |= int(f)
            assert acc == r["status"] & ~0xFF, (kw, r["imf_flags"], hex(r["status"]))
    s = signals.component_signal(52, 3, 1024).astype(np.float64)
    base = oracle_mod.direct(s, delta=3e-2, max_inner=100, max_imfs=3)
    k = 1
    delta = float(base["sd_m"][k]) * (1 + 1e-7)     # SD_m of IMF 1 within the tie band
    r = oracle_mod.direct(s, delta=delta, max_inner=100, max_imfs=3)
    assert r["m"][k] == base["m"][k]
    assert r["imf_flags"][k] & oracle_mod.FLAG_NEAR_DELTA_TIE
