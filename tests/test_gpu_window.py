"""GPU parity of shape-generated windows (FIF_WIN_SHAPE: the window is h * h,
h sampled from a shape g; Theorem 4's double convolution, eq. W_m) on the
fused batch path, the staged single-signal path and the multi-pass path."""
import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = {
    "sine": np.sin(np.pi * np.linspace(0.0, 1.0, 33)),
    "ramp": np.array([0.2, 1.0]),
    "rough": np.random.default_rng(11).uniform(0.1, 1.0, 7),
}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_01359_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def _pack(sigs, dev):
    lens = np.array([s.size for s in sigs], dtype=np.int64)
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    return torch.from_numpy(np.concatenate(sigs).astype(np.float32)).to(dev), offs


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_shape_batch_matches_oracle(dev, oracle_mod, name):
    g = SHAPES[name]
    lens = [4096, 3072, 2187, 1024, 729, 256, 4096]
    sigs = [signals.component_signal(98, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=4096, max_imfs=6, window_shape=g) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=6, shape=g)
        parity.compare(res.signal(i), ref)


@pytest.mark.parametrize("n", [4096, 8192])
def test_shape_staged_single_matches_oracle(dev, oracle_mod, n):
    g = SHAPES["sine"]
    s = signals.component_signal(99, 3, n)
    with fif.Plan(max_n=n, max_imfs=5, window_shape=g) as plan:
        d = plan.decompose(torch.from_numpy(s).to(dev), diag=True)
    parity.compare(d, oracle_mod.direct(s.astype(np.float64), max_imfs=5, shape=g))


def test_shape_with_threshold_and_peak_mask(dev, oracle_mod):
    """The binary64 window row also serves the threshold's tie-break."""
    g = SHAPES["rough"]
    lens = [2048, 1536, 729]
    sigs = [signals.component_signal(97, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    kw = dict(max_imfs=5, gamma=0.05, peak_mask=True)
    with fif.Plan(max_n=2048, window_shape=g, **kw) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        parity.compare(res.signal(i), oracle_mod.direct(s.astype(np.float64), shape=g, **kw))


def test_constant_shape_matches_the_triangle(dev):
    """A constant shape generates the triangle: same integers, IMFs equal to
    FP32 rounding of the two tables."""
    sigs = [signals.component_signal(96, i, 2048) for i in range(12)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=2048, max_imfs=6) as a, fif.Plan(max_n=2048, max_imfs=6,
                                                          window_shape=[1.0]) as b:
        ra = a.decompose_batch(x, offs)
        rb = b.decompose_batch(x, offs)
        torch.cuda.synchronize()
    tie = fif.FLAG_NEAR_DELTA_TIE | fif.FLAG_EXTREMA_TIE
    for i in range(len(sigs)):
        da, db = ra.signal(i), rb.signal(i)
        if (da.status | db.status) & tie:
            continue
        assert da.n_imfs == db.n_imfs
        assert np.array_equal(_np(da.m), _np(db.m))
        assert np.array_equal(_np(da.mask_len), _np(db.mask_len))
        A, B = _np(da.imfs), _np(db.imfs)
        for k in range(da.n_imfs):
            assert parity.rel_l2(B[k], A[k]) < 1e-5


def test_shape_pure_tone_eigenvalue(dev, oracle_mod):
    """A tone at bin k0 with forced L comes out scaled by (1 - w_hat_k0)^m,
    w_hat from the oracle's DFT of the shape window's taps."""
    n, k0, L = 4096, 36, 150
    g = SHAPES["sine"]
    s = np.cos(2 * np.pi * k0 * np.arange(n) / n + 0.4)
    lam = oracle_mod.shape_spectrum(n, L, g)[k0]
    assert 1e-3 < lam < 0.05                 # SD_j = lam > delta: m = max_inner, scale ~0.37
    with fif.Plan(max_n=n, max_imfs=1, max_inner=120, force_L=True, window_shape=g) as plan:
        d = plan.decompose(torch.from_numpy(s.astype(np.float32)).to(dev), mask_len=[L])
    assert int(d.m[0]) == 120 and int(d.mask_len[0]) == L
    want = (1 - lam) ** 120 * s
    assert parity.rel_l2(_np(d.imfs)[0].astype(np.float64), want) < 1e-5


def test_shape_multipass_forced_matches_oracle(dev, oracle_mod):
    """The multi-pass path builds each IMF's row from a float-float transform of h."""
    g = SHAPES["sine"]
    lens = [256, 729, 1024, 2048, 4096]
    sigs = [signals.component_signal(92, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=4096, max_imfs=5, window_shape=g, multipass=True) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        parity.compare(res.signal(i), oracle_mod.direct(s.astype(np.float64), max_imfs=5, shape=g))


@pytest.mark.parametrize("count", [1, 9])  # grid-wide m search; one CTA per signal
def test_shape_long_signals_match_oracle(dev, oracle_mod, count):
    g = SHAPES["ramp"]
    n = 1 << 15
    sigs = [signals.component_signal(93, i, n) for i in range(count)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=n, max_imfs=4, window_shape=g) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i in range(min(count, 2)):
        ref = oracle_mod.direct(sigs[i].astype(np.float64), max_imfs=4, shape=g)
        parity.compare(res.signal(i), ref)


def test_shape_long_single_with_threshold(dev, oracle_mod):
    """The threshold's binary64 decisions read the signal's own binary64 row."""
    g = SHAPES["rough"]
    n = 1 << 15
    s = signals.component_signal(94, 0, n, sigma=0.0)
    kw = dict(max_imfs=4, gamma=0.05)
    with fif.Plan(max_n=n, window_shape=g, **kw) as plan:
        d = plan.decompose(torch.from_numpy(s).to(dev), diag=True)
    parity.compare(d, oracle_mod.direct(s.astype(np.float64), shape=g, **kw))
