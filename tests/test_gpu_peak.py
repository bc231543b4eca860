"""GPU parity of the Fourier-peak mask length (FIF_PEAK_MASK; end of Sec. 2) on every path."""
import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_01359_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _pack(sigs, dev):
    lens = np.array([s.size for s in sigs], dtype=np.int64)
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    return torch.from_numpy(np.concatenate(sigs).astype(np.float32)).to(dev), offs


@pytest.mark.parametrize("multipass", [False, True])
def test_peak_mask_batch_matches_oracle(dev, oracle_mod, multipass):
    lens = [4096, 3072, 2187, 1024, 729, 4096]
    sigs = [signals.component_signal(98, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=4096, max_imfs=6, peak_mask=True, multipass=multipass) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=6, peak_mask=True)
        parity.compare(res.signal(i), ref)


def test_peak_mask_long_single_noalloc(dev, oracle_mod):
    s = signals.component_signal(99, 0, 20736)
    x = torch.from_numpy(s).to(dev)
    with fif.Plan(max_n=20736, max_imfs=4, peak_mask=True) as plan:
        d = plan.decompose(x, diag=True)
    parity.compare(d, oracle_mod.direct(s.astype(np.float64), max_imfs=4, peak_mask=True))
    s2 = signals.component_signal(99, 1, 4096)
    x2 = torch.from_numpy(s2).to(dev)
    d2 = fif.decompose_noalloc(x2, max_imfs=4, peak_mask=True, diag=True)
    parity.compare(d2, oracle_mod.direct(s2.astype(np.float64), max_imfs=4, peak_mask=True))


def test_peak_mask_pure_tone_gives_the_extrema_rule(dev, oracle_mod):
    n, k0 = 4096, 37
    s = np.cos(2 * np.pi * k0 * np.arange(n) / n + 0.2).astype(np.float32)
    x, offs = _pack([s], dev)
    with fif.Plan(max_n=n, max_imfs=1, peak_mask=True) as a, fif.Plan(max_n=n, max_imfs=1) as b:
        ra = a.decompose_batch(x, offs)
        rb = b.decompose_batch(x, offs)
        torch.cuda.synchronize()
    assert int(ra.mask_len[0, 0]) == int(rb.mask_len[0, 0]) == oracle_mod.mask_length(n, 2 * k0)
