"""GPU parity of the thresholded IMF (fif_plan_desc.gamma; eq. I_gamma,
eq. IMF_cont_stop_threshold) on every path against the oracle's direct method."""
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


@pytest.mark.parametrize("gamma", [0.05, 0.3])
@pytest.mark.parametrize("multipass", [False, True])
def test_threshold_batch_matches_oracle(dev, oracle_mod, gamma, multipass):
    lens = [4096, 3072, 2187, 1024, 729]
    sigs = [signals.component_signal(95, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=4096, max_imfs=6, gamma=gamma, multipass=multipass) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=6, gamma=gamma)
        parity.compare(res.signal(i), ref)


def test_threshold_long_single_and_noalloc(dev, oracle_mod):
    s = signals.component_signal(96, 0, 20736)
    x = torch.from_numpy(s).to(dev)
    with fif.Plan(max_n=20736, max_imfs=4, gamma=0.1) as plan:
        d = plan.decompose(x, diag=True)
    parity.compare(d, oracle_mod.direct(s.astype(np.float64), max_imfs=4, gamma=0.1))
    s2 = signals.component_signal(96, 1, 4096)
    x2 = torch.from_numpy(s2).to(dev)
    d2 = fif.decompose_noalloc(x2, max_imfs=4, gamma=0.1, diag=True)
    parity.compare(d2, oracle_mod.direct(s2.astype(np.float64), max_imfs=4, gamma=0.1))


def test_threshold_changes_the_imfs(dev, oracle_mod):
    """gamma > 0 really moves bins: the thresholded first IMF differs from the plain one
    by the energy of the bins that pass whole."""
    s = signals.component_signal(97, 0, 4096)
    x, offs = _pack([s], dev)
    with fif.Plan(max_n=4096, max_imfs=2) as a, fif.Plan(max_n=4096, max_imfs=2, gamma=0.3) as b:
        ra = a.decompose_batch(x, offs)
        rb = b.decompose_batch(x, offs)
        torch.cuda.synchronize()
    ia = ra.signal(0).imfs[0].cpu().numpy()
    ib = rb.signal(0).imfs[0].cpu().numpy()
    assert parity.rel_l2(ia, ib) > 1e-3
