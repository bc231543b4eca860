"""GPU parity of the a-priori N0 mode (FIF_APRIORI_N0, Theorem 5 / eq. N0_discrete) on
every path: fused batch, staged single signal, multi-pass, allocation-free."""
import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KW = dict(max_inner=1 << 16, max_imfs=6)


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


@pytest.mark.parametrize("delta", [2.0, 10.0])
@pytest.mark.parametrize("multipass", [False, True])
def test_apriori_batch_matches_oracle(dev, oracle_mod, delta, multipass):
    lens = [4096, 3072, 2187, 4096, 1024, 729]
    sigs = [signals.component_signal(91, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=4096, delta=delta, apriori_n0=True, multipass=multipass, **KW) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), apriori=True, delta=delta, **KW)
        parity.compare(res.signal(i), ref)


def test_apriori_long_signals_match_oracle(dev, oracle_mod):
    lens = [20736, 32768]
    sigs = [signals.component_signal(92, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 15, delta=5.0, apriori_n0=True, **KW) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), apriori=True, delta=5.0, **KW)
        parity.compare(res.signal(i), ref)


def test_apriori_single_and_noalloc_match_oracle(dev, oracle_mod):
    s = signals.component_signal(93, 0, 4096)
    x = torch.from_numpy(s).to(dev)
    ref = oracle_mod.direct(s.astype(np.float64), apriori=True, delta=2.0, **KW)
    with fif.Plan(max_n=4096, delta=2.0, apriori_n0=True, **KW) as plan:
        d = plan.decompose(x, diag=True)
    parity.compare(d, ref)
    d2 = fif.decompose_noalloc(x, delta=2.0, apriori_n0=True, diag=True, **KW)
    parity.compare(d2, ref)


def test_apriori_cap_sets_max_inner_hit(dev, oracle_mod):
    s = signals.component_signal(94, 0, 4096)
    x, offs = _pack([s], dev)
    with fif.Plan(max_n=4096, delta=1e-3, apriori_n0=True, max_inner=100, max_imfs=2) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    d = res.signal(0)
    assert np.all(d.m.cpu().numpy()[:d.n_imfs] == 100)
    assert d.status & fif.FLAG_MAX_INNER_HIT
    ref = oracle_mod.direct(s.astype(np.float64), apriori=True, delta=1e-3, max_inner=100, max_imfs=2)
    parity.compare(d, ref)
