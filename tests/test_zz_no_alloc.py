"""The allocation-free entry point fif_decompose_noalloc against fif_decompose.

fif_decompose_noalloc serves callers that cannot allocate device memory when
they decompose; it keeps its working arrays in one fixed device array of the
library instead of a plan.  Two calls in a row (different signals and lengths,
so the second call finds the first call's data in that array) must each give
the same integers as fif_decompose and IMFs within the parity tolerance.
"""
import ctypes

import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_plan_entry_point_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_01359_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    for seed, n in ((0, 4096), (1, 3072)):
        s = signals.component_signal(61, seed, n)
        x = torch.from_numpy(s).to(dev)
        with fif.Plan(max_n=n) as plan:
            ref = plan.decompose(x, diag=True)
        got = fif.decompose_noalloc(x, diag=True)
        path_flag = fif.FLAG_FP64_TIEBREAK  # which screen decisions went to binary64
        assert got.n_imfs == ref.n_imfs and (got.status & ~path_flag) == (ref.status & ~path_flag)
        K = got.n_imfs
        assert np.array_equal(got.m.cpu().numpy()[:K], ref.m.cpu().numpy()[:K])
        assert np.array_equal(got.mask_len.cpu().numpy()[:K], ref.mask_len.cpu().numpy()[:K])
        assert np.array_equal(got.diag["k_extrema"][:K + 1], ref.diag["k_extrema"][:K + 1])
        a = got.imfs.cpu().numpy().astype(np.float64)
        b = ref.imfs.cpu().numpy().astype(np.float64)
        for k in range(K + 1):
            assert parity.rel_l2(a[k], b[k]) < parity.IMF_TOL, (n, k)


def test_noalloc_rejects_lengths_above_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = fif.load_library()
    n = fif.NOALLOC_MAX_N * 2
    x = torch.zeros(n, device="cuda:0")
    out = torch.zeros(11 * n, device="cuda:0")
    ints = torch.zeros(32, dtype=torch.int32, device="cuda:0")
    desc = fif.PlanDesc(0, 1.6, 1, 1e-3, 200, 10, 0, n, 0)
    rc = lib.fif_decompose_noalloc(ctypes.byref(desc), x.data_ptr(), n, out.data_ptr(),
                                   ints.data_ptr(), ints.data_ptr() + 64, ints.data_ptr() + 40,
                                   ints.data_ptr() + 44, None, None)
    assert rc == fif.FIF_EUNSUPPORTED
