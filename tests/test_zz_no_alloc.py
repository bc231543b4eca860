"""The allocation-free entry point fif_decompose_noalloc against fif_decompose
and the FP64 oracle.

fif_decompose_noalloc serves callers that cannot allocate device memory when
they decompose (latency-critical code that cannot afford cudaMalloc's device
synchronisation, hosts that give all device memory to their own pool at
start-up, plug-ins that may only allocate during setup); it keeps its working
arrays in one fixed device array of the library instead of a plan.  Calls in a
row (different signals and lengths, so every call finds the previous call's
data in that array) must each give the integers of fif_decompose and of the
oracle, and IMFs within the parity tolerance; the lengths cover an even n, an
odd n (3^8, the odd-length epilogue) and the largest supported n.
"""
import ctypes

import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LENGTHS = ((0, 4096), (1, 3072), (2, 6561), (3, fif.NOALLOC_MAX_N))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_01359_gb300 import build
    build.build()
    return torch.device("cuda:0")


def test_noalloc_matches_plan_entry_point_and_oracle(dev, oracle_mod):
    for seed, n in LENGTHS:
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
        # and directly against the FP64 oracle (direct method)
        rep = parity.compare(got, oracle_mod.direct(s.astype(np.float64)))
        assert rep["diverged_at"] is None, (n, rep)


def test_noalloc_allocates_no_device_memory(dev):
    s = signals.component_signal(62, 0, 4096)
    x = torch.from_numpy(s).to(dev)
    fif.decompose_noalloc(x)        # first call: address lookup, module load
    torch.cuda.synchronize()
    imfs = torch.zeros(11 * 4096, device=dev)
    ints = torch.zeros(64, dtype=torch.int32, device=dev)
    desc = fif.PlanDesc(0, 1.6, 1, 1e-3, 200, 10, 0, 4096, 0)
    lib = fif.load_library()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        rc = lib.fif_decompose_noalloc(ctypes.byref(desc), x.data_ptr(), 4096, imfs.data_ptr(),
                                       ints.data_ptr(), ints.data_ptr() + 64,
                                       ints.data_ptr() + 128, ints.data_ptr() + 132, None, None)
        assert rc == fif.FIF_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0


def test_noalloc_rejects_lengths_above_its_maximum(dev):
    lib = fif.load_library()
    n = fif.NOALLOC_MAX_N * 2
    x = torch.zeros(n, device=dev)
    out = torch.zeros(11 * n, device=dev)
    ints = torch.zeros(32, dtype=torch.int32, device=dev)
    desc = fif.PlanDesc(0, 1.6, 1, 1e-3, 200, 10, 0, n, 0)
    rc = lib.fif_decompose_noalloc(ctypes.byref(desc), x.data_ptr(), n, out.data_ptr(),
                                   ints.data_ptr(), ints.data_ptr() + 64, ints.data_ptr() + 40,
                                   ints.data_ptr() + 44, None, None)
    assert rc == fif.FIF_EUNSUPPORTED
