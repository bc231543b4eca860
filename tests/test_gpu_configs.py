"""GPU parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (the whole batch in one fif_decompose_batch call), on sampled
signals against the FP64 oracle (direct method).

  - the large uniform batch: 65536 signals, n = 4096, max_imfs = 12,
    delta = 1e-3 and 1e-4: 64 sampled signals each;
  - the uneven batch: 4096 signals, n log-uniform in [256, 2^20]: its first
    2^20 signal and a spread of others;
  - the long signal: one n = 2^24 signal, all ten IMFs.

A divergence is allowed only where a tie flag of that step excuses it
(parity.compare; a flagged extrema count that leaves L and the stop test
unchanged is not a divergence); the fraction of sampled signals that diverge
must stay at or below MAX_FLAGGED (observed: 1 of 64, 0 of 29, 0 of 1).
The fraction of all signals that raise each tie flag is printed.
The oracle runs on host threads (the C oracle releases the GIL) while the GPU
works.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_FLAGGED = 0.10
TC_TOL = 1e-4  # the split-BF16 variant's stated IMF bound (tests/test_gpu_tc.py)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_01359_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def pool():
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        yield ex


def _oracle_jobs(pool, oracle_mod, data, offs, idx, **kw):
    return {int(i): pool.submit(oracle_mod.direct, data[offs[i]:offs[i + 1]].astype(np.float64), **kw)
            for i in idx}


def _check_sampled(res, jobs, bound=None):
    """parity.compare on every sampled signal; flagged divergences at most
    bound (default MAX_FLAGGED) of the sample (at least two allowed in small
    samples)."""
    bound = MAX_FLAGGED if bound is None else bound
    flagged = []
    for i, fut in sorted(jobs.items()):
        rep = parity.compare(res.signal(i), fut.result())
        if rep["diverged_at"] is not None:
            flagged.append((i, int(res.lengths[i]), rep["diverged_at"], rep["diverged_on"]))
    print(f"flagged divergences {len(flagged)} of {len(jobs)}: {flagged}")
    assert len(flagged) <= max(2, int(np.ceil(bound * len(jobs)))), flagged
    return len(flagged)


@pytest.mark.parametrize("delta", [1e-3, 1e-4])
def test_large_uniform_batch_4096(dev, oracle_mod, pool, delta):
    import bench
    B, n, K = 65536, 4096, 12
    data, offs = bench.generate(signals.W_BATCH_4096, np.full(B, n))
    idx = np.unique(np.linspace(0, B - 1, 64).astype(np.int64))
    jobs = _oracle_jobs(pool, oracle_mod, data, offs, idx, delta=delta, max_imfs=K)
    x = torch.from_numpy(data).to(dev)
    with fif.Plan(max_n=n, delta=delta, max_imfs=K) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        st = res.status.cpu().numpy()
        assert ((st & 0xFF) > 0).all()
        # every signal: the rows reconstruct the input (Algorithm 1 telescopes)
        imfs = res.imfs.view(B, K + 1, n)
        rows = torch.arange(K + 1, device=dev)[None, :, None]
        mask = rows <= res.n_imfs.to(torch.int64)[:, None, None]
        for a in range(0, B, 8192):
            part = torch.where(mask[a:a + 8192], imfs[a:a + 8192].double(),
                               torch.zeros((), dtype=torch.float64, device=dev)).sum(1)
            err = (part - x.view(B, n)[a:a + 8192].double()).abs().max().item()
            assert err < 1e-5 * x.abs().max().item()
        _check_sampled(res, jobs)
    # how often the tie flags are raised at all (most raised flags change nothing:
    # the sampled divergences above stay within MAX_FLAGGED)
    print(f"delta={delta}: tie-flag fractions over all {B} signals:", parity.tie_fractions(st))


def test_uneven_batch_top_length(dev, oracle_mod, pool):
    """The first 2^20 signal and 12 others of the multi-pass lengths (above the fused
    limit, up to 2^17), 16 of the fused lengths.  On long smooth remainders the FP32
    extrema count often differs from binary64's by a flagged tie (near each true
    extremum the first differences fall below the remainder's FP32 error); such a
    count ends the comparison only when it changes L or the stop test."""
    import bench
    lens = signals.uneven_lengths(4096)
    data, offs = bench.generate(signals.W_UNEVEN, lens)
    top = int(np.where(lens == lens.max())[0][0])
    assert lens[top] == 1 << 20
    rng = np.random.default_rng(5)
    fmax = fif.fused_max_n()
    short = rng.choice(np.where(lens <= fmax)[0], 16, replace=False)
    long_ = rng.choice(np.where((lens > fmax) & (lens <= 1 << 17))[0], 12, replace=False)
    jobs_s = _oracle_jobs(pool, oracle_mod, data, offs, short)
    jobs_l = _oracle_jobs(pool, oracle_mod, data, offs, np.concatenate([[top], long_]))
    x = torch.from_numpy(data).to(dev)
    with fif.Plan(max_n=int(lens.max())) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        _check_sampled(res, jobs_s)
        _check_sampled(res, jobs_l)
        assert ((res.status.cpu().numpy() & 0xFF) > 0).all()


def test_long_signal_2p24(dev, oracle_mod, pool):
    s = signals.long_signal()
    n = s.size
    assert n == 1 << 24
    fut = pool.submit(oracle_mod.direct, s.astype(np.float64))
    x = torch.from_numpy(s).to(dev)
    offs = np.array([0, n], dtype=np.int64)
    with fif.Plan(max_n=n) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        d = res.signal(0)
        ref = fut.result()
        rep = parity.compare(d, ref)
    # the split-BF16 variant (tensor-core radix-16 passes in both inverse levels)
    # against the same oracle result, within its own stated bound
    with fif.Plan(max_n=n, precision=fif.PREC_SPLIT_BF16) as plan:
        ms = plan.multipass_schedule(n)
        assert ms["E1"] == 16 and ms["E2"] == 16, ms
        rt = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        rep_tc = parity.compare(rt.signal(0), ref, tol=TC_TOL)
    print("long signal, split-BF16:", {k: v for k, v in rep_tc.items() if k != "errors"},
          "IMF errors", [f"{e:.2e}" for e in rep_tc["errors"]])
    assert len(rep_tc["errors"]) >= 3, rep_tc
    # a divergence is allowed only as a flagged tie (parity.compare); every IMF before
    # it is compared element by element
    print("long signal:", {k: v for k, v in rep.items() if k != "errors"},
          "IMF errors", [f"{e:.2e}" for e in rep["errors"]])
    assert rep["diverged_at"] is not None or d.n_imfs == 10
    assert len(rep["errors"]) >= 3, rep
    rec = d.imfs[:d.n_imfs + 1].double().sum(0)
    assert (rec - x.double()).abs().max().item() < 1e-5 * x.abs().max().item()
