"""GPU parity of the multi-pass path (FFTs through global memory) used for long signals."""
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


MP_LENGTHS = [8, 12, 18, 27, 64, 96, 243, 256, 729, 1024, 1536, 2187, 4096, 6144, 6561, 16384]


def test_multipass_forced_small_lengths_match_oracle(dev, oracle_mod):
    sigs = [signals.component_signal(70, i, n) for i, n in enumerate(MP_LENGTHS)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=16384, max_imfs=5, multipass=True) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=5)
        parity.compare(res.signal(i), ref)


def test_multipass_and_fused_agree(dev):
    sigs = [signals.component_signal(71, i, n) for i, n in enumerate([2048, 4096, 12288, 16384])]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=16384) as a, fif.Plan(max_n=16384, multipass=True) as b:
        ra = a.decompose_batch(x, offs, diag=True)
        rb = b.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i in range(len(sigs)):
        da, db = ra.signal(i), rb.signal(i)
        # FP64_TIEBREAK records which screen decisions went to binary64: it
        # depends on each path's reduction order, the results do not
        path_flag = fif.FLAG_FP64_TIEBREAK
        assert da.n_imfs == db.n_imfs and (da.status & ~path_flag) == (db.status & ~path_flag)
        K = da.n_imfs
        assert np.array_equal(da.m.cpu().numpy()[:K], db.m.cpu().numpy()[:K])
        assert np.array_equal(da.mask_len.cpu().numpy()[:K], db.mask_len.cpu().numpy()[:K])
        A = da.imfs.cpu().numpy().astype(np.float64)
        B = db.imfs.cpu().numpy().astype(np.float64)
        for k in range(K + 1):
            assert parity.rel_l2(B[k], A[k]) < 2 * parity.IMF_TOL


LONG = [20736, 32768, 39366, 59049, 65536, 131072]


def test_long_lengths_match_oracle(dev, oracle_mod):
    sigs = [signals.component_signal(72, i, n) for i, n in enumerate(LONG)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 17, max_imfs=4) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=4)
        parity.compare(res.signal(i), ref)


def test_mixed_short_and_long_batch(dev, oracle_mod):
    lens = [4096, 24576, 729, 20736, 16384, 46656]
    sigs = [signals.component_signal(73, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 16, max_imfs=3) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=3)
        parity.compare(res.signal(i), ref)


def test_single_signal_entry_long(dev, oracle_mod):
    n = 1 << 18
    s = signals.component_signal(74, 0, n)
    with fif.Plan(max_n=n, max_imfs=2) as plan:
        d = plan.decompose(torch.from_numpy(s).to(dev), diag=True)
    ref = oracle_mod.direct(s.astype(np.float64), max_imfs=2)
    parity.compare(d, ref)
    # sum of IMFs and remainder reconstructs the input
    imfs = d.imfs.cpu().numpy().astype(np.float64)
    rec = imfs[:d.n_imfs + 1].sum(0)
    assert np.abs(rec - s).max() < 1e-5 * np.abs(s).max()


def test_long_degenerate_inputs(dev):
    n = 32768
    z = np.zeros(n, np.float32)
    nanv = np.ones(n, np.float32)
    nanv[1234] = np.nan
    x, offs = _pack([z, nanv], dev)
    with fif.Plan(max_n=n) as plan:
        res = plan.decompose_batch(x, offs)
        torch.cuda.synchronize()
    assert res.signal(0).stop == fif.STOP_EXTREMA and res.signal(0).n_imfs == 0
    assert res.signal(1).stop == fif.STOP_NONFINITE and res.signal(1).n_imfs == 0
    assert np.array_equal(res.signal(1).imfs[0].cpu().numpy(), nanv, equal_nan=True)


def test_batch_graph_replay_and_recapture(dev):
    """Repeated calls with one layout replay the captured graph; new output pointers
    re-capture; both give bit-identical results."""
    lens = [4096, 24576, 729, 20736, 16384]
    sigs = [signals.component_signal(75, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 15, max_imfs=4) as plan:
        r1 = plan.decompose_batch(x, offs)
        torch.cuda.synchronize()
        first = [r1.signal(i).imfs[:r1.signal(i).n_imfs + 1].clone() for i in range(len(lens))]
        m1 = r1.m.clone()
        r1.imfs.fill_(0.0)
        plan.decompose_batch(x, offs, out=r1)          # same pointers: graph replay
        r2 = plan.decompose_batch(x, offs)             # new outputs: re-capture
        torch.cuda.synchronize()
        for r in (r1, r2):
            assert torch.equal(r.m, m1)
            for i in range(len(lens)):
                d = r.signal(i)
                assert torch.equal(d.imfs[:d.n_imfs + 1], first[i])


def test_batch_inside_callers_cuda_graph(dev):
    """With the plan's stream set to a capturing stream, the call is recorded into the
    caller's graph (its layout was prepared by an earlier call)."""
    lens = [2048, 20736]
    sigs = [signals.component_signal(76, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 15, max_imfs=3) as plan:
        ref = plan.decompose_batch(x, offs)
        torch.cuda.synchronize()
        out = plan.alloc_batch_outputs(np.diff(offs), dev)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.set_stream(torch.cuda.current_stream())
                plan.decompose_batch(x, offs, out=out)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out.m, ref.m) and torch.equal(out.n_imfs, ref.n_imfs)
        for i in range(len(lens)):
            a, b = out.signal(i), ref.signal(i)
            assert torch.equal(a.imfs[:a.n_imfs + 1], b.imfs[:b.n_imfs + 1])


@pytest.mark.parametrize("max_inner", [1, 2, 15, 16, 17, 40, 200, 289, 290, 1000])
def test_multipass_m_search_any_max_inner(dev, oracle_mod, max_inner):
    """The grid-wide search for m (rounds of up to 16 candidates j) closes its
    bracket for every cap: m and every other integer match the oracle."""
    lens = [4096, 6561, 20736]
    sigs = [signals.component_signal(77, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 15, max_imfs=4, max_inner=max_inner, delta=1e-4,
                  multipass=True) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=4, max_inner=max_inner, delta=1e-4)
        parity.compare(res.signal(i), ref)


def test_long_classes_of_many_signals_match_oracle(dev, oracle_mod):
    """Classes of 8 or more long signals take m from one CTA per signal (bisection);
    smaller classes from the grid-wide search.  Both match the oracle."""
    lens = [20736] * 8 + [24576] * 9 + [32768] * 2
    sigs = [signals.component_signal(78, i, n) for i, n in enumerate(lens)]
    x, offs = _pack(sigs, dev)
    with fif.Plan(max_n=1 << 15, max_imfs=3) as plan:
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
    for i, s in enumerate(sigs):
        ref = oracle_mod.direct(s.astype(np.float64), max_imfs=3)
        parity.compare(res.signal(i), ref)


def test_batch_launch_count(dev):
    """fif_plan_batch_launches: the fused lengths of one E share a persistent
    launch while their shared memory stays within 2x (1024 and 2048 here: one
    launch; 256 with 2048: two); a multi-pass class adds its fixed launch
    sequence (counted independently here from the structure of one outer
    iteration)."""
    short = [signals.component_signal(71, i, n) for i, n in enumerate([1024, 2048, 1024])]
    x, offs = _pack(short, dev)
    with fif.Plan(max_n=1 << 15, max_imfs=3, max_inner=8) as plan:
        assert plan.batch_launches() == 0
        plan.decompose_batch(x, offs)
        torch.cuda.synchronize()
        assert plan.schedule(1024)[0] == plan.schedule(2048)[0]
        assert plan.batch_launches() == 1
        far = [signals.component_signal(71, 5, 256), signals.component_signal(71, 6, 2048)]
        xf, offf = _pack(far, dev)
        plan.decompose_batch(xf, offf)
        torch.cuda.synchronize()
        assert plan.batch_launches() == 2
        sigs = short + [signals.component_signal(71, 9, 1 << 15)]
        x2, offs2 = _pack(sigs, dev)
        plan.decompose_batch(x2, offs2)
        torch.cuda.synchronize()
        # one long signal: grid-wide m search; max_inner = 8 fits one round of 8 candidates
        per_it = 2 + 2 * 1 + 1 + 2 + 1
        assert plan.batch_launches() == 1 + 4 + 1 + (3 + 1) * per_it
