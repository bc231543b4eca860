"""GPU: schedule autotuning per length class (fif_plan_tune and the tuning file)."""
import numpy as np
import pytest

import parity
from paper_1802_01359_gb300 import fif, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VALID_E = {2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_01359_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _batch(seed, lens, dev):
    sigs = [signals.component_signal(seed, i, n) for i, n in enumerate(lens)]
    offs = np.zeros(len(lens) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    return sigs, torch.from_numpy(np.concatenate(sigs).astype(np.float32)).to(dev), offs


def test_tune_picks_valid_schedules_and_keeps_results(dev, oracle_mod, tmp_path):
    lens = [4096] * 12 + [3072] * 6 + [2187] * 4 + [16384] * 3 + [20736]
    sigs, x, offs = _batch(80, lens, dev)
    with fif.Plan(max_n=1 << 15, max_imfs=4) as plan:
        before = {n: plan.schedule(n) for n in (4096, 3072, 2187, 16384)}
        assert all(not t for _, _, t in before.values())
        ref = plan.decompose_batch(x, offs)
        torch.cuda.synchronize()
        res = plan.tune(x, offs)
        torch.cuda.synchronize()
        after = {n: plan.schedule(n) for n in (4096, 3072, 2187, 16384)}
        for n, (E, T, tuned) in after.items():
            assert tuned and E in VALID_E and 32 <= T <= 1024
        with pytest.raises(fif.FifError):
            plan.schedule(20736)                     # multi-pass length: no fused schedule
        # the tuned plan decomposes the same batch correctly
        again = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        path = str(tmp_path / "tuning.txt")
        plan.save_tuning(path)
    for i in (0, 12, 18, 22, 25):
        ref_i = oracle_mod.direct(sigs[i].astype(np.float64), max_imfs=4)
        parity.compare(again.signal(i), ref_i)
    # every schedule the tuner ran takes the same integer decisions on this batch
    assert torch.equal(res.m, again.m) and torch.equal(res.n_imfs, again.n_imfs)
    assert torch.equal(res.n_imfs, ref.n_imfs)
    lines = [ln.split() for ln in open(path).read().split("\n") if ln.strip()]
    assert {int(ln[0]) for ln in lines if len(ln) == 2} == {4096, 3072, 2187, 16384}
    assert {int(ln[0]) for ln in lines if len(ln) == 5} == {20736}   # the multi-pass length
    with fif.Plan(max_n=1 << 15, max_imfs=4) as p2:
        p2.load_tuning(path)
        for n, (E, T, tuned) in after.items():
            assert p2.schedule(n) == (E, T, True)
        assert p2.multipass_schedule(20736)["tuned"]


def test_multipass_tuning_keeps_results(dev, oracle_mod, tmp_path):
    """The multi-pass classes' inverse-level schedules (E, TJ per level) are tuned,
    valid, kept by save/load, and the tuned plan still matches the oracle."""
    lens = [20736] * 4 + [32768] * 3 + [65536] * 2
    sigs, x, offs = _batch(81, lens, dev)
    with fif.Plan(max_n=1 << 16, max_imfs=3) as plan:
        before = {n: plan.multipass_schedule(n) for n in (20736, 32768, 65536)}
        assert not any(v["tuned"] for v in before.values())
        plan.tune(x, offs)
        after = {n: plan.multipass_schedule(n) for n in (20736, 32768, 65536)}
        for n, v in after.items():
            assert v["tuned"] and v["R1"] * v["R2"] == n // 2
            assert v["E1"] in VALID_E and v["E2"] in VALID_E
            assert 1 <= v["TJ1"] <= 4 and 1 <= v["TJ2"] <= 4
        res = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        path = str(tmp_path / "mp.txt")
        plan.save_tuning(path)
    print("multi-pass schedules: before", before, "after", after)
    for i in (0, 4, 7, 8):
        parity.compare(res.signal(i), oracle_mod.direct(sigs[i].astype(np.float64), max_imfs=3))
    with fif.Plan(max_n=1 << 16, max_imfs=3) as p2:
        p2.load_tuning(path)
        assert p2.multipass_schedule(32768) == after[32768]


def test_load_tuning_skips_unusable_lines_and_rejects_garbage(dev, tmp_path):
    good = tmp_path / "t.txt"
    good.write_text("4096 8\n\n5000 8\n4096000 8\n2048 5\n")
    bad = tmp_path / "bad.txt"
    bad.write_text("4096 eight\n")
    with fif.Plan(max_n=16384) as plan:
        plan.load_tuning(str(good))
        assert plan.schedule(4096)[0] == 8 and plan.schedule(4096)[2]
        assert not plan.schedule(2048)[2]            # E = 5 is not a valid schedule
        with pytest.raises(fif.FifError):
            plan.load_tuning(str(bad))
        with pytest.raises(fif.FifError):
            plan.load_tuning(str(tmp_path / "missing.txt"))
