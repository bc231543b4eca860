"""Benchmark: decomposed samples/s of FFT-based Iterative Filtering on GB300.

Default workload (the large uniform batch): 65536 independent float32 signals
of n = 4096 samples, each 2-5 chirped, amplitude-modulated components plus
N(0, 0.01^2) noise (seeded, synthetic), triangle window, nu = 1.6,
delta = 1e-3, max_inner = 200, max_imfs = 12.  One step = the full
decomposition of the batch (every IMF and the remainder) through
fif_decompose_batch.  Other workloads: --workload (see WORKLOADS).

Prints ONE JSON line (rank 0).  value = whole-job samples/s of the batch path
with inputs resident in HBM; e2e = the same through fif_decompose_batch_host
with pinned host buffers (the host-link transfers inside the timed region);
plain = the staged one-launch-per-step path on a subset of signals; roofline =
the fused kernel's algorithmic HBM bytes per launch / its measured duration
against the measured copy bandwidth; cpu_baseline = the FP64 oracle (direct
method) on a bounded sample, timed on the host cores, whose outputs also give
the parity summary of the sampled signals.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decomposed samples/s (batched FIF vs plain) at stated IMF error; HBM roofline %"
UNIT = "samples/s"
PARAMS = dict(nu=1.6, mask_scale=1, delta=1e-3, max_inner=200, max_imfs=10)
DEFAULT_WORKLOAD = "batch4096"

# Other synthetic workloads (not the default line): name -> description, generator args
WORKLOADS = {
    "batch4096": dict(desc="65536 float32 signals, n=4096, 2-5 chirped AM components + "
                           "N(0,0.01^2) noise; triangle window, nu=1.6, delta=1e-3, max_inner=200, "
                           "max_imfs=12"),
    "batch4096_d1e-4": dict(desc="65536 float32 signals, n=4096, as batch4096 with delta=1e-4"),
    "batch4096_bf16": dict(desc="the batch4096 signals with the split-BF16 tensor-core variant "
                                "(FIF_PREC_SPLIT_BF16: radix-16 inverse-FFT passes as BF16 hi+lo "
                                "mma products, FP32 accumulation); delta=1e-3, max_imfs=12"),
    "batch16384": dict(desc="1024 float32 signals, n=16384, 2-5 chirped AM components + "
                            "N(0,0.01^2) noise; triangle window, nu=1.6, delta=1e-3, "
                            "max_inner=200, max_imfs=10"),
    "single4096": dict(desc="one n=4096 three-component test signal (noise from default_rng(0)); "
                            "delta=1e-3, max_inner=200, max_imfs=10"),
    "uneven": dict(desc="4096 float32 signals, n log-uniform in [256, 2^20] rounded to 2^a 3^b, "
                        "2-5 chirped AM components + noise; delta=1e-3, max_imfs=10"),
    "long": dict(desc="one float32 signal, n=2^24, 6 components f0=10^{0..6}, noise 1e-3; "
                      "delta=1e-3, max_imfs=10"),
    "long_bf16": dict(desc="the long signal with the split-BF16 tensor-core variant (radix-16 "
                           "passes of both multi-pass inverse levels as BF16 hi+lo mma "
                           "products, FP32 accumulation); delta=1e-3, max_imfs=10"),
    "batch16384_n0": dict(desc="the batch16384 signals with m from the a-priori bound of "
                               "Theorem 5 (eq. N0_discrete; absolute delta=2.0, "
                               "max_inner=65536, max_imfs=10)"),
    "batch16384_th": dict(desc="the batch16384 signals, thresholded IMFs (eq. I_gamma, "
                               "gamma=0.05; delta=1e-3, max_inner=200, max_imfs=10)"),
    "batch16384_pk": dict(desc="the batch16384 signals, mask length from the spectral peak "
                               "(end of Sec. 2; delta=1e-3, max_inner=200, max_imfs=10)"),
    "batch16384_sh": dict(desc="the batch16384 signals, window generated by the shape "
                               "g(x) = sin(pi x) (33 samples; Theorem 4's h * h); delta=1e-3, "
                               "max_inner=200, max_imfs=10"),
    "uneven_sh": dict(desc="the uneven signals with the window generated by g(x) = sin(pi x) "
                           "(a float-float transform of h per IMF on the multi-pass path); "
                           "delta=1e-3, max_imfs=10"),
}

# generating shape of the batch16384_sh workload
SINE_SHAPE = np.sin(np.pi * np.linspace(0.0, 1.0, 33))


def _gen_chunk(args):
    wid, first, lens = args
    sys.path.insert(0, ROOT)
    from paper_1802_01359_gb300 import signals
    return [signals.component_signal(wid, first + i, int(n)) for i, n in enumerate(lens)]


def generate(wid, lens, first=0):
    """Signals first.. of workload wid with the given lengths, generated on a spawn process
    pool (started before any CUDA call).  Returns (float32 data, int64 offsets)."""
    import multiprocessing as mp
    lens = np.asarray(lens, dtype=np.int64)
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    data = np.empty(int(offs[-1]), dtype=np.float32)
    chunk = max(1, lens.size // 64)
    jobs = [(wid, first + a, lens[a:a + chunk]) for a in range(0, lens.size, chunk)]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    procs = max(1, min(16, (os.cpu_count() or 1) // max(world, 1)))
    with mp.get_context("spawn").Pool(procs) as pool:
        pos = 0
        for part in pool.map(_gen_chunk, jobs):
            for s in part:
                data[pos:pos + s.size] = s
                pos += s.size
    return data, offs


# uniform batches: workload -> (seed stream, signals per rank, n); rank r decomposes signals
# r*count .. r*count+count-1 of the stream (weak scaling, disjoint batches)
UNIFORM = {"batch4096": ("W_BATCH_4096", 65536, 4096), "batch4096_d1e-4": ("W_BATCH_4096", 65536, 4096),
           "batch4096_bf16": ("W_BATCH_4096", 65536, 4096),
           "batch16384": ("W_BATCH_16384", 1024, 16384), "batch16384_n0": ("W_BATCH_16384", 1024, 16384),
           "batch16384_th": ("W_BATCH_16384", 1024, 16384), "batch16384_pk": ("W_BATCH_16384", 1024, 16384),
           "batch16384_sh": ("W_BATCH_16384", 1024, 16384)}


def first_signal(name, rank):
    """Index of rank's first signal in the workload's seed stream."""
    return rank * UNIFORM[name][1] if name in UNIFORM else 0


def make_workload(name, rank=0):
    """(data, offsets, params) of a named workload."""
    from paper_1802_01359_gb300 import signals
    params = dict(PARAMS)
    if name in ("batch16384", "batch16384_n0", "batch16384_th", "batch16384_pk",
                "batch16384_sh"):
        data, offs = generate(signals.W_BATCH_16384, np.full(1024, 16384),
                              first=first_signal(name, rank))
        if name == "batch16384_n0":
            params.update(delta=2.0, max_inner=1 << 16, apriori_n0=True)
        if name == "batch16384_th":
            params.update(gamma=0.05)
        if name == "batch16384_pk":
            params.update(peak_mask=True)
        if name == "batch16384_sh":
            params.update(window_shape=SINE_SHAPE)
    elif name == "single4096":
        s = signals.single_4096()
        data, offs = s, np.array([0, s.size], dtype=np.int64)
    elif name in ("uneven", "uneven_sh"):
        lens = signals.uneven_lengths(4096)
        data, offs = generate(signals.W_UNEVEN, lens)
        if name == "uneven_sh":
            params.update(window_shape=SINE_SHAPE)
    elif name in ("long", "long_bf16"):
        s = signals.long_signal()
        data, offs = s, np.array([0, s.size], dtype=np.int64)
        if name == "long_bf16":
            params["precision"] = 1  # FIF_PREC_SPLIT_BF16
    elif name in ("batch4096", "batch4096_d1e-4", "batch4096_bf16"):
        data, offs = generate(signals.W_BATCH_4096, np.full(65536, 4096),
                              first=first_signal(name, rank))
        params["max_imfs"] = 12
        if name == "batch4096_d1e-4":
            params["delta"] = 1e-4
        if name == "batch4096_bf16":
            params["precision"] = 1  # FIF_PREC_SPLIT_BF16
    else:
        raise SystemExit(f"unknown workload {name}")
    return data, offs, params
L2_FLUSH_BYTES = 512 << 20
FUSED_SOURCES = ("paper_1802_01359_gb300/csrc/fif_device.cuh",
                 "paper_1802_01359_gb300/csrc/fif_fused.cu",
                 "paper_1802_01359_gb300/csrc/fif_internal.h",
                 "paper_1802_01359_gb300/csrc/fif_tc.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_kernel_traffic.json")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def fused_source_hash() -> str:
    h = hashlib.sha256()
    for rel in FUSED_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(n_units: int, key: str):
    """DRAM bytes per launch from the committed ncu record of this kernel and length (key
    "n" or "n_bf16"), scaled from the captured launch to this launch's signal count, if the
    kernel sources still match the profiled ones; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        t = json.load(f)
    if t.get("source_hash") != fused_source_hash():
        return None
    rec = t.get("records", {}).get(key)
    return None if rec is None else float(rec["dram_bytes_per_signal"]) * n_units


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(seconds: float, dist, device) -> float:
    """The largest of every rank's timed seconds (each rank's own device clock)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(samples_per_rank: int, world: int, seconds: float) -> float:
    """Samples all ranks decomposed (each rank its own batch) per second of the slowest."""
    return samples_per_rank * world / seconds


def oracle_sample(data, offs, idx, threads, params=None):
    """The FP64 oracle (direct method, tier B) on signals idx, one signal per task on a
    thread pool (the C oracle releases the GIL).  Returns (results, seconds)."""
    import concurrent.futures as cf

    import oracle
    oracle.build()

    prm = dict(params or PARAMS)
    prm.pop("precision", None)  # the oracle is binary64 throughout
    if prm.pop("apriori_n0", False):
        prm["apriori"] = True
    if "window_shape" in prm:
        prm["shape"] = prm.pop("window_shape")

    def one(i):
        return oracle.direct(data[offs[i]:offs[i + 1]].astype(np.float64), **prm)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, idx))
    return res, time.perf_counter() - t0


def _step_divergence(g, r):
    """First outer step where the GPU result g (with diag records) and the oracle result r
    part, as (step, what, excused): excused when the side-specific tie flag of THAT step
    (the GPU's diag[k].flags or the oracle's imf_flags[k]) allows it.  An extrema count
    that differs (flagged) but leaves the stop test and L unchanged does not part them.
    None if the decisions agree everywhere (stop tests, L, m, IMF count, stop reason)."""
    EXT, NDT = 1 << 9, 1 << 8
    K_g, K_r = g.n_imfs, r["n_imfs"]
    m = g.m.cpu().numpy() if hasattr(g.m, "cpu") else np.asarray(g.m)
    L = g.mask_len.cpu().numpy() if hasattr(g.mask_len, "cpu") else np.asarray(g.mask_len)
    for k in range(min(K_g, K_r) + 1):
        fl = int(g.diag[k]["flags"]) | int(r["imf_flags"][k])
        ke_g, ke_r = int(g.diag[k]["k_extrema"]), int(r["kext"][k])
        if ke_g != ke_r and (not (fl & EXT) or (ke_g < 2) != (ke_r < 2)):
            return k, "extrema", bool(fl & EXT)
        if k == K_g or k == K_r:
            break
        if L[k] != r["L"][k]:
            return k, "L", bool(fl & EXT)
        if m[k] != r["m"][k]:
            return k, "m", bool(fl & NDT)
    if K_g != K_r or g.stop != r["stop"]:
        return min(K_g, K_r), "count", False
    return None


def parity_summary(res_gpu, refs, idx, statuses):
    """Parity of the sampled signals against the oracle, with the per-step tie rule of the
    tests: integers exact, a divergence counted as flagged only when a tie flag of that
    step excuses it; IMF and remainder relative L2 errors of every compared row; and the
    fraction of all signals of the batch whose status carries each tie flag."""
    exact, flagged, unflagged, errs, rerrs = 0, 0, 0, [], []
    for r, i in zip(refs, idx):
        g = res_gpu.signal(int(i))
        div = _step_divergence(g, r)
        upto = g.n_imfs if div is None else div[0]
        imfs = g.imfs.cpu().numpy().astype(np.float64)
        for k in range(upto):
            errs.append(float(np.linalg.norm(imfs[k] - r["imfs"][k]) / np.linalg.norm(r["imfs"][k])))
        if div is None:
            exact += 1
            nr = np.linalg.norm(r["remainder"])
            rerrs.append(float(np.linalg.norm(imfs[g.n_imfs] - r["remainder"]) / nr) if nr > 0
                         else float(np.linalg.norm(imfs[g.n_imfs])))
        elif div[2]:
            flagged += 1
        else:
            unflagged += 1
    st = np.asarray(statuses, dtype=np.int64)
    frac = lambda b: float(((st & b) != 0).mean()) if st.size else 0.0
    return {"signals": len(idx), "exact": exact, "diverged_flagged": flagged,
            "int_mismatch_unflagged": unflagged,
            "max_imf_rel_l2": max(errs) if errs else None,
            "median_imf_rel_l2": float(np.median(errs)) if errs else None,
            "max_remainder_rel_l2": max(rerrs) if rerrs else None,
            "rule": "per-step flags (GPU diag record or oracle step record)",
            "tie_fraction_all_signals": {"extrema_tie": frac(1 << 9), "near_delta_tie": frac(1 << 8),
                                         "fp64_tiebreak": frac(1 << 11)}}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, on bounded samples of the same
    workload.  The per-step sample is sized from the warm-up steps so that the K timed
    steps take about a minute in total."""
    if rank != 0:
        return
    data, offs, params = make_workload(args.workload)
    lens = np.diff(offs)
    threads = os.cpu_count() or 1
    order = [int(i) for i in np.random.default_rng(777).permutation(lens.size)]
    first = order[:threads]
    t_warm = None
    for _ in range(args.warmup):
        _, dt = oracle_sample(data, offs, first, threads, params)
        t_warm = dt if t_warm is None else min(t_warm, dt)
    rate = float(lens[first].sum()) / t_warm          # samples/s on all cores
    want = rate * 60.0 / max(args.steps, 1)           # samples per timed step
    idx, tot = [], 0
    for i in order:
        if idx and tot + lens[i] > want:
            break
        idx.append(i)
        tot += int(lens[i])
    used = min(threads, len(idx))
    t = 0.0
    for _ in range(args.steps):
        _, dt = oracle_sample(data, offs, idx, used, params)
        t += dt
    value = tot * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "name": args.workload,
                   "signals": int(lens.size), "samples": int(offs[-1]),
                   "step_sample_signals": len(idx)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{len(idx)} random signals of the workload ({tot} samples) "
                                   "per step, FP64 direct method (tier B), one signal per thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fif")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample", type=int, default=48)
    ap.add_argument("--plain-signals", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="fixed schedules, no autotuning")
    ap.add_argument("--schedule", default="",
                    help="schedules to load instead of autotuning, in the plan's tuning-file line "
                         "format ('n E' fused, 'n E1 TJ1 E2 TJ2' multi-pass), lines separated by "
                         "';' (reproduces a tuned run under a profiler, whose timings would "
                         "mislead the tuner)")
    ap.add_argument("--signals", type=int, default=0,
                    help="decompose only the first N signals of the workload (reduced cases for "
                         "profiler captures); 0 = all")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    # ranks exist only under torchrun; a plain run is one GPU whatever --gpus says
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world and rank == 0:
        print(f"bench.py: --gpus {args.gpus} but {world} rank(s) launched; timing {world}",
              file=sys.stderr)

    if args.impl == "reference":
        dist = None
        if world > 1 and "RANK" in os.environ:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    # inputs first: the generator pool is spawned before any CUDA call
    data, offs, params = make_workload(args.workload, rank)
    if 0 < args.signals < offs.size - 1:
        offs = offs[:args.signals + 1].copy()
        data = data[:int(offs[-1])]
    lens = np.diff(offs)
    nsig = lens.size

    dist = None
    import torch
    if world > 1 and "RANK" in os.environ:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")

    from paper_1802_01359_gb300 import build, fif
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    x = torch.from_numpy(data).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    plan = fif.Plan(max_n=int(lens.max()), stream=stream, **params)
    plan.prepare(sorted(set(int(v) for v in lens)))
    out = plan.alloc_batch_outputs(lens, dev)
    tune_s = None
    if args.schedule:
        import tempfile
        with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as f:
            f.write("\n".join(ln.strip() for ln in args.schedule.split(";")) + "\n")
        plan.load_tuning(f.name)
        os.unlink(f.name)
    elif not args.no_tune:
        # schedule autotuning per length class, before (and outside) the timed region
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            plan.tune(x, offs, out=out)
        stream.synchronize()
        tune_s = time.perf_counter() - t0

    chosen = []  # fused schedule of the first few lengths, multi-pass of the largest
    ulens = sorted(set(int(v) for v in lens))
    for n in ulens[:4]:
        try:
            E, T, _ = plan.schedule(n)
            chosen.append(f"n={n}: E={E}, {T} threads")
        except fif.FifError:
            pass
    for n in ulens[-3:]:
        if n <= fif.fused_max_n():
            continue
        ms = plan.multipass_schedule(n)
        chosen.append(f"n={n}: {ms['R1']}x{ms['R2']}, level 1 E={ms['E1']} TJ={ms['TJ1']}, "
                      f"level 2 E={ms['E2']} TJ={ms['TJ2']}{' (tuned)' if ms['tuned'] else ''}")

    def step():
        plan.decompose_batch(x, offs, out=out)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()

    # ---- timed region: K steps, L2 flushed between steps, events on the plan's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = whole_job_rate(int(offs[-1]) * args.steps, world, t_total)

    # ---- algorithmic bytes of one step: read s, write K_i IMFs + remainder, ints
    nim = out.n_imfs.cpu().numpy().astype(np.int64)
    K = params["max_imfs"]
    alg_bytes = int((4 * lens + 4 * lens * (nim + 1)).sum() + nsig * (8 * K + 8))
    kern_s = statistics.mean(step_ms) / 1e3
    peak, peak_kind = peaks()
    achieved = alg_bytes / kern_s / 1e9
    fused_only = args.workload.startswith("batch") or args.workload == "single4096"
    traffic = None
    if args.workload in UNIFORM:
        tkey = str(UNIFORM[args.workload][2]) + ("_bf16" if params.get("precision") else "")
        traffic = recorded_traffic(nsig, tkey)

    desc = WORKLOADS[args.workload]["desc"]
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if not params.get("precision") else "f32 (radix-16 inverse stages: bf16 hi+lo products, f32 accumulation)",
        "data": "synthetic",
        "config": {"workload": desc, "name": args.workload, "signals": nsig,
                   "samples": int(offs[-1]),
                   "path": "fused batch (one CTA per signal, shared-memory resident)" if fused_only
                   else "batch: fused for short signals, multi-pass for long ones, one CUDA graph",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "schedule": ("loaded (--schedule)" if args.schedule
                                else "fixed rule" if tune_s is None
                                else f"autotuned per length class (fif_plan_tune, {tune_s:.2f} s "
                                     "before timing)") + ("; " + "; ".join(chosen) if chosen else ""),
                   "mean_imfs": float(nim.mean())},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "kernel": "fused_kernel (one launch per step)" if fused_only
                     else "whole step (all kernels of the graph)",
                     "alg_bytes_per_launch": alg_bytes},
        # kernels of one graph replay (fif_plan_batch_launches) times the timed steps
        "gpu_launches": plan.batch_launches() * args.steps,
        "clocks": clk.summary(),
    }

    # ---- e2e through the host-buffer C entry point (pinned host memory)
    if not args.no_e2e:
        K1 = K + 1
        h_in = torch.from_numpy(data).pin_memory().numpy()
        h_out = dict(imfs=torch.empty(int(offs[-1]) * K1, dtype=torch.float32).pin_memory().numpy(),
                     m=np.zeros((nsig, K), np.int32), mask_len=np.zeros((nsig, K), np.int32),
                     n_imfs=np.zeros(nsig, np.int32), status=np.zeros(nsig, np.int32), diag=None)
        for _ in range(2):
            plan.decompose_batch_host(h_in, offs, out=h_out)
        if dist is not None:
            dist.barrier()
        e2e_steps = max(3, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.decompose_batch_host(h_in, offs, out=h_out)
        te = max_over_ranks(time.perf_counter() - t0, dist, dev)
        result["e2e"] = {"value": whole_job_rate(int(offs[-1]) * e2e_steps, world, te),
                         "unit": UNIT,
                         "h2d_bytes_per_step": int(h_in.nbytes),
                         "d2h_bytes_per_step": int(h_out["imfs"].nbytes + 4 * nsig * (2 * K + 2))}

    # ---- plain staged path (one launch per step of the method) on a subset
    if rank == 0 and args.plain_signals > 0 and fused_only:
        P = min(args.plain_signals, nsig)
        n0 = int(lens[0])
        with torch.cuda.stream(stream):
            plan.decompose(x[:n0])            # warm
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        views = [x[int(offs[i]):int(offs[i + 1])] for i in range(P)]
        lib = fif.load_library()
        imfs = torch.empty((K + 1) * n0, dtype=torch.float32, device=dev)
        mm = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
        LL = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
        ni = torch.empty(1, dtype=torch.int32, device=dev)
        ss = torch.empty(1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        e0.record(stream)
        for v in views:
            rc = lib.fif_decompose(plan.handle, v.data_ptr(), n0, imfs.data_ptr(), mm.data_ptr(),
                                   LL.data_ptr(), ni.data_ptr(), ss.data_ptr(), None)
            assert rc == 0, fif.status_string(rc)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        result["plain"] = {"value": P * n0 / tp, "unit": UNIT, "signals_timed": P,
                           "launches_per_signal": 1 + 3 * (K + 1),
                           "path": "staged, one kernel launch per step per outer iteration"}
        result["batched_over_plain"] = value / world / result["plain"]["value"]

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N=1), plus parity
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        threads = os.cpu_count() or 1
        rng = np.random.default_rng(12345)
        # a bounded sample: about 30 s of oracle work on the machine's cores
        order = rng.permutation(nsig)
        budget = 16 * threads * 16384 if not args.workload.startswith("long") else 1 << 24
        idx, tot = [], 0
        for i in order[:max(args.cpu_sample, 1)]:
            if tot + lens[i] > budget and idx:
                continue
            idx.append(int(i))
            tot += int(lens[i])
        idx.sort()
        refs, tc = oracle_sample(data, offs, idx, threads, params)
        # the sampled signals' per-IMF diag records come from one more (untimed) call with
        # diagnostics on; the timed outputs give the batch's status words
        dres = plan.decompose_batch(x, offs, diag=True)
        torch.cuda.synchronize()
        result["cpu_baseline"] = {"value": tot / tc, "unit": UNIT, "cores": min(threads, len(idx)),
                                  "kind": "oracle",
                                  "sample": f"{len(idx)} random signals of the workload "
                                            f"({tot} samples), FP64 direct method (tier B), one "
                                            "signal per thread"}
        result["parity"] = parity_summary(dres, refs, idx, out.status.cpu().numpy())
        del dres

    plan.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
