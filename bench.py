"""Benchmark: decomposed samples/s of FFT-based Iterative Filtering on GB300.

Workload: 1024 independent float32 signals of n = 16384 samples, each 2-5
chirped, amplitude-modulated components plus N(0, 0.01^2) noise (seeded,
synthetic), triangle window, nu = 1.6, delta = 1e-3, max_inner = 200,
max_imfs = 10.  One step = the full decomposition of the batch (every IMF and
the remainder) through fif_decompose_batch.

Prints ONE JSON line (rank 0).  value = whole-job samples/s of the fused batch
path with inputs resident in HBM; e2e = the same through
fif_decompose_batch_host with pinned host buffers (copies inside the timed
region); plain = the staged one-launch-per-step path on a subset of signals;
roofline = the fused kernel's algorithmic HBM bytes per launch / its measured
duration against the measured copy bandwidth; cpu_baseline = the FP64 oracle
(direct method) on a bounded sample, timed on the host cores, whose outputs
also give the parity summary of the sampled signals.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
BATCH, N = 1024, 16384
PARAMS = dict(nu=1.6, mask_scale=1, delta=1e-3, max_inner=200, max_imfs=10)
WORKLOAD = (f"batch of {BATCH} float32 signals, n={N}, 2-5 chirped AM components + N(0,0.01^2) "
            "noise; triangle window, nu=1.6, delta=1e-3, max_inner=200, max_imfs=10")
L2_FLUSH_BYTES = 512 << 20
FUSED_SOURCES = ("paper_1802_01359_gb300/csrc/fif_device.cuh",
                 "paper_1802_01359_gb300/csrc/fif_fused.cu",
                 "paper_1802_01359_gb300/csrc/fif_internal.h")
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


def recorded_traffic(n_units: int):
    """DRAM bytes per launch from the committed ncu summary, scaled to this launch's
    signal count, if the kernel sources still match the profiled ones."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        t = json.load(f)
    if t.get("source_hash") != fused_source_hash():
        return None
    return float(t["dram_bytes_per_signal"]) * n_units


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


def oracle_sample(data, offs, idx, threads):
    """The FP64 oracle (direct method, tier B) on signals idx, one signal per task on a
    thread pool (the C oracle releases the GIL).  Returns (results, seconds)."""
    import concurrent.futures as cf

    import oracle
    oracle.build()

    def one(i):
        return oracle.direct(data[offs[i]:offs[i + 1]].astype(np.float64), **PARAMS)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, idx))
    return res, time.perf_counter() - t0


def parity_summary(res_gpu, refs, idx):
    int_mismatch, errs, flagged = 0, [], 0
    for r, i in zip(refs, idx):
        g = res_gpu.signal(int(i))
        K = g.n_imfs
        m = g.m.cpu().numpy()[:K]
        L = g.mask_len.cpu().numpy()[:K]
        same = (K == r["n_imfs"] and np.array_equal(m, r["m"]) and np.array_equal(L, r["L"]))
        if not same:
            if g.status & (3 << 8):
                flagged += 1
            else:
                int_mismatch += 1
            continue
        imfs = g.imfs.cpu().numpy().astype(np.float64)
        for k in range(K):
            errs.append(float(np.linalg.norm(imfs[k] - r["imfs"][k]) / np.linalg.norm(r["imfs"][k])))
    return {"signals": len(idx), "int_mismatch_unflagged": int_mismatch,
            "diverged_flagged": flagged,
            "max_imf_rel_l2": max(errs) if errs else None,
            "median_imf_rel_l2": float(np.median(errs)) if errs else None}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, on bounded samples of the workload.
    The per-step sample is sized from a warm-up step so that the K timed steps take
    about a minute in total."""
    if rank != 0:
        return
    from paper_1802_01359_gb300 import signals
    threads = os.cpu_count() or 1
    pool = 4 * threads
    data, offs = signals.batch(signals.W_BATCH_16384, pool, N)
    t_warm = None
    for _ in range(args.warmup):
        _, dt = oracle_sample(data, offs, list(range(threads)), threads)
        t_warm = dt if t_warm is None else min(t_warm, dt)
    per_step = int(threads * 60.0 / (max(args.steps, 1) * t_warm))
    per_step = max(1, min(pool, per_step))
    idx = list(range(per_step))
    used = min(threads, per_step)
    t = 0.0
    for _ in range(args.steps):
        _, dt = oracle_sample(data, offs, idx, used)
        t += dt
    value = per_step * N * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "batch": BATCH, "n": N,
                                        "step_sample_signals": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{per_step} signals of the workload per step, FP64 direct "
                                   "method (tier B), one signal per thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fif")
    ap.add_argument("--cpu-sample", type=int, default=48)
    ap.add_argument("--plain-signals", type=int, default=64)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1 and "RANK" in os.environ:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")

    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch

    from paper_1802_01359_gb300 import build, fif, signals
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    # weak scaling: every rank decomposes its own batch of the workload
    data, offs = signals.batch(signals.W_BATCH_16384, BATCH, N, first=rank * BATCH)
    x = torch.from_numpy(data).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    plan = fif.Plan(max_n=N, stream=stream, **PARAMS)
    plan.prepare([N])
    out = plan.alloc_batch_outputs(np.diff(offs), dev)

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
    t_total = sum(step_ms) / 1e3
    if dist is not None:
        tt = torch.tensor([t_total], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt.item())
    samples_per_step = int(offs[-1]) * world
    value = samples_per_step * args.steps / t_total

    # ---- algorithmic bytes of one launch: read s, write K_i IMFs + remainder, ints
    nim = out.n_imfs.cpu().numpy().astype(np.int64)
    lens = np.diff(offs)
    alg_bytes = int((4 * lens + 4 * lens * (nim + 1)).sum() + BATCH * (8 * PARAMS["max_imfs"] + 8))
    kern_s = statistics.mean(step_ms) / 1e3
    peak, peak_kind = peaks()
    achieved = alg_bytes / kern_s / 1e9
    traffic = recorded_traffic(BATCH)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "n": N, "path": "fused batch (one CTA "
                   "per signal, shared-memory resident)", "l2": "flushed between steps "
                   f"({L2_FLUSH_BYTES >> 20} MiB write); inputs 64 MiB, outputs > L2",
                   "mean_imfs": float(nim.mean())},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "kernel": "fused_kernel<16>", "alg_bytes_per_launch": alg_bytes},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }

    # ---- e2e through the host-buffer C entry point (pinned host memory)
    K1 = PARAMS["max_imfs"] + 1
    h_in = torch.from_numpy(data).pin_memory().numpy()
    h_out = dict(imfs=torch.empty(int(offs[-1]) * K1, dtype=torch.float32).pin_memory().numpy(),
                 m=np.zeros((BATCH, K1 - 1), np.int32), mask_len=np.zeros((BATCH, K1 - 1), np.int32),
                 n_imfs=np.zeros(BATCH, np.int32), status=np.zeros(BATCH, np.int32), diag=None)
    for _ in range(2):
        plan.decompose_batch_host(h_in, offs, out=h_out)
    if dist is not None:
        dist.barrier()
    e2e_steps = max(3, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.decompose_batch_host(h_in, offs, out=h_out)
    te = time.perf_counter() - t0
    if dist is not None:
        tt = torch.tensor([te], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
    result["e2e"] = {"value": samples_per_step * e2e_steps / te, "unit": UNIT,
                     "h2d_bytes_per_step": int(h_in.nbytes),
                     "d2h_bytes_per_step": int(h_out["imfs"].nbytes + 4 * BATCH * (2 * (K1 - 1) + 2))}

    # ---- plain staged path (one launch per step of the method) on a subset
    if rank == 0 and args.plain_signals > 0:
        P = min(args.plain_signals, BATCH)
        with torch.cuda.stream(stream):
            plan_out = plan.decompose(x[:N])            # warm
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        views = [x[int(offs[i]):int(offs[i + 1])] for i in range(P)]
        lib = fif.load_library()
        K = PARAMS["max_imfs"]
        imfs = torch.empty((K + 1) * N, dtype=torch.float32, device=dev)
        mm = torch.empty(K, dtype=torch.int32, device=dev)
        LL = torch.empty(K, dtype=torch.int32, device=dev)
        ni = torch.empty(1, dtype=torch.int32, device=dev)
        ss = torch.empty(1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        e0.record(stream)
        for v in views:
            rc = lib.fif_decompose(plan.handle, v.data_ptr(), N, imfs.data_ptr(), mm.data_ptr(),
                                   LL.data_ptr(), ni.data_ptr(), ss.data_ptr(), None)
            assert rc == 0, fif.status_string(rc)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        result["plain"] = {"value": P * N / tp, "unit": UNIT, "signals_timed": P,
                           "launches_per_signal": 1 + 3 * (K + 1),
                           "path": "staged, one kernel launch per step per outer iteration"}
        result["batched_over_plain"] = value / world / result["plain"]["value"]

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N=1), plus parity
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        threads = os.cpu_count() or 1
        rng = np.random.default_rng(12345)
        idx = sorted(rng.choice(BATCH, size=min(args.cpu_sample, BATCH), replace=False).tolist())
        refs, tc = oracle_sample(data, offs, idx, threads)
        result["cpu_baseline"] = {"value": len(idx) * N / tc, "unit": UNIT, "cores": threads,
                                  "kind": "oracle",
                                  "sample": f"{len(idx)} random signals of the workload, FP64 "
                                            "direct method (tier B), one signal per thread"}
        result["parity"] = parity_summary(out, refs, idx)

    plan.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
