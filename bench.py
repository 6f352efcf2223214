#!/usr/bin/env python3
"""Benchmark of the unbalanced Beckmann-OT proximal hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload prox|rpca]

Prints ONE JSON line (rank 0).  Workloads (synthetic, seeded):

* ``prox`` -- Algorithm 1 on the 63 frame pairs of a 64-frame 256x256 blob
  video (the prox batch of line 11 of Algorithm 3).  A step is one check
  interval: 10 fused iterations, the last computing the FP64 stopping sums,
  and the read-back of those sums.

The metric is prox pixel-iterations per second (B * H * W * iterations / s).
Multi-GPU (torchrun): every rank solves its own batch (replicas, weak
scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "OT-prox pixel-iters/s"
UNIT = "pixel-iter/s"
BYTES_PER_PIXEL_ITER = {"prox": 56, "fixed_first": 48, "eval": 40}
ITERS_PER_STEP = 10


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1909_00149_gb300", "csrc", "prox_tma.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_tag: str) -> float | None:
    """DRAM bytes per launch of the tiled iteration kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "prox_tma_63x256x256.md")
    if not os.path.exists(path):
        return None
    src_hash, traffic = None, None
    for line in open(path):
        if line.startswith("source_sha256_16:"):
            src_hash = line.split(":", 1)[1].strip()
        if line.startswith(f"traffic_bytes_per_launch[{kernel_tag}]:"):
            traffic = float(line.split(":", 1)[1].strip())
    if src_hash != kernel_source_hash():
        return None
    return traffic


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip() not in ("Not Active", "0", "[N/A]"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- workloads
def prox_inputs(rank: int):
    from synth import blob_video, rng_for
    v = blob_video(rng_for(1, 100 + rank), 64, 256, 256, n_blobs=8)
    return np.ascontiguousarray(v[:-1]), np.ascontiguousarray(v[1:])


PROX_KW = dict(mu=3.0, rho=0.01, kernel="tma", use_graph=True, check_every=ITERS_PER_STEP)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1909_00149_gb300 as otp

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    p0, p1 = prox_inputs(rank)
    B, H, W = p0.shape
    px = B * H * W
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        s = otp.OtProx(B, H, W, stream=stream, **PROX_KW)
        d0 = torch.from_numpy(p0).cuda()
        d1 = torch.from_numpy(p1).cuda()
        s.set_input(d0, d1)
        torch.cuda.synchronize()

        # ---- device-resident throughput
        for _ in range(args.warmup):
            s.check_interval(ITERS_PER_STEP)
        sampler = ClockSampler(local_rank)
        barrier()
        torch.cuda.synchronize()
        sampler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            s.check_interval(ITERS_PER_STEP)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1)

        # ---- the iteration kernel alone (events on the library's stream)
        kernel_ms = []
        for _ in range(max(args.steps, 3)):
            kernel_ms.append(s.step_timed(ITERS_PER_STEP) / ITERS_PER_STEP)
        k_ms = statistics.median(kernel_ms)

        # ---- end to end through the C ABI with pinned host buffers
        h0 = torch.from_numpy(p0).pin_memory()
        h1 = torch.from_numpy(p1).pin_memory()
        for _ in range(max(1, args.warmup // 2)):
            s.set_input(h0, h1)
            s.check_interval(ITERS_PER_STEP)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            s.set_input(h0, h1)            # H2D of this step's inputs
            s.check_interval(ITERS_PER_STEP)   # D2H of the step's stopping sums
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        s.close()

    if dist:
        t = torch.tensor([ms, e2e_ms, k_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, e2e_ms, k_ms = t.tolist()
    if rank != 0:
        return None

    units = px * ITERS_PER_STEP * args.steps * world
    value = units / (ms / 1e3)
    e2e_value = units / (e2e_ms / 1e3)
    peaks = measured_peaks()
    alg_bytes = BYTES_PER_PIXEL_ITER["prox"] * px
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "prox_63_pairs_256x256 (64-frame 256x256 blob video, Algorithm 1)",
                   "B": B, "H": H, "W": W, "iters_per_step": ITERS_PER_STEP, "mu": PROX_KW["mu"],
                   "rho": PROX_KW["rho"], "kernel": PROX_KW["kernel"], "cuda_graph": True,
                   "l2": "inputs larger than L2 (11 state planes = %.0f MB; 231 MB moved per iteration)" % (11 * px * 4 / 1e6)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic("nored"),
                     "kernel": "prox_tma_kernel (Algorithm 1 iteration, no reduction)",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": k_ms,
                     "peak_source": peaks["source"] + " copy bandwidth (of measured)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * px * 4, "d2h_bytes_per_step": 8 * 8},
        "gpu_launches": (ITERS_PER_STEP + 1) * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p0, p1, budget_s=args.cpu_seconds)
    return line


# --------------------------------------------------------------------- oracle timing
def oracle_sample_rate(p0, p1, budget_s: float, n_pairs: int = 2):
    """Pixel-iterations/s of the FP64 oracle's Algorithm 1 on the first
    ``n_pairs`` pairs of the batch, run until ``budget_s`` seconds pass."""
    from oracle import prox as P
    a0 = p0[:n_pairs].astype(np.float64)
    a1 = p1[:n_pairs].astype(np.float64)
    prm = P.default_steps(a0.shape[1], a0.shape[2], P.ProxParams(mu=PROX_KW["mu"], rho=PROX_KW["rho"]))
    st = P.zero_state(a0, a1, "prox")
    t0 = time.perf_counter()
    n = 0
    while True:
        st = P.alg1_iteration(st, a0, a1, prm)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s and n >= 3:
            break
    return a0.size * n / el, n, el


def cpu_baseline(p0, p1, budget_s: float) -> dict:
    rate, n, el = oracle_sample_rate(p0, p1, budget_s)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 NumPy oracle, Algorithm 1, {n} iterations on 2 of the 63 pairs "
                      f"(2x256x256) in {el:.1f} s, single thread"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    p0, p1 = prox_inputs(0)
    from oracle import prox as P
    a0 = p0[:2].astype(np.float64)
    a1 = p1[:2].astype(np.float64)
    prm = P.default_steps(256, 256, P.ProxParams(mu=PROX_KW["mu"], rho=PROX_KW["rho"]))
    st = P.zero_state(a0, a1, "prox")
    per_step = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(ITERS_PER_STEP):
            st = P.alg1_iteration(st, a0, a1, prm)
        el = time.perf_counter() - t0
        if k >= args.warmup:
            per_step.append(el)
    tot = sum(per_step)
    units = 2 * 256 * 256 * ITERS_PER_STEP * args.steps
    value = units / tot
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "prox_63_pairs_256x256 (64-frame 256x256 blob video, Algorithm 1)",
                       "iters_per_step": ITERS_PER_STEP, "sample": "2 of 63 pairs"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"FP64 NumPy oracle, {ITERS_PER_STEP} Algorithm 1 iterations on 2 of the 63 "
                                       "256x256 pairs per step, single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["prox"], default="prox")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
