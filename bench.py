"""Benchmark: Billiard steps/s on the paper's random spectrahedron S-200-200
(n = m = 200, Sec. 4 generator), 8192 independent chains, one GPU per rank.

A bench "step" is one Billiard step (Alg. 5) of every chain: each chain draws
a direction and a length and runs the boundary oracle (form F, V; Cholesky;
extreme eigenpair; normal; reflect) until the length is used up.  Chains are
independent, so N GPUs run N replicas on disjoint chain ranges (weak scaling,
no collective on the data path).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(test infrastructure) on the host cores instead, on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DIM, M_DIM, CHAINS = 200, 200, 8192
SEED_SPEC = 2010_03817 + 6   # S-200-200 workload seed
SEED_WALK = 1234
RHO, KAPPA = 1000, 1e-6
# tau ~ diam(S) (Alg. 5).  For this workload: the longest chord through the
# origin over 256 seeded random directions (a pilot run of the boundary
# oracle), fixed here so that every arm uses the same value.
TAU = 0.3752
WORKLOAD = "Dabbene S-200-200 (n=m=200), 8192 chains, Billiard walk"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="fp64")
    p.add_argument("--chains", type=int, default=CHAINS)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--tau-scale", type=float, default=1.0,
                   help="scale the length scale tau (a small value gives short steps, "
                        "for profiling captures)")
    return p.parse_args()


def workload():
    from paper_2010_03817_gb300 import workloads as W
    return W.dabbene(N_DIM, M_DIM, seed=SEED_SPEC)


def start_points(A, C, rank):
    # a small random cloud around the interior point x = 0
    from paper_2010_03817_gb300 import workloads as W
    return W.random_directions(N_DIM, C, seed=SEED_WALK + rank) * 1e-3


def estimate_tau(spec, torch, C=256):
    """tau ~ diameter (Alg. 5): the longest chord through 0 over random directions."""
    from paper_2010_03817_gb300 import workloads as W
    V = torch.tensor(W.random_directions(N_DIM, C, seed=99), device="cuda")
    X = torch.zeros_like(V)
    tm, tp, _, st = spec.intersect(X, V)
    return float((tp - tm).max())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU baseline: the oracle on the host cores
# ----------------------------------------------------------------------------
def cpu_oracle_rate(A, tau, chains=32, steps=1):
    import oracle
    X0 = start_points(A, chains, 0)
    t0 = time.perf_counter()
    _, stats = oracle.walk("billiard", A, X0, steps, tau=tau, rho=RHO, kappa=KAPPA,
                           seed=SEED_WALK)
    dt = time.perf_counter() - t0
    return dict(value=chains * steps / dt, unit="steps/s", cores=oracle.num_threads(),
                kind="oracle",
                sample="%d chains x %d Billiard step(s) of the same workload (%d segments), "
                       "%.1f s on %d threads" % (chains, steps, stats["segments"], dt,
                                                 oracle.num_threads()),
                segments=stats["segments"], seconds=dt)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    A = workload()
    tau = TAU
    times, segs = [], 0
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(A, tau, chains=16, steps=1)
        if i >= args.warmup:
            times.append(r["seconds"])
            segs += r["segments"]
    total = sum(times)
    value = 16 * args.steps / total
    line = {
        "impl": "reference", "metric": "billiard steps/s at n=m=200", "value": value,
        "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (oracle sample: 16 chains x 1 step per bench step)"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "16 chains x 1 Billiard step per bench step, %d segments"
                                   % segs},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def alg_flops_fp64(n, m, stats, steps):
    """Algorithmic FP64 flops of the plain path: per segment 2nP (V) +
    m^3/3 (Cholesky) + 2(n+1)P (w); 2nP per step for F(x) at the step start,
    2P per reflection for the carried F; 4m^2 per Lanczos iteration."""
    P = m * (m + 1) / 2
    per_seg = 2 * n * P + m ** 3 / 3 + 2 * (n + 1) * P
    return (stats["segments"] * per_seg + steps * 2 * n * P + stats["reflections"] * 2 * P
            + stats["lanczos_iters"] * 4 * m * m)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_2010_03817_gb300 import build, spectra

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    lib = spectra.lib()
    A = workload()
    spec = spectra.Spectrahedron(A)
    tau = TAU * args.tau_scale
    C = args.chains
    X0 = start_points(A, C, rank)
    chains = spectra.Chains(spec, C, x0=X0, seed=SEED_WALK, chain0=rank * C)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        chains.billiard(1, tau=tau, rho=RHO, kappa=KAPPA, mode=args.mode)
    torch.cuda.synchronize()
    _, s0 = chains.status()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            evs[i][0].record(stream)
            chains.billiard(1, tau=tau, rho=RHO, kappa=KAPPA, mode=args.mode)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_ms = float(sum(step_ms))
    _, s1 = chains.status()
    seg_stats = {k: s1[k] - s0[k] for k in s1}
    t_max = dev_ms
    if world > 1:
        t = torch.tensor([dev_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = world * C * args.steps / (t_max / 1e3)

    # roofline of the dominant (and only) kernel: FP64 ALU bound
    flops = alg_flops_fp64(N_DIM, M_DIM, seg_stats, C * args.steps)
    achieved = flops / (dev_ms / 1e3) / 1e12
    peak = 152 * 2 * 2 * 2.07e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        xh, step = chains.state_host()
        xh = np.ascontiguousarray(xh)
        out = np.empty_like(xh)
        k = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            chains.set_state(xh, step)
            chains.billiard(1, tau=tau, rho=RHO, kappa=KAPPA, mode=args.mode)
            out, step = chains.state_host(out)
            xh, out = out, xh
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": C * k / e2e_s * world, "unit": "steps/s",
               "h2d_bytes_per_step": int(xh.nbytes), "d2h_bytes_per_step": int(xh.nbytes)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            r = cpu_oracle_rate(A, tau, chains=32, steps=1)
            cpu = {k: r[k] for k in ["value", "unit", "cores", "kind", "sample"]}
        except Exception as exc:  # the baseline must not sink the GPU number
            cpu = {"value": None, "unit": "steps/s", "cores": None, "kind": "oracle",
                   "sample": "failed: %s" % exc}

    if rank == 0:
        line = {
            "metric": "billiard steps/s at n=m=200",
            "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_DIM, "m": M_DIM, "chains_per_gpu": C,
                       "path": args.mode, "tau": tau, "rho": RHO, "kappa": KAPPA,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "replicas x%d" % world},
            "segments_per_step": seg_stats["segments"] / (C * args.steps),
            "oracle_calls_per_s": seg_stats["segments"] * world / (t_max / 1e3),
            "lanczos_iters_per_segment": seg_stats["lanczos_iters"] / max(1, seg_stats["segments"]),
            "shift_retry_rate": seg_stats["shift_retries"] / max(1, seg_stats["segments"]),
            "bad_steps": seg_stats["bad_steps"],
            "roofline": {"bound": "alu", "kernel": "walk_fp64_kernel", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s (FP64)", "frac": achieved / peak,
                         "traffic": None},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
