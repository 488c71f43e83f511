"""Benchmark: Billiard steps/s on the paper's random spectrahedron S-200-200
(n = m = 200, Sec. 4 generator), 8192 independent chains per GPU.

A bench "step" is one Billiard step (Alg. 5) of every chain: each chain draws
a direction and a length and runs the boundary oracle (pencil, Cholesky,
extreme eigenpair, normal, reflection) until the length is used up.

First --burn-in mixed-precision steps take the chains from their start cloud
into the body (recording the learned path's training tuples on the way) and
the warm-start network is trained on the GPU; all of this is outside the
timed region.  Then every path starts from that same state and is timed for
--steps steps after --warmup steps (the same step window for all): the
headline path (--mode, default "learned") and, for context, the others
("fp64": every step in FP64; "mixed": tensor-core formation and normals,
FP32 estimate, double-float refinement next to the boundary).  Every path's
t+ and normal are checked against the FP64 CPU oracle on sampled walk
states.

Chains are independent, so N GPUs run N replicas on disjoint chain ranges
(weak scaling, no collective on the data path).  Prints one JSON line (rank
0).  `--impl reference` times the FP64 CPU oracle (test infrastructure) on
the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
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
SEED_TRAIN = 4321
RHO, KAPPA = 1000, 1e-6
# tau ~ diam(S) (Alg. 5).  For this workload: the longest chord through the
# origin over 256 seeded random directions (a pilot run of the boundary
# oracle), fixed here so that every arm uses the same value.
TAU = 0.3752
T_SCALE = 0.05     # normalisation of log t+ for the warm-start network
WORKLOAD = "Dabbene S-200-200 (n=m=200), 8192 chains, Billiard walk"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--burn-in", type=int, default=4,
                   help="mixed Billiard steps from the start cloud before any path is timed; "
                        "every path then starts from that state (the same step window)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="learned", choices=["fp64", "mixed", "learned"])
    p.add_argument("--workload", default="s200",
                   choices=["s200", "batch", "hmc", "ball10", "ball40", "cube40"],
                   help="s200: the headline (S-200-200, 8192 chains); batch: 64 spectrahedra "
                        "of uneven n, m in one persistent launch")
    p.add_argument("--walk", default="billiard", choices=["billiard", "hnr", "cdhr"],
                   help="the walk timed (the headline is the Billiard walk; Hit-and-Run and "
                        "CDHR are context lines: CDHR reads V = A_j instead of forming it)")
    p.add_argument("--only", action="store_true", help="time the --mode path alone")
    p.add_argument("--chains", type=int, default=None,
                   help="chains per GPU (default: the workload's, 8192 for S-200-200)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-check", action="store_true", help="skip the sampled oracle check")
    p.add_argument("--stage-timers", action="store_true",
                   help="report the mixed path's per-stage cycle shares")
    p.add_argument("--tau-scale", type=float, default=1.0,
                   help="scale tau (a small value gives short steps, for profiling captures)")
    p.add_argument("--tol32", type=float, default=None,
                   help="stage-1 FP32 Lanczos tolerance of the mixed paths (library default 1e-5)")
    p.add_argument("--tol64", type=float, default=None,
                   help="stage-2 relative residual of the mixed paths (library default 1e-12)")
    p.add_argument("--delta1", type=float, default=None,
                   help="stage-2 shift of the mixed paths, sigma1 = sigma0 + (t~ - sigma0)(1 - "
                        "delta1) (library default 2e-4)")
    p.add_argument("--dump-checked", default=None,
                   help="save the checked calls and their errors to PREFIX_<path>.npz")
    p.add_argument("--check-samples", type=int, default=384,
                   help="boundary-oracle calls of each timed walk checked against the oracle")
    p.add_argument("--train-tuples", type=int, default=262144)
    p.add_argument("--train-epochs", type=int, default=24)
    return p.parse_args()


# The smaller bodies of the same walk (every path, same flow and checks):
# name -> (body, n, m, chains, tau = diam(S), description)
def _sized_workloads():
    from paper_2010_03817_gb300 import workloads as W
    return {
        "ball10": (lambda: W.ball_random(10, 10, 3.0, seed=W.BASE_SEED + 500), 10, 21, 64, 6.0,
                   "ball block r=3 + random block k=10 (n=10, m=21), 64 chains, Billiard walk"),
        "ball40": (lambda: W.ball_random(40, 40, 3.0, seed=W.BASE_SEED + 501), 40, 81, 4096, 6.0,
                   "ball block r=3 + random block k=40 (n=40, m=81), 4096 chains, Billiard walk"),
        "cube40": (lambda: W.rotated_cube(40, seed=W.BASE_SEED + 502), 40, 80, 4096,
                   2.0 * math.sqrt(40.0),
                   "rotated cube [-1,1]^40 (n=40, m=80), 4096 chains, Billiard walk"),
    }


_BODY = None


def workload():
    from paper_2010_03817_gb300 import workloads as W
    if _BODY is not None:
        return _BODY()
    return W.dabbene(N_DIM, M_DIM, seed=SEED_SPEC)


def metric_name(walk):
    if _BODY is None:
        return "%s steps/s at n=m=200" % walk
    return "%s steps/s at n=%d, m=%d" % (walk, N_DIM, M_DIM)


def use_workload(name):
    """Switch the module's workload constants to one of the smaller bodies."""
    global N_DIM, M_DIM, CHAINS, TAU, WORKLOAD, _BODY
    body, n, m, chains, tau, desc = _sized_workloads()[name]
    N_DIM, M_DIM, CHAINS, TAU, WORKLOAD, _BODY = n, m, chains, tau, desc, body


def replica_plan(rank, world, C):
    """Replicas: rank r runs chains [r C, (r + 1) C) (Philox chain offset) from
    its own start cloud; no collective on the data path."""
    return {"chain0": rank * C, "chains": C, "start_seed": SEED_WALK + rank}


def aggregate(ms_per_rank, world, C, steps):
    """Whole-job steps/s: all ranks' chain-steps over the slowest rank's time."""
    t = max(ms_per_rank)
    return world * C * steps / (t / 1e3), t


def start_points(C, rank):
    # a small random cloud around the interior point x = 0
    from paper_2010_03817_gb300 import workloads as W
    return W.random_directions(N_DIM, C, seed=replica_plan(rank, 1, C)["start_seed"]) * 1e-3


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
def cpu_oracle_rate(A, tau, X, step0, chains=32, steps=1):
    """The oracle's Billiard walk on chains 0..chains-1 from the points X
    (chains x n, host) over steps step0 .. step0+steps-1: the same chains,
    states and Philox draws as the GPU arms' first timed steps."""
    import oracle
    t0 = time.perf_counter()
    _, stats = oracle.walk("billiard", A, np.ascontiguousarray(X[:chains]), steps, tau=tau,
                           rho=RHO, kappa=KAPPA, seed=SEED_WALK, step0=step0, chain0=0)
    dt = time.perf_counter() - t0
    return dict(value=chains * steps / dt, unit="steps/s", cores=oracle.num_threads(),
                kind="oracle", segments_per_s=stats["segments"] / dt,
                sample="chains 0-%d of the burned-in state, steps %d-%d (the GPU arms' first "
                       "timed steps), %d segments, %.1f s on %d threads"
                       % (chains - 1, step0, step0 + steps - 1, stats["segments"], dt,
                          oracle.num_threads()),
                segments=stats["segments"], seconds=dt)


def run_reference(args):
    """The oracle (FP64, Cholesky + Jacobi, OpenMP over chains) on the GPU
    arms' workload and step window: chains 0..15 from the same start cloud
    walk the same burn-in and warm-up steps (untimed), then the --steps timed
    steps, each a bounded sample of the bench step (16 of the 8192 chains)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    A = workload()
    chains = 16  # one chain per host core of the box: 20 steps end in about 3 minutes
    X = start_points(CHAINS, 0)[:chains]
    X, _ = oracle.walk("billiard", A, X, args.burn_in + args.warmup, tau=TAU, rho=RHO,
                       kappa=KAPPA, seed=SEED_WALK, step0=0, chain0=0)
    times, segs = [], 0
    step = args.burn_in + args.warmup
    for _ in range(args.steps):
        t0 = time.perf_counter()
        X, st = oracle.walk("billiard", A, X, 1, tau=TAU, rho=RHO, kappa=KAPPA, seed=SEED_WALK,
                            step0=step, chain0=0)
        times.append(time.perf_counter() - t0)
        segs += st["segments"]
        step += 1
    total = sum(times)
    value = chains * args.steps / total
    line = {
        "impl": "reference", "metric": metric_name("billiard"), "value": value,
        "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (oracle sample: chains 0-%d, the GPU arms' timed "
                               "steps %d-%d)" % (chains - 1, args.burn_in + args.warmup,
                                                 step - 1)},
        "oracle_calls_per_s": segs / total,
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "chains 0-%d x %d burned-in Billiard steps (%d segments, "
                                   "%.1f segments per chain-step), %.1f s"
                                   % (chains - 1, args.steps, segs, segs / (chains * args.steps),
                                      total),
                         "segments_per_s": segs / total},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# algorithmic work
# ----------------------------------------------------------------------------
def alg_flops_fp64(n, m, stats, steps):
    """FP64 flops of the plain path: per segment 2nP (V) + m^3/3 (Cholesky) +
    2(n+1)P (normal); 2nP per step for F(x) at the step start, 2P per
    reflection for the carried F; 4m^2 per Lanczos iteration."""
    P = m * (m + 1) / 2
    per_seg = 2 * n * P + m ** 3 / 3 + 2 * (n + 1) * P
    return (stats["segments"] * per_seg + steps * 2 * n * P + stats["reflections"] * 2 * P
            + stats["lanczos_iters"] * 4 * m * m)


def alg_flops_wave(n, m, stats):
    """The method's own work in the mixed wave kernel (the factorisation and
    the eigen-solve of INTERSECTION): one Cholesky (m^3/3) per segment and
    4m^2 per iteration of the eigen-solve (two triangular solves and a product
    with V), counting the FP32 Lanczos and the double-float power iterations.
    The mixed path's second factorisation (double-float, next to the
    boundary) and its fills are overhead of the precision scheme, reported
    apart (alg_overhead_wave)."""
    return (stats["segments"] * m ** 3 / 3
            + (stats["lanczos_iters"] + stats["power_iters"]) * 4 * m * m)


def alg_overhead_wave(n, m, stats):
    """Flops the mixed wave kernel spends beyond the method's work: the
    second (double-float) factorisation per segment and the fills of both
    (2P each) and the carried-F update (2P)."""
    P = m * (m + 1) / 2
    return stats["segments"] * (m ** 3 / 3 + 6 * P)


def alg_flops_contraction(n, m, segments):
    """Tensor-core flops of the digit-split normal contraction: 28 digit pairs
    of a (rows x 16-padded m) x (m x (n+1) 32-padded m) product per segment."""
    Kp = (m + 15) // 16 * 16
    Q = (n + 1) * ((m + 31) // 32 * 32)
    return segments * 28 * 2 * Kp * Q


def alg_flops_formation(n, m, segments):
    """Tensor-core flops of the digit-split formation of V: 28 digit pairs of a
    (rows x 16-padded K) x (K x P) product per segment."""
    P = m * (m + 1) / 2
    Kp = (n + 15) // 16 * 16
    return segments * 28 * 2 * Kp * P


def alg_flops_fp64_formation(n, m, segments):
    """FP64-quality flops of V = sum v_j A_j (2nP per segment): what the
    digit-split tensor-core formation delivers."""
    return segments * 2 * n * m * (m + 1) / 2


def alg_flops_fp64_contraction(n, m, segments):
    """FP64-quality flops of w_j = u^T A_j u (2(n+1)P per normal)."""
    return segments * 2 * (n + 1) * m * (m + 1) / 2


# ALU peaks from the unit counts and the 2.07 GHz maximum SM clock of GB300
# (152 SMs): FP32 128 FFMA / clk / SM, FP64 2 DFMA / clk / SM; a dependent-FMA
# probe on this GPU measured 69.8 (FP32) and 1.19 (FP64) TFLOP/s.
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
PROBE_FP32_TFLOPS, PROBE_FP64_TFLOPS = 69.8, 1.19
# dram__bytes_read.sum + dram__bytes_write.sum per segment from one ncu
# capture of the current kernels (profiles/): walk_fp64_kernel on one step
# of 152 chains (149.90 + 137.19 MB); mixed_wave_kernel (816 KB per segment
# on one wave of 152 single-segment lines) has changed since its capture;
# None once a kernel changes until the next capture
WAVE_DRAM_BYTES_PER_SEGMENT = None  # changed since its capture (the correction's sum)
FP64_DRAM_BYTES_PER_SEGMENT = (149.895168e6 + 137.188608e6) / 152


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained",
                                                     d["bf16_tflops"])),
                "hbm_gbs": float(d.get("hbm_gbs", 6800.0)), "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
                "source": "fallback"}


# ----------------------------------------------------------------------------
# the walk on one path
# ----------------------------------------------------------------------------
def burn_in(spectra, torch, spec, C, rank, steps, tau, record=None):
    """Mixed Billiard steps from the start cloud (recording training tuples
    when `record` = (X, Y, counter)); returns the host state (x, step)."""
    chains = spectra.Chains(spec, C, x0=start_points(C, rank), seed=SEED_WALK,
                            chain0=replica_plan(rank, 1, C)["chain0"])
    if record is not None:
        chains.record(*record)
    for _ in range(steps):
        chains.billiard(1, tau=tau, rho=RHO, kappa=KAPPA, mode="mixed")
    if record is not None:
        chains.record()
    torch.cuda.synchronize()
    return chains.state_host()


WALK = "billiard"  # set from --walk


def walk(chains, steps, tau, mode):
    """`steps` steps of the bench's walk (Alg. 5 Billiard by default; Alg. 4
    Hit-and-Run or CDHR with --walk) on every chain."""
    if WALK == "billiard":
        chains.billiard(steps, tau=tau, rho=RHO, kappa=KAPPA, mode=mode)
    elif WALK == "hnr":
        chains.hnr(steps, mode=mode)
    else:
        chains.cdhr(steps, mode=mode)


def time_path(spectra, torch, spec, mode, C, rank, steps, warmup, tau, flush, state,
              stage_timers=False, record=0):
    """Warm-up steps, then the timed steps as one walk call.  record > 0:
    about that many of the timed walk's boundary-oracle calls are recorded
    (sp_record_segments, evenly sampled by arrival) for the oracle check."""
    chains = spectra.Chains(spec, C, x0=start_points(C, rank), seed=SEED_WALK,
                            chain0=replica_plan(rank, 1, C)["chain0"])
    chains.set_state(state[0], state[1])
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        walk(chains, 1, tau, mode)
    torch.cuda.synchronize()
    _, s0 = chains.status()
    warm_state = chains.state_host()
    seg = None
    if record > 0:
        # sampling stride from the warm-up's segments per step
        est = max(1, s0["segments"] * steps // max(1, warmup))
        every = max(1, est // record)
        buf = torch.zeros((2 * record, 3 * spec.n + 8), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        chains.record_segments(buf, cnt, every)
        seg = (buf, cnt, every)
    timers = None
    if stage_timers and mode != "fp64":
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        timers = torch.zeros((sms, 16), dtype=torch.int64, device="cuda")
        spec.set_stage_timers(timers)
    chains.kernel_timing(1)
    flush.zero_()  # cold L2 at the start of the timed region
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # the timed steps as one walk call: chains move on to their next step as
    # soon as they finish one (no step barrier); the per-chain state the
    # steps stream through (F and V, 2 x 8192 x 160 KB) is far larger than
    # the L2, so no flush is needed between steps
    ev0.record(stream)
    walk(chains, steps, tau, mode)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if seg is not None:
        chains.record_segments()
        seg = spectra.decode_segments(seg[0], int(seg[1].item()), seg[2], spec.n)
    evs = [(ev0, ev1)]
    kt = chains.kernel_timing(0)
    dev_ms = float(sum(a.elapsed_time(b) for a, b in evs))
    _, s1 = chains.status()
    stats = {k: s1[k] - s0[k] for k in s1}
    share = None
    if timers is not None:
        spec.set_stage_timers(None)
        tot = timers.sum(0).double()
        names = ["stage1_fill+fp32_cholesky", "stage1_fp32_lanczos", "stage2_fill+factorisation",
                 "stage2_iterations", "fp64_lanczos_fallback", "normal_contraction",
                 "bookkeeping"]
        stages = tot[:7]
        share = {nm: float(stages[i] / stages.sum()) for i, nm in enumerate(names)}
        share["cycles_per_segment"] = float(stages.sum()) / max(1, stats["segments"])
        lz = tot[8:12]
        if float(lz.sum()) > 0:
            share["lanczos_split"] = {nm: float(lz[i] / lz.sum()) for i, nm in
                                      enumerate(["apply", "reorth", "check", "final"])}
        s2 = tot[12:16]
        if float(s2.sum()) > 0:
            share["stage2_iteration_split"] = {
                nm: float(s2[i] / s2.sum()) for i, nm in
                enumerate(["solve_upper", "symv_V", "solve_lower", "reductions"])}
    return dict(chains=chains, dev_ms=dev_ms, wall=wall, stats=stats, kt=kt, share=share,
                steps=steps, warm_state=warm_state, segments=seg)


def oracle_check(A, seg, tol, dump=None):
    """t+ and the unit normal of the timed walk's own recorded boundary-oracle
    calls (sp_record_segments, sampled over the whole timed window) against
    the FP64 oracle on the same lines.  The normal is compared for segments
    that reflected, where the eigengap allows (relative gap > 1e-6)."""
    import oracle
    ok = seg["status"] == 0
    P, V = seg["p"][ok], seg["v"][ok]
    ref = oracle.reflect_batch(A, P, V)
    good = ref["status"] == 0
    et = np.abs(seg["t_plus"][ok][good] - ref["t_plus"][good]) / np.abs(ref["t_plus"][good])
    refl = seg["reflected"][ok][good] & (ref["rel_gap"][good] > 1e-6)
    ew = np.abs(seg["w_hat"][ok][good][refl] - ref["w_hat"][good][refl]).max(axis=1) \
        if refl.any() else np.zeros(0)
    out = {"samples": int(good.sum()), "reflected_samples": int(refl.sum()),
           "t_rel_err_max": float(et.max()) if len(et) else None,
           "t_rel_err_p99": float(np.quantile(et, 0.99)) if len(et) else None,
           "t_rel_err_median": float(np.median(et)) if len(et) else None,
           "normal_err_max": float(ew.max()) if len(ew) else None,
           "normal_err_p99": float(np.quantile(ew, 0.99)) if len(ew) else None,
           "oracle_failures": int((~good).sum()), "gpu_non_ok": int((~ok).sum()),
           "tolerance": tol}
    # chord walks: the other end of the chord too
    chord = np.isfinite(seg["t_minus"][ok])
    if chord.any():
        ri = oracle.intersect_batch(A, P[chord], V[chord])
        gm = ri["status"] == 0
        em = (np.abs(seg["t_minus"][ok][chord][gm] - ri["t_minus"][gm])
              / np.abs(ri["t_minus"][gm]))
        out["t_minus_rel_err_max"] = float(em.max()) if len(em) else None
        out["t_minus_rel_err_p99"] = float(np.quantile(em, 0.99)) if len(em) else None
    else:
        em = np.zeros(0)
    out["pass"] = bool(len(et) >= 256 and et.max() <= tol and
                       (len(ew) == 0 or ew.max() <= tol) and (len(em) == 0 or em.max() <= tol))
    if dump:
        # every checked call with its error and the solver-path flags, for
        # looking at the worst ones against the oracle
        np.savez(dump, p=P[good], v=V[good], t_gpu=seg["t_plus"][ok][good],
                 t_oracle=ref["t_plus"][good], err=et, flags=seg["flags"][ok][good],
                 chain=seg["chain"][ok][good], step=seg["step"][ok][good],
                 k=seg["k"][ok][good], rel_gap=ref["rel_gap"][good])
    return out


def train_network(spectra, torch, spec, X, Y, cnt, epochs, record_s, walk_steps):
    """Train the warm-start network on the GPU on the (x, v) -> (log t+, u)
    tuples that the mixed walk recorded on the same spectrahedron."""
    net = spectra.MLP(2 * N_DIM, 512, 1 + M_DIM, seed=SEED_TRAIN)
    spec.attach_mlp(net, x_scale=1.0 / TAU, t_scale=T_SCALE, margin=0.05, iters=12)
    got = min(int(cnt.item()), X.shape[0])
    t0 = t1 = time.perf_counter()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    perm = torch.randperm(got, device="cuda", generator=g)
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    nval = max(8, got // 16 // 8 * 8)
    ntr = (got - nval) // 1024 * 1024
    losses = net.train(X[nval:nval + ntr].contiguous(), Y[nval:nval + ntr].contiguous(),
                       epochs=epochs, batch=1024, lr=1e-3)
    t2 = time.perf_counter()
    Yp = net.forward(X[:nval].contiguous())
    lt_err = (Yp[:, 0] - Y[:nval, 0]).abs()
    # margin of the stage-1 shift sigma0 = (1 - margin) t^: below the true t+
    # for 90 % of the validation lines (a shift beyond t+ costs a failed
    # factorisation)
    ratio = torch.exp(Y[:nval, 0] - Yp[:, 0])  # t+ / t^
    margin = float(min(0.9, max(0.02, 1.0 - float(ratio.quantile(0.1)))))
    spec.attach_mlp(net, x_scale=1.0 / TAU, t_scale=T_SCALE, margin=margin, iters=12)
    cos = ((Yp[:, 1:] * Y[:nval, 1:]).sum(1).abs()
           / (Yp[:, 1:].norm(dim=1) * Y[:nval, 1:].norm(dim=1)))
    return net, {"tuples": got, "walk_steps": walk_steps, "record_s": record_s,
                 "train_s": t2 - t1, "epochs": epochs, "final_loss": float(losses[-1]),
                 "val_rel_err_t_median": float(torch.expm1(lt_err).median()),
                 "val_rel_err_t_p90": float(torch.expm1(lt_err).quantile(0.9)),
                 "val_cos_u_median": float(cos.median()), "shift_margin": margin}


def batch_workload():
    """The uneven batch: 64 spectrahedra ball block (r = 3) + random block
    with n, k = round(log-uniform[20, 200]) (seeded), 10,000 chains split in
    proportion to n (the remainder to the largest n)."""
    from paper_2010_03817_gb300 import workloads as W
    pairs = W.uneven_batch()
    bodies = [W.ball_random(n, k, 3.0, seed=W.BASE_SEED + 300 + i)
              for i, (n, k) in enumerate(pairs)]
    ns = np.array([n for n, _ in pairs], dtype=np.int64)
    chains = np.maximum(1, np.floor(10000 * ns / ns.sum())).astype(np.int64)
    chains[int(np.argmax(ns))] += 10000 - int(chains.sum())
    return pairs, bodies, chains.tolist()


def run_batch(args):
    """The uneven batch in one persistent launch (sp_batch_billiard, FP64
    path, autotuned Cholesky panel widths), against the same work as one
    launch per body; the oracle on a sample of the same bodies as the CPU
    baseline."""
    import tempfile

    import torch
    from paper_2010_03817_gb300 import build, spectra
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    pairs, bodies, chains = batch_workload()
    specs = [spectra.Spectrahedron(A, fp64_only=True) for A in bodies]
    b = spectra.Batch(specs, chains, seed=SEED_WALK)
    t0 = time.perf_counter()
    panels, ptimes = b.tune(os.path.join(tempfile.gettempdir(), "spectra_gb_panels.tsv"))
    tune_s = time.perf_counter() - t0
    tau = 6.0  # 2 r: every body lies in the ball block's ball of radius 3
    b.billiard(args.warmup, tau)
    torch.cuda.synchronize()
    s0 = b.stats()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ev0.record(stream)
        b.billiard(args.steps, tau)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    s1 = b.stats()
    segs = sum(s1[i]["segments"] - s0[i]["segments"] for i in range(len(bodies)))
    total = sum(chains)
    value = total * args.steps / (ms / 1e3)
    # the same steps as one launch per body, from the batch's state
    per_body_ms = 0.0
    for i, sp in enumerate(specs):
        n, m, c, c0 = b.dims(i)
        ch = spectra.Chains(sp, c, x0=b.state(i), seed=SEED_WALK, chain0=c0)
        ch.set_state(b.state(i), args.warmup + args.steps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ch.billiard(args.steps, tau=tau, rho=100, kappa=KAPPA)
        e1.record(stream)
        torch.cuda.synchronize()
        per_body_ms += e0.elapsed_time(e1)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pick = list(range(0, len(bodies), 4))  # 16 bodies, 2 chains each, 1 step
        t0 = time.perf_counter()
        osegs = 0
        for i in pick:
            n, m, c, c0 = b.dims(i)
            _, st = oracle.walk("billiard", bodies[i], b.state(i)[:2], 1, tau=tau, rho=100,
                                kappa=KAPPA, seed=SEED_WALK, step0=args.warmup, chain0=c0)
            osegs += st["segments"]
        dt = time.perf_counter() - t0
        cpu = {"value": 2 * len(pick) / dt, "unit": "chain-steps/s", "cores": oracle.num_threads(),
               "kind": "oracle", "segments_per_s": osegs / dt,
               "sample": "2 chains of each of 16 of the 64 bodies (every 4th), 1 burned-in step, "
                         "%.1f s" % dt}
    if rank == 0:
        ms_ = [pairs[i][0] + 1 + pairs[i][1] for i in range(len(pairs))]
        line = {
            "metric": "uneven batch billiard chain-steps/s (64 spectrahedra, one launch)",
            "value": value, "unit": "chain-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "64 spectrahedra, ball block r=3 + random block, n, k "
                                   "log-uniform in [20, 200] (m %d-%d), 10,000 chains split "
                                   "in proportion to n, Billiard walk, FP64 path, one "
                                   "persistent launch with autotuned Cholesky panels"
                                   % (min(ms_), max(ms_)),
                       "tau": tau, "rho": 100, "kappa": KAPPA},
            "oracle_calls_per_s": segs / (ms / 1e3),
            "per_body_launches": {"ms_per_step": per_body_ms / args.steps,
                                  "speedup_of_one_launch": per_body_ms / ms},
            "panels": {str(w): int((panels == w).sum()) for w in (4, 8, 16)},
            "tune_s": tune_s,
            "cpu_baseline": cpu,
            "gpu_launches": 1,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def hmc_workload():
    """HMC with reflections (Alg. 6) for exp(-c.x / T) on Dabbene S-60-60 (the
    largest S-n-m of the paper's annealing study, Table 4), c a seeded unit
    vector, T = 1."""
    from paper_2010_03817_gb300 import workloads as W
    A = W.dabbene(60, 60, seed=W.BASE_SEED + 400)
    g = np.random.default_rng(W.BASE_SEED + 401)
    c = g.normal(size=60)
    return A, c / np.linalg.norm(c), 1.0


def run_hmc(args):
    """HMC-r chain-steps/s on one GPU (sp_step_hmc, FP64 curve oracle), the
    oracle's HMC on a sample of the same chains as the CPU baseline."""
    import torch
    from paper_2010_03817_gb300 import build, spectra
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    A, c, T = hmc_workload()
    n, m = A.shape[0] - 1, A.shape[1]
    spec = spectra.Spectrahedron(A, fp64_only=True)
    # tau ~ diam(S): the longest chord through the origin over 256 directions
    from paper_2010_03817_gb300 import workloads as W
    D = torch.tensor(W.random_directions(n, 256, seed=W.BASE_SEED + 402), device="cuda")
    tm, tp, _, _ = spec.intersect(torch.zeros_like(D), D)
    tau = float((tp - tm).max().item())
    C = args.chains or 8192
    ch = spectra.Chains(spec, C, seed=SEED_WALK, chain0=rank * C)
    ch.hmc(args.warmup, c, T, tau, rho=100, kappa=KAPPA)
    torch.cuda.synchronize()
    X0, step0 = ch.state_host()
    _, s0 = ch.status()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        ch.hmc(args.steps, c, T, tau, rho=100, kappa=KAPPA)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    _, s1 = ch.status()
    segs = s1["segments"] - s0["segments"]
    value = C * args.steps / (ms / 1e3)
    P = m * (m + 1) / 2
    N = 2 * m
    # per segment: eigenvalues of the 2m companion matrix (Hessenberg + Francis
    # QR, 10 N^3), two Cholesky factorisations, the triangular solves that
    # build it (2 m^3), F(p), V, F(Phi(sigma)), F(Phi(t)) and the normal
    flops_seg = 10.0 * N ** 3 + 2 * m ** 3 / 3 + 2 * m ** 3 + 8 * n * P + 2 * (n + 1) * P
    achieved = flops_seg * segs / (ms / 1e3) / 1e12
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        from oracle import hmc as ohmc
        k, t0, osegs = 0, time.perf_counter(), 0
        while k < C and (k < 2 or time.perf_counter() - t0 < 20.0):
            x, st, refl = ohmc.hmc_step(A, X0[k], c, T, tau=tau, rho=100, kappa=KAPPA,
                                        seed=SEED_WALK, chain=k, step=step0)
            osegs += refl + 1
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": k / dt, "unit": "chain-steps/s", "cores": 1, "kind": "oracle",
               "segments_per_s": osegs / dt,
               "sample": "chains 0-%d of the warmed-up state, step %d (the GPU's first timed "
                         "step), oracle/hmc.py (numpy), %.1f s" % (k - 1, step0, dt)}
    if rank == 0:
        line = {
            "metric": "HMC-r Boltzmann chain-steps/s (S-60-60)",
            "value": value, "unit": "chain-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Dabbene S-60-60 (n=m=60), HMC with reflections for "
                                   "exp(-c.x/T), c a seeded unit vector, T=1, %d chains" % C,
                       "tau": tau, "rho": 100, "kappa": KAPPA,
                       "l2": "per-chain state 8 KB; inputs L2-resident (no flush)"},
            "oracle_calls_per_s": segs / (ms / 1e3),
            "segments_per_step": segs / (C * args.steps),
            "bad_steps": s1["bad_steps"] - s0["bad_steps"],
            "roofline": {"bound": "alu", "kernel": "curve_kernel", "launches": 1,
                         "achieved": achieved, "peak": PEAK_FP64_TFLOPS,
                         "unit": "TFLOP/s (FP64 pipe)", "frac": achieved / PEAK_FP64_TFLOPS,
                         "peak_source": "derived: 152 SMs x unit count x 2.07 GHz",
                         "algorithmic_flops_per_segment": flops_seg, "traffic": None},
            "cpu_baseline": cpu,
            "gpu_launches": 2,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_reference_sized(args):
    """The reference arm (the oracle on the host cores) of the uneven batch and
    of the HMC workload: the same bodies, chains, Philox draws and steps as
    the GPU line, on a bounded sample of the chains."""
    import oracle
    oracle.build()
    t_all = time.perf_counter()
    if args.workload == "batch":
        pairs, bodies, chains = batch_workload()
        chain0 = np.concatenate([[0], np.cumsum(chains)[:-1]]).astype(int)
        pick = list(range(0, len(bodies), 4))  # 16 of the 64 bodies, 2 chains each
        tau, steps, segs, dt = 6.0, max(1, args.steps), 0, 0.0
        for i in pick:
            X = np.zeros((2, pairs[i][0]))
            X, _ = oracle.walk("billiard", bodies[i], X, args.warmup, tau=tau, rho=100,
                               kappa=KAPPA, seed=SEED_WALK, step0=0, chain0=int(chain0[i]))
            t0 = time.perf_counter()
            _, st = oracle.walk("billiard", bodies[i], X, steps, tau=tau, rho=100, kappa=KAPPA,
                                seed=SEED_WALK, step0=args.warmup, chain0=int(chain0[i]))
            dt += time.perf_counter() - t0
            segs += st["segments"]
            if time.perf_counter() - t_all > 150.0:
                pick = pick[:pick.index(i) + 1]
                break
        value = 2 * len(pick) * steps / dt
        metric = "uneven batch billiard chain-steps/s (64 spectrahedra, one launch)"
        sample = ("2 chains of each of %d of the 64 bodies (every 4th), steps %d-%d, %.1f s"
                  % (len(pick), args.warmup, args.warmup + steps - 1, dt))
        cores = oracle.num_threads()
    else:
        from oracle import hmc as ohmc
        A, c, T = hmc_workload()
        n = A.shape[0] - 1
        # the GPU line's tau: the longest chord through the origin over the
        # same 256 directions, here from the oracle's own intersection
        from paper_2010_03817_gb300 import workloads as W
        D = W.random_directions(n, 256, seed=W.BASE_SEED + 402)
        r = oracle.intersect_batch(A, np.zeros_like(D), D)
        tau = float(np.max(r["t_plus"] - r["t_minus"]))
        k, segs, dt = 0, 0, 0.0
        while k < 2 or dt < 20.0:
            x = np.zeros(n)
            for j in range(args.warmup):
                x, _, _ = ohmc.hmc_step(A, x, c, T, tau=tau, rho=100, kappa=KAPPA,
                                        seed=SEED_WALK, chain=k, step=j)
            t0 = time.perf_counter()
            x, _, refl = ohmc.hmc_step(A, x, c, T, tau=tau, rho=100, kappa=KAPPA,
                                       seed=SEED_WALK, chain=k, step=args.warmup)
            dt += time.perf_counter() - t0
            segs += refl + 1
            k += 1
        value = k / dt
        metric = "HMC-r Boltzmann chain-steps/s (S-60-60)"
        sample = ("chains 0-%d, step %d (the GPU line's first timed step), oracle/hmc.py "
                  "(numpy), %.1f s" % (k - 1, args.warmup, dt))
        cores = 1
    line = {"impl": "reference", "metric": metric, "value": value, "unit": "chain-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload + " (oracle sample)"},
            "oracle_calls_per_s": segs / dt,
            "cpu_baseline": {"value": value, "unit": "chain-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample, "segments_per_s": segs / dt},
            "e2e": {"value": value, "unit": "chain-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    global WALK
    args = parse()
    if args.impl == "reference" and args.workload in ("batch", "hmc"):
        if int(os.environ.get("RANK", "0")) == 0:
            run_reference_sized(args)
        return
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "hmc":
        return run_hmc(args)
    if args.workload in ("ball10", "ball40", "cube40"):
        use_workload(args.workload)
    if args.chains is None:
        args.chains = CHAINS
    WALK = args.walk
    if WALK != "billiard" and args.mode == "learned":
        args.mode = "mixed"  # the warm start predicts Billiard segments only
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
    spectra.lib()
    A = workload()
    spec = spectra.Spectrahedron(A)
    if args.tol32 is not None or args.tol64 is not None or args.delta1 is not None:
        spec.set_mixed_solver(tol32=args.tol32 or 1e-4, tol64=args.tol64 or 1e-10,
                              delta1=args.delta1 or 2e-4)
    tau = TAU * args.tau_scale
    C = args.chains
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # burn-in (mixed walk from the start cloud; it records the training tuples
    # of the learned path), then the network's training on the GPU
    learned = args.mode == "learned" or not args.only
    record = None
    if learned:
        record = (torch.zeros((args.train_tuples, 2 * N_DIM), dtype=torch.float32, device="cuda"),
                  torch.zeros((args.train_tuples, 1 + M_DIM), dtype=torch.float32, device="cuda"),
                  torch.zeros(1, dtype=torch.int32, device="cuda"))
    if learned:
        # the recorded tuples carry the scales the network will be used with
        spec.attach_mlp(None, x_scale=1.0 / TAU, t_scale=T_SCALE)
    t0 = time.perf_counter()
    state = burn_in(spectra, torch, spec, C, rank, args.burn_in, tau, record)
    burn_s = time.perf_counter() - t0
    train_info = None
    if learned:
        _net, train_info = train_network(spectra, torch, spec, *record, args.train_epochs,
                                         burn_s, args.burn_in)

    # every path from the same state over the same step window: context paths
    # first, then the headline path under the clock sampler
    context = {}
    if not args.only:
        for mode in ["fp64", "mixed", "learned"]:
            if mode == args.mode or (mode == "learned" and WALK != "billiard"):
                continue
            context[mode] = time_path(spectra, torch, spec, mode, C, rank, args.steps,
                                      args.warmup, tau, flush, state,
                                      record=0 if args.no_check else args.check_samples)
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        head = time_path(spectra, torch, spec, args.mode, C, rank, args.steps, args.warmup, tau,
                         flush, state, stage_timers=args.stage_timers,
                         record=0 if args.no_check else args.check_samples)
    if world > 1:
        dist.barrier()
    times = [head["dev_ms"]]
    if world > 1:
        g = [torch.zeros(1, device="cuda") for _ in range(world)]
        dist.all_gather(g, torch.tensor([head["dev_ms"]], device="cuda"))
        times = [float(t.item()) for t in g]
    value, t_max = aggregate(times, world, C, args.steps)
    st = head["stats"]
    kt = head["kt"]

    # roofline of the dominant kernel of the headline path: the method's own
    # work (one factorisation and the eigen-solve iterations per segment, plus
    # formation and normal on the FP64 path) over its CUDA-event time, against
    # the ALU peak from the unit counts and the maximum clock
    P = M_DIM * (M_DIM + 1) / 2
    if args.mode == "fp64":
        flops = alg_flops_fp64(N_DIM, M_DIM, st, C * args.steps)
        ms = kt["fp64_ms"] or head["dev_ms"]
        roof = {"bound": "alu", "kernel": "walk_fp64_kernel",
                "launches": int(kt["fp64_launches"])}
        peak, probe, unit = PEAK_FP64_TFLOPS, PROBE_FP64_TFLOPS, "TFLOP/s (FP64 pipe)"
        dram = FP64_DRAM_BYTES_PER_SEGMENT
        overhead = 0.0
    else:
        flops = alg_flops_wave(N_DIM, M_DIM, st)
        ms = kt["wave_ms"] or head["dev_ms"]
        roof = {"bound": "alu", "kernel": "mixed_wave_kernel",
                "launches": int(kt["wave_launches"])}
        peak, probe, unit = PEAK_FP32_TFLOPS, PROBE_FP32_TFLOPS, "TFLOP/s (FP32 pipe)"
        dram = WAVE_DRAM_BYTES_PER_SEGMENT
        overhead = alg_overhead_wave(N_DIM, M_DIM, st)
    achieved = flops / (ms / 1e3) / 1e12
    launches = max(1, roof["launches"])
    roof.update({
        "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
        "peak_source": "derived: 152 SMs x unit count x 2.07 GHz", "peak_probe": probe,
        "frac_of_probe": achieved / probe,
        "traffic": (dram * st["segments"] / launches) if dram else None,
        "traffic_unit": "bytes per launch (DRAM read + write)",
        "algorithmic_flops_per_segment": flops / max(1, st["segments"]),
        "overhead_flops_per_segment": overhead / max(1, st["segments"]),
        "kernel_ms_per_step": ms / args.steps,
        "share_of_step": ms / max(1e-9, head["dev_ms"])})
    peaks = _peaks()
    formation = None
    if args.mode != "fp64" and kt["form_ms"] > 0:
        ff = alg_flops_formation(N_DIM, M_DIM, st["segments"])
        fa = ff / (kt["form_ms"] / 1e3) / 1e12
        f64 = alg_flops_fp64_formation(N_DIM, M_DIM, st["segments"]) / (kt["form_ms"] / 1e3) / 1e12
        formation = {"bound": "tensor", "kernel": "ozaki_form_kernel (+ digit slicing)",
                     "achieved": fa, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                     "frac": fa / peaks["bf16_tflops_sustained"],
                     "peak_source": peaks["source"] + " (bf16, sustained)",
                     "fp64_quality_tflops": f64, "fp64_quality_frac_of_fp64_peak":
                         f64 / PEAK_FP64_TFLOPS,
                     "share_of_step": kt["form_ms"] / max(1e-9, head["dev_ms"])}
    contraction = None
    if args.mode != "fp64" and kt.get("contract_ms", 0) > 0:
        cf = alg_flops_contraction(N_DIM, M_DIM, st["segments"])
        ca = cf / (kt["contract_ms"] / 1e3) / 1e12
        c64 = (alg_flops_fp64_contraction(N_DIM, M_DIM, st["reflections"])
               / (kt["contract_ms"] / 1e3) / 1e12)
        contraction = {"bound": "tensor", "kernel": "ozaki_kernel<contract> (+ digit slicing)",
                       "achieved": ca, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                       "frac": ca / peaks["bf16_tflops_sustained"],
                       "peak_source": peaks["source"] + " (bf16, sustained)",
                       "fp64_quality_tflops": c64,
                       "share_of_step": kt["contract_ms"] / max(1e-9, head["dev_ms"]),
                       "finish_share_of_step": kt["finish_ms"] / max(1e-9, head["dev_ms"])}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        chains = head["chains"]
        xh, step = chains.state_host()
        xh = np.ascontiguousarray(xh)
        out = np.empty_like(xh)
        k = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            chains.set_state(xh, step)
            walk(chains, 1, tau, args.mode)
            out, step = chains.state_host(out)
            xh, out = out, xh
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": C * k / e2e_s * world, "unit": "steps/s",
               "h2d_bytes_per_step": int(xh.nbytes), "d2h_bytes_per_step": int(xh.nbytes),
               "note": "set_state from host, one Billiard step, get_state to host"}

    checks = {}
    if rank == 0 and not args.no_check:
        try:
            import oracle
            oracle.build()
            for mode, r in list(context.items()) + [(args.mode, head)]:
                if r["segments"] is not None:
                    checks[mode] = oracle_check(
                        A, r["segments"], 1e-10 if mode == "fp64" else 1e-9,
                        dump=(args.dump_checked + "_" + mode + ".npz") if args.dump_checked
                        else None)

        except Exception as exc:
            checks = {"failed": str(exc)}
    parity_pass = bool(checks) and all(isinstance(c, dict) and c.get("pass") is not False
                                       for c in checks.values())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            wx, wstep = head["warm_state"]
            r = cpu_oracle_rate(A, tau, wx, wstep, chains=32, steps=2)
            cpu = {k: r[k] for k in ["value", "unit", "cores", "kind", "sample",
                                     "segments_per_s"]}
        except Exception as exc:  # the baseline must not sink the GPU number
            cpu = {"value": None, "unit": "steps/s", "cores": None, "kind": "oracle",
                   "sample": "failed: %s" % exc}

    def summary(r):
        s = r["stats"]
        segs = max(1, s["segments"])
        return {"steps_per_s": C * r["steps"] / (r["dev_ms"] / 1e3),
                "segments_per_s": s["segments"] / (r["dev_ms"] / 1e3),
                "ms_per_step": r["dev_ms"] / r["steps"],
                "segments_per_step": s["segments"] / (C * r["steps"]),
                "iters_per_segment": s["lanczos_iters"] / segs,
                "power_iters_per_segment": s["power_iters"] / segs,
                "fp64_fallback_rate": s["fp64_fallbacks"] / segs,
                "shift_retries_per_segment": s["shift_retries"] / segs,
                "warm_start_accept_rate": s["learned_ok"] / segs,
                "bad_steps": s["bad_steps"], "steps": r["steps"]}

    if rank == 0:
        paths = {m: summary(r) for m, r in context.items()}
        paths[args.mode] = summary(head)
        speedup = None
        if "fp64" in paths and args.mode != "fp64":
            speedup = paths[args.mode]["steps_per_s"] / paths["fp64"]["steps_per_s"]
        launches = int(kt["fp64_launches"] + kt["form_launches"] + kt["wave_launches"]
                       + kt["mlp_launches"] + kt["other_launches"] + kt["contract_launches"]
                       + kt["finish_launches"])
        line = {
            "metric": metric_name(WALK),
            "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.mode == "fp64" else "f64+f32+bf16",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("Billiard", {"billiard": "Billiard",
                                                                 "hnr": "Hit-and-Run",
                                                                 "cdhr": "CDHR"}[WALK]),
                       "n": N_DIM, "m": M_DIM, "chains_per_gpu": C,
                       "path": args.mode, "tau": tau, "rho": RHO, "kappa": KAPPA,
                       "l2": "inputs larger than L2 (per-chain F and V, 2.6 GB); flushed "
                             "once before the timed steps",
                       "parallelism": "replicas x%d" % world},
            "oracle_calls_per_s": st["segments"] * world / (t_max / 1e3),
            "parity_pass": parity_pass,
            "paths": paths,
            "speedup_vs_fp64": speedup,
            "oracle_check": checks,
            "training": train_info,
            "stage_share": head["share"],
            "roofline": roof,
            "roofline_formation": formation,
            "roofline_contraction": contraction,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "wall_s_timed": head["wall"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
