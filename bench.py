"""Throughput benchmark of the GB300 CFET/Krylov propagator.

Workload: the driven XXZ chain with N = 20 sites (dim 2^20, complex128),
J = 1, Delta = 0.5, h_i ~ U[-1, 1] (seed 1), drive 1.0 cos(2 t) sum_i X_i,
random normalised complex Gaussian psi0 (seed 2), CFET order 6 (CF6:5Opt),
dt = 0.02, Krylov tolerance 1e-10, m <= 16.  One bench step = one CFET time
step (5 stage exponentials, each a full device Lanczos loop with adaptive
Krylov dimension, error estimate and reconstruction).

Metric: Hamiltonian applications per second (= Lanczos iterations per second,
the paper's unit of effort), also reported as CFET steps per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank propagates
its own replica (the path does not shard: replicas only); value is the total
over ranks divided by the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_SITES = 20
ORDER = 6
SCHEME = "CF6:5Opt"
DT = 0.02
TOL = 1e-10
M_MAX = 16
PSI_SEED = 2
METRIC = "Hamiltonian applies/sec and CFET steps/sec at fixed final-state error; HBM GB/s vs peak"
UNIT = "H_applies/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock


# DRAM bytes (read + write) per Lanczos iteration of the persistent kernel,
# from one ncu capture of the same kernel build on the 2-step case (76
# iterations): see profiles/.  Must be reset to None whenever the kernel
# changes and re-measured.
DRAM_BYTES_PER_ITERATION = {"fx": (1.207240448e9 + 1.633021184e9) / 76, "c64": (191.0784e6 + 649.152256e6) / 76,
                            "f64": None}

# ncu DRAM read+write bytes per term of the Chebyshev kernel (2-step capture: 66 terms)
DRAM_BYTES_PER_TERM_CHEB = (17.067008e6 + 21.68192e6) / 66

# trace slots of the control-warp kernels (cfet_stats.phase_ns)
PHASES = ("apply_loops", "apply_control", "orth_loops", "orth_control", "reconstruct_loops", "barrier_wait",
          "overlapped_control", "worker_wait")


def workload_config():
    return {
        "workload": f"driven XXZ chain N={N_SITES} (dim 2^{N_SITES}), {SCHEME} dt={DT}, Krylov tol={TOL}, "
                    f"m_max={M_MAX}, random complex Gaussian psi0 (seed {PSI_SEED})",
        "model": "driven XXZ spin chain (matrix-free Pauli apply)",
        "hilbert_dim": 1 << N_SITES,
        "scheme": SCHEME,
        "order": ORDER,
        "dt": DT,
        "krylov_tol": TOL,
        "m_max": M_MAX,
        "l2": "inputs larger than L2: Krylov basis (m_max vectors x 16 MiB) + psi exceed the 129 MB L2",
        "parallelism": "replicas",
    }


def problem():
    pr = W.spin_chain(N_SITES)
    psi0 = W.random_state(PSI_SEED, 1 << N_SITES)
    return pr, psi0


def algorithmic_counts(stats, dim, N=N_SITES, elem_bytes=16.0):
    """Algorithmic bytes and FP64 flops of the persistent kernel for the
    Lanczos iterations and reconstructions reported in stats.

    bytes: 48 B per element per Lanczos iteration (read v_k, v_{k-1}, write
      v_{k+1}) + 16 B per element per basis vector read in the reconstruction
      + 16 B per element for the reconstructed psi: 16 dim (4 n_app + n_sub)
      (8 B instead of 16 B per vector element for complex64 vectors).
    flops: per element and iteration 5N+7 for the spin apply (diagonal 4,
      (N-1)/2 complex hop additions on average, 2 complex FMA for the hop
      scale, N complex FMA for the transverse field) + 16 for the three-term
      recurrence and the two reductions; per reconstruction 8k + 4.
    """
    n_app, n_sub = stats["n_applies"], stats["n_substeps"]
    bytes_ = elem_bytes * dim * (4 * n_app + n_sub)
    flops = dim * ((5 * N + 7 + 16 + 8) * n_app + 4 * n_sub)
    return bytes_, flops


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def cpu_baseline_sample():
    """The oracle, as it stands, on a bounded sample of the same workload: one
    stage exponential of the first CF6:5Opt step with a fixed Krylov dimension
    of 6 (6 H applications on the 2^20 chain)."""
    from oracle import cfet as OC, krylov as OK, operators as O, schemes as OS
    pr, psi0 = problem()
    op = O.SpinChain(N_SITES, pr.J, pr.Delta, pr.h, [pr.xfield])
    c = OC.stage_coefficients(OS.get(SCHEME), 0.0, DT, [pr.drive])[-1]
    k = 6
    t = time.perf_counter()
    _, log, na = OK.expv(lambda v: op.apply(c, v), psi0, DT, 0.0, k)
    el = time.perf_counter() - t
    return {"value": na / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle expv, first stage exponential of {SCHEME} on the N={N_SITES} chain, "
                      f"fixed Krylov dimension {k} ({na} H applies, {el:.1f} s, numpy single thread, "
                      f"{platform.machine()} {os.cpu_count()} cores)"}


def aggregate_over_ranks(ms, units, device="cuda"):
    """Whole-job figures of a replicated run: (slowest rank's time in ms, sum of
    the units over ranks).  With one process it returns its own numbers; under
    torch.distributed every rank contributes (any backend: nccl on the GPU,
    gloo in the host tests)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    from oracle import cfet as OC, krylov as OK, operators as O, schemes as OS
    pr, psi0 = problem()
    op = O.SpinChain(N_SITES, pr.J, pr.Delta, pr.h, [pr.xfield])
    c = OC.stage_coefficients(OS.get(SCHEME), 0.0, DT, [pr.drive])[-1]
    k = 2   # bounded sample per step: two Lanczos iterations on the full vector
    psi = psi0
    for _ in range(args.warmup):
        psi, _, _ = OK.expv(lambda v: op.apply(c, v), psi, DT, 0.0, k)
    t = time.perf_counter()
    na_tot = 0
    for _ in range(args.steps):
        psi, _, na = OK.expv(lambda v: op.apply(c, v), psi, DT, 0.0, k)
        na_tot += na
    el = time.perf_counter() - t
    value = na_tot / el
    sample = (f"each step: oracle expv with fixed Krylov dimension {k} on the N={N_SITES} chain "
              f"({k} H applies), numpy single thread, {platform.machine()} {os.cpu_count()} cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1102_5071_gb300 as P
    P.build()
    pr, psi0 = problem()
    dim = 1 << N_SITES
    cheb = args.expm == "chebyshev"
    prop = P.Propagator(P.XXZChain(N_SITES, pr.J, pr.Delta, pr.h), [P.XField(N_SITES, pr.xfield)], [pr.drive],
                        m_max=M_MAX, max_substeps=64, precision=args.precision, block_size=args.block_size,
                        grid_size=args.grid_size, expm=args.expm)
    psi = torch.from_numpy(psi0).cuda()
    t0 = 0.0
    # warm-up steps (untimed)
    st = prop.propagate(psi, t0, DT, args.warmup, order=ORDER, tol=TOL)
    t0 += args.warmup * DT

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        stats = prop.propagate(psi, t0, DT, args.steps, order=ORDER, tol=TOL)
        ev1.record(stream)
        barrier()
    t0 += args.steps * DT
    ms = ev0.elapsed_time(ev1)
    kernel_ms = prop.kernel_time_ms()
    clocks = clk.summary()
    n_app = stats["n_applies"]
    ms_max, app_total = aggregate_over_ranks(ms, n_app)
    value = app_total / (ms_max * 1e-3)

    # roofline of the persistent kernel (one launch per 256 steps)
    bytes_, flops = algorithmic_counts(stats, dim, elem_bytes=8.0 if args.precision == "c64" else 16.0)
    if cheb:
        # per element and term: read v_k, v_{k-1}, the sum; write v_{k+1}, the sum (80 B); the first
        # term of an exponential reads v_0 and writes v_1 and the sum (48 B), the last writes v_0 only (64 B)
        bytes_ = dim * (80.0 * n_app - 48.0 * stats["n_exp"])
    achieved_tflops = flops / (kernel_ms * 1e-3) / 1e12
    achieved_gbs = bytes_ / (kernel_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    # end-to-end through the host-buffer entry point: each step uploads psi
    # from pinned host memory, runs one CFET step, downloads psi
    host = torch.empty(dim, dtype=torch.complex128, pin_memory=True)
    host.copy_(psi.cpu())
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps, 10))
    if e2e_steps:
        prop.propagate_host(host, t0, DT, 1, order=ORDER, tol=TOL)   # warm the staging buffer
        t0 += DT
    barrier()
    te = time.perf_counter()
    e2e_app = 0
    for _ in range(e2e_steps):
        s2 = prop.propagate_host(host, t0, DT, 1, order=ORDER, tol=TOL)
        e2e_app += s2["n_applies"]
        t0 += DT
    barrier()
    e2e_s = time.perf_counter() - te
    e2e_val = e2e_app / e2e_s if e2e_steps else None
    if ws > 1 and e2e_steps:
        s_max, app_all = aggregate_over_ranks(e2e_s, e2e_app)
        e2e_val = app_all / s_max

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    if cheb:
        per_t = DRAM_BYTES_PER_TERM_CHEB
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak,
                    "traffic": per_t * n_app / math.ceil(args.steps / 256) if per_t is not None else None,
                    "traffic_note": "per launch: ncu DRAM read+write bytes per Chebyshev term (2-step capture) x "
                                    "the launch's terms; algorithmic bytes per launch: %.4g"
                                    % (bytes_ / math.ceil(args.steps / 256)),
                    "kernel": "k_cheb_fx (persistent Chebyshev recurrence, int64 fixed-point vectors)",
                    "kernel_ms": kernel_ms, "launches": math.ceil(args.steps / 256),
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst figure"}
    elif args.precision in ("fx", "c64"):
        per_it = DRAM_BYTES_PER_ITERATION[args.precision]
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak,
                    "traffic": per_it * n_app / math.ceil(args.steps / 256) if per_it is not None else None,
                    "traffic_note": "per launch: ncu DRAM read+write bytes per Lanczos iteration (2-step "
                                    "capture) x the launch's iterations; algorithmic bytes per launch: %.4g"
                                    % (bytes_ / math.ceil(args.steps / 256)),
                    "kernel": "k_propagate_fx (persistent Lanczos, int64 fixed-point vectors)"
                    if args.precision == "fx" else
                    "k_propagate_c64 (persistent Lanczos, complex64 vectors, FP64-class reductions)",
                    "kernel_ms": kernel_ms, "launches": math.ceil(args.steps / 256),
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst figure",
                    "fp64_equivalent_tflops": achieved_tflops}
    else:
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                    "kernel": "k_propagate (persistent Lanczos, FP64)", "kernel_ms": kernel_ms,
                    "launches": math.ceil(args.steps / 256),
                    "hbm_algorithmic_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak,
                    "hbm_frac": achieved_gbs / hbm_peak,
                    "peak_note": "FP64 peak from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fx": "i64", "c64": "f32", "f64": "f64"}[args.precision],
            "data": "synthetic", "config": dict(workload_config(), precision=args.precision, expm=args.expm),
            "cfet_steps_per_s": args.steps * ws / (ms_max * 1e-3),
            "krylov": {"applies_per_step": n_app / args.steps, "substeps": stats["n_substeps"],
                       "max_k": stats["max_k"], "max_err_est": stats["max_err_est"],
                       # SM clock cycles per CTA (mean, max over CTAs), in millions
                       "phase_Mcycles": {k: v * 1e-6 for k, v in zip(PHASES, stats.get("phase_ns", [0] * 8))},
                       "phase_max_Mcycles": {k: v * 1e-6 for k, v in zip(PHASES,
                                                                           stats.get("phase_max_ns", [0] * 8))}},
            "roofline": roofline,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 16 * dim, "d2h_bytes_per_step": 16 * dim,
                    "steps": e2e_steps},
            "gpu_launches": math.ceil(args.steps / 256),
            "clocks": clocks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    prop.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--precision", default="fx", choices=["fx", "f64", "c64"],
                    help="Krylov vector format: int64 fixed point (default), FP64, or complex64 (mixed precision)")
    ap.add_argument("--expm", default="krylov", choices=["krylov", "chebyshev"],
                    help="stage exponentials: Krylov (default) or the Chebyshev expansion (fixed point only)")
    ap.add_argument("--grid-size", type=int, default=0,
                    help="CTAs of the persistent kernel (0 = co-resident maximum)")
    ap.add_argument("--block-size", type=int, default=0,
                    help="threads per CTA of the FP64 kernel; the fixed-point kernel uses 2x this many workers + 1 control warp")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
