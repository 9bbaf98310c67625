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


def run_sweep(args):
    """Accuracy study behind "at fixed final-state error": the N=20 chain over
    T = 20 with orders 4, 6, 8 (default schemes) and dt in {0.05, 0.02, 0.01},
    each compared with a reference run (CF8:11, dt = 0.0025, tol 1e-13, m <= 24)
    by ||psi - psi_ref||_2.  Prints one JSON line per run and a summary line."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    pr, psi0 = problem()
    T = args.sweep_T

    def make(m_max, precision):
        return P.Propagator(P.XXZChain(N_SITES, pr.J, pr.Delta, pr.h), [P.XField(N_SITES, pr.xfield)],
                            [pr.drive], m_max=m_max, max_substeps=64, precision=precision)

    ref_prop = make(24, "fx")   # the reference is always an FP64-class run
    ref = torch.from_numpy(psi0).cuda()
    dt_ref = 0.0025
    n_ref = int(round(T / dt_ref))
    t = time.perf_counter()
    st_ref = ref_prop.propagate(ref, 0.0, dt_ref, n_ref, order=8, tol=1e-13)
    ref_s = time.perf_counter() - t
    ref_prop.close()
    rows = []
    prop = make(M_MAX, args.precision)
    for order in (4, 6, 8):
        for dt in (0.05, 0.02, 0.01):
            n = int(round(T / dt))
            psi = torch.from_numpy(psi0).cuda()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            st = prop.propagate(psi, 0.0, dt, n, order=order, tol=TOL)
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            err = torch.linalg.vector_norm(psi - ref).item()
            row = {"order": order, "dt": dt, "steps": n, "final_state_error": err,
                   "H_applies": st["n_applies"], "H_applies_per_s": st["n_applies"] / (ms * 1e-3),
                   "cfet_steps_per_s": n / (ms * 1e-3), "time_s": ms * 1e-3,
                   "norm_drift": abs(torch.linalg.vector_norm(psi).item() - 1.0)}
            rows.append(row)
            print(json.dumps(row))
    prop.close()
    summary = {"sweep": "driven XXZ chain N=20, T=%g, tol %g, m_max %d, precision %s" % (T, TOL, M_MAX, args.precision),
               "reference": {"scheme": "CF8:11", "dt": dt_ref, "tol": 1e-13, "m_max": 24,
                             "H_applies": st_ref["n_applies"], "time_s": ref_s},
               "cheapest_for_error": {}}
    for target in (1e-4, 1e-6, 1e-8):
        ok = [r for r in rows if r["final_state_error"] <= target]
        if ok:
            best = min(ok, key=lambda r: r["time_s"])
            summary["cheapest_for_error"][f"{target:g}"] = {k: best[k] for k in ("order", "dt", "time_s",
                                                                                 "final_state_error")}
    print(json.dumps(summary))
    return 0


def _roofline_study_line(prop, stats, ms, dim, bytes_per_app, elem, label, extra):
    """bytes_per_app: algorithmic bytes per element of one Lanczos iteration;
    elem: bytes per vector element (reconstruction reads k vectors, writes 1)."""
    n_app, n_sub = stats["n_applies"], stats["n_substeps"]
    kernel_ms = prop.kernel_time_ms()
    bytes_ = dim * (bytes_per_app * n_app + elem * (n_app + n_sub))
    line = {"study": label, "H_applies": n_app, "substeps": n_sub, "exponentials": stats["n_exp"],
            "substeps_per_exponential": n_sub / max(1, stats["n_exp"]), "max_k": stats["max_k"],
            "H_applies_per_s": n_app / (ms * 1e-3), "ms": ms, "kernel_ms": kernel_ms,
            "algorithmic_GBps": bytes_ / (kernel_ms * 1e-3) / 1e9,
            "phase_Mcycles": {k: v * 1e-6 for k, v in zip(PHASES, stats.get("phase_ns", [0] * 8))}}
    line.update(extra)
    print(json.dumps(line))


def run_study_atom(args):
    """The grid atom (Nr = 2000, l < 100, dim 200 000, CF8:11, dt = 0.1, m <= 64,
    tol 1e-10) for --steps steps from t0 = 500 (peak of the pulse envelope),
    starting from the discrete 1s state: H applies/s, substeps per stage
    exponential and the projected cost of the full T = 1000 pulse."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    a = W.ATOM
    p = W.grid_atom(Nr=a["Nr"], L=a["L"], dr=a["dr"], E0=a["E0"], omega=a["omega"], Tp=a["Tp"])
    psi0, e0 = W.atom_ground_state(p)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                        m_max=a["m_max"], max_substeps=4000, precision=args.precision, grid_size=args.grid_size)
    psi = torch.from_numpy(psi0).cuda()
    t0 = 500.0
    # warm-up: one apply (context, tables and graph set-up); a full atom step
    # takes seconds, so the timed steps are not preceded by one
    prop.apply(np.array([1.0, 0.0]), psi, torch.empty_like(psi))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    st = prop.propagate(psi, t0, a["dt"], args.steps, order=a["order"], tol=a["tol"])
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    nfull = int(round(a["Tp"] / a["dt"]))
    # per element and iteration: q_k, q_{k-1} read, u written + 5 real diagonals
    elem, val = (8.0, 4.0) if args.precision == "c64" else (16.0, 8.0)
    _roofline_study_line(prop, st, ms, p.dim, 3 * elem + 5 * val, elem, "grid atom Nr=2000 L=100 CF8:11 dt=0.1 m<=64 tol 1e-10",
                         {"steps": args.steps, "t0": t0, "precision": args.precision,
                          "norm_drift": abs(torch.linalg.vector_norm(psi).item() - 1.0),
                          "full_pulse_steps": nfull,
                          "full_pulse_projected_s": ms * 1e-3 / args.steps * nfull})
    prop.close()
    return 0


def run_study_sizes(args):
    """The driven chain of the bench at N = 20, 22, 24, 26 (vectors 16 MiB to
    1 GiB, the larger ones far beyond L2): H applies/s and algorithmic HBM
    GB/s of the persistent kernel for --steps CFET steps each."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    for n in (20, 22, 24, 26):
        pr = W.spin_chain(n)
        prop = P.Propagator(P.XXZChain(n, pr.J, pr.Delta, pr.h), [P.XField(n, pr.xfield)], [pr.drive],
                            m_max=M_MAX, max_substeps=64, precision=args.precision)
        psi = torch.from_numpy(W.random_state(PSI_SEED, 1 << n)).cuda()
        prop.propagate(psi, 0.0, DT, 1, order=ORDER, tol=TOL)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = prop.propagate(psi, DT, DT, args.steps, order=ORDER, tol=TOL)
        ev1.record()
        torch.cuda.synchronize()
        elem = 8.0 if args.precision == "c64" else 16.0
        _roofline_study_line(prop, st, ev0.elapsed_time(ev1), 1 << n, 3 * elem, elem,
                             f"driven XXZ chain N={n} {SCHEME} dt={DT} tol {TOL}",
                             {"N": n, "steps": args.steps, "precision": args.precision})
        prop.close()
        del psi
        torch.cuda.empty_cache()
    return 0


def run_study_batch(args):
    """256 driven XXZ chains with N uniform in {10..16} (dims 1024..65536),
    per-instance fields, A ~ U[0.5, 2], omega ~ U[1, 3], CF6:5Opt, dt = 0.02,
    --steps steps (500 = T 10), tol 1e-10: the batched launch in FP64 and
    complex64 after the autotuner picked each plan, against the single-instance
    FP64 propagator run instance by instance (timed over --baseline-steps steps
    and scaled per step).  Final-state error of the complex64 batch is stated
    against the FP64 batch."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    cfg = W.BATCH
    insts = W.chain_batch(cfg["n"], cfg["n_lo"], cfg["n_hi"])
    chains = [P.Chain(c.N, c.J, c.Delta, c.h, c.xfield, None, c.A, c.omega, 0.0) for c in insts]
    host = [W.random_state(c.psi_seed, 1 << c.N) for c in insts]
    dims = np.array([1 << c.N for c in insts], dtype=np.float64)
    order, dt, tol, nsteps = cfg["order"], cfg["dt"], cfg["tol"], args.steps
    out = {}
    finals = {}
    for prec in ("f64", "c64"):
        bp = P.BatchPropagator(chains, m_max=cfg["m_max"], precision=prec)
        t = time.perf_counter()
        plan = bp.tune(0.0, dt, order=order, tol=tol, nsteps=1)
        tune_s = time.perf_counter() - t
        dev = [torch.from_numpy(h).cuda() for h in host]
        bp.propagate(dev, 0.0, dt, 1, order=order, tol=tol)        # warm-up step
        dev = [torch.from_numpy(h).cuda() for h in host]
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = bp.propagate(dev, 0.0, dt, nsteps, order=order, tol=tol)
        wall = time.perf_counter() - t
        kms = bp.kernel_time_ms()
        n_app = np.array([x["n_applies"] for x in st], dtype=np.float64)
        finals[prec] = [d.cpu().numpy() for d in dev]
        out[prec] = {"plan": plan, "tune_s": tune_s, "kernel_ms": kms, "wall_s": wall,
                     "H_applies": float(n_app.sum()), "H_applies_per_s": float(n_app.sum()) / (kms * 1e-3),
                     "element_applies_per_s": float((n_app * dims).sum()) / (kms * 1e-3),
                     "cfet_steps_per_s": nsteps * len(insts) / (kms * 1e-3),
                     "max_k": max(x["max_k"] for x in st)}
        bp.close()
        del dev
    err = max(np.linalg.norm(a - b) for a, b in zip(finals["c64"], finals["f64"]))
    out["c64"]["final_state_error_vs_f64_batch_max"] = float(err)
    # single-instance FP64 propagator, instance by instance
    nb = args.baseline_steps
    tot_ms, tot_app = 0.0, 0.0
    for c, h in zip(insts, host):
        prop = P.Propagator(P.XXZChain(c.N, c.J, c.Delta, c.h), [P.XField(c.N, c.xfield)], [c.drive],
                            m_max=cfg["m_max"], precision="f64")
        x = torch.from_numpy(h).cuda()
        prop.propagate(x, 0.0, dt, 1, order=order, tol=tol)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        s2 = prop.propagate(x, dt, dt, nb, order=order, tol=tol)
        ev1.record()
        torch.cuda.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        tot_app += s2["n_applies"]
        prop.close()
    single_ms_per_step = tot_ms / nb
    out["single_instance_f64"] = {"ms_per_batch_step": single_ms_per_step, "steps_timed": nb,
                                  "H_applies_per_s": tot_app / (tot_ms * 1e-3)}
    for prec in ("f64", "c64"):
        out[prec]["speedup_vs_single_instance_f64"] = single_ms_per_step * nsteps / out[prec]["kernel_ms"]
    print(json.dumps({"study": "batch: %d driven XXZ chains N=%d..%d, CF6:5Opt dt=%g, %d steps, tol %g, m<=%d"
                      % (len(insts), cfg["n_lo"], cfg["n_hi"], dt, nsteps, tol, cfg["m_max"]),
                      "sum_dims": float(dims.sum()), **out}))
    return 0


def run_study_adjoint(args):
    """Gradient of the fidelity loss for the N=18 chain (dim 2^18), 64
    piecewise-constant amplitude segments ~ U[-1, 1] over T = 16, CF4:2,
    dt = 0.01, drive A_k cos(2 t) sum_i X_i, tol 1e-10: the adjoint sweep
    (forward with checkpoints every 25 steps + FP64 backward) against the
    gradient by central differences with the plain FP64 propagator
    (2 x 64 forward runs, timed on one and scaled)."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    N, nseg, T, dt, omega, tol = 18, 64, 16.0, 0.01, 2.0, 1e-10
    nsteps = int(round(T / dt))
    pr = W.spin_chain(N)
    psi0 = torch.from_numpy(W.random_state(3, 1 << N)).cuda()
    phi = torch.from_numpy(W.random_state(13, 1 << N)).cuda()
    amps = W.uniform(7, nseg, -1.0, 1.0)
    out = {}
    for prec in ("fx", "f64"):
        prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, np.ones(N))], [lambda t: 0.0],
                            m_max=16, precision=prec)
        prop.fidelity_grad(psi0, phi, 0.0, dt, 50, amps[:2], omega, tol=tol, checkpoint_every=25)   # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        L, g, st = prop.fidelity_grad(psi0, phi, 0.0, dt, nsteps, amps, omega, tol=tol, checkpoint_every=25)
        wall = time.perf_counter() - t
        out["adjoint_forward_" + prec] = {"loss": L, "wall_s": wall, **st, "grad_norm": float(np.linalg.norm(g))}
        prop.close()
    # one plain FP64 forward propagation (a central-difference gradient needs 2 x 64 of them)
    sps = nsteps // nseg

    def f(t):   # the same piecewise-constant drive, segment of the step containing t
        return amps[min(int(math.floor(t / dt)) // sps, nseg - 1)] * math.cos(omega * t)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, np.ones(N))], [f], m_max=16,
                        precision="f64")
    x = psi0.clone()
    prop.propagate(x, 0.0, dt, 10, order=4, tol=tol)
    x = psi0.clone()
    torch.cuda.synchronize()
    t = time.perf_counter()
    prop.propagate(x, 0.0, dt, nsteps, order=4, tol=tol)
    torch.cuda.synchronize()
    fwd_s = time.perf_counter() - t
    prop.close()
    out["f64_forward_s"] = fwd_s
    out["central_difference_gradient_s"] = 2 * nseg * fwd_s
    for prec in ("fx", "f64"):
        out["adjoint_forward_" + prec]["speedup_vs_central_differences_f64"] = (
            2 * nseg * fwd_s / out["adjoint_forward_" + prec]["wall_s"])
    print(json.dumps({"study": "fidelity gradient: N=18 chain, 64 segments, T=16, CF4:2 dt=0.01, tol 1e-10",
                      **out}))
    return 0


def run_study_expm(args):
    """Krylov (Sec. 8.1, the default) against the Chebyshev technique (Sec. 8.1/8.2)
    for the stage exponentials, both in the fixed-point format at the same
    tolerance: the N=20 chain over T = --sweep-T with CF6:5Opt at dt in
    {0.05, 0.02, 0.01}, each run compared with a reference (CF8:11, dt 0.0025,
    tol 1e-13, Krylov) by ||psi - psi_ref||_2 (Chebyshev also at tolerances
    1e-12 and 1e-14); then the grid atom (CF8:11,
    dt 0.1, from t = 500) for --steps steps with both methods.  One JSON line
    per run.  Chebyshev algorithmic bytes per element and term: read v_k,
    v_{k-1} and the partial sum, write v_{k+1} and the partial sum (80 B)."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    pr, psi0 = problem()
    T = args.sweep_T

    def chain(expm, m_max=M_MAX):
        return P.Propagator(P.XXZChain(N_SITES, pr.J, pr.Delta, pr.h), [P.XField(N_SITES, pr.xfield)],
                            [pr.drive], m_max=m_max, max_substeps=64, expm=expm)

    def timed(prop, psi, *a, **kw):
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = prop.propagate(psi, *a, **kw)
        ev1.record()
        torch.cuda.synchronize()
        return st, ev0.elapsed_time(ev1)

    ref_prop = chain("krylov", 24)
    ref = torch.from_numpy(psi0).cuda()
    ref_prop.propagate(ref, 0.0, 0.0025, int(round(T / 0.0025)), order=8, tol=1e-13)
    ref_prop.close()
    dim = 1 << N_SITES
    # the Chebyshev tail bound is nearly attained and its stage errors add up,
    # while the Krylov estimate is pessimistic: Chebyshev runs at three tolerances
    for expm, tols in (("krylov", (TOL,)), ("chebyshev", (TOL, 1e-12, 1e-14))):
        prop = chain(expm)
        for dt, tol in [(dt, tol) for dt in (0.05, 0.02, 0.01) for tol in tols]:
            n = int(round(T / dt))
            psi = torch.from_numpy(psi0).cuda()
            prop.propagate(psi, 0.0, dt, 2, order=6, tol=tol)        # warm-up (graph, tables)
            psi = torch.from_numpy(psi0).cuda()
            st, ms = timed(prop, psi, 0.0, dt, n, order=6, tol=tol)
            kms = prop.kernel_time_ms()
            row = {"study": "expm", "workload": "driven XXZ chain N=20 CF6:5Opt T=%g tol %g" % (T, tol),
                   "expm": expm, "dt": dt, "steps": n, "H_applies": st["n_applies"],
                   "applies_per_exponential": st["n_applies"] / st["n_exp"], "max_k": st["max_k"],
                   "H_applies_per_s": st["n_applies"] / (ms * 1e-3), "cfet_steps_per_s": n / (ms * 1e-3),
                   "time_s": ms * 1e-3, "final_state_error": torch.linalg.vector_norm(psi - ref).item()}
            if expm == "chebyshev":
                row["algorithmic_GBps"] = dim * 80.0 * st["n_applies"] / (kms * 1e-3) / 1e9
            print(json.dumps(row))
        prop.close()
    a = W.ATOM
    p = W.grid_atom(Nr=a["Nr"], L=a["L"], dr=a["dr"], E0=a["E0"], omega=a["omega"], Tp=a["Tp"])
    psi0a, _ = W.atom_ground_state(p)
    outs = {}
    for expm in ("krylov", "chebyshev"):
        prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                            m_max=a["m_max"], max_substeps=4000, expm=expm)
        psi = torch.from_numpy(psi0a).cuda()
        prop.apply(np.array([1.0, 0.0]), psi, torch.empty_like(psi))
        st, ms = timed(prop, psi, 500.0, a["dt"], args.steps, order=a["order"], tol=a["tol"])
        outs[expm] = psi
        print(json.dumps({"study": "expm", "workload": "grid atom Nr=2000 L=100 CF8:11 dt=0.1 tol %g from t=500"
                          % a["tol"], "expm": expm, "steps": args.steps, "H_applies": st["n_applies"],
                          "applies_per_exponential": st["n_applies"] / st["n_exp"], "max_k": st["max_k"],
                          "H_applies_per_s": st["n_applies"] / (ms * 1e-3), "time_s": ms * 1e-3,
                          "ms_per_step": ms / args.steps}))
        prop.close()
    print(json.dumps({"study": "expm", "atom_krylov_vs_chebyshev_difference":
                      torch.linalg.vector_norm(outs["krylov"] - outs["chebyshev"]).item()}))
    return 0


def run_study_timestep(args):
    """Time-step selection (Sec. 6.6) on the N=20 chain over T = --sweep-T,
    order 4 (CF4:2), Krylov tol 1e-12: (a) cfet_select_dt with c probed over
    T/10 for goals 1e-6, 1e-8, 1e-10, then the run with the selected step,
    its error against a reference (CF8:11, dt T/1600, tol 1e-13) and the cost
    including the probe; (b) a chirped drive 0.8 cos(0.5 t + 0.15 t^2):
    cfet_propagate_adaptive for goal 1e-8 against a uniform grid with as many
    steps as the adaptive run took (trial steps included)."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    pr, psi0 = problem()
    T = args.sweep_T

    def chain(drive):
        return P.Propagator(P.XXZChain(N_SITES, pr.J, pr.Delta, pr.h), [P.XField(N_SITES, pr.xfield)], [drive],
                            m_max=M_MAX, max_substeps=64)

    def reference(prop):
        ref = torch.from_numpy(psi0).cuda()
        prop.propagate(ref, 0.0, T / 1600, 1600, order=8, tol=1e-13)
        return ref

    prop = chain(pr.drive)
    ref = reference(prop)
    for target in (1e-6, 1e-8, 1e-10):
        x = torch.from_numpy(psi0).cuda()
        torch.cuda.synchronize()
        t = time.perf_counter()
        dt, n, c = prop.select_dt(x, 0.0, T, target, T / 10, 8, order=4, tol=1e-12)
        tp = time.perf_counter() - t
        st = prop.propagate(x, 0.0, dt, n, order=4, tol=1e-12)
        torch.cuda.synchronize()
        tt = time.perf_counter() - t
        print(json.dumps({"study": "timestep", "workload": "driven XXZ chain N=20 CF4:2 T=%g" % T, "goal": target,
                          "c": c, "dt": dt, "steps": n, "final_state_error": torch.linalg.vector_norm(x - ref).item(),
                          "probe_s": tp, "total_s": tt, "H_applies": st["n_applies"]}))
    prop.close()

    def chirp(t):
        return 0.8 * math.cos(0.5 * t + 0.15 * t * t)

    prop = chain(chirp)
    ref = reference(prop)
    x = torch.from_numpy(psi0).cuda()
    torch.cuda.synchronize()
    t = time.perf_counter()
    hs, trials, st = prop.propagate_adaptive(x, 0.0, T, 1e-8, 0.05, 1e-4, 1.0, order=4, tol=1e-12)
    torch.cuda.synchronize()
    ta = time.perf_counter() - t
    err_a = torch.linalg.vector_norm(x - ref).item()
    n_uni = 3 * trials        # every trial costs one step of h and two of h/2
    y = torch.from_numpy(psi0).cuda()
    prop.propagate(y, 0.0, T / n_uni, n_uni, order=4, tol=1e-12)
    err_u = torch.linalg.vector_norm(y - ref).item()
    print(json.dumps({"study": "timestep", "workload": "driven XXZ chain N=20, chirped drive, CF4:2 T=%g" % T,
                      "goal": 1e-8, "accepted_steps": len(hs), "trial_steps": trials,
                      "h_first_last": [hs[0], hs[len(hs) // 2], hs[-1]], "adaptive_error": err_a, "adaptive_s": ta,
                      "uniform_steps_same_cost": n_uni, "uniform_error": err_u}))
    prop.close()
    return 0


def run_study_pauli(args):
    """The N=20 driven chain through the general Pauli-sum kernel (97 strings:
    XX, YY, ZZ per bond, Z and X per site) against the FP64 chain kernel,
    CF6:5Opt, dt 0.02, tol 1e-10, m <= 16, --steps steps: H applies/s of each
    and the difference of their final states."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    N = N_SITES
    pr = W.spin_chain(N)
    terms = []
    for i in range(N - 1):
        terms += [(pr.J, {i: "X", i + 1: "X"}), (pr.J, {i: "Y", i + 1: "Y"}), (pr.J * pr.Delta, {i: "Z", i + 1: "Z"})]
    terms += [(float(pr.h[i]), {i: "Z"}) for i in range(N)]
    forms = {
        "chain kernel (FP64)": lambda: P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)],
                                                    [pr.drive], m_max=M_MAX, precision="f64"),
        "Pauli-sum kernel (FP64)": lambda: P.Propagator(P.PauliSum(N, terms),
                                                        [P.PauliSum(N, [(float(pr.xfield[i]), {i: "X"})
                                                                        for i in range(N)])],
                                                        [pr.drive], m_max=M_MAX),
    }
    outs = []
    for name, make in forms.items():
        prop = make()
        psi = torch.from_numpy(W.random_state(PSI_SEED, 1 << N)).cuda()
        prop.propagate(psi, 0.0, DT, 1, order=ORDER, tol=TOL)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = prop.propagate(psi, DT, DT, args.steps, order=ORDER, tol=TOL)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        outs.append(psi)
        print(json.dumps({"study": "pauli", "workload": f"driven XXZ chain N={N} {SCHEME} dt={DT} tol {TOL}",
                          "form": name, "steps": args.steps, "H_applies": st["n_applies"], "ms": ms,
                          "H_applies_per_s": st["n_applies"] / ms * 1e3}))
        prop.close()
    print(json.dumps({"study": "pauli", "final_state_difference": torch.linalg.vector_norm(outs[0] - outs[1]).item()}))
    return 0


def run_study_reorth(args):
    """Cost of full re-orthogonalisation: the N=20 chain in FP64 (CF6:5Opt,
    dt 0.02, tol 1e-10, m <= 16) with the plain three-term recurrence and with
    one classical Gram-Schmidt sweep per Lanczos vector, --steps steps: H
    applies/s of each and the difference of their final states."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    pr = W.spin_chain(N_SITES)
    outs = []
    for reorth in (False, True):
        prop = P.Propagator(P.XXZChain(N_SITES, pr.J, pr.Delta, pr.h), [P.XField(N_SITES, pr.xfield)], [pr.drive],
                            m_max=M_MAX, precision="f64", reorth=reorth)
        psi = torch.from_numpy(W.random_state(PSI_SEED, 1 << N_SITES)).cuda()
        prop.propagate(psi, 0.0, DT, 1, order=ORDER, tol=TOL)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = prop.propagate(psi, DT, DT, args.steps, order=ORDER, tol=TOL)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        outs.append(psi)
        print(json.dumps({"study": "reorth", "workload": f"driven XXZ chain N={N_SITES} {SCHEME} dt={DT} tol {TOL}",
                          "reorth": reorth, "steps": args.steps, "H_applies": st["n_applies"], "ms": ms,
                          "H_applies_per_s": st["n_applies"] / ms * 1e3}))
        prop.close()
    print(json.dumps({"study": "reorth", "final_state_difference": torch.linalg.vector_norm(outs[0] - outs[1]).item()}))
    return 0


def run_study_picture(args):
    """Interaction against Schroedinger picture (Secs. 9.3, 9.4), FP64 Krylov,
    N=20 chain, CF6:5Opt, tol 1e-10, m <= 16, over T = --sweep-T: the default
    chain (|h_i| <= 1, J Delta = 0.5) and one with a strong diagonal (h_i in
    [-8, 8], Delta = 4): Krylov applies per exponential, time, and the error of
    each against a fine Schroedinger-picture reference (fixed point, CF8:11,
    dt T/400, tol 1e-13)."""
    import torch
    import paper_1102_5071_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    T = args.sweep_T
    psi0 = W.random_state(PSI_SEED, 1 << N_SITES)
    for label, h_scale, Delta in (("default chain", 1.0, 0.5), ("strong diagonal", 8.0, 4.0)):
        pr = W.spin_chain(N_SITES, Delta=Delta)
        h = pr.h * h_scale

        def make(picture, m_max=M_MAX, precision="f64"):
            return P.Propagator(P.XXZChain(N_SITES, pr.J, Delta, h), [P.XField(N_SITES, pr.xfield)], [pr.drive],
                                m_max=m_max, max_substeps=200, precision=precision, picture=picture)

        ref_p = make("schroedinger", 30, "fx")
        ref = torch.from_numpy(psi0).cuda()
        ref_p.propagate(ref, 0.0, T / 400, 400, order=8, tol=1e-13)
        ref_p.close()
        for picture in ("schroedinger", "interaction"):
            prop = make(picture)
            for dt in (0.02, 0.005):
                n = int(round(T / dt))
                x = torch.from_numpy(psi0).cuda()
                torch.cuda.synchronize()
                t = time.perf_counter()
                st = prop.propagate(x, 0.0, dt, n, order=6, tol=TOL)
                torch.cuda.synchronize()
                el = time.perf_counter() - t
                print(json.dumps({"study": "picture", "workload": "N=20 chain, %s, CF6:5Opt T=%g" % (label, T),
                                  "picture": picture, "dt": dt, "steps": n,
                                  "applies_per_exponential": st["n_applies"] / st["n_exp"],
                                  "substeps_per_exponential": st["n_substeps"] / st["n_exp"],
                                  "time_s": el, "final_state_error": torch.linalg.vector_norm(x - ref).item()}))
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
    ap.add_argument("--sweep", action="store_true",
                    help="accuracy study: final-state error and throughput per (order, dt) over T")
    ap.add_argument("--sweep-T", type=float, default=20.0)
    ap.add_argument("--study", choices=["atom", "sizes", "batch", "adjoint", "expm", "timestep", "picture", "pauli",
                                        "reorth"],
                    help="extra measurements: the grid atom, the chain at N = 20..26, the 256-chain batch, "
                         "the fidelity gradient, Krylov against Chebyshev stage exponentials, time-step selection, "
                         "interaction against Schroedinger picture")
    ap.add_argument("--baseline-steps", type=int, default=10,
                    help="batch study: steps of the single-instance baseline per instance")
    ap.add_argument("--grid-size", type=int, default=0,
                    help="CTAs of the persistent kernel (0 = co-resident maximum)")
    ap.add_argument("--block-size", type=int, default=0,
                    help="threads per CTA of the FP64 kernel; the fixed-point kernel uses 2x this many workers + 1 control warp")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.study == "atom":
        return run_study_atom(args)
    if args.study == "sizes":
        return run_study_sizes(args)
    if args.study == "batch":
        return run_study_batch(args)
    if args.study == "adjoint":
        return run_study_adjoint(args)
    if args.study == "expm":
        return run_study_expm(args)
    if args.study == "timestep":
        return run_study_timestep(args)
    if args.study == "picture":
        return run_study_picture(args)
    if args.study == "pauli":
        return run_study_pauli(args)
    if args.study == "reorth":
        return run_study_reorth(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
