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
DRAM_BYTES_PER_ITERATION = {"fx": (1.192853248e9 + 1.631790848e9) / 76, "c64": None, "f64": None}

# ncu L2 (lts__t_bytes) bytes per Lanczos iteration of the element-wise fixed-point
# kernel (2-step capture: 76 iterations, see profiles/); None where not measured
LTS_BYTES_PER_ITERATION = {"fx": 31846678688 / 76, "c64": None, "f64": None}

# final-state error: horizon, and the reference run (CF8:11 at REF_DT, REF_TOL)
ERR_T = 1.0
REF_DT = 0.0025
REF_TOL = 1e-13

# L2 copy probe: two buffers of this size (together far below the 129 MB L2)
L2_PROBE_BYTES = 16 << 20
L2_PROBE_REPS = 2000

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


# ---------------------------------------------------------------- oracle on the host cores
# Worker processes (started with "spawn": the parent has already touched the
# GPU) each build the problem once and run the oracle's Lanczos exponential on
# it; the parent adds their H applications and divides by the wall time.
_ORACLE = {}


def _oracle_init():
    from oracle import cfet as OC, operators as O, schemes as OS
    pr, psi0 = problem()
    _ORACLE["op"] = O.SpinChain(N_SITES, pr.J, pr.Delta, pr.h, [pr.xfield])
    _ORACLE["psi0"] = psi0
    _ORACLE["drive"] = pr.drive
    _ORACLE["OC"], _ORACLE["OS"] = OC, OS


def _oracle_task(args):
    """One bounded sample: the first stage exponential (exp(Omega_s)) of the
    CF6:5Opt step at t = step * DT, either adaptive (tol, m_max of the bench)
    or with a fixed Krylov dimension k_fixed; returns the H applications."""
    from oracle import krylov as OK
    step, k_fixed = args
    OC, OS, op = _ORACLE["OC"], _ORACLE["OS"], _ORACLE["op"]
    c = OC.stage_coefficients(OS.get(SCHEME), step * DT, DT, [_ORACLE["drive"]])[-1]
    tol, m = (0.0, k_fixed) if k_fixed else (TOL, M_MAX)
    _, _, na = OK.expv(lambda v: op.apply(c, v), _ORACLE["psi0"], DT, tol, m)
    return na


class OraclePool:
    """The oracle, as it stands, on `workers` host processes (one thread each)."""

    def __init__(self, workers):
        import importlib
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        # fail here, not in the workers: a pool whose initializer raises keeps
        # replacing its workers and never returns
        importlib.import_module("oracle.cfet")
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init)

    def run(self, step, k_fixed=0):
        t = time.perf_counter()
        na = sum(self.pool.map(_oracle_task, [(step, k_fixed)] * self.workers, chunksize=1))
        return na, time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def host_desc():
    return f"{platform.machine()}, {os.cpu_count()} cores"


def cpu_baseline_sample():
    """The oracle on a bounded sample of the same workload: the first stage
    exponential of CF6:5Opt on the N=20 chain with a fixed Krylov dimension of
    6 (6 H applications), once on one core and once on every host core at the
    same time (one process per core, each doing the same sample)."""
    k = 6
    one = OraclePool(1)
    one.run(0, k)                        # warm: imports, problem set-up
    na1, el1 = one.run(0, k)
    one.close()
    P = os.cpu_count() or 1
    allc = OraclePool(P)
    allc.run(0, 2)
    naP, elP = allc.run(0, k)
    allc.close()
    return {"value": naP / elP, "unit": UNIT, "cores": P, "kind": "oracle",
            "single_core_value": na1 / el1,
            "sample": f"oracle expv, first stage exponential of {SCHEME} on the N={N_SITES} chain, fixed Krylov "
                      f"dimension {k} ({k} H applies per process): {P} processes with one numpy thread each, "
                      f"{elP:.1f} s; alone on one core {el1:.1f} s ({host_desc()})"}


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
    """The reference arm: the oracle on every host core.  Each step is one
    bounded sample per core: the first stage exponential of the CF6:5Opt step
    at t = step * dt with a fixed Krylov dimension of 2 (two H applications on
    the full 2^20 vector; an adaptive exponential takes ~7 and would make the
    run last many minutes)."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    P = os.cpu_count() or 1
    pool = OraclePool(P)
    k_fixed = 2
    for w in range(args.warmup):
        pool.run(w, k_fixed)
    na_tot, el = 0, 0.0
    for k in range(args.steps):
        na, t = pool.run(args.warmup + k, k_fixed)
        na_tot += na
        el += t
    pool.close()
    value = na_tot / el
    sample = (f"each step: on each of {P} processes (one numpy thread each) the oracle's Krylov exponential "
              f"of the first stage of a {SCHEME} step of the N={N_SITES} chain with fixed dimension {k_fixed} "
              f"({k_fixed} H applies per process); {host_desc()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- device measurements
def make_chain(P, pr, N, precision, m_max=M_MAX, **kw):
    return P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [pr.drive], m_max=m_max,
                        max_substeps=64, precision=precision, **kw)


def final_state_error(P, torch, pr, psi0, N, precision, T, order, dt, tol, ref_state=None):
    """||psi - psi_ref||_2 after time T from psi0 for (order, dt, tol) against
    the FP64-class reference CF8:11, dt = REF_DT, tol REF_TOL, m <= 24 (computed
    once and passed back in ref_state)."""
    if ref_state is None:
        ref = torch.from_numpy(psi0).cuda()
        rp = make_chain(P, pr, N, "fx", m_max=24)
        rp.propagate(ref, 0.0, REF_DT, int(round(T / REF_DT)), order=8, tol=REF_TOL)
        rp.close()
        ref_state = ref
    x = torch.from_numpy(psi0).cuda()
    p = make_chain(P, pr, N, precision)
    p.propagate(x, 0.0, dt, int(round(T / dt)), order=order, tol=tol)
    p.close()
    return torch.linalg.vector_norm(x - ref_state).item(), ref_state


def timed_reps(prop, psi, t0, K, barrier, min_ms, reps=None):
    """Propagations of exactly K steps, each between barriers and CUDA events
    on the launching stream, repeated until at least min_ms have been timed
    (or `reps` times): [(ms, kernel_ms, stats)], t0 after them."""
    import torch
    stream = torch.cuda.current_stream()
    out = []
    total = 0.0
    while (reps is None and (total < min_ms or len(out) < 3)) or (reps is not None and len(out) < reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        st = prop.propagate(psi, t0, DT, K, order=ORDER, tol=TOL)
        ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1)
        out.append((ms, prop.kernel_time_ms(), st))
        total += ms
        t0 += K * DT
    return out, t0


def roofline_of(precision, reps, dim, hbm_peak, per_launch_div):
    """Roofline object of the persistent kernel from the median rep."""
    elem = 8.0 if precision == "c64" else 16.0
    ach_gbs, ach_tf, bytes_l, kms_l = [], [], [], []
    for ms, kms, st in reps:
        b, f = algorithmic_counts(st, dim, elem_bytes=elem)
        ach_gbs.append(b / (kms * 1e-3) / 1e9)
        ach_tf.append(f / (kms * 1e-3) / 1e12)
        bytes_l.append(b / per_launch_div)
        kms_l.append(kms)
    gbs, tf = statistics.median(ach_gbs), statistics.median(ach_tf)
    n_app_med = statistics.median([st["n_applies"] for _, _, st in reps])
    if precision in ("fx", "c64"):
        per_it = DRAM_BYTES_PER_ITERATION[precision]
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": per_it * n_app_med / per_launch_div if per_it is not None else None,
                "traffic_note": "per launch: ncu DRAM read+write bytes per Lanczos iteration (2-step capture) x "
                                "the launch's iterations (median rep); algorithmic bytes per launch: %.4g"
                                % statistics.median(bytes_l),
                "kernel": "k_propagate_fx (persistent Lanczos, int64 fixed-point vectors)" if precision == "fx"
                else "k_propagate_c64 (persistent Lanczos, complex64 vectors, FP64-class reductions)",
                "kernel_ms": statistics.median(kms_l), "launches": per_launch_div,
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst figure",
                "fp64_equivalent_tflops": tf}
    return {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": tf / FP64_PEAK_TFLOPS, "traffic": None,
            "kernel": "k_propagate (persistent Lanczos, FP64)", "kernel_ms": statistics.median(kms_l),
            "launches": per_launch_div, "hbm_algorithmic_gbs": gbs, "hbm_peak_gbs": hbm_peak,
            "hbm_frac": gbs / hbm_peak,
            "peak_note": "FP64 peak from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}


def l2_roofline(P, torch, precision, roof):
    """L2 view of the N = 20 kernel (its vector and most of its basis are
    L2-resident): the L2-served copy rate measured here as the peak, the
    kernel's ncu L2 traffic (lts bytes) and its algorithmic bytes per second."""
    nb = L2_PROBE_BYTES
    a = torch.empty(nb // 16, dtype=torch.complex128, device="cuda")
    b = torch.empty_like(a)
    a.zero_()
    peak = max(P.probe_copy_gbs(a, b, reps=L2_PROBE_REPS) for _ in range(3))
    del a, b
    out = {"unit": "GB/s", "peak": peak,
           "peak_note": f"cfet_probe_copy_gbs: {L2_PROBE_REPS} alternating copies between two "
                        f"{nb >> 20} MiB buffers in one launch (read + write bytes), best of 3, measured in this run",
           "achieved_algorithmic": roof["achieved"] if roof["unit"] == "GB/s" else roof["hbm_algorithmic_gbs"]}
    out["frac_algorithmic"] = out["achieved_algorithmic"] / peak
    per_it = LTS_BYTES_PER_ITERATION.get(precision)
    if per_it is not None and roof.get("kernel_ms"):
        n_it = roof["_n_app"]
        out["traffic"] = per_it * n_it
        out["achieved"] = per_it * n_it / (roof["kernel_ms"] * 1e-3) / 1e9
        out["frac"] = out["achieved"] / peak
        out["traffic_note"] = "ncu lts__t_bytes per Lanczos iteration (2-step capture) x the launch's iterations"
    else:
        out["traffic"] = out["achieved"] = out["frac"] = None
    return out


def small_chain_line(P, torch):
    """The N = 8 chain (dim 256): Neel state, CF4:2, dt 0.01, T 10 (1000 steps),
    tol 1e-12, m <= 16; CFET steps/s of one 1000-step propagation and its
    final-state error against CF8:11 at dt 0.0025, tol 1e-14."""
    cfg = W.CHAIN_SMALL
    N = cfg["N"]
    pr = W.spin_chain(N)
    psi0 = W.neel_state(N)
    n = int(round(cfg["T"] / cfg["dt"]))
    prop = make_chain(P, pr, N, "fx", m_max=cfg["m_max"])
    x = torch.from_numpy(psi0).cuda()
    prop.propagate(x, 0.0, cfg["dt"], 10, order=cfg["order"], tol=cfg["tol"])   # warm-up
    x = torch.from_numpy(psi0).cuda()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    st = prop.propagate(x, 0.0, cfg["dt"], n, order=cfg["order"], tol=cfg["tol"])
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    kms = prop.kernel_time_ms()
    prop.close()
    ref = torch.from_numpy(psi0).cuda()
    rp = make_chain(P, pr, N, "fx", m_max=24)
    rp.propagate(ref, 0.0, 0.0025, int(round(cfg["T"] / 0.0025)), order=8, tol=1e-14)
    rp.close()
    return {"workload": f"driven XXZ chain N={N} (dim {1 << N}), Neel state, CF4:2 dt={cfg['dt']}, T={cfg['T']}, "
                        f"tol {cfg['tol']}, m_max {cfg['m_max']}", "precision": "fx",
            "cfet_steps_per_s": n / (ms * 1e-3), "H_applies_per_s": st["n_applies"] / (ms * 1e-3),
            "us_per_apply": 1e3 * kms / st["n_applies"], "ms": ms, "kernel_ms": kms, "H_applies": st["n_applies"],
            "final_state_error": torch.linalg.vector_norm(x - ref).item(),
            "reference": "CF8:11, dt 0.0025, tol 1e-14, m_max 24 (fixed point)",
            "grid": None if not st.get("phase_ns") else "see phase_Mcycles",
            "phase_Mcycles": {k: v * 1e-6 for k, v in zip(PHASES, st.get("phase_ns", [0] * 8))}}


def grid_atom_line(P, torch):
    """The grid atom (Nr 2000, l < 100, dim 200 000, CF8:11, dt 0.1, m <= 64,
    tol 1e-10) for one step from t = 500 (pulse maximum), starting from the
    discrete 1s state: H applies/s, substeps per stage exponential and the
    projected time of the full T = 1000 pulse."""
    a = W.ATOM
    p = W.grid_atom(Nr=a["Nr"], L=a["L"], dr=a["dr"], E0=a["E0"], omega=a["omega"], Tp=a["Tp"])
    psi0, _ = W.atom_ground_state(p)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                        m_max=a["m_max"], max_substeps=4000)
    x = torch.from_numpy(psi0).cuda()
    prop.apply(np.array([1.0, 0.0]), x, torch.empty_like(x))   # context, tables
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    st = prop.propagate(x, 500.0, a["dt"], 1, order=a["order"], tol=a["tol"])
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    kms = prop.kernel_time_ms()
    prop.close()
    nfull = int(round(a["Tp"] / a["dt"]))
    return {"workload": "grid atom Nr=2000 dr=0.1 l<100 (dim 200000), E0=0.05, omega=0.057, Tp=1000, CF8:11 dt=0.1, "
                        "m_max 64, tol 1e-10, one step from t=500, 1s state", "precision": "fx",
            "H_applies_per_s": st["n_applies"] / (ms * 1e-3), "ms_per_step": ms, "kernel_ms": kms,
            "H_applies": st["n_applies"], "substeps_per_exponential": st["n_substeps"] / max(1, st["n_exp"]),
            "max_k": st["max_k"], "norm_drift": abs(torch.linalg.vector_norm(x).item() - 1.0),
            "full_pulse_projected_h": ms * 1e-3 * nfull / 3600.0}


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
    # the host-core oracle runs first, before this process touches the GPU
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()
    pr, psi0 = problem()
    dim = 1 << N_SITES
    cheb = args.expm == "chebyshev"
    prop = make_chain(P, pr, N_SITES, args.precision, block_size=args.block_size, grid_size=args.grid_size,
                      expm=args.expm, apply_form=args.apply_form)
    psi = torch.from_numpy(psi0).cuda()
    t0 = 0.0
    # warm-up steps (untimed)
    prop.propagate(psi, t0, DT, args.warmup, order=ORDER, tol=TOL)
    t0 += args.warmup * DT

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # the number of timed repetitions of the K-step call: enough for
    # args.min_timed_ms on the slowest rank, the same on every rank
    cal, t0 = timed_reps(prop, psi, t0, args.steps, barrier, 0.0, reps=1)
    cal_ms, _ = aggregate_over_ranks(cal[0][0], 0.0)
    nrep = max(3, int(math.ceil(args.min_timed_ms / max(cal_ms, 1e-3))))
    with ClockSampler(local) as clk:
        reps, t0 = timed_reps(prop, psi, t0, args.steps, barrier, 0.0, reps=nrep)
    clocks = clk.summary()
    per_rep = [aggregate_over_ranks(ms, st["n_applies"]) for ms, _, st in reps]
    values = [u / (m * 1e-3) for m, u in per_rep]
    value = statistics.median(values)
    ms_med = statistics.median([m for m, _ in per_rep])
    launches = math.ceil(args.steps / 256)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if cheb:
        kms = statistics.median([k for _, k, _ in reps])
        n_app = statistics.median([st["n_applies"] for _, _, st in reps])
        n_exp = reps[0][2]["n_exp"]
        # per element and term: read v_k, v_{k-1}, the sum; write v_{k+1}, the sum (80 B); the first
        # term of an exponential reads v_0 and writes v_1 and the sum (48 B), the last writes v_0 only (64 B)
        bytes_ = dim * (80.0 * n_app - 48.0 * n_exp)
        gbs = bytes_ / (kms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "traffic": DRAM_BYTES_PER_TERM_CHEB * n_app / launches,
                    "traffic_note": "per launch: ncu DRAM read+write bytes per Chebyshev term (2-step capture) x "
                                    "the launch's terms; algorithmic bytes per launch: %.4g" % (bytes_ / launches),
                    "kernel": "k_cheb_fx (persistent Chebyshev recurrence, int64 fixed-point vectors)",
                    "kernel_ms": kms, "launches": launches,
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst figure"}
    else:
        roofline = roofline_of(args.precision, reps, dim, hbm_peak, launches)

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
    prop.close()

    if rank == 0:
        st_all = [st for _, _, st in reps]
        med = sorted(range(len(reps)), key=lambda i: values[i])[len(reps) // 2]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_med / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fx": "i64", "c64": "f32", "f64": "f64"}[args.precision],
            "data": "synthetic", "config": dict(workload_config(), precision=args.precision, expm=args.expm,
                                                apply_form=args.apply_form),
            "timed_repeats": len(reps),
            "timing_note": f"the {args.steps}-step call timed {len(reps)} times back to back (CUDA events, "
                           f"barrier and synchronize around each); value and ms_per_step are the medians",
            "cfet_steps_per_s": args.steps * ws / (ms_med * 1e-3),
            "krylov": {"applies_per_step": statistics.median([s["n_applies"] for s in st_all]) / args.steps,
                       "substeps": st_all[med]["n_substeps"], "max_k": max(s["max_k"] for s in st_all),
                       "max_err_est": max(s["max_err_est"] for s in st_all),
                       # SM clock cycles per CTA of the median rep (mean, max over CTAs), in millions
                       "phase_Mcycles": {k: v * 1e-6 for k, v in zip(PHASES, st_all[med].get("phase_ns", [0] * 8))},
                       "phase_max_Mcycles": {k: v * 1e-6 for k, v in zip(PHASES,
                                                                           st_all[med].get("phase_max_ns", [0] * 8))}},
            "roofline": roofline,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 16 * dim, "d2h_bytes_per_step": 16 * dim,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if not args.quick:
            # accuracy of the benchmarked setting, outside the timed region
            err, ref_state = final_state_error(P, torch, pr, psi0, N_SITES, args.precision, ERR_T, ORDER, DT, TOL)
            line["final_state_error"] = {
                "value": err, "T": ERR_T, "steps": int(round(ERR_T / DT)),
                "reference": f"CF8:11, dt {REF_DT}, tol {REF_TOL}, m_max 24 (fixed point), same psi0",
                "note": "||psi - psi_ref||_2 of the benchmarked scheme, dt, tolerance and precision from t = 0"}
            if not cheb and args.precision != "f64":
                # the complex128 (FP64) form of the same workload, as a secondary arm
                fp = make_chain(P, pr, N_SITES, "f64")
                x = torch.from_numpy(psi0).cuda()
                fp.propagate(x, 0.0, DT, args.warmup, order=ORDER, tol=TOL)
                r64, _ = timed_reps(fp, x, args.warmup * DT, args.steps, torch.cuda.synchronize,
                                    args.min_timed_ms / 4)
                roof64 = roofline_of("f64", r64, dim, hbm_peak, launches)
                fp.close()
                e64, _ = final_state_error(P, torch, pr, psi0, N_SITES, "f64", ERR_T, ORDER, DT, TOL, ref_state)
                line["f64_arm"] = {
                    "value": statistics.median([st["n_applies"] / (ms * 1e-3) for ms, _, st in r64]),
                    "unit": UNIT, "cfet_steps_per_s": args.steps / (statistics.median([m for m, _, _ in r64]) * 1e-3),
                    "ms_per_step": statistics.median([m for m, _, _ in r64]) / args.steps, "timed_repeats": len(r64),
                    "dtype": "f64", "roofline": roof64, "final_state_error": e64}
            roof = dict(roofline, _n_app=statistics.median([s["n_applies"] for s in st_all]) / launches)
            if not cheb:
                line["l2_roofline"] = l2_roofline(P, torch, args.precision, roof)
            line["small_chain"] = small_chain_line(P, torch)
            line["grid_atom"] = grid_atom_line(P, torch)
            del ref_state
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
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
    ap.add_argument("--apply-form", default="auto", choices=["auto", "elementwise", "tiled"],
                    help="XXZ-chain apply form of the fixed-point and complex64 kernels")
    ap.add_argument("--min-timed-ms", type=float, default=2000.0,
                    help="the K-step call is repeated until at least this much has been timed (median reported)")
    ap.add_argument("--quick", action="store_true",
                    help="headline figures only (no final-state error, FP64 arm, L2 probe, N=8 or atom line)")
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
