#!/usr/bin/env python
"""Benchmark of the RMHMC hot path on GB300.

Workload (32^4 full RMHMC): periodic 32^4 lattice, Wilson beta = 6.0, 12-pole mass term with
kappa = 0.9, tau = 1 with 20 implicit-leapfrog steps, kinetic + gauge forces, Metropolis in float64,
mixed precision (float32 Krylov, float64 link update, reductions and Hamiltonian).  One step = one
trajectory followed by the per-mode power spectrum of the new configuration's Wilson and Iwasaki
gauge forces (degree-200 Chebyshev filters over 64 windows, 16 noise vectors, one batched launch per
recurrence step).  Links: seeded random start exp(i 0.3 sum r_a T_a), thermalised by plain HMC before
timing.  Every input is synthetic; the working set (~30 GB) exceeds the 129 MB L2, so no flush is
needed between steps.

Besides the timed steps the line carries: the roofline of the CG stencil (CUDA events around its
launches in the host-driven solves; DRAM traffic from an ncu capture of the same launch shape), the
lap_apply block (float32 18/12-real, float64, four fields in one launch; 32^4 and 24^3 x 48), the
split of a step into trajectory and spectrum, the same steps through host buffers (e2e), float64
and mixed trajectories from the same links and momenta at the workload's 20 steps and at the
accepting 40 steps (fp64_compare), three Metropolis trajectories at 40 steps (accepting), SM
clocks sampled during the timed region, and the float64 CPU oracle on a bounded sample
(cpu_baseline).

Prints one JSON line (rank 0).  --impl reference times the float64 CPU oracle instead.
"""
import argparse
import json
import re
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Laplacian GB/s & % HBM peak; RMHMC traj/s at 32^4, mixed vs FP64 at fixed ΔH"
DIMS = (32, 32, 32, 32)
BETA = 6.0
KAPPA = 0.9
NPOLE = 12
TAU = 1.0
NSTEPS = 20
CHEB_DEGREE = 200
CHEB_WINDOWS = 64
CHEB_NOISE = 16
# mixed-precision MD settings of the headline: float32 Krylov forces to MIXED_TOL_MD, fixed points to a max-norm
# change of MIXED_FP_TOL followed by MIXED_FP_EXTRA further iterations, which remove the systematic part of
# the fixed points' error (float32 rounding noise stays); float64 runs use FP64_TOL for both
MIXED_TOL_MD = 3e-7
MIXED_FP_TOL = 1e-6
MIXED_FP_EXTRA = 4
FP64_TOL = 1e-10
DH_BAR = 1e-3
# step counts at 32^4 (tau = 1) beyond the workload's 20: at 20 steps (eps = 0.05) the leapfrog is near its
# stability edge for this mass term (dH ~ 200, every trajectory rejected); at 40 steps dH ranges from 0.1 to ~20
# over momentum draws (the float64-vs-mixed comparison at fixed dH runs there, PAIR_NSTEPS), and the accepting
# setting's trajectories use 64 steps
PAIR_NSTEPS = 40
ACCEPT_NSTEPS = 64
# DRAM bytes (read + write) of one k_cg_A<float,18> launch at 32^4, mean of three consecutive CG iterations of
# one ncu capture per launch shape (dram__bytes_read.sum + dram__bytes_write.sum;
# profiles/k_cg_A_fp32_32x32x32x32.md), keyed by the tuned shape (components per lane, threads per block); a
# shape without a capture reports null
CG_TRAFFIC_32 = {(1, 256): 880.3e6, (2, 256): 885.9e6, (1, 128): 877.0e6, (0, 128): 936.9e6, (0, 256): 936.9e6}
# algorithmic bytes per site of the conjugate-gradient stencil k_cg_A<float,18> (float32, 18-real links):
# read r_k (128 B) and q_{k-1} (128 B), write q_k (128 B), four links of 72 B
CG_BYTES_PER_SITE = 3 * 128 + 4 * 72
IWASAKI_C1 = -0.331
# float32 FMA rate of the GB300 (measured with a register-resident FMA loop on this machine: 37.4 TFMA/s; the nominal
# 152 SMs x 128 lanes x 2.07 GHz = 40.3 TFMA/s)
FP32_FMA_PEAK = 37.4


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(x, dist, device="cpu"):
    """Largest value of x over all ranks (the timed region of the slowest replica)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank):
    """Per-replica seeds: link start, thermalisation momenta, trajectory momenta."""
    return {"links": rank, "therm": 7 + rank, "traj": 100 + rank}


def oracle_sample(seconds_cap=30.0):
    """Time the float64 CPU oracle on a bounded sample of the workload (about 10 s): kinetic-force
    evaluations (two 12-shift rational solves by per-shift CG, plus the link gradient) and Laplacian
    applications at 8^4 with the workload's mass term and link recipe."""
    import numpy as np

    import oracle
    from oracle import fit
    from paper_2112_04556_gb300 import inputs
    oracle.build()
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.3, seed=0)
    P = inputs.gaussian_fields(L, 1, seed=1)[0]
    m = fit.mass_term(NPOLE, KAPPA)
    # repeat the kinetic evaluation until about 8 s of CPU work (at least twice) and average
    t0 = time.perf_counter()
    nkin = 0
    while nkin < 2 or time.perf_counter() - t0 < 8.0:
        oracle.kinetic(L, U, P, m, tol=1e-6)
        nkin += 1
    t_kin = (time.perf_counter() - t0) / nkin
    t0 = time.perf_counter()
    nlap = 0
    while time.perf_counter() - t0 < 2.0:
        oracle.lap(L, U, P)
        nlap += 1
    t_lap = (time.perf_counter() - t0) / nlap
    return {"t_kin_8": t_kin, "t_lap_8": t_lap, "cores": oracle.num_threads(),
            "scale": float(np.prod(DIMS)) / float(np.prod(L))}


def oracle_traj_seconds(s, md_solves):
    """Oracle seconds per step at 32^4, scaled linearly in volume (iteration counts do not depend on the
    volume at fixed condition number): (md_solves + 3) kinetic-equivalents for the trajectory (MD plus
    heatbath and the two Hamiltonians) and (18 fields x 100 applications) for the spectrum."""
    return s["scale"] * ((md_solves + 3) * s["t_kin_8"] + 18 * CHEB_DEGREE // 2 * s["t_lap_8"])


def workload_config(nsteps, world):
    return {"workload": "32^4 full RMHMC (Wilson beta 6.0, 12-pole mass kappa 0.9, tau 1, %d steps, "
                        "mixed precision) + gauge-force spectrum (degree 200, 64 windows, 16 noise)" % nsteps,
            "lattice": "x".join(str(d) for d in DIMS), "l2": "working set > L2, no flush",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    """The float64 CPU oracle as the reference arm.  Each step is one bounded sample (the oracle_sample work, about
    10 s); ms_per_step is that sample's measured time, and value = the fraction of a 32^4 step the sample covers
    divided by that time, i.e. 32^4 steps per second at the oracle's measured per-operation costs."""
    if rank != 0:
        return 0
    s0 = time.perf_counter()
    md_solves = md_solves_estimate(args.nsteps)
    secs, trajs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = oracle_sample()
        if i >= args.warmup:
            secs.append(time.perf_counter() - t0)
            trajs.append(oracle_traj_seconds(s, md_solves))
    sec_step = sum(secs) / len(secs)
    traj_sec = sum(trajs) / len(trajs)
    value = 1.0 / traj_sec
    units = sec_step / traj_sec
    sample = ("oracle kinetic-force evaluations + Laplacians at 8^4 per step (%.1f s), a fraction %.3g of one 32^4 "
              "step: V(32^4)/V(8^4) = 256 x (%d kinetic evaluations + 3 for heatbath and Hamiltonians + 1800 "
              "spectrum applications)" % (sec_step, units, md_solves))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "traj/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_step * 1e3, "units_per_step": units,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.nsteps, world),
            "cpu_baseline": {"value": value, "unit": "traj/s", "cores": s["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "traj/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - s0}
    print(json.dumps(line), flush=True)
    return 0


def md_solves_estimate(nsteps):
    """Kinetic evaluations of one trajectory at the headline settings: 4 fixed-point iterations to the tolerance
    plus MIXED_FP_EXTRA, for each of the two fixed points of every step (each iterate of either needs a Krylov
    run: a kinetic force or a velocity), and the first force (the GPU runs count these; at 20 steps 161 + 160)."""
    return 2 * nsteps * (4 + MIXED_FP_EXTRA) + 1


# algorithmic bytes per site of lap_apply: links once (4 x 18 or 12 reals) + every field read once and written
# once (2 x 32 reals per field)
def lap_bytes_per_site(prec_bytes, linkfmt, nf):
    return 4 * linkfmt * prec_bytes + 2 * 32 * prec_bytes * nf


def lap_fma_per_site(form, nf, linkfmt=18):
    """FP32 pipe operations (FMA, or a single add or multiply) per site: the 3x3 form does 8 hops x 4 components
    x 108 FMA per field (traceless conjugations; +24 per hop to rebuild the third row of 12-real links); the
    adjoint form builds 8 adjoint matrices (~270 operations each, +24 for 12-real links) and does 64 FMA per
    component hop."""
    if form == "3x3":
        return 3456 * nf + (8 * 24 if linkfmt == 12 else 0)
    return 8 * (270 + (24 if linkfmt == 12 else 0)) + 8 * 4 * 64 * nf


def lap_block(rm, torch, inputs, dims, ctx=None, U=None, reps=20):
    """lap_apply timed with CUDA events on the launching stream (warm-up 3, then reps calls): float32 with 18-
    and 12-real links, float64, and the 18 float32 fields of the spectrum in one launch (the adjoint form).  The
    inputs (links and fields) are larger than L2 at these sizes, so no flush is needed between calls."""
    import numpy as np
    V = int(np.prod(dims))
    own = ctx is None
    if own:
        ctx = rm.Context(dims)
        U = torch.from_numpy(inputs.random_links(dims, eps=0.3, seed=0)).cuda()
    rm.set_links(ctx, U)
    X64 = torch.from_numpy(inputs.gaussian_fields(dims, 1, seed=1)[0]).cuda()
    X32 = X64.float()
    XM = torch.randn((18,) + tuple(X64.shape), dtype=torch.float32, device=X64.device)
    peak, kind = measured_peaks()
    out = {"lattice": "x".join(map(str, dims)), "peak_gbs": peak, "peak_kind": kind, "fp32_fma_peak_tfma_s": FP32_FMA_PEAK,
           "l2": "inputs larger than L2, no flush", "variants": []}
    st = torch.cuda.current_stream()
    for name, X, prec, lf, nf, form in [("fp32_18", X32, rm.FP32, 18, 1, "3x3"), ("fp32_12", X32, rm.FP32, 12, 1, "3x3"),
                                        ("fp64_18", X64, rm.FP64, 18, 1, "3x3"),
                                        ("fp32_18_x18", XM, rm.FP32, 18, 18, "adjoint")]:
        Y = torch.empty_like(X)
        for _ in range(3):
            rm.lap_apply(ctx, None, X, Y, prec=prec, linkfmt=lf)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            rm.lap_apply(ctx, None, X, Y, prec=prec, linkfmt=lf)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        pb = 8 if prec == rm.FP64 else 4
        gbs = lap_bytes_per_site(pb, lf, nf) * V / (ms * 1e-3) / 1e9
        fma = lap_fma_per_site(form, nf, lf) * V / (ms * 1e-3) / 1e12
        d = {"variant": name, "ms": ms, "bytes_per_site": lap_bytes_per_site(pb, lf, nf), "gbs_alg": gbs,
             "frac_hbm": gbs / peak, "form": form}
        if prec == rm.FP32:
            d["tfma_s"] = fma
            d["frac_fp32_fma"] = fma / FP32_FMA_PEAK
        else:
            d["tflop_s_fp64"] = 2 * fma
        out["variants"].append(d)
        del Y
    if own:
        ctx.close()
    return out


def run_kernel(args):
    """Kernel microbenchmark: lap_apply (float32, 18-real links) or one mixed kinetic-force evaluation
    (the conjugate-gradient stencil in the tuned shape) on the chosen lattice, timed with CUDA events."""
    import numpy as np
    import torch

    import paper_2112_04556_gb300 as rm
    from paper_2112_04556_gb300 import inputs
    V = int(np.prod(DIMS))
    lat = rm.Context(DIMS)
    U = torch.from_numpy(inputs.random_links(DIMS, eps=0.3, seed=0)).cuda()
    rm.set_links(lat, U)
    X = torch.from_numpy(inputs.gaussian_fields(DIMS, 1, seed=1)[0]).cuda()
    X32 = X.float()
    Y32 = torch.empty_like(X32)
    mass = rm.mass_fit(NPOLE, KAPPA)
    if args.shape:
        nmu, block = (int(v) for v in args.shape.split(","))
        rm.set_stencil_shape(lat, rm.SHAPE_LAP, rm.FP32, 18, nmu, block)
        rm.set_stencil_shape(lat, rm.SHAPE_CG, rm.FP32, 18, nmu, block)
    nf = 1
    if args.kernel == "lap":
        op = lambda: rm.lap_apply(lat, None, X32, Y32, prec=rm.FP32, linkfmt=18)
    elif args.kernel == "lapmulti":
        # the 18 fields of the spectrum in one launch (the adjoint form)
        nf = 18
        XM = torch.randn((nf,) + tuple(X32.shape), dtype=torch.float32, device="cuda")
        YM = torch.empty_like(XM)
        op = lambda: rm.lap_apply(lat, None, XM, YM, prec=rm.FP32, linkfmt=18)
    else:
        op = lambda: rm.kinetic_force(lat, None, X, mass, tol=1e-6, prec=rm.MIXED)
    for _ in range(args.warmup):
        op()
    rm.counters(lat, reset=True)
    rm.set_profiling(lat, True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        op()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    cnt = rm.counters(lat)
    peak, kind = measured_peaks()
    line = {"kernel": args.kernel, "lattice": "x".join(map(str, DIMS)), "ms_per_call": ms, "autotune": rm.tuning(lat)}
    if args.kernel in ("lap", "lapmulti"):
        line["gbs_alg"] = lap_bytes_per_site(4, 18, nf) * V / (ms * 1e-3) / 1e9
        line["frac_hbm"] = line["gbs_alg"] / peak
    else:
        avg = cnt["cg_ms"] / max(cnt["cg_count"], 1)
        line["cg_launches"] = cnt["cg_count"]
        line["cg_avg_ms"] = avg
        line["cg_gbs_alg"] = CG_BYTES_PER_SITE * V / (avg * 1e-3) / 1e9
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=["lap", "cg", "lapmulti"], default=None,
                    help="time one kernel family instead of the workload (for profiling)")
    ap.add_argument("--shape", default=None,
                    help="pin the float32 stencil shape of --kernel lap/cg as nmu,block (8,256: the link-centric kernel)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 comparison trajectory")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--dims", default="32,32,32,32")
    ap.add_argument("--nsteps", type=int, default=NSTEPS)
    ap.add_argument("--therm", type=int, default=20, help="plain-HMC thermalisation trajectories")
    ap.add_argument("--graphs", choices=["on", "off"], default="on",
                    help="run the mixed-precision MD as one CUDA graph per trajectory")
    ap.add_argument("--no-lap", action="store_true", help="skip the lap_apply block")
    ap.add_argument("--no-accept", action="store_true", help="skip the accepting-setting trajectories")
    ap.add_argument("--compare-tau", type=float, default=TAU,
                    help="trajectory length of the float64-vs-mixed comparison (same number of steps)")
    args = ap.parse_args()
    global DIMS
    DIMS = tuple(int(v) for v in args.dims.split(","))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.kernel:
        return run_kernel(args)

    # the CPU oracle sample runs before any GPU work (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample()

    import numpy as np
    import torch

    import paper_2112_04556_gb300 as rm
    from paper_2112_04556_gb300 import inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    V = int(np.prod(DIMS))
    lat = rm.Context(DIMS, device=local)
    rm.set_graphs(lat, args.graphs == "on")
    mass = rm.mass_fit(NPOLE, KAPPA)
    seeds = replica_seeds(rank)
    U = torch.from_numpy(inputs.random_links(DIMS, eps=0.3, seed=seeds["links"])).cuda()

    # thermalise with plain HMC, every trajectory accepted (not timed)
    ident = {"c": 1.0, "alpha": [], "sigma": [], "kappa": 0.0}
    therm = []
    for n in range(args.therm):
        p = rm.make_params(beta=BETA, mass=ident, tau=1.0, nsteps=20, tol_md=1e-6, tol_h=1e-11, fp_tol=1e-6,
                           prec=rm.MIXED, seed=seeds["therm"], traj_index=1000 + n, metropolis=False)
        therm.append(rm.rmhmc_trajectory(lat, U, p)["plaq"])

    def params(idx, prec, tau=TAU, nsteps=None, metropolis=True):
        mixed = prec == rm.MIXED
        return rm.make_params(beta=BETA, mass=mass, tau=tau, nsteps=nsteps or args.nsteps,
                              tol_md=MIXED_TOL_MD if mixed else FP64_TOL, tol_h=1e-12,
                              fp_tol=MIXED_FP_TOL if mixed else FP64_TOL, fp_extra=MIXED_FP_EXTRA if mixed else 0,
                              fp_maxit=50, maxiter=400, prec=prec, seed=seeds["traj"], traj_index=idx,
                              metropolis=metropolis)

    F2 = torch.empty((2, V, 4, 8), dtype=torch.float64, device="cuda")
    edges = inputs.equal_windows(CHEB_WINDOWS)
    results = []
    ev = {"traj": [], "spec": []}

    def step(idx, Ulinks, timed=False):
        if timed:
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
        r = rm.rmhmc_trajectory(lat, Ulinks, params(idx, rm.MIXED))
        if timed:
            b.record(stream)
        rm.gauge_force(lat, None, BETA, 0.0, prec=rm.FP32, F=F2[0])
        rm.gauge_force(lat, None, BETA, IWASAKI_C1, prec=rm.FP32, F=F2[1])
        spec = rm.cheb_filter_spectrum(lat, None, F2, None, CHEB_DEGREE, edges, prec=rm.MIXED,
                                       nnoise=CHEB_NOISE, seed=idx)[0]
        if timed:
            c.record(stream)
            ev["traj"].append((a, b))
            ev["spec"].append((b, c))
        r["spec_low"] = float(spec[0, 0])
        r["spec_high"] = float(spec[0, -1])
        return r

    U_start = U.clone()
    for w in range(args.warmup):
        step(w, U)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    rm.counters(lat, reset=True)
    rm.set_profiling(lat, True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        results.append(step(args.warmup + k, U, timed=True))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    rm.set_profiling(lat, False)
    ms = e0.elapsed_time(e1)
    cnt = rm.counters(lat, reset=True)
    ms = max_over_ranks(ms, dist, "cuda")
    value = world * args.steps / (ms / 1e3)
    split = {"trajectory_s": sum(a.elapsed_time(b) for a, b in ev["traj"]) / 1e3 / args.steps,
             "spectrum_s": sum(a.elapsed_time(b) for a, b in ev["spec"]) / 1e3 / args.steps}
    split["traj_per_s_trajectory_only"] = 1.0 / split["trajectory_s"]

    # live roofline of the conjugate-gradient stencil (float32, 18-real links):
    # per site 3 field passes of 128 B (read r_k and q_{k-1}, write q_k) + 4 links x 72 B = 672 B
    peak, peak_kind = measured_peaks()
    cg_bytes = CG_BYTES_PER_SITE * V
    cg_avg_ms = cnt["cg_ms"] / max(cnt["cg_count"], 1)
    achieved = cg_bytes / (cg_avg_ms * 1e-3) / 1e9 if cnt["cg_count"] else None
    alu_fma = 3600.0 * V   # per site: 8 hops x 4 components x 108 FMA + the fused axpy and epilogue
    m = re.search(r"cg fp32 -> nmu (\d+) block (\d+)", rm.tuning(lat))
    shape = (int(m.group(1)), int(m.group(2))) if m else None
    traffic = CG_TRAFFIC_32.get(shape) if DIMS == (32, 32, 32, 32) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "k_cg_A<float,18> (CG stencil)", "shape": shape, "launches": cnt["cg_count"],
                "avg_launch_ms": cg_avg_ms, "alu_tfma_s": alu_fma / (cg_avg_ms * 1e-3) / 1e12 if cnt["cg_count"] else None,
                "alu_peak_tfma_s": FP32_FMA_PEAK}

    # end to end through the public API with host buffers: pinned H2D of the links, D2H of the result
    e2e = None
    if not args.no_e2e:
        Uh = U.cpu().pin_memory()
        Uout = torch.empty_like(Uh).pin_memory()
        Ud = torch.empty_like(U)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            Ud.copy_(Uh, non_blocking=True)
            step(10000 + k, Ud)
            Uout.copy_(Ud, non_blocking=True)
            torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        sec = max_over_ranks(sec, dist, "cuda")
        nb = Uh.numel() * Uh.element_size()
        e2e = {"value": world * args.steps / sec, "unit": "traj/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb + 8 * 16}

    # the Laplacian (first half of the metric): 32^4 on the workload's thermalised links, and 24^3 x 48
    lap = None
    if rank == 0 and not args.no_lap:
        lap = [lap_block(rm, torch, inputs, DIMS, lat, U)]
        if DIMS == (32, 32, 32, 32):
            lap.append(lap_block(rm, torch, inputs, (24, 24, 24, 48)))

    def timed_traj(Ulinks, p):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rm.rmhmc_trajectory(lat, Ulinks, p)
        torch.cuda.synchronize()
        r["seconds"] = time.perf_counter() - t0
        return r

    def pair(tau, nsteps, idx):
        """one float64 and one mixed trajectory (the headline's mixed settings) from the same links and momenta"""
        ra = timed_traj(U_start.clone(), params(idx, rm.FP64, tau, nsteps))
        rb = timed_traj(U_start.clone(), params(idx, rm.MIXED, tau, nsteps))
        d = abs(ra["dH"] - rb["dH"])
        return {"tau": tau, "nsteps": nsteps, "dH_fp64": ra["dH"], "dH_mixed": rb["dH"], "abs_dH_diff": d,
                "meets_dH_bar": bool(d <= DH_BAR), "accepted_fp64": ra["accepted"], "accepted_mixed": rb["accepted"],
                "seconds_fp64": ra["seconds"], "seconds_mixed": rb["seconds"],
                "traj_per_s_fp64": 1.0 / ra["seconds"], "traj_per_s_mixed": 1.0 / rb["seconds"],
                "speedup_mixed_over_fp64": ra["seconds"] / rb["seconds"], "plaq_fp64": ra["plaq"],
                "plaq_mixed": rb["plaq"], "md_iters_fp64": ra["md_iters"], "md_iters_mixed": rb["md_iters"],
                "fp_iters_fp64": [ra["fp_iters_p"], ra["fp_iters_u"]],
                "fp_iters_mixed": [rb["fp_iters_p"], rb["fp_iters_u"]]}

    # mixed vs float64 at fixed dH: at the workload's 20 steps and at 40 steps (tau = 1 both)
    fp64 = None
    if world == 1 and not args.no_fp64:
        fp64 = {"dH_bar": DH_BAR, "mixed": {"tol_md": MIXED_TOL_MD, "fp_tol": MIXED_FP_TOL, "fp_extra": MIXED_FP_EXTRA},
                "fp64": {"tol_md": FP64_TOL, "fp_tol": FP64_TOL},
                "workload_steps": pair(args.compare_tau, args.nsteps, 0)}
        if not args.no_accept:
            fp64["stable_steps"] = pair(args.compare_tau, PAIR_NSTEPS, 0)

    # the accepting setting at 32^4 (tau = 1 in ACCEPT_NSTEPS steps, the headline's mixed tolerances): three
    # consecutive trajectories with Metropolis from the thermalised start
    accept = None
    if rank == 0 and not args.no_accept:
        Ua = U_start.clone()
        runs = [timed_traj(Ua, params(20000 + i, rm.MIXED, TAU, ACCEPT_NSTEPS)) for i in range(3)]
        accept = {"tau": TAU, "nsteps": ACCEPT_NSTEPS, "dH": [r["dH"] for r in runs],
                  "accepted": [r["accepted"] for r in runs], "seconds": [r["seconds"] for r in runs],
                  "traj_per_s": len(runs) / sum(r["seconds"] for r in runs),
                  "acceptance_expected": [min(1.0, math.exp(-r["dH"])) for r in runs]}

    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": "traj/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(args.nsteps, world),
            "thermalisation_plaq": therm[-3:] if therm else None,
            "autotune": rm.tuning(lat),
            "roofline": roofline, "clocks": clk, "gpu_launches": cnt["launches"],
            "krylov_iters": cnt["krylov_iters"], "e2e": e2e, "split": split, "lap_apply": lap,
            "accepting": accept,
            "mixed_settings": {"tol_md": MIXED_TOL_MD, "fp_tol": MIXED_FP_TOL, "fp_extra": MIXED_FP_EXTRA},
            "trajectories": [{k: r[k] for k in ("dH", "accepted", "plaq", "md_solves", "md_iters", "fp_iters_p",
                                                "fp_iters_u", "spec_low", "spec_high")} for r in results]}
    if fp64:
        line["fp64_compare"] = fp64
    if cpu:
        md_solves = int(np.mean([r["md_solves"] for r in results]))
        sec = oracle_traj_seconds(cpu, md_solves)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "traj/s", "cores": cpu["cores"], "kind": "oracle",
                                "sample": "oracle kinetic-force evaluation (%.1f s) and Laplacian at 8^4, scaled by "
                                          "V(32^4)/V(8^4) = 256 and by %d + 3 kinetic evaluations + 1800 spectrum "
                                          "applications per step" % (cpu["t_kin_8"], md_solves)}
    print(json.dumps(line), flush=True)
    lat.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
