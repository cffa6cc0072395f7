"""Benchmark: HMC trajectories per second for the pseudofermion HMC of the O(3) spin-fermion
model on an 80 x 80 x 160 lattice (dtau = 0.1), Yukawa coupling lambda = 1 in D's on-site term,
8 pseudofermion right-hand sides per chain, n_leap = 40, complex64 CG with FP64 reliable updates
(tolerance 1e-10 on the FP64 true residual), one chain per GPU.

Before the timed region the chain is thermalised and its HMC hyperparameters are tuned as the
paper's warm-up does: the start is an ordered field (the mean-field amplitude along one component
plus free-boson fluctuations), N_THERM trajectories at a small step with the free-boson metric,
sigma-hat from Eq. (covest) over the last N_COVEST of them, then eps by Eq. (acc_ineq). The timed
trajectories use the tuned sigma-hat and eps.

A step is one full trajectory (heatbath, momentum draw, 41 force evaluations, Metropolis).
The line also reports the fused A = D D^dagger matvec (complex64, 8 RHS) against the measured
HBM copy bandwidth, one solve in FP64 vs mixed precision at equal true residual, the trajectory
measured end to end from host buffers, and the FP64 oracle's throughput on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (replicas, weak scaling): torchrun --nproc-per-node N bench.py --gpus N ...
"""

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HMC traj/s and M†M matvec GB/s at 80×80; mixed vs FP64 at equal CG residual"
L, NT, NRHS, NLEAP, TOL, MAXIT = 80, 160, 8, 40, 1e-10, 20000
GUESS = 4   # force solves start from the degree-4 extrapolation of the previous solutions (same stopping test)
LAMBDA = 1.0   # Yukawa coupling: D's on-site term is dtau * LAMBDA * (-1)^(x+y) phi.sigma sigma^x
COUPLINGS = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=LAMBDA, r=0.5, u=1.0, c=3.0)
# Ordered start: the uniform amplitude that minimises S_B - 8 log det(D D^dagger) over uniform
# fields of this lattice (mean field for eight right-hand sides), plus free-boson fluctuations.
AMP = 2.8
EPS0 = 0.01                 # thermalisation step
# Eq. (covest) about the batch mean: the ordered chain keeps its condensate over the warm-up, and
# the uncentered moment would book V |phi-bar|^2 on the zero mode as a fluctuation (a leapfrog
# frequency ~ 4500 for that mode, far past any usable step)
SIGMA_CENTERED = True
N_THERM, N_COVEST = 12, 8   # thermalisation trajectories; the last N_COVEST feed Eq. (covest)
# Eq. (acc_ineq): rounds of TUNE_WINDOW single-step proposals at eps and eps/2, eps scaled by
# TUNE_GROW each round, until it has turned TUNE_TURNS times (at most TUNE_ROUNDS rounds)
TUNE_ROUNDS, TUNE_WINDOW, TUNE_GROW, TUNE_TURNS = 24, 2, 1.5, 2
# Solver: plain CG. On this ordered workload the fermions are gapped and the preconditioner of
# Eq. (precon), exact for the free Fermi surface, saves few iterations (69 against 58 per solve
# measured on GB300) while each preconditioned iteration streams about 1.4x the bytes.
PRECOND = False
WORKLOAD_BASE = (f"L={L}x{L}, Nt={NT} (dtau=0.1), 2 bands x 2 spins, {NRHS} pseudofermion RHS (N_f={2 * NRHS}), "
                 f"Yukawa lambda={LAMBDA} (D coefficient dtau*lambda), n_leap={NLEAP}, "
                 f"complex64 {'PCG' if PRECOND else 'CG'} with FP64 reliable updates to true residual {TOL}, "
                 f"degree-{GUESS} chronological initial guess; start: ordered field (amplitude {AMP} on one "
                 f"component + free-boson fluctuations), {N_THERM} thermalisation trajectories at eps={EPS0}, "
                 f"sigma-hat from Eq. (covest){' about the batch mean' if SIGMA_CENTERED else ''} over the last "
                 f"{N_COVEST}, eps by Eq. (acc_ineq) then backed off until a {NLEAP}-step trajectory is stable")
# DRAM bytes (read + write) of one launch of the roofline kernel, the plain fused A on 8 RHS at
# 80x80x160, from one ncu capture of `bench.py --profile-matvec 3` (324.3 MB read + 220.5 MB
# written); set to None when that kernel changes until it is captured again.
ROOFLINE_TRAFFIC_BYTES = 544_735_488
# CG iterations per solve of this workload with the degree-4 chronological start at the tuned step
# (92.0 measured on a GB300), used only to
# scale the oracle's timed sample (a few iterations) to a trajectory when no GPU run is available
# in the process.
ITERS_PER_SOLVE_DEFAULT = 92


def kt():
    return 2.0 / (COUPLINGS["c"] ** 2 * COUPLINGS["dtau"] ** 2)


def synthetic_inputs(seed):
    """phi: the ordered start (AMP on component 3 plus a Gaussian field with the free-boson
    spectrum 1/(dtau B(k))); sigma-hat: that spectrum (the thermalisation metric)."""
    from paper_2204_14241_gb300 import inputs as I
    dt = COUPLINGS["dtau"]
    phi = I.ordered_field(seed, L, NT, COUPLINGS["r"], kt(), 1.0 / np.sqrt(dt), AMP)
    sig = np.broadcast_to(I.spectrum(L, NT, COUPLINGS["r"], kt())[None] / dt, (3, NT, L, L)).copy()
    return phi, sig


# ---- distributed helpers (replicas; tested on CPU with gloo) ------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws, device=None):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def chain_seed(base, rank):
    """Independent chain per rank: distinct synthetic field and Philox key."""
    return int(base) * 1000003 + 7919 * int(rank) + 1


# ---- clocks ------------------------------------------------------------------------------------------
CLOCK_LOG_DIR = None   # --clock-log DIR keeps the raw nvidia-smi samples there (default: a temp file)


def clock_log_path(gpu_index):
    import tempfile
    d = CLOCK_LOG_DIR or tempfile.gettempdir()
    return os.path.join(d, f"hmc_bench_clocks_gpu{gpu_index}_{os.getpid()}.csv")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.path = clock_log_path(gpu_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- the oracle on the host cores (cpu_baseline / reference arm) -------------------------------------
_ORACLE_INPUTS = {}


def oracle_iteration_time(n_iter=2):
    """Seconds per solver iteration of the FP64 oracle on the full lattice, one right-hand side:
    one A apply, the preconditioner when the workload uses it, the vector updates and the dot
    products. Returns (seconds per iteration, threads used)."""
    from oracle.model import Params
    from oracle import solver, fermion
    from paper_2204_14241_gb300 import inputs as I
    if not _ORACLE_INPUTS:
        phi, _ = synthetic_inputs(1)
        _ORACLE_INPUTS["phi"] = I.to_paper_boson(phi)
        _ORACLE_INPUTS["b"] = I.to_paper_fermion(I.fermion_noise(2, 1, L, NT)[0])
    P = Params(L=L, Nt=NT, **COUPLINGS)
    phi_o, b = _ORACLE_INPUTS["phi"], _ORACLE_INPUTS["b"]
    x, r, pdir = np.zeros_like(b), b.copy(), b.copy()
    t0 = time.perf_counter()
    for _ in range(n_iter):
        q = fermion.apply_A(P, phi_o, pdir)
        a = solver.vdot(r, r).real / solver.vdot(pdir, q).real
        x = x + a * pdir
        r = r - a * q
        z = solver.apply_precond(P, r) if PRECOND else r
        pdir = z + 0.5 * pdir
        solver.vdot(r, z)
    dt = (time.perf_counter() - t0) / n_iter
    return dt, 1


def oracle_traj_per_s(iters_per_solve, n_iter=2):
    t_it, threads = oracle_iteration_time(n_iter)
    t_traj = (NLEAP + 1) * NRHS * iters_per_solve * t_it
    return 1.0 / t_traj, t_it, threads


def solver_name():
    return "PCG" if PRECOND else "CG"


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_iteration_time(1)
    vals, t0 = [], time.perf_counter()
    for _ in range(args.steps):
        v, t_it, threads = oracle_traj_per_s(ITERS_PER_SOLVE_DEFAULT, 1)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    sample = (f"per step: 1 {solver_name()} iteration of the FP64 numpy oracle (A apply + updates) on one RHS "
              f"at {L}x{L}x{NT}, scaled to a trajectory as {NLEAP + 1} solves x {NRHS} RHS x "
              f"{ITERS_PER_SOLVE_DEFAULT} iterations per solve")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "traj/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_BASE},
            "cpu_baseline": {"value": value, "unit": "traj/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "host_cpus": os.cpu_count()},
            "e2e": {"value": value, "unit": "traj/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- our arm --------------------------------------------------------------------------------------------
def time_matvec(ctx, torch, phi32, x, reps=20):
    """Average duration of the fused A apply (complex64, NRHS) with CUDA events on ctx's stream."""
    y = torch.empty_like(x)
    st = ctx.stream
    for _ in range(3):
        ctx.apply_MdagM(phi32, x, out=y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        ctx.apply_MdagM(phi32, x, out=y)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps


def run_ours(args):
    import torch
    from paper_2204_14241_gb300.hmc import Context
    from paper_2204_14241_gb300 import inputs as I

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    seed = chain_seed(args.seed, rank)
    phi_np, sig_np = synthetic_inputs(seed)
    phi = torch.from_numpy(phi_np).to(dev)
    sig = torch.from_numpy(sig_np).to(dev)
    ctx = Context(L, NT, solver="mixed", nrhs_max=NRHS, cg_tol=TOL, cg_maxit=MAXIT, device=dev, initial_guess=GUESS,
                  **COUPLINGS)
    st = ctx.stream

    # warm-up as in the paper (Sections "Online metric estimation" and "Online HMC hyperparameter
    # tuning"): thermalisation with the free-boson metric, sigma-hat by Eq. (covest) over the last
    # N_COVEST states, then eps by Eq. (acc_ineq); none of it is timed
    from paper_2204_14241_gb300.tuning import SigmaEstimator, Tuner
    t_w0 = time.perf_counter()
    est = SigmaEstimator(ctx, sig, centered=SIGMA_CENTERED)
    therm = []
    for w in range(N_THERM):
        o = ctx.trajectory([phi], [sig], EPS0, NLEAP, nrhs=NRHS, precond=PRECOND, seed=seed, counter=w, check=False)
        therm.append(o)
        if w >= N_THERM - N_COVEST:
            est.add(phi)
    sig_free = sig.clone()
    sig = est.value()
    sigma_ratio = (sig / sig_free)
    tuner = Tuner(ctx, phi, sig, nrhs=NRHS, precond=PRECOND, seed=seed + 1)
    eps_single, eps_hist = tuner.tune_eps(EPS0, TUNE_ROUNDS, TUNE_WINDOW, grow=TUNE_GROW,
                                          stop_after_turns=TUNE_TURNS)
    # Eq. (acc_ineq) judges single steps; back off until a 40-step trajectory integrates stably
    eps, eps_tries = tuner.stabilize_eps(eps_single, NLEAP, shrink=TUNE_GROW)
    warm = []
    for w in range(args.warmup):
        o = ctx.trajectory([phi], [sig], eps, NLEAP, nrhs=NRHS, precond=PRECOND, seed=seed, counter=500 + w,
                           check=False)
        warm.append(o)
    t_warm = time.perf_counter() - t_w0
    sig_np = sig.cpu().numpy()
    workload = WORKLOAD_BASE + f"; tuned eps={eps:.4g}"

    # timed trajectories. Each step: H2D copy of the step's inputs (phi, sigma-hat) from pinned
    # host memory, the trajectory (CUDA events around it give the device-resident value), D2H
    # copy of the new phi and dH (the host clock around all of it gives the end-to-end value).
    h_phi = torch.from_numpy(phi.cpu().numpy()).pin_memory()
    h_sig = torch.from_numpy(sig_np).pin_memory()
    h_out = torch.empty_like(h_phi).pin_memory()
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    l0 = ctx.launches()
    outs, t_dev, t_e2e = [], 0.0, 0.0
    for k in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        phi.copy_(h_phi, non_blocking=True)
        sig.copy_(h_sig, non_blocking=True)
        e0.record(st)
        o = ctx.trajectory([phi], [sig], eps, NLEAP, nrhs=NRHS, precond=PRECOND, seed=seed, counter=1000 + k,
                           check=False)
        e1.record(st)
        h_out.copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e += time.perf_counter() - h0
        t_dev += e0.elapsed_time(e1) / 1000.0
        h_phi.copy_(h_out)          # the chain continues from the new state
        outs.append(o)
    barrier(ws)
    launches = ctx.launches() - l0
    clk = clocks.stop()
    t_max = max_over_ranks(t_dev, ws, dev)
    value = ws * args.steps / t_max
    t_e2e = max_over_ranks(t_e2e, ws, dev)
    V = L * L * NT
    e2e = {"value": ws * args.steps / t_e2e, "unit": "traj/s", "h2d_bytes_per_step": 2 * 3 * V * 8,
           "d2h_bytes_per_step": 3 * V * 8 + 8}
    iters = [o["cg_iterations"][0] for o in outs]
    iters_per_solve = float(np.mean(iters)) / (NLEAP + 1)

    # dominant kernel: the fused A = D D^dagger matvec, complex64, NRHS right-hand sides (> L2)
    phi32 = phi.float()
    x = torch.from_numpy(I.fermion_noise(seed + 1, NRHS, L, NT)).to(dev).to(torch.complex64)
    t_mv = time_matvec(ctx, torch, phi32, x)
    mv_bytes = NRHS * V * 64 + V * 12         # x read + y written per RHS, phi (fp32) read once
    achieved = mv_bytes / t_mv / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # mixed vs FP64 at equal final true residual: one 8-RHS solve each of A X = D chi (the
    # right-hand side of a force solve)
    chi = torch.from_numpy(I.fermion_noise(seed + 2, NRHS, L, NT)).to(dev)
    b = ctx.apply_M(phi, chi)
    solve = {}
    for mode in ("mixed", "fp64"):
        c2 = ctx if mode == "mixed" else Context(L, NT, solver="fp64", nrhs_max=NRHS, cg_tol=TOL, cg_maxit=MAXIT,
                                                   device=dev, **COUPLINGS)
        c2.cg_solve(phi, b, precond=PRECOND, maxit=16, raise_on_noconv=False)   # warm (first launches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, s = c2.cg_solve(phi, b, precond=PRECOND, raise_on_noconv=False)
        torch.cuda.synchronize()
        solve[mode] = {"seconds": time.perf_counter() - t0, "iterations": s["iterations"],
                       "true_rel_resid": s["true_rel_resid"], "reliable_updates": s["reliable_updates"]}
        if c2 is not ctx:
            c2.close()

    # FP64 arithmetic peak of this GPU's CUDA cores (the roofline of the FP64 operator passes of the
    # reliable updates and of the force), measured by the library's FMA-chain kernel
    from paper_2204_14241_gb300.hmc import fma_peak, FP64
    fp64_peak = fma_peak(FP64, dev) / 1e12

    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            v, t_it, threads = oracle_traj_per_s(iters_per_solve, 2)
            cpu = {"value": v, "unit": "traj/s", "cores": threads, "kind": "oracle", "host_cpus": os.cpu_count(),
                   "sample": (f"2 {solver_name()} iterations of the FP64 numpy oracle on one RHS at {L}x{L}x{NT} "
                              f"({t_it:.2f} s each), scaled to a trajectory as {NLEAP + 1} solves x {NRHS} RHS x "
                              f"{iters_per_solve:.0f} iterations per solve (the GPU run's count)")}
        acc_rate = float(np.mean([bool(o["accepted"][0]) for o in outs]))
        sr = sigma_ratio.flatten()
        line = {"metric": METRIC, "value": value, "unit": "traj/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": workload, "l2": "inputs larger than L2 (8 x 33 MB fermion fields + "
                           "workspace per solve; matvec timed on 537 MB in/out)", "parallelism": f"replicas x{ws}"},
                "matvec_gbs": achieved,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": ROOFLINE_TRAFFIC_BYTES,
                             "kernel": "k_apply_A_strip<80> (complex64 A = D D^dagger, 8 RHS)",
                             "peak_source": peak_src, "algorithmic_bytes": mv_bytes,
                             "launch_us": t_mv * 1e6},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "hmc": {"acceptance_rate": acc_rate, "eps": eps, "n_leap": NLEAP, "solver": solver_name(),
                        "cg_iters_per_solve": iters_per_solve,
                        "accept": [bool(o["accepted"][0]) for o in outs], "dH": [o["dH"][0] for o in outs],
                        "status": [o["status"] for o in outs],
                        "max_true_resid": max(o["max_true_resid"][0] for o in outs),
                        "phi_mean_component3": float(phi[2].mean().item()),
                        "thermalisation": {"trajectories": N_THERM, "eps": EPS0,
                                           "dH": [o["dH"][0] for o in therm], "status": [o["status"] for o in therm],
                                           "cg_iters_per_solve": [o["cg_iterations"][0] / (NLEAP + 1) for o in therm]},
                        "sigma_hat_over_free_spectrum": {"median": float(sr.median().item()),
                                                          "mean": float(sr.mean().item()),
                                                          "max": float(sr.max().item())},
                        "eps_tuning": [list(h) for h in eps_hist], "eps_single_step": eps_single,
                        "eps_stability_tries": [list(t) for t in eps_tries],
                        "warmup_dH": [o["dH"][0] for o in warm], "warmup_status": [o["status"] for o in warm],
                        "untimed_warmup_seconds": t_warm},
                "fp64_fma_peak_tflops": fp64_peak,
                "solve_mixed_vs_fp64": solve}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_profile_solve(args):
    """A capture-sized sample of the workload for ncu: on the full lattice, one 8-RHS solve of
    the workload's solver (the paper's preconditioned CG with --pcg) cut at a fixed iteration
    count, run twice (the second is the one to capture), plus one fused A apply. Prints the solve
    statistics."""
    import torch
    from paper_2204_14241_gb300.hmc import Context
    from paper_2204_14241_gb300 import inputs as I
    phi_np, _ = synthetic_inputs(chain_seed(args.seed, 0))
    phi = torch.from_numpy(phi_np).cuda()
    b = torch.from_numpy(I.fermion_noise(2, NRHS, L, NT)).cuda()
    ctx = Context(L, NT, solver="mixed", nrhs_max=NRHS, cg_tol=TOL, **COUPLINGS)
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = ctx.cg_solve(phi, b, precond=PRECOND or args.pcg, maxit=args.profile_solve, raise_on_noconv=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_solve": args.profile_solve, "seconds": time.perf_counter() - t0, **st}))
    x = b.to(torch.complex64)
    ctx.apply_MdagM(phi.float(), x)
    torch.cuda.synchronize()
    ctx.close()


def run_profile_trajectory(args):
    """One benchmark trajectory for an ncu launch list: the workload of the default mode (inputs,
    coupling, eps, n_leap, chronological start), one warm-up trajectory, then one inside the NVTX
    range "trajectory" (capture it with ncu --nvtx --nvtx-include "trajectory/")."""
    import torch
    from paper_2204_14241_gb300.hmc import Context
    phi_np, sig_np = synthetic_inputs(chain_seed(args.seed, 0))
    phi = torch.from_numpy(phi_np).cuda()
    sig = torch.from_numpy(sig_np).cuda()
    ctx = Context(L, NT, solver="mixed", nrhs_max=NRHS, cg_tol=TOL, cg_maxit=MAXIT, initial_guess=GUESS, **COUPLINGS)
    for rep in range(2):
        if rep == 1:
            torch.cuda.nvtx.range_push("trajectory")
        n0 = ctx.launches()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = ctx.trajectory([phi], [sig], EPS0, NLEAP, nrhs=NRHS, precond=PRECOND, seed=args.seed, counter=rep,
                           check=False)
        torch.cuda.synchronize()
        if rep == 1:
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_trajectory": rep, "seconds": time.perf_counter() - t0,
                          "launches": ctx.launches() - n0, "cg_iterations": o["cg_iterations"][0],
                          "dH": o["dH"][0]}))
    ctx.close()


def run_profile_force(args):
    """One force evaluation of the workload (solve + force kernel), for an ncu capture of the FP64
    force kernel and of the FP64 operator passes of the solve's reliable updates."""
    import torch
    from paper_2204_14241_gb300.hmc import Context
    from paper_2204_14241_gb300 import inputs as I
    phi_np, _ = synthetic_inputs(chain_seed(args.seed, 0))
    phi = torch.from_numpy(phi_np).cuda()
    pf = torch.from_numpy(I.fermion_noise(4, NRHS, L, NT)).cuda()
    ctx = Context(L, NT, solver="mixed", nrhs_max=NRHS, cg_tol=TOL, cg_maxit=MAXIT, **COUPLINGS)
    F, spf, sb, st = ctx.force(phi, pf, include_boson=True, precond=PRECOND)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_force": 1, "S_pf": spf, **st}))


def run_profile_matvec(args):
    """Only the dominant kernel: N launches of the fused A = D D^dagger (complex64, NRHS) on the
    benchmark's lattice, for an ncu capture of the last one."""
    import torch
    from paper_2204_14241_gb300.hmc import Context
    from paper_2204_14241_gb300 import inputs as I
    phi_np, _ = synthetic_inputs(chain_seed(args.seed, 0))
    phi32 = torch.from_numpy(phi_np).cuda().float()
    x = torch.from_numpy(I.fermion_noise(3, NRHS, L, NT)).cuda().to(torch.complex64)
    y = torch.empty_like(x)
    ctx = Context(L, NT, solver="mixed", nrhs_max=NRHS, cg_tol=TOL, **COUPLINGS)
    for _ in range(args.profile_matvec):
        ctx.apply_MdagM(phi32, x, out=y)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_matvec": args.profile_matvec}))


# ---- the batched configuration: 64 uneven chains ---------------------------------------------------
B_NCHAINS, B_NRHS, B_EPS, B_NLEAP, B_GUESS = 64, 2, 0.02, 10, 3
# ordered start: the uniform amplitude minimising S_B - 2 log det(D D^dagger) for two right-hand
# sides is 1.5-1.7 across r in [0.2, 1] on these lattices
B_AMP = 1.6


def batched_chains():
    """Chain i: L = {12, 16, 20, 24}[i mod 4], Nt = {24, 32, 48}[(i div 4) mod 3], r ~ U[0.2, 1]."""
    from paper_2204_14241_gb300 import inputs as I
    out = []
    for i in range(B_NCHAINS):
        L = (12, 16, 20, 24)[i % 4]
        Nt = (24, 32, 48)[(i // 4) % 3]
        out.append((L, Nt, 0.2 + 0.8 * I.uniform(900 + i)))
    return out


def run_batched_bench(args):
    """64 independent chains of uneven lattices with 2 RHS each, every force solve of all chains in
    one persistent launch and the leapfrog replayed as a CUDA graph; value = chain-trajectories per
    second. The same chains with the leapfrog's kernels launched one by one, and through the serial
    path (one chain after another, same solver), are timed for comparison."""
    import torch
    from paper_2204_14241_gb300.hmc import Context
    from paper_2204_14241_gb300 import inputs as I
    chains = batched_chains()
    dt = COUPLINGS["dtau"]
    phis, sigs = [], []
    for i, (L, Nt, r) in enumerate(chains):
        phis.append(torch.from_numpy(I.ordered_field(5000 + i, L, Nt, r, kt(), 1.0 / np.sqrt(dt), B_AMP)).cuda())
        sigs.append(torch.from_numpy(np.broadcast_to(I.spectrum(L, Nt, r, kt())[None] / dt, (3, Nt, L, L)).copy()).cuda())
    kw = dict(solver="mixed", nrhs_max=B_NRHS, cg_tol=TOL, cg_maxit=MAXIT, chains=chains, initial_guess=B_GUESS,
              **COUPLINGS)
    res = {}
    for mode, steps in (("batched", args.steps), ("batched_direct", args.steps), ("serial", max(1, min(args.steps, 2)))):
        ctx = Context(12, 24, batch_chains=0 if mode == "serial" else 1, batch_graph=1 if mode == "batched" else 0,
                      **kw)
        ph = [p.clone() for p in phis]
        for w in range(args.warmup):
            ctx.trajectory(ph, sigs, B_EPS, B_NLEAP, nrhs=B_NRHS, precond=False, seed=args.seed, counter=w, check=False)
        torch.cuda.synchronize()
        st = ctx.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ctx.launches()
        e0.record(st)
        outs = [ctx.trajectory(ph, sigs, B_EPS, B_NLEAP, nrhs=B_NRHS, precond=False, seed=args.seed,
                               counter=100 + k, check=False) for k in range(steps)]
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1000.0
        res[mode] = {"chain_traj_per_s": B_NCHAINS * steps / sec, "ms_per_step": 1000.0 * sec / steps, "steps": steps,
                     "launches_per_step": (ctx.launches() - l0) / steps,
                     "acceptance_rate": float(np.mean([a for o in outs for a in o["accepted"]])),
                     "cg_iters_per_solve": float(np.mean([i for o in outs for i in o["cg_iterations"]])) / (B_NLEAP + 1),
                     "status": sorted(set(o["status"] for o in outs))}
        ctx.close()
    line = {"metric": "chain trajectories/s, 64 uneven chains (batched configuration)",
            "value": res["batched"]["chain_traj_per_s"], "unit": "chain-traj/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{B_NCHAINS} chains, L in {{12,16,20,24}} x Nt in {{24,32,48}}, r ~ U[0.2,1], "
                                   f"{B_NRHS} RHS, Yukawa lambda={LAMBDA}, eps={B_EPS}, n_leap={B_NLEAP}, ordered start "
                                   f"(amplitude {B_AMP}), free-boson sigma-hat, complex64 CG with FP64 reliable "
                                   f"updates to {TOL}, degree-{B_GUESS} chronological start",
                       "total_sites": int(sum(L * L * Nt for L, Nt, _ in chains))},
            "batched": res["batched"], "batched_direct": res["batched_direct"], "serial": res["serial"],
            "speedup_vs_serial": res["batched"]["chain_traj_per_s"] / res["serial"]["chain_traj_per_s"],
            "graph_speedup": res["batched"]["chain_traj_per_s"] / res["batched_direct"]["chain_traj_per_s"]}
    print(json.dumps(line), flush=True)


def run_profile_batched(args):
    """One trajectory of the batched configuration for an ncu launch list: 64 uneven chains, one
    warm-up trajectory, then one inside the NVTX range "batched" (the leapfrog's kernels launched
    one by one, so that each appears in the list)."""
    import torch
    from paper_2204_14241_gb300.hmc import Context
    from paper_2204_14241_gb300 import inputs as I
    chains = batched_chains()
    dt = COUPLINGS["dtau"]
    phis, sigs = [], []
    for i, (L_, Nt_, r) in enumerate(chains):
        phis.append(torch.from_numpy(I.ordered_field(5000 + i, L_, Nt_, r, kt(), 1.0 / np.sqrt(dt), B_AMP)).cuda())
        sigs.append(torch.from_numpy(np.broadcast_to(I.spectrum(L_, Nt_, r, kt())[None] / dt,
                                                     (3, Nt_, L_, L_)).copy()).cuda())
    ctx = Context(12, 24, solver="mixed", nrhs_max=B_NRHS, cg_tol=TOL, cg_maxit=MAXIT, chains=chains,
                  initial_guess=B_GUESS, batch_chains=1, batch_graph=0, **COUPLINGS)
    for t in range(2):
        if t == 1:
            torch.cuda.nvtx.range_push("batched")
        t0 = time.perf_counter()
        o = ctx.trajectory(phis, sigs, B_EPS, B_NLEAP, nrhs=B_NRHS, precond=False, seed=args.seed, counter=t,
                           check=False)
        torch.cuda.synchronize()
        if t == 1:
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_batched": t, "seconds": time.perf_counter() - t0,
                          "cg_iterations_per_chain": float(np.mean(o["cg_iterations"])), "status": o["status"]}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clock-log", default=None, help="directory for the raw nvidia-smi clock samples")
    ap.add_argument("--profile-solve", type=int, default=0,
                    help="run only a capture-sized sample: one solve cut at this many iterations")
    ap.add_argument("--pcg", action="store_true",
                    help="with --profile-solve: the preconditioned CG (the preconditioner's passes) instead")
    ap.add_argument("--profile-trajectory", action="store_true",
                    help="run only two trajectories of the workload, the second inside an NVTX range")
    ap.add_argument("--profile-matvec", type=int, default=0,
                    help="run only this many launches of the fused A kernel (the roofline kernel)")
    ap.add_argument("--profile-force", action="store_true",
                    help="run only one force evaluation of the workload (for a capture of the FP64 kernels)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="run only two trajectories of the batched configuration, the second inside an NVTX range")
    ap.add_argument("--config", choices=["largest", "batched64"], default="largest",
                    help="largest: the 80x80x160 chain (default); batched64: 64 uneven chains in batched launches")
    args = ap.parse_args()
    global CLOCK_LOG_DIR
    CLOCK_LOG_DIR = args.clock_log
    if args.profile_batched:
        run_profile_batched(args)
    elif args.config == "batched64":
        run_batched_bench(args)
    elif args.profile_force:
        run_profile_force(args)
    elif args.profile_trajectory:
        run_profile_trajectory(args)
    elif args.profile_matvec:
        run_profile_matvec(args)
    elif args.profile_solve:
        run_profile_solve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
