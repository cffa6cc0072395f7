"""Preconditioner speedup in the shape of Supplementary Note 5 ("Preconditioner performance").

The paper fixes N_tau = 100 and reports, against the lattice extent L, the average speedup that
the preconditioner P of Eq. (26) gives the CG solve of D D^dagger x = b, in CG iterations and in
wall-clock time; a second figure repeats it at N_tau = 50 for several Trotter steps dtau. Model
parameters: u = 0, g = 0.7 sqrt(2), c = 3, nesting v_2, r = 1.26 (``presets.paper_nesting(2)``).

Reading: the paper averages over the configurations of an HMC run. Here each point averages over
seeded configurations drawn from the free-boson Gaussian with the same r and dtau (the
benchmark's input recipe), which is what a thermalised g = 0, u = 0 configuration looks like.
Solves are the library's complex64 CG with FP64 reliable updates, stopped at the FP64 true
residual tol; both arms solve the same right-hand sides.

Run: ``python -m paper_2204_14241_gb300.experiments [--quick]`` (prints one JSON line per point).

``precision_report`` (``--precision``) measures the error of the mixed-precision solver against
the FP64 one on the 20 x 20 x 40 chain: S_PF, force, dH and phi' per trajectory.
"""

import argparse
import json
import math
import time

import numpy as np


def _field(seed, L, Nt, kw):
    from . import inputs as I
    kt = 2.0 / (kw["c"] ** 2 * kw["dtau"] ** 2)
    return I.smooth_field(seed, L, Nt, kw["r"], kt) / math.sqrt(kw["dtau"])


def precond_point(L, Nt, dtau=0.1, n_cfg=3, nrhs=1, tol=1e-10, nesting=2, seed=0):
    """Mean CG iterations and seconds per solve without and with P at one (L, Nt, dtau)."""
    import torch
    from . import inputs as I
    from .hmc import Context
    from .presets import paper_nesting
    kw = paper_nesting(nesting)
    kw["dtau"] = dtau
    ctx = Context(L, Nt, solver="mixed", nrhs_max=nrhs, cg_tol=tol, cg_maxit=200000, **kw)
    it = {False: [], True: []}
    sec = {False: [], True: []}
    for c in range(n_cfg + 1):   # configuration 0 warms the context up and is not counted
        phi = torch.from_numpy(_field(seed * 1000 + c, L, Nt, kw)).cuda()
        b = torch.from_numpy(I.fermion_noise(seed * 1000 + 500 + c, nrhs, L, Nt)).cuda()
        for precond in (False, True):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = ctx.cg_solve(phi, b, precond=precond)
            torch.cuda.synchronize()
            if c > 0:
                it[precond].append(st["iterations"])
                sec[precond].append(time.perf_counter() - t0)
    ctx.close()
    out = {"L": L, "Nt": Nt, "dtau": dtau, "configs": n_cfg,
           "cg_iterations": float(np.mean(it[False])), "pcg_iterations": float(np.mean(it[True])),
           "cg_seconds": float(np.mean(sec[False])), "pcg_seconds": float(np.mean(sec[True]))}
    out["speedup_iterations"] = out["cg_iterations"] / out["pcg_iterations"]
    out["speedup_time"] = out["cg_seconds"] / out["pcg_seconds"]
    return out


def precision_report(L=20, Nt=40, n_traj=100, n_leap=20, eps=0.05, nrhs=1, tol=1e-10, seed=7, g=1.0):
    """Mixed precision against FP64 on one chain (the 20 x 20 x 40 single-chain configuration):
    complex64 CG with FP64 reliable updates against complex128 CG, both preconditioned and
    stopped at the FP64 true residual tol, on identical Philox noise.

    Each trajectory starts both solver modes from the same phi (the FP64 chain's state, which the
    chain then continues from), so the errors are per trajectory and do not compound. Per
    trajectory: relative error of S_PF at the end, |dH_mixed - dH_fp64|, relative error of phi'
    (max entry), and of the force F = -dS/dphi evaluated at the starting phi with the
    pseudofermions varphi = D chi of that trajectory's noise. Returns a dict of maxima and means
    plus the per-trajectory lists."""
    import torch
    from . import inputs as I
    from .hmc import Context
    kw = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=g, r=0.5, u=1.0, c=3.0)
    ctx = {m: Context(L, Nt, solver=m, nrhs_max=nrhs, cg_tol=tol, **kw) for m in ("fp64", "mixed")}
    phi = torch.from_numpy(I.gaussian_field(seed, L, Nt)).cuda()
    sig = torch.ones_like(phi)
    rows = []
    for t in range(n_traj):
        chi = ctx["fp64"].philox_normal(seed, 1_000_000 + t, nrhs * Nt * L * L * 4, complex_out=True)
        chi = chi.reshape(nrhs, Nt, L, L, 2, 2)
        pf = ctx["fp64"].apply_M(phi, chi)
        F = {m: ctx[m].force(phi, pf, include_boson=True, precond=True)[0] for m in ctx}
        res = {}
        for m in ctx:
            ph = phi.clone()
            o = ctx[m].trajectory([ph], [sig], eps, n_leap, nrhs=nrhs, precond=True, seed=seed, counter=t,
                                  check=False)
            res[m] = (ph, o)
        (p64, o64), (p32, o32) = res["fp64"], res["mixed"]
        e64, e32 = o64["energies"][0], o32["energies"][0]
        rows.append({
            "dH_fp64": o64["dH"][0], "dH_err": abs(o32["dH"][0] - o64["dH"][0]),
            "S_pf_rel_err": abs(e32[5] - e64[5]) / abs(e64[5]),
            "force_rel_err": float((F["mixed"] - F["fp64"]).abs().max() / F["fp64"].abs().max()),
            "phi_rel_err": float((p32 - p64).abs().max() / p64.abs().max()),
            "accepted": o64["accepted"][0], "same_accept": o32["accepted"][0] == o64["accepted"][0],
            "status": (o64["status"], o32["status"]),
        })
        phi = p64
    for c in ctx.values():
        c.close()
    keys = ("dH_err", "S_pf_rel_err", "force_rel_err", "phi_rel_err")
    out = {"L": L, "Nt": Nt, "n_traj": n_traj, "n_leap": n_leap, "eps": eps, "tol": tol, "nrhs": nrhs,
           "accept_rate": float(np.mean([r["accepted"] for r in rows])),
           "accept_agree": all(r["same_accept"] for r in rows)}
    for k in keys:
        v = [r[k] for r in rows]
        out[k + "_max"] = float(np.max(v))
        out[k + "_mean"] = float(np.mean(v))
    out["rows"] = rows
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="two lattice sizes per sweep")
    ap.add_argument("--configs", type=int, default=3)
    ap.add_argument("--precision", action="store_true",
                    help="mixed vs FP64 on the 20 x 20 x 40 chain (100 trajectories) instead of the speedup sweep")
    ap.add_argument("--tol", type=float, default=1e-10, help="solver tolerance of the precision report")
    ap.add_argument("--trajectories", type=int, default=100)
    args = ap.parse_args()
    if args.precision:
        r = precision_report(n_traj=args.trajectories, tol=args.tol)
        print(json.dumps({k: v for k, v in r.items() if k != "rows"}), flush=True)
        return
    Ls = (8, 16) if args.quick else (8, 12, 16, 20, 24, 32, 40)
    for L in Ls:   # N_tau = 100, dtau = 0.1
        print(json.dumps(precond_point(L, 100, 0.1, args.configs)), flush=True)
    for dtau in (0.05, 0.1, 0.2):   # N_tau = 50
        for L in ((8, 16) if args.quick else (8, 16, 24, 32)):
            print(json.dumps(precond_point(L, 50, dtau, args.configs)), flush=True)


if __name__ == "__main__":
    main()
