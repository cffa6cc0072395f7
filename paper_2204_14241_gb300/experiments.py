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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="two lattice sizes per sweep")
    ap.add_argument("--configs", type=int, default=3)
    args = ap.parse_args()
    Ls = (8, 16) if args.quick else (8, 12, 16, 20, 24, 32, 40)
    for L in Ls:   # N_tau = 100, dtau = 0.1
        print(json.dumps(precond_point(L, 100, 0.1, args.configs)), flush=True)
    for dtau in (0.05, 0.1, 0.2):   # N_tau = 50
        for L in ((8, 16) if args.quick else (8, 16, 24, 32)):
            print(json.dumps(precond_point(L, 50, dtau, args.configs)), flush=True)


if __name__ == "__main__":
    main()
