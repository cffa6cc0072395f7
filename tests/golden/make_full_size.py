"""Writes full_size_80x80x160.json: oracle values for the largest configuration (80 x 80 x 160,
dtau = 0.1, Yukawa coupling 1), computed by the FP64 oracle alone on seeded inputs from
paper_2204_14241_gb300.inputs (draws and layouts only).

Two cases, one pseudofermion right-hand side each (the oracle's preconditioned CG at this size
takes about two minutes per solve on one core):
* force: F = -d(S_B + S_PF)/dphi and S_PF at phi (Eq. hamiltonseq with S_PF of Eq. Z with pfs),
  varphi a standard complex Gaussian vector; F sampled at 512 seeded entries;
* trajectory: heatbath varphi = D chi, momentum from z, two leapfrog steps of eps = 0.01
  (three force evaluations), energies, dH and the proposed phi' sampled at the same entries
  (Section "HMC", Eq. hmc Hamiltonian).
The field is an ordered configuration: the mean-field amplitude 2.8 along component 3 (the
minimum over a uniform amplitude of S_B - 8 log det(D D^dagger) for eight right-hand sides)
plus a free-boson Gaussian field. sigma-hat is the free-boson spectrum.

Run from the repository root: python tests/golden/make_full_size.py
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.model import Params  # noqa: E402
from oracle import hmc as ohmc  # noqa: E402
from paper_2204_14241_gb300 import inputs as I  # noqa: E402

L, NT = 80, 160
COUPLINGS = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5, u=1.0, c=3.0)
KT = 2.0 / (COUPLINGS["c"] ** 2 * COUPLINGS["dtau"] ** 2)
AMP = 2.8
SEEDS = dict(phi=801, pf=802, chi=803, z=804, samples=805)
EPS, NLEAP, U, TOL = 0.01, 2, 0.5, 1e-12
NSAMP = 512


def inputs():
    """Library-layout inputs of both cases (shared with the GPU test)."""
    dt = COUPLINGS["dtau"]
    phi = I.ordered_field(SEEDS["phi"], L, NT, COUPLINGS["r"], KT, 1.0 / np.sqrt(dt), AMP)
    sig = np.broadcast_to(I.spectrum(L, NT, COUPLINGS["r"], KT)[None] / dt, (3, NT, L, L)).copy()
    pf = I.fermion_noise(SEEDS["pf"], 1, L, NT)
    chi = I.fermion_noise(SEEDS["chi"], 1, L, NT)
    z = I.gaussian_field(SEEDS["z"], L, NT)
    idx = I.rng(SEEDS["samples"]).choice(3 * NT * L * L, size=NSAMP, replace=False)
    return phi, sig, pf, chi, z, np.sort(idx)


def main():
    phi, sig, pf, chi, z, idx = inputs()
    P = Params(L=L, Nt=NT, **COUPLINGS)
    out = {"L": L, "Nt": NT, "couplings": COUPLINGS, "amp": AMP, "seeds": SEEDS, "eps": EPS, "n_leap": NLEAP,
           "u": U, "oracle_tol": TOL, "indices": [int(i) for i in idx]}
    t0 = time.time()
    F, spf, iters = ohmc.force(P, I.to_paper_boson(phi), [I.to_paper_fermion(pf[0])], method="pcg", tol=TOL)
    Fl = I.from_paper_boson(F).ravel()
    out["force"] = {"S_pf": spf, "F_samples": [float(Fl[i]) for i in idx], "F_max_abs": float(np.abs(F).max()),
                    "pcg_iterations": iters, "seconds": time.time() - t0}
    print("force done", out["force"]["seconds"], iters, flush=True)
    t0 = time.time()
    tr = ohmc.trajectory(P, I.to_paper_boson(phi), I.to_paper_boson(sig), [I.to_paper_fermion(chi[0])],
                         I.to_paper_boson(z), U, EPS, NLEAP, method="pcg", tol=TOL)
    php = I.from_paper_boson(tr["phi_proposed"]).ravel()
    out["trajectory"] = {"dH": tr["dH"], "accept": tr["accept"], "kinetic": list(tr["kinetic"]),
                         "S_B": list(tr["S_B"]), "S_PF": list(tr["S_PF"]),
                         "phi_samples": [float(php[i]) for i in idx], "phi_max_abs": float(np.abs(php).max()),
                         "pcg_iterations": tr["cg_iters"], "seconds": time.time() - t0}
    print("trajectory done", out["trajectory"]["seconds"], tr["dH"], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_80x80x160.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
