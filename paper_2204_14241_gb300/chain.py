"""A Markov chain of libhmc trajectories with per-trajectory JSONL records and checkpoint/resume.

Every trajectory draws its noise from the library's Philox4x32-10 stream with key ``seed`` and
counter ``index`` (the trajectory's position in the chain), and starts its force solves afresh, so
the state (phi, sigma-hat, eps, n_leap or n_max, seed, index) determines the rest of the chain bit
for bit: a chain saved after n trajectories and resumed in a new process produces the same fields
and records as one that ran straight through.

Trajectory length: a fixed ``n_leap``, or, when ``n_max`` is set, n_leap ~ U{1 .. n_max} drawn
from (jitter_seed, index) as in Section "Online HMC hyperparameter tuning" (Eq. ESJD).

Each ``step`` appends one JSON line to ``log`` (a path or an open text file), with dH, the
acceptance, the energies, the iterations and final true residual of every force solve, the FP64
reliable updates and the per-phase GPU times of the trajectory (hmc_trajectory_stats).
"""

import json

import numpy as np
import torch

from .tuning import uniform_jitter

ENERGY_KEYS = ("kinetic_start", "S_B_start", "S_PF_start", "kinetic_end", "S_B_end", "S_PF_end")


class Chain:
    def __init__(self, ctx, phi, sigma, eps, n_leap=None, nrhs=1, precond=True, seed=0, index=0, n_max=None,
                 jitter_seed=None, log=None, accepted=0):
        if (n_leap is None) == (n_max is None):
            raise ValueError("give exactly one of n_leap and n_max")
        self.ctx, self.phi, self.sigma = ctx, phi, sigma
        self.eps, self.n_leap, self.n_max = float(eps), n_leap, n_max
        self.nrhs, self.precond, self.seed = int(nrhs), bool(precond), int(seed)
        self.index, self.accepted = int(index), int(accepted)
        self.jitter_seed = int(seed if jitter_seed is None else jitter_seed)
        self._jitter = uniform_jitter(self.jitter_seed)
        self.log = log

    def trajectory_length(self, index):
        return self.n_leap if self.n_max is None else self._jitter(index, self.n_max)

    def step(self):
        """One HMC update; returns (and logs) its record."""
        n = self.trajectory_length(self.index)
        o = self.ctx.trajectory([self.phi], [self.sigma], self.eps, n, nrhs=self.nrhs, precond=self.precond,
                                seed=self.seed, counter=self.index, check=False)
        rec = {"index": self.index, "status": o["status"], "dH": o["dH"][0], "accepted": bool(o["accepted"][0]),
               "eps": self.eps, "n_leap": n, "energies": dict(zip(ENERGY_KEYS, o["energies"][0])),
               "cg_iterations": o["cg_iterations"][0], "max_true_resid": o["max_true_resid"][0]}
        if o["status"] == 0:
            st = self.ctx.trajectory_stats(0)
            rec.update({"solve_iterations": st["iterations"], "solve_true_resid": st["true_resid"],
                        "reliable_updates": st["reliable_updates"], "phase_ms": st["phase_ms"]})
        self.index += 1
        self.accepted += int(rec["accepted"])
        self._write(rec)
        return rec

    def run(self, n):
        return [self.step() for _ in range(n)]

    def _write(self, rec):
        if self.log is None:
            return
        line = json.dumps(rec) + "\n"
        if hasattr(self.log, "write"):
            self.log.write(line)
            self.log.flush()
        else:
            with open(self.log, "a") as f:
                f.write(line)

    # ---- checkpoint -----------------------------------------------------------------------------
    def state_dict(self):
        return {"phi": self.phi.detach().cpu().numpy(), "sigma": self.sigma.detach().cpu().numpy(),
                "eps": self.eps, "n_leap": -1 if self.n_leap is None else int(self.n_leap),
                "n_max": -1 if self.n_max is None else int(self.n_max), "nrhs": self.nrhs,
                "precond": int(self.precond), "seed": self.seed, "jitter_seed": self.jitter_seed,
                "index": self.index, "accepted": self.accepted}

    def save(self, path):
        sd = self.state_dict()
        np.savez(path, **{k: np.asarray(v) for k, v in sd.items()})

    @classmethod
    def load(cls, path, ctx, log=None, device=None):
        z = np.load(path)
        dev = torch.device(device) if device is not None else getattr(ctx, "device", torch.device("cuda"))
        n_leap, n_max = int(z["n_leap"]), int(z["n_max"])
        return cls(ctx, torch.from_numpy(z["phi"]).to(dev), torch.from_numpy(z["sigma"]).to(dev), float(z["eps"]),
                   n_leap=None if n_leap < 0 else n_leap, nrhs=int(z["nrhs"]), precond=bool(int(z["precond"])),
                   seed=int(z["seed"]), index=int(z["index"]), n_max=None if n_max < 0 else n_max,
                   jitter_seed=int(z["jitter_seed"]), log=log, accepted=int(z["accepted"]))
