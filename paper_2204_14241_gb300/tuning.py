"""Warm-up auto-tuning of the HMC hyperparameters (Section "Online HMC hyperparameter tuning"
and Section "Online metric estimation"), driving libhmc trajectories on the GPU.

* Step size (Eq. acc_ineq): from the current state, alternate single-step proposals
  (n_leap = 1) of size eps and eps / 2, average their acceptance probabilities
  alpha = min(1, exp(-dH)) over a window, then grow eps by ``grow`` if
  alpha(eps/2)^2 <= 2 alpha(eps) and shrink it by ``grow`` otherwise. Reading of the printed
  inequality (1 - alpha(eps/2))^2 <= 2 (1 - alpha(eps)), which holds for every acceptance curve
  that falls with eps and so never stops eps from growing: the passage describes its two
  sides as the probability of accepting two half steps and one full step, the full step
  costing half as many solves, i.e. alpha(eps/2)^2 against 2 alpha(eps).
* Trajectory length (Eq. ESJD): for each candidate n, run proposals with n_leap = n and average
  (phi' - phi)^T M (phi' - phi) * alpha (the library reports the proposal's M-norm jump,
  accepted or not); n_max is the maximiser. Production runs draw n_leap ~ U{1 .. n_max}.
* Metric (Eq. covest): sigma-hat <- mean over a batch of samples of |F phi|^2.
Every proposal is a full libhmc trajectory (heatbath, momentum, leapfrog, Metropolis), so the
chain keeps moving while the statistics are gathered.

Randomness: ``noise(t)`` returns the explicit (chi, z, u) for proposal t (GPU tensors and a
float), or None to use the library's Philox stream with counter t.
"""

import math

import torch

from .hmc import METRIC_ACCUM


class Tuner:
    def __init__(self, ctx, phi, sigma, nrhs=1, precond=True, seed=0, noise=None):
        self.ctx, self.phi, self.sigma = ctx, phi, sigma
        self.nrhs, self.precond, self.seed, self.noise = nrhs, precond, seed, noise
        self.t = 0
        self.log = []

    def propose(self, eps, n_leap):
        """One HMC update; returns (alpha, jump2, dH, accepted)."""
        nz = self.noise(self.t) if self.noise else None
        if nz is None:
            o = self.ctx.trajectory([self.phi], [self.sigma], eps, n_leap, nrhs=self.nrhs,
                                    precond=self.precond, seed=self.seed, counter=self.t)
        else:
            chi, z, u = nz
            o = self.ctx.trajectory([self.phi], [self.sigma], eps, n_leap, nrhs=self.nrhs,
                                    precond=self.precond, chi=[chi], z=[z], u=[u])
        self.t += 1
        dH = o["dH"][0]
        alpha = 1.0 if dH <= 0 else math.exp(-dH)
        self.log.append((eps, n_leap, dH, o["accepted"][0]))
        return alpha, o["jump2"][0], dH, o["accepted"][0]

    def tune_eps(self, eps, rounds, window, grow=1.2):
        """Eq. (acc_ineq); returns the final eps and the history of (eps, a_eps, a_half)."""
        hist = []
        for _ in range(rounds):
            a1 = a2 = 0.0
            for _ in range(window):
                a1 += self.propose(eps, 1)[0]
                a2 += self.propose(0.5 * eps, 1)[0]
            a1, a2 = a1 / window, a2 / window
            hist.append((eps, a1, a2))
            eps = eps * grow if a2 ** 2 <= 2.0 * a1 else eps / grow
        return eps, hist

    def tune_nmax(self, eps, candidates, per_candidate):
        """Eq. (ESJD); returns n_max and {n: ESJD(n)}."""
        esjd = {}
        for n in candidates:
            acc = 0.0
            for _ in range(per_candidate):
                alpha, jump2, _, _ = self.propose(eps, n)
                acc += jump2 * alpha
            esjd[n] = acc / per_candidate
        n_max = max(candidates, key=lambda n: esjd[n])
        return n_max, esjd

    def estimate_sigma(self, eps, n_max, samples, jitter):
        """Eq. (covest) over `samples` production updates (n_leap ~ U{1..n_max} via jitter(t))."""
        acc = torch.zeros_like(self.sigma)
        for _ in range(samples):
            self.propose(eps, jitter(self.t, n_max))
            self.ctx.metric(METRIC_ACCUM, self.sigma, self.phi, out=acc)
        return acc / samples


def uniform_jitter(seed):
    """n_leap ~ U{1 .. n_max}, reproducible per update index t."""
    def draw(t, n_max):
        g = torch.Generator().manual_seed(int(seed) * 1000003 + int(t))
        return int(torch.randint(1, n_max + 1, (1,), generator=g).item())
    return draw
