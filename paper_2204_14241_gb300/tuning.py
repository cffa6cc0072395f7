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
* Metric (Eq. covest): sigma-hat <- mean over a batch of samples of |F phi|^2, or (centered)
  the batch covariance mean |F phi|^2 - |F phi-bar|^2 about the batch mean phi-bar. Reading:
  Sigma_true = <phi phi^T> is the covariance of a target whose mean vanishes by O(3) symmetry;
  a warm-up batch of an ordered chain keeps its condensate, which the uncentered moment books on
  the zero mode as a fluctuation of variance V |phi-bar|^2; the centered estimate equals
  Eq. (covest) when the batch mean vanishes.
* A proposal that fails (non-finite energy, solver failure) counts as alpha = 0; when alpha(eps)
  is 0 the inequality is vacuous and eps shrinks.
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
                                    precond=self.precond, seed=self.seed, counter=self.t, check=False)
        else:
            chi, z, u = nz
            o = self.ctx.trajectory([self.phi], [self.sigma], eps, n_leap, nrhs=self.nrhs,
                                    precond=self.precond, chi=[chi], z=[z], u=[u], check=False)
        self.t += 1
        dH = o["dH"][0]
        if o["status"] != 0 or not math.isfinite(dH):
            alpha = 0.0   # the library restored phi
        else:
            alpha = 1.0 if dH <= 0 else math.exp(-dH)
        self.log.append((eps, n_leap, dH, o["accepted"][0]))
        return alpha, o["jump2"][0], dH, o["accepted"][0]

    def tune_eps(self, eps, rounds, window, grow=1.2, stop_after_turns=None):
        """Eq. (acc_ineq); returns the final eps and the history of (eps, a_eps, a_half). With
        stop_after_turns = n the rounds end once eps has changed direction n times (it then
        oscillates around the largest step the inequality admits) and the step returned is the
        last one for which the inequality held."""
        hist = []
        turns, last, last_ok = 0, 0, None
        for _ in range(rounds):
            a1 = a2 = 0.0
            for _ in range(window):
                a1 += self.propose(eps, 1)[0]
                a2 += self.propose(0.5 * eps, 1)[0]
            a1, a2 = a1 / window, a2 / window
            hist.append((eps, a1, a2))
            up = a1 > 0.0 and a2 ** 2 <= 2.0 * a1
            if up:
                last_ok = eps
            eps = eps * grow if up else eps / grow
            d = 1 if up else -1
            if last and d != last:
                turns += 1
            last = d
            if stop_after_turns is not None and turns >= stop_after_turns:
                return (last_ok if last_ok is not None else eps), hist
        return eps, hist

    def stabilize_eps(self, eps, n_leap, max_tries=8, shrink=1.5, max_abs_dH=1.0):
        """Back eps off until a production-length trajectory (n_leap steps) integrates stably:
        Eq. (acc_ineq) judges single steps, and a step that single steps tolerate can still drive
        a long leapfrog trajectory unstable (non-finite energies or a solver failure). Each try is
        one full update; eps is divided by `shrink` until a try ends with status 0 and
        |dH| <= max_abs_dH. Returns (eps, list of (eps, dH, status))."""
        tries = []
        for _ in range(max_tries):
            alpha, _, dH, _ = self.propose(eps, n_leap)   # alpha = 0 when the update failed
            ok = math.isfinite(dH) and alpha > 0.0 and abs(dH) <= max_abs_dH
            tries.append((eps, dH, ok))
            if ok:
                return eps, tries
            eps /= shrink
        return eps, tries

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

    def estimate_sigma(self, eps, n_max, samples, jitter, centered=False):
        """Eq. (covest) over `samples` production updates (n_leap ~ U{1..n_max} via jitter(t))."""
        est = SigmaEstimator(self.ctx, self.phi, centered)
        for _ in range(samples):
            self.propose(eps, jitter(self.t, n_max))
            est.add(self.phi)
        return est.value()


class SigmaEstimator:
    """Running Eq. (covest): the library accumulates |F phi|^2 over the samples (METRIC_ACCUM);
    with centered=True the batch mean phi-bar is kept as well and |F phi-bar|^2 is subtracted."""

    def __init__(self, ctx, like, centered=False, chain=0):
        self.ctx, self.centered, self.chain = ctx, centered, chain
        self.acc = torch.zeros_like(like)
        self.sum = torch.zeros_like(like) if centered else None
        self.unused_sig = torch.ones_like(like)   # the accumulate op takes no metric
        self.n = 0

    def add(self, phi):
        self.ctx.metric(METRIC_ACCUM, self.unused_sig, phi, out=self.acc, chain=self.chain)
        if self.centered:
            self.sum.add_(phi)
        self.n += 1

    def value(self):
        m2 = self.acc / self.n
        if not self.centered:
            return m2
        mean = self.sum / self.n
        mm = self.ctx.metric(METRIC_ACCUM, self.unused_sig, mean, chain=self.chain)   # |F phi-bar|^2
        return m2 - mm


def uniform_jitter(seed):
    """n_leap ~ U{1 .. n_max}, reproducible per update index t."""
    def draw(t, n_max):
        g = torch.Generator().manual_seed(int(seed) * 1000003 + int(t))
        return int(torch.randint(1, n_max + 1, (1,), generator=g).item())
    return draw
