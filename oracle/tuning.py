"""Warm-up auto-tuning, plainly (Section "Online HMC hyperparameter tuning").

Step size, Eq. (acc_ineq): alpha(eps) is the mean acceptance probability min(1, e^{-dH}) of
single-step proposals (n_leap = 1) of size eps, estimated over a window of recent proposals,
alternating sizes eps and eps/2 from the current chain state; eps grows by a factor when
alpha(eps/2)^2 <= 2 alpha(eps) holds and shrinks by the same factor otherwise. (Reading: the
printed form (1 - alpha(eps/2))^2 <= 2 (1 - alpha(eps)) holds for any acceptance curve that
falls with eps; the passage itself compares the probability of accepting two half steps,
alpha(eps/2)^2, with that of one full step at half the cost, 2 alpha(eps).) When no proposal
of size eps is accepted (alpha(eps) = 0) the comparison is vacuous and eps shrinks: the rule is
to take eps as large as possible without losing the acceptance.

Trajectory length, Eq. (ESJD): ESJD(n) = < (phi - phi')^T M (phi - phi') alpha > over proposals
with n_leap = n, M = Sigma^{-1} (so the norm is sum |F (phi' - phi)|^2 / sigma-hat); n_max is
the candidate with the largest ESJD.

Randomness is explicit: noise(t) returns (list of chi, z, u) for proposal t.
"""

import numpy as np

from . import hmc


def jump_norm2(sigma_hat, d):
    """(phi' - phi)^T M (phi' - phi) with M = Sigma^{-1} = F^{-1} diag(1/sigma-hat) F."""
    return float(np.sum(np.abs(hmc.fourier(d)) ** 2 / sigma_hat))


class Tuner:
    def __init__(self, p, phi, sigma_hat, noise, method="dense", tol=1e-12):
        self.p, self.phi, self.sigma_hat, self.noise = p, phi.copy(), sigma_hat, noise
        self.method, self.tol = method, tol
        self.t = 0

    def propose(self, eps, n_leap):
        chis, z, u = self.noise(self.t)
        self.t += 1
        out = hmc.trajectory(self.p, self.phi, self.sigma_hat, chis, z, u, eps, n_leap, self.method, self.tol)
        alpha = min(1.0, float(np.exp(-out["dH"]))) if np.isfinite(out["dH"]) else 0.0
        jump2 = jump_norm2(self.sigma_hat, out["phi_proposed"] - self.phi)
        self.phi = out["phi"]
        return alpha, jump2, out["dH"], out["accept"]

    def tune_eps(self, eps, rounds, window, grow=1.2):
        hist = []
        for _ in range(rounds):
            a_eps = np.mean([self.propose_pair(eps, k) for k in range(window)], axis=0)
            hist.append((eps, a_eps[0], a_eps[1]))
            eps = eps * grow if (a_eps[0] > 0.0 and a_eps[1] ** 2 <= 2.0 * a_eps[0]) else eps / grow
        return eps, hist

    def propose_pair(self, eps, _k):
        a1 = self.propose(eps, 1)[0]
        a2 = self.propose(0.5 * eps, 1)[0]
        return a1, a2

    def tune_nmax(self, eps, candidates, per_candidate):
        esjd = {}
        for n in candidates:
            vals = []
            for _ in range(per_candidate):
                alpha, jump2, _, _ = self.propose(eps, n)
                vals.append(jump2 * alpha)
            esjd[n] = float(np.mean(vals))
        return max(candidates, key=lambda n: esjd[n]), esjd
