"""Pins for the oracle's warm-up tuner (Eqs. acc_ineq and ESJD) on a Gaussian target, where the
dynamics with the exact metric are harmonic with unit frequency in every Fourier mode:
* acceptance -> 1 as eps -> 0, so Eq. (acc_ineq) (read as alpha(eps/2)^2 <= 2 alpha(eps)) holds
  and eps grows from a small value; at eps = 1 a single step is accepted with probability ~0.16
  against ~0.86 for eps/2, the inequality fails and eps shrinks;
* the expected squared M-norm jump after time T = n eps is 2 (1 - cos T) per real mode
  (displacement phi0 (cos T - 1) + sigma pi0 sin T), so ESJD(n) peaks near n eps = pi."""

import numpy as np

from oracle.model import Params
from oracle import tuning


def gaussian_setup(L=4, Nt=4):
    p = Params(L=L, Nt=Nt, g=0.0, u=0.0)
    w = 2 * np.pi * np.arange(Nt) / Nt
    k = 2 * np.pi * np.arange(L) / L
    B = p.dtau * (2.0 / (p.c ** 2 * p.dtau ** 2) * (2 - 2 * np.cos(w))[:, None, None]
                  + (2 - 2 * np.cos(k))[None, :, None] + (2 - 2 * np.cos(k))[None, None, :] + p.r)
    sig = np.broadcast_to(1.0 / B, (3, Nt, L, L)).copy()
    rng = np.random.default_rng(0)
    # equilibrium draw: phi = F^-1(sigma^1/2 F z)
    z = rng.standard_normal((3, Nt, L, L))
    phi = np.fft.ifftn(np.fft.fftn(z, axes=(1, 2, 3), norm="ortho") * np.sqrt(sig), axes=(1, 2, 3),
                       norm="ortho").real
    return p, phi, sig


def noise_for(p, seed):
    def noise(t):
        g = np.random.default_rng(seed * 100003 + t)
        return [], g.standard_normal((3, p.Nt, p.L, p.L)), g.random()
    return noise


def test_step_size_rule_directions():
    p, phi, sig = gaussian_setup()
    tu = tuning.Tuner(p, phi, sig, noise_for(p, 1))
    eps, hist = tu.tune_eps(0.05, rounds=3, window=16)
    assert eps > 0.05 and all(h[1] > 0.99 for h in hist)
    tu = tuning.Tuner(p, phi, sig, noise_for(p, 2))
    eps, hist = tu.tune_eps(1.0, rounds=1, window=16)
    assert eps < 1.0 and hist[0][1] < 0.5 < hist[0][2]


def test_esjd_peaks_near_half_period():
    p, phi, sig = gaussian_setup()
    tu = tuning.Tuner(p, phi, sig, noise_for(p, 3))
    eps = 0.3
    n_max, esjd = tu.tune_nmax(eps, [2, 5, 10, 15, 20], per_candidate=30)
    nmodes = phi.size
    w_eff = 2 / eps * np.arcsin(eps / 2)        # leapfrog frequency of a unit oscillator
    for n, v in esjd.items():
        ref = nmodes * 2 * (1 - np.cos(w_eff * eps * n))   # unweighted; ESJD weights by alpha <= 1
        assert v < ref + 0.2 * nmodes, (n, v, ref)
    assert esjd[10] > 0.7 * nmodes * 2 * (1 - np.cos(w_eff * eps * 10))
    assert n_max == 10


def test_step_size_shrinks_when_nothing_is_accepted():
    # Eq. (acc_ineq) is vacuous when neither size is ever accepted (0 <= 0): eps must shrink.
    # A step far above the leapfrog stability limit of the Gaussian target (omega eps >> 2) gives
    # dH ~ exp(huge), never accepted.
    p, phi, sig = gaussian_setup()
    tu = tuning.Tuner(p, phi, sig, noise_for(p, 4))
    eps, hist = tu.tune_eps(40.0, rounds=2, window=4)
    assert all(h[1] == 0.0 and h[2] == 0.0 for h in hist)
    assert abs(eps - 40.0 / 1.2 ** 2) < 1e-12


def test_centered_metric_estimate_removes_the_batch_mean():
    # Samples phi_s = mu + Gaussian field with Fourier variance sigma: the centered estimate
    # approaches sigma on every mode (the mean enters only the zero mode, as V |mu|^2 in the
    # uncentered moment of Eq. covest); with mu = 0 the two estimates differ by |F phi-bar|^2,
    # which is O(sigma / S).
    from oracle import hmc
    p, _, sig = gaussian_setup(L=4, Nt=4)
    rng = np.random.default_rng(5)
    S = 4000
    mu = np.array([0.3, -0.2, 2.5])[:, None, None, None]
    samples = []
    for _ in range(S):
        z = rng.standard_normal(sig.shape)
        f = np.fft.ifftn(np.fft.fftn(z, axes=(1, 2, 3), norm="ortho") * np.sqrt(sig), axes=(1, 2, 3),
                         norm="ortho").real
        samples.append(f + mu)
    c = hmc.sigma_estimate_centered(samples)
    u = hmc.sigma_estimate(samples)
    V = sig[0].size
    assert np.abs(c / sig - 1).max() < 0.15
    assert abs(u[2, 0, 0, 0] - (sig[2, 0, 0, 0] + V * 2.5 ** 2)) < 0.05 * V * 2.5 ** 2
    zero = [s - mu for s in samples[:50]]
    assert np.abs(hmc.sigma_estimate_centered(zero) - hmc.sigma_estimate(zero)).max() < 5 * sig.max()
