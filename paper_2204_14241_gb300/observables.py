"""Observables on the GPU (Section "Estimation of observables").

Fermionic: ``hmc.Context.green_estimate`` (libhmc's green_estimate) gives the randomized
diagonal estimate of F~^* D^{-1} F~ from Rademacher probes; ``rademacher_probes`` draws them.
Bosonic: ``SdwSusceptibility`` below, ``binder_cumulant`` and ``tau_int``.

``SdwSusceptibility`` accumulates Eq. (SDWsus), chi(omega, q) = < |F phi|^2 > dtau summed over the
three components, with the library's Fourier accumulation (metric_apply, HMC_METRIC_ACCUM):
one unitary 3-D FFT per sample. It also keeps the per-sample series of chi(0, 0) and of
|Phi|^2 = V sum_a phi-hat_a(0, 0)^2 (Phi = the field summed over the lattice), read from the
accumulator's zero mode (three doubles per sample).

``binder_cumulant`` (Supplementary Note 1): B_c = 1 - 3 <|Phi|^4> / (5 <|Phi|^2>^2); 0 for a
Gaussian order parameter, 0.4 for one of fixed length.

``tau_int`` (Supplementary Note 6, tau_int of chi(0, 0)): the estimator is not printed; reading:
tau_int = 1 + 2 sum_{t <= W} rho(t), rho from the FFT of the centred series, window W the
smallest with W >= c tau_int(W) (Sokal, c = 5); 1 for independent samples.
"""

import numpy as np
import torch

from .hmc import METRIC_ACCUM


def rademacher_probes(seed, K, L, Nt, device="cuda"):
    """K vectors with independent +-1 entries (complex128, imaginary part 0), fermion layout."""
    v = np.random.default_rng(seed).choice([-1.0, 1.0], size=(K, Nt, L, L, 2, 2)).astype(np.complex128)
    return torch.from_numpy(v).to(device)


class SdwSusceptibility:
    def __init__(self, ctx, chain=0):
        L, Nt = ctx.dims(chain)
        self.ctx, self.chain = ctx, chain
        self.acc = torch.zeros((3, Nt, L, L), dtype=torch.float64, device=ctx.device)
        self.ones = torch.ones_like(self.acc)
        self.n = 0
        self.volume = Nt * L * L
        self.phi2 = []    # |Phi|^2 per sample
        self.chi00 = []   # chi(0, 0) per sample

    def add(self, phi):
        before = self.acc[:, 0, 0, 0].clone()
        self.ctx.metric(METRIC_ACCUM, self.ones, phi, out=self.acc, chain=self.chain)
        zero = float((self.acc[:, 0, 0, 0] - before).sum().item())   # sum_a phi-hat_a(0, 0)^2
        self.phi2.append(zero * self.volume)
        self.chi00.append(zero * self.ctx.params.dtau)
        self.n += 1

    def value(self):
        """chi as a (Nt, L, L) float64 tensor indexed [n_tau, m_y, m_x]."""
        dtau = self.ctx.params.dtau
        return self.acc.sum(dim=0) * (dtau / max(self.n, 1))


def binder_cumulant(phi2):
    """B_c from the per-sample |Phi|^2 series."""
    m2 = np.asarray(phi2, dtype=float)
    return float(1.0 - 3.0 * np.mean(m2 * m2) / (5.0 * np.mean(m2) ** 2))


def tau_int(series, c=5.0):
    """Integrated autocorrelation time, automatic window (module header)."""
    x = np.asarray(series, dtype=float)
    n = len(x)
    d = x - x.mean()
    f = np.fft.rfft(d, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    rho = acf / acf[0]
    tau = 1.0 + 2.0 * np.cumsum(rho[1:])
    W = np.arange(1, n)
    ok = np.nonzero(W >= c * tau)[0]
    return float(tau[ok[0]] if len(ok) else tau[-1])
