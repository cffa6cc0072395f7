"""Observables on the GPU (Section "Estimation of observables").

Fermionic: ``hmc.Context.green_estimate`` (libhmc's green_estimate) gives the randomized
diagonal estimate of F~^* D^{-1} F~ from Rademacher probes; ``rademacher_probes`` draws them.
Bosonic: ``SdwSusceptibility`` below.

``SdwSusceptibility`` accumulates Eq. (SDWsus), chi(omega, q) = < |F phi|^2 > dtau summed over the
three components, with the library's Fourier accumulation (metric_apply, HMC_METRIC_ACCUM):
one unitary 3-D FFT per sample, no host round trip.
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

    def add(self, phi):
        self.ctx.metric(METRIC_ACCUM, self.ones, phi, out=self.acc, chain=self.chain)
        self.n += 1

    def value(self):
        """chi as a (Nt, L, L) float64 tensor indexed [n_tau, m_y, m_x]."""
        dtau = self.ctx.params.dtau
        return self.acc.sum(dim=0) * (dtau / max(self.n, 1))
