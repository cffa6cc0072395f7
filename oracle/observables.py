"""Bosonic observables (Section "Estimation of observables").

Eq. (SDWsus): chi(omega, q) = < |phi-hat(omega, q)|^2 > dtau, phi-hat = F phi with F the unitary
space-time DFT, summed over the three components (phi . phi); the expectation is the sample mean.
"""

import numpy as np


def sdw_susceptibility(samples, dtau):
    acc = None
    for phi in samples:
        ph = np.fft.fftn(phi, axes=(1, 2, 3), norm="ortho")
        term = np.sum(np.abs(ph) ** 2, axis=0)
        acc = term if acc is None else acc + term
    return acc * dtau / len(samples)
