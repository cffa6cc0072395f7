"""Bosonic observables (Section "Estimation of observables", Supplementary Notes 1 and 6).

Eq. (SDWsus): chi(omega, q) = < |phi-hat(omega, q)|^2 > dtau, phi-hat = F phi with F the unitary
space-time DFT, summed over the three components (phi . phi); the expectation is the sample mean.

Binder cumulant (Supplementary Note 1): B_c = 1 - 3 <|Phi|^4> / (5 <|Phi|^2>^2), Phi = sum over
(tau, x, y) of the three-component field phi; expectations are sample means.

Integrated autocorrelation time of a series (the paper's tau_int of chi(0, 0); the estimator is
not printed, reading): tau_int = 1 + 2 sum_{t=1}^{W} rho(t) with the sample autocorrelation rho
and the automatic window W = the smallest W with W >= c tau_int(W) (Sokal; c = 5), so that
independent samples give tau_int = 1.
"""

import numpy as np


def sdw_susceptibility(samples, dtau):
    acc = None
    for phi in samples:
        ph = np.fft.fftn(phi, axes=(1, 2, 3), norm="ortho")
        term = np.sum(np.abs(ph) ** 2, axis=0)
        acc = term if acc is None else acc + term
    return acc * dtau / len(samples)


def twisted_fourier(p, v, inverse):
    """F~ v = T F v (inverse = True: T times the inverse unitary DFT) or F~^* v = F^* (T^* v)
    over (tau, x, y), T = diag(e^{i pi tau / Nt}) (Eqs. twist, Kdiag)."""
    from .solver import twist
    T = twist(p)
    if inverse:
        return T * np.fft.ifftn(v, axes=(2, 3, 4), norm="ortho")
    return np.fft.fftn(np.conj(T) * v, axes=(2, 3, 4), norm="ortho")


def green_diagonal(p, phi, probes, method="dense", tol=1e-12):
    """Randomized diagonal estimator (Section "Fermionic observables"): diag(O) = E[v . O v]
    for Rademacher v, with O = F~^* D^{-1} F~ and D^{-1} = D^dagger (D D^dagger)^{-1}.
    probes: list of real +-1 arrays of fermion shape; returns the sample mean of v . O v."""
    from . import fermion, solver
    acc = None
    for v in probes:
        w = twisted_fourier(p, v.astype(complex), inverse=True)
        if method == "dense":
            u = solver.dense_solve(p, phi, w)
        else:
            u, _, _ = solver.pcg(p, phi, w, tol=tol)
        ov = twisted_fourier(p, fermion.apply_Ddag(p, phi, u), inverse=False)
        term = v * ov
        acc = term if acc is None else acc + term
    return acc / len(probes)


def binder_cumulant(samples):
    """B_c from a list of phi samples ([3][Nt][L][L] arrays)."""
    m2 = np.array([np.sum(np.sum(phi, axis=(1, 2, 3)) ** 2) for phi in samples])
    return 1.0 - 3.0 * np.mean(m2 ** 2) / (5.0 * np.mean(m2) ** 2)


def tau_int(series, c=5.0):
    """Integrated autocorrelation time with Sokal's automatic window (see the module header)."""
    x = np.asarray(series, dtype=float)
    n = len(x)
    d = x - x.mean()
    var = np.dot(d, d) / n
    tau = 1.0
    for W in range(1, n):
        rho = np.dot(d[:n - W], d[W:]) / (n * var)   # plain sum, one lag at a time
        tau += 2.0 * rho
        if W >= c * tau:
            break
    return tau
