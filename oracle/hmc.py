"""Pseudofermion HMC on phi (Section "HMC" and "Scale-invariant sampling").

One update (Gibbs alternation, Section "HMC"):
  1. heatbath: varphi = D(phi) chi with chi a standard complex Gaussian vector;
  2. momentum pi ~ N(0, M), M = Sigma^{-1}, Sigma = F diag(sigma-hat) F^* (Eq. covest ff.);
  3. leapfrog integration of Eq. (hamiltonseq) for the Hamiltonian of Eq. (hmc Hamiltonian)
     H = (1/2) pi^T M^{-1} pi + S_B(phi) + S_PF(phi, varphi);
  4. Metropolis: accept with probability min(1, e^{-(H' - H)}).
All random numbers (chi, z, u) are inputs, so the update is a deterministic function.

Readings (the paper is silent):
* "standard complex Gaussian": real and imaginary parts independent N(0, 1/2), so
  E|chi_i|^2 = 1 and S_PF at the start of a trajectory equals chi^dagger chi.
* F is the unitary DFT over (tau, x, y) applied per boson component (numpy fftn,
  norm="ortho"); sigma-hat is even in the wave vector (it is estimated from |F phi|^2
  of real fields), so Sigma = F^* diag(sigma-hat) F = F diag(sigma-hat) F^* is real
  symmetric. The momentum is drawn as pi = F^{-1}(sigma-hat^{-1/2} . F z) with z real
  N(0, 1): real, with covariance M. Kinetic energy (1/2) pi^T Sigma pi =
  (1/2) sum sigma-hat |F pi|^2; drift d phi/dt = Sigma pi = F^{-1}(sigma-hat . F pi).
* Leapfrog is kick(eps/2) - [drift(eps) - kick(eps)] x n_leap with the last kick eps/2,
  i.e. n_leap + 1 force evaluations.
* k pseudofermion right-hand sides: S_PF = sum_i varphi_i^dagger A^{-1} varphi_i (k = 1 is
  the paper's N_f = 2).
"""

import numpy as np

from .model import Params, stagger, pauli
from . import fermion, boson, solver

AXES = (1, 2, 3)


def heatbath(p: Params, phi, chi):
    """varphi = D(phi) chi (Section "HMC": exact draw from N(0, D D^dagger))."""
    return fermion.apply_D(p, phi, chi)


def solve(p: Params, phi, b, method="dense", tol=1e-12):
    """A^{-1} b by the chosen method; returns (x, iterations)."""
    if method == "dense":
        return solver.dense_solve(p, phi, b), 0
    if method == "cg":
        x, it, _ = solver.cg(p, phi, b, tol=tol)
        return x, it
    if method == "pcg":
        x, it, _ = solver.pcg(p, phi, b, tol=tol)
        return x, it
    raise ValueError(method)


def pseudofermion_action(p: Params, phi, varphis, method="dense", tol=1e-12):
    """S_PF = sum_i varphi_i^dagger (D D^dagger)^{-1} varphi_i (Eq. Z with pfs)."""
    s = 0.0
    for vp in varphis:
        x, _ = solve(p, phi, vp, method, tol)
        s += solver.vdot(vp, x).real
    return float(s)


def fermion_force(p: Params, X, Y):
    """-dS_PF/dphi_a(tau, r) for one right-hand side, given X = A^{-1} varphi and Y = D^dagger X.

    dS_PF = -X^dagger (dD D^dagger + D dD^dagger) X = -2 Re[X^dagger dD Y], and
    dD/dphi_a(tau, r) = dtau g eta(r) sigma^a (spin) x sigma^x (band) on site (tau, r)
    (Eq. D_formula), so the force is 2 dtau g eta Re[X^dagger (sigma^x x sigma^a) Y] per site.
    """
    eta = stagger(p)[None]
    sig = pauli()
    F = np.empty((3, p.Nt, p.L, p.L))
    for a in range(3):
        acc = np.zeros((p.Nt, p.L, p.L), dtype=complex)
        for alpha in range(2):
            for s in range(2):
                for sp in range(2):
                    if sig[a][s, sp] != 0:
                        acc += np.conj(X[alpha, s]) * sig[a][s, sp] * Y[1 - alpha, sp]
        F[a] = 2.0 * p.dtau * p.g * eta * acc.real
    return F


def force(p: Params, phi, varphis, method="dense", tol=1e-12, include_boson=True):
    """F = -d(S_B + S_PF)/dphi and S_PF = sum varphi^dagger X, solving A X = varphi per RHS."""
    F = -boson.grad(p, phi) if include_boson else np.zeros((3, p.Nt, p.L, p.L))
    s_pf = 0.0
    iters = []
    for vp in varphis:
        X, it = solve(p, phi, vp, method, tol)
        Y = fermion.apply_Ddag(p, phi, X)
        F += fermion_force(p, X, Y)
        s_pf += solver.vdot(vp, X).real
        iters.append(it)
    return F, float(s_pf), iters


def fourier(v):
    """Unitary DFT over (tau, x, y) per boson component."""
    return np.fft.fftn(v, axes=AXES, norm="ortho")


def inverse_fourier(vh):
    return np.fft.ifftn(vh, axes=AXES, norm="ortho")


def momentum(sigma_hat, z):
    """pi = F^{-1}(sigma-hat^{-1/2} . F z): pi ~ N(0, M) for z ~ N(0, 1) (Section "Online
    metric estimation"); real because sigma-hat is even."""
    return inverse_fourier(fourier(z) / np.sqrt(sigma_hat)).real


def kinetic(sigma_hat, pi):
    """(1/2) pi^T M^{-1} pi = (1/2) sum sigma-hat |F pi|^2 (Eq. hmc Hamiltonian)."""
    return float(0.5 * np.sum(sigma_hat * np.abs(fourier(pi)) ** 2))


def velocity(sigma_hat, pi):
    """d phi / dt = M^{-1} pi = F^{-1}(sigma-hat . F pi) (Eq. hamiltonseq)."""
    return inverse_fourier(sigma_hat * fourier(pi)).real


def leapfrog(p: Params, phi, pi, varphis, sigma_hat, eps, n_leap, method="dense", tol=1e-12):
    """Kick-drift-kick leapfrog; returns (phi', pi', S_PF(phi'), cg iteration list)."""
    phi = phi.copy()
    F, s_pf, iters = force(p, phi, varphis, method, tol)
    pi = pi + 0.5 * eps * F
    all_iters = [iters]
    for i in range(1, n_leap + 1):
        phi = phi + eps * velocity(sigma_hat, pi)
        F, s_pf, iters = force(p, phi, varphis, method, tol)
        all_iters.append(iters)
        pi = pi + (eps if i < n_leap else 0.5 * eps) * F
    return phi, pi, s_pf, all_iters


def trajectory(p: Params, phi, sigma_hat, chis, z, u, eps, n_leap, method="dense", tol=1e-12):
    """One Gibbs sweep with explicit noise (chi list, z, u). Returns a dict with the new
    phi, dH, the acceptance flag and the energy pieces."""
    varphis = [heatbath(p, phi, chi) for chi in chis]
    pi0 = momentum(sigma_hat, z)
    k0 = kinetic(sigma_hat, pi0)
    sb0 = boson.action(p, phi)
    spf0 = float(sum(solver.vdot(chi, chi).real for chi in chis))   # = varphi^dag A^-1 varphi
    phi1, pi1, spf1, iters = leapfrog(p, phi, pi0, varphis, sigma_hat, eps, n_leap, method, tol)
    k1 = kinetic(sigma_hat, pi1)
    sb1 = boson.action(p, phi1)
    dH = (k1 + sb1 + spf1) - (k0 + sb0 + spf0)
    accept = bool(u < np.exp(-dH))
    return {
        "phi": phi1 if accept else phi.copy(), "phi_proposed": phi1, "pi_final": pi1,
        "dH": float(dH), "accept": accept, "H0": k0 + sb0 + spf0, "H1": k1 + sb1 + spf1,
        "kinetic": (k0, k1), "S_B": (sb0, sb1), "S_PF": (spf0, spf1), "cg_iters": iters,
    }


def sigma_estimate_centered(samples):
    """Covariance of the batch about its own mean, per Fourier mode:
    sigma-hat = (1/S) sum_s |F phi_s|^2 - |F phi-bar|^2 with phi-bar the batch mean.

    Reading of Section "Online metric estimation": Sigma_true = <phi phi^T> is the covariance of
    the target, whose mean vanishes by O(3) symmetry, and the metric is to rescale the target to
    unit covariance. A warm-up batch of an ordered chain does not turn its condensate, so the
    uncentered moment of Eq. (covest) books the condensate V |phi-bar|^2 on the zero mode as a
    fluctuation; this estimate equals Eq. (covest) whenever the batch mean vanishes."""
    S = len(samples)
    mean = sum(samples) / S
    mh = fourier(mean)
    return sigma_estimate(samples) - (mh * np.conj(mh)).real


def sigma_estimate(samples):
    """Eq. (covest): sigma-hat = (1/S) sum_s F phi_s . conj(F phi_s)."""
    acc = None
    for phi in samples:
        ph = fourier(phi)
        term = (ph * np.conj(ph)).real
        acc = term if acc is None else acc + term
    return acc / len(samples)
