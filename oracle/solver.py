"""Solving A eta = varphi, A = D D^dagger (Eq. linsys), plainly.

* ``dense_solve``: the exact solution through numpy's dense solver (tiny lattices).
* ``cg``: the conjugate-gradient method (Section "Solving the linear system") in its
  textbook form, zero initial guess, stopping when the recursive residual norm drops
  below tol * ||b||; the true residual is reported.
* ``pcg``: the same with the preconditioner P = (K K^dagger)^{-1} of Eq. (precon),
  applied as P = F~ P-hat F~^* with the twisted DFT F~ = T F of Eq. (twist).

Readings (Section "Choice of preconditioner"):
* The twist printed as e^{pi i tau} cannot map periodic to antiperiodic fields; the
  operator that does is T = diag(e^{i pi tau / Nt}).
* "P-hat = K-hat K-hat^dagger" contradicts P = (K K^dagger)^{-1}; the symbol consistent
  with P = (K K^dagger)^{-1} is P-hat = 1 / |K-hat|^2.
* F is the unitary DFT over (tau, x, y) whose columns are e^{+2 pi i (n tau/Nt + m.r/L)};
  F^* is numpy's forward FFT with norm="ortho".
"""

import numpy as np

from .model import Params
from . import fermion


def vdot(a, b):
    """<a, b> = sum conj(a) b over all entries."""
    return np.vdot(a.ravel(), b.ravel())


def dense_solve(p: Params, phi, b):
    """eta = A^{-1} b with A = D D^dagger built densely."""
    D = fermion.dense_D(p, phi)
    A = D @ D.conj().T
    return np.linalg.solve(A, b.ravel()).reshape(b.shape)


def cg(p: Params, phi, b, tol=1e-12, maxit=100000):
    """Conjugate gradient on A x = b. Returns (x, iterations, true relative residual)."""
    bnorm = np.sqrt(vdot(b, b).real)
    x = np.zeros_like(b)
    r = b.copy()
    pdir = r.copy()
    rr = vdot(r, r).real
    it = 0
    while np.sqrt(rr) > tol * bnorm and it < maxit:
        Ap = fermion.apply_A(p, phi, pdir)
        alpha = rr / vdot(pdir, Ap).real
        x = x + alpha * pdir
        r = r - alpha * Ap
        rr_new = vdot(r, r).real
        pdir = r + (rr_new / rr) * pdir
        rr = rr_new
        it += 1
    res = b - fermion.apply_A(p, phi, x)
    return x, it, float(np.sqrt(vdot(res, res).real) / bnorm)


def twist(p: Params):
    """Diagonal of T: e^{i pi tau / Nt} on the tau axis, broadcast over (alpha, s, tau, x, y)."""
    return np.exp(1j * np.pi * np.arange(p.Nt) / p.Nt)[None, None, :, None, None]


def precond_symbol(p: Params):
    """P-hat = 1 / |K-hat|^2 per (alpha, n, m_x, m_y), broadcast over spin."""
    kh = fermion.free_symbol(p)
    return (1.0 / np.abs(kh) ** 2)[:, None]


def apply_precond(p: Params, v):
    """P v = F~ P-hat F~^* v with F~ = T F (Eqs. twist, Kdiag, precon)."""
    T = twist(p)
    vh = np.fft.fftn(np.conj(T) * v, axes=(2, 3, 4), norm="ortho")   # F~^* v
    return T * np.fft.ifftn(precond_symbol(p) * vh, axes=(2, 3, 4), norm="ortho")


def pcg(p: Params, phi, b, tol=1e-12, maxit=100000):
    """Preconditioned CG with z = P r; stops on the unpreconditioned recursive residual."""
    bnorm = np.sqrt(vdot(b, b).real)
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_precond(p, r)
    pdir = z.copy()
    rz = vdot(r, z).real
    it = 0
    while np.sqrt(vdot(r, r).real) > tol * bnorm and it < maxit:
        Ap = fermion.apply_A(p, phi, pdir)
        alpha = rz / vdot(pdir, Ap).real
        x = x + alpha * pdir
        r = r - alpha * Ap
        z = apply_precond(p, r)
        rz_new = vdot(r, z).real
        pdir = z + (rz_new / rz) * pdir
        rz = rz_new
        it += 1
    res = b - fermion.apply_A(p, phi, x)
    return x, it, float(np.sqrt(vdot(res, res).real) / bnorm)
