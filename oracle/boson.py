"""Lattice boson action S_B(phi) and its gradient.

The paper prints only the continuum form (Eq. sign-problem-free action, boson line):
    int dtau sum_r [ (1/c^2)(d_tau phi)^2 + (1/2)(grad phi)^2 + (r/2) phi^2 + (u/4)(phi^2)^2 ].
Reading used here (forward differences, periodic in tau and in space, Riemann sum in tau):
    S_B = dtau sum_{tau, r} [ (1/c^2) |phi(tau+1, r) - phi(tau, r)|^2 / dtau^2
                              + (1/2) sum_{d = x, y} |phi(tau, r + d) - phi(tau, r)|^2
                              + (r/2) |phi(tau, r)|^2 + (u/4) |phi(tau, r)|^4 ]
phi has shape (3, Nt, L, L) indexed [a, tau, x, y]; |.| is the O(3) norm.
"""

import numpy as np

from .model import Params


def action(p: Params, phi: np.ndarray) -> float:
    """S_B(phi) summed site by site from the reading above."""
    dt = p.dtau
    d_tau = np.roll(phi, -1, axis=1) - phi
    d_x = np.roll(phi, -1, axis=2) - phi
    d_y = np.roll(phi, -1, axis=3) - phi
    phi2 = np.sum(phi * phi, axis=0)
    dens = (np.sum(d_tau * d_tau, axis=0) / (p.c ** 2 * dt ** 2)
            + 0.5 * np.sum(d_x * d_x + d_y * d_y, axis=0)
            + 0.5 * p.r * phi2 + 0.25 * p.u * phi2 * phi2)
    return float(dt * np.sum(dens))


def grad(p: Params, phi: np.ndarray) -> np.ndarray:
    """dS_B/dphi_a(tau, r), differentiated term by term from ``action``."""
    dt = p.dtau
    lap_tau = 2 * phi - np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)
    lap_xy = (4 * phi - np.roll(phi, -1, axis=2) - np.roll(phi, 1, axis=2)
              - np.roll(phi, -1, axis=3) - np.roll(phi, 1, axis=3))
    phi2 = np.sum(phi * phi, axis=0)[None]
    return dt * (2.0 / (p.c ** 2 * dt ** 2) * lap_tau + lap_xy + p.r * phi + p.u * phi2 * phi)
