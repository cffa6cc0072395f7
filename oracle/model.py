"""Parameters of the lattice spin-fermion model.

Section "Sign-problem-free UV completion", Eq. (sign-problem-free action): two bands
alpha in {x, y}, two spins, band-dependent nearest-neighbour hopping t_{alpha,r,r'},
chemical potential mu_alpha, boson mass r, quartic u, boson velocity c, Yukawa g.
Section "QMC path integral with fermions": L x L periodic lattice, Nt time slices of
width dtau (0.1 in the paper), fermions antiperiodic and the boson periodic in time.

Readings (the paper is silent or ambiguous):
* t_h[alpha], t_v[alpha] are the signed nearest-neighbour amplitudes along x and y
  for band alpha; the hop enters D as -dtau * t (Eq. D_formula).
* t2_h[alpha], t2_v[alpha] are the amplitudes of hops of distance two along x and y (zero by
  default): the paper's "next-nearest-neighbour" t~_{v,x} = -t~_{h,y} of the five nesting sets,
  read as the hop of distance two along each band's weak direction, because that reading gives
  the nesting parameters v_1 ... v_5 the paper prints for those sets (the nearest-neighbour
  reading gives Fermi lines crossing at ~88 degrees). They enter D like t.
* e^{i Q_AF . r} with Q_AF = (pi, pi) is (-1)^{x+y}; L must be even.
"""

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Params:
    L: int
    Nt: int
    dtau: float = 0.1
    t_h: tuple = (1.0, 0.5)   # hopping along x for bands (x, y)
    t_v: tuple = (0.5, 1.0)   # hopping along y for bands (x, y)
    mu: tuple = (-0.5, -0.5)  # chemical potential per band
    g: float = 1.0            # Yukawa coupling in D's on-site term
    r: float = 0.5            # boson mass term (r/2) phi^2
    u: float = 1.0            # quartic (u/4) phi^4
    c: float = 3.0            # boson velocity: (1/c^2) (d_tau phi)^2
    t2_h: tuple = (0.0, 0.0)  # hopping of distance two along x for bands (x, y)
    t2_v: tuple = (0.0, 0.0)  # hopping of distance two along y for bands (x, y)

    def __post_init__(self):
        if self.L < 2 or self.L % 2:
            raise ValueError("L must be even and >= 2 (Q_AF = (pi, pi) needs even L)")
        if self.Nt < 2:
            raise ValueError("Nt must be >= 2")

    @property
    def V(self):
        """Number of space-time sites Nt * L^2."""
        return self.Nt * self.L * self.L

    @property
    def n(self):
        """Dimension of D: 2 bands x 2 spins x Nt x L x L (Section QMC path integral)."""
        return 4 * self.V


def stagger(p: Params) -> np.ndarray:
    """e^{i Q_AF . (x, y)} = (-1)^{x+y} as an (L, L) array indexed [x, y]."""
    x = np.arange(p.L)
    return np.where((x[:, None] + x[None, :]) % 2 == 0, 1.0, -1.0)


def pauli():
    """Pauli matrices sigma^1, sigma^2, sigma^3 (spin) as 2x2 complex arrays."""
    s1 = np.array([[0, 1], [1, 0]], dtype=complex)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
    s3 = np.array([[1, 0], [0, -1]], dtype=complex)
    return s1, s2, s3
