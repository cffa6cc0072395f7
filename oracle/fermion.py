"""The fermion matrix D(phi), its adjoint and the normal operator A = D D^dagger.

Eq. (D_formula): for row (alpha, s, tau, x, y) and column (alpha', s', tau', x', y'),

    D = delta_{alpha alpha'} delta_{s s'} { delta_{r r'} ( delta_{tau tau'} [-1 - dtau mu_alpha]
                                                       + delta_{tau+1, tau'} [1 - 2 delta_{tau, Nt-1}] )
                                         - delta_{tau tau'} dtau t_{alpha, r, r'} }
      + delta_{r r'} delta_{tau tau'} dtau g e^{i Q_AF . r} phi(tau, r) . sigma_{s s'} sigma^x_{alpha alpha'}

with tau + 1 taken modulo Nt (the -1 at the wrap makes the fermions antiperiodic) and
x, y periodic. sigma are the Pauli matrices on spin (the paper's "generators" with the
factor 1/2 absorbed into g); sigma^x acts on the band index.

Two implementations, cross-checked by the tests:
* ``dense_D`` writes the matrix entry by entry from the formula above (tiny lattices);
* ``apply_D`` / ``apply_Ddag`` / ``apply_A`` are the same operator written matrix-free
  with np.roll, for lattices too large to store D.
Vectors are complex arrays of shape (2, 2, Nt, L, L) indexed [alpha, s, tau, x, y];
the flattened row index of the dense matrix is the C-order flattening of that shape.
"""

import numpy as np

from .model import Params, stagger, pauli


def index(p: Params, alpha, s, tau, x, y):
    """Row/column index of (alpha, s, tau, x, y) in the dense D (C-order of the paper's tuple)."""
    return (((alpha * 2 + s) * p.Nt + tau) * p.L + x) * p.L + y


def hop(p: Params, alpha, x, y, xp, yp):
    """t_{alpha, (x,y), (x',y')}: sum of the bond amplitudes joining the two sites on the
    periodic L x L lattice, nearest-neighbour (t) and of distance two along an axis (t2); each
    bond of a site counted once, so on L = 2 the +x and -x bonds join the same pair and the
    distance-two bonds return to the site itself (and on L = 4 the +2 and -2 bonds coincide)."""
    L = p.L
    t = 0.0
    if yp == y:
        t += p.t_h[alpha] * (((xp - x) % L == 1) + ((x - xp) % L == 1))
        t += p.t2_h[alpha] * (((xp - x - 2) % L == 0) + ((x - xp - 2) % L == 0))
    if xp == x:
        t += p.t_v[alpha] * (((yp - y) % L == 1) + ((y - yp) % L == 1))
        t += p.t2_v[alpha] * (((yp - y - 2) % L == 0) + ((y - yp - 2) % L == 0))
    return t


def dense_D(p: Params, phi: np.ndarray) -> np.ndarray:
    """D(phi) as a dense complex matrix, written term by term from Eq. (D_formula)."""
    L, Nt, dt = p.L, p.Nt, p.dtau
    n = p.n
    D = np.zeros((n, n), dtype=complex)
    sig = pauli()
    sigx_band = np.array([[0.0, 1.0], [1.0, 0.0]])
    eta = stagger(p)
    for alpha in range(2):
        for s in range(2):
            for tau in range(Nt):
                for x in range(L):
                    for y in range(L):
                        i = index(p, alpha, s, tau, x, y)
                        # diagonal in (alpha, s, r): -1 - dtau mu_alpha
                        D[i, i] += -1.0 - dt * p.mu[alpha]
                        # forward time hop with the antiperiodic sign at the wrap
                        tp = (tau + 1) % Nt
                        D[i, index(p, alpha, s, tp, x, y)] += 1.0 - 2.0 * (tau == Nt - 1)
                        # spatial hopping within the time slice
                        for xp in range(L):
                            for yp in range(L):
                                t = hop(p, alpha, x, y, xp, yp)
                                if t != 0.0:
                                    D[i, index(p, alpha, s, tau, xp, yp)] += -dt * t
                        # on-site Yukawa term
                        for alphap in range(2):
                            if sigx_band[alpha, alphap] == 0.0:
                                continue
                            for sp in range(2):
                                phisig = sum(phi[a, tau, x, y] * sig[a][s, sp] for a in range(3))
                                D[i, index(p, alphap, sp, tau, x, y)] += (
                                    dt * p.g * eta[x, y] * phisig * sigx_band[alpha, alphap])
    return D


def _coupling(p: Params, phi, v):
    """On-site term dtau g eta (phi . sigma) sigma^x_band applied to v (Hermitian block)."""
    eta = stagger(p)[None, :, :]
    f = p.dtau * p.g * eta
    out = np.empty_like(v)
    for alpha in range(2):
        w = v[1 - alpha]  # sigma^x swaps the bands
        out[alpha, 0] = f * (phi[2] * w[0] + (phi[0] - 1j * phi[1]) * w[1])
        out[alpha, 1] = f * ((phi[0] + 1j * phi[1]) * w[0] - phi[2] * w[1])
    return out


def _spatial_hop(p: Params, alpha, v):
    """sum_{r'} t_{alpha, r, r'} v(r') on the periodic lattice; axes -2 = x, -1 = y."""
    out = (p.t_h[alpha] * (np.roll(v, 1, axis=-2) + np.roll(v, -1, axis=-2))
           + p.t_v[alpha] * (np.roll(v, 1, axis=-1) + np.roll(v, -1, axis=-1)))
    if p.t2_h[alpha] != 0.0:   # hops of distance two (absent unless set)
        out = out + p.t2_h[alpha] * (np.roll(v, 2, axis=-2) + np.roll(v, -2, axis=-2))
    if p.t2_v[alpha] != 0.0:
        out = out + p.t2_v[alpha] * (np.roll(v, 2, axis=-1) + np.roll(v, -2, axis=-1))
    return out


def time_sign(p: Params):
    """b(tau) = 1 - 2 delta_{tau, Nt-1}: the coefficient of the forward time hop."""
    b = np.ones(p.Nt)
    b[-1] = -1.0
    return b


def apply_D(p: Params, phi, v):
    """D(phi) v, matrix-free (Eq. D_formula)."""
    b = time_sign(p)[None, :, None, None]
    out = _coupling(p, phi, v)
    for alpha in range(2):
        va = v[alpha]
        out[alpha] += ((-1.0 - p.dtau * p.mu[alpha]) * va
                       + b * np.roll(va, -1, axis=1)          # + b(tau) v(tau+1)
                       - p.dtau * _spatial_hop(p, alpha, va))
    return out


def apply_Ddag(p: Params, phi, v):
    """D(phi)^dagger v: the time hop runs backwards with coefficient b(tau-1); the
    hopping is real symmetric and the on-site block is Hermitian."""
    b_prev = np.roll(time_sign(p), 1)[None, :, None, None]   # b(tau - 1)
    out = _coupling(p, phi, v)
    for alpha in range(2):
        va = v[alpha]
        out[alpha] += ((-1.0 - p.dtau * p.mu[alpha]) * va
                       + b_prev * np.roll(va, 1, axis=1)      # + b(tau-1) v(tau-1)
                       - p.dtau * _spatial_hop(p, alpha, va))
    return out


def apply_A(p: Params, phi, v):
    """A v = D D^dagger v, the Hermitian positive definite operator of Eq. (linsys)."""
    return apply_D(p, phi, apply_Ddag(p, phi, v))


def apply_K(p: Params, v):
    """K v: the phi-independent part of D (Eq. Dsplit)."""
    return apply_D(p, np.zeros((3, p.Nt, p.L, p.L)), v)


def free_symbol(p: Params):
    """K-hat of Eq. (Kdiag) on the twisted Fourier grid, shape (2, Nt, L, L) indexed
    [alpha, n, m_x, m_y]: e^{i w_n} - 1 - dtau (mu_alpha + 2 t_h cos k_x + 2 t_v cos k_y
    + 2 t2_h cos 2k_x + 2 t2_v cos 2k_y) with antiperiodic w_n = (2n + 1) pi / Nt and
    k = 2 pi m / L.
    """
    w = (2 * np.arange(p.Nt) + 1) * np.pi / p.Nt
    k = 2 * np.pi * np.arange(p.L) / p.L
    out = np.empty((2, p.Nt, p.L, p.L), dtype=complex)
    for alpha in range(2):
        eps = (2 * p.t_h[alpha] * np.cos(k)[:, None] + 2 * p.t_v[alpha] * np.cos(k)[None, :]
               + 2 * p.t2_h[alpha] * np.cos(2 * k)[:, None] + 2 * p.t2_v[alpha] * np.cos(2 * k)[None, :])
        out[alpha] = (np.exp(1j * w)[:, None, None] - 1.0
                      - p.dtau * (p.mu[alpha] + eps[None, :, :]))
    return out
