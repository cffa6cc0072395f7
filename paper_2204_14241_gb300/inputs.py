"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds random-number draws and array layout only: no part of the method's
arithmetic (no fermion matrix, action, force, solver or integrator).

Layouts (the library's device layout):
* boson field and momenta: real ``[3][Nt][L][L]`` indexed ``[a, tau, y, x]`` (x fastest);
* fermion vectors: complex ``[nrhs][Nt][L][L][2][2]`` indexed ``[k, tau, y, x, alpha, s]``.
The helpers ``to_paper_*`` / ``from_paper_*`` permute to and from the paper's index order
``[a, tau, x, y]`` and ``[alpha, s, tau, x, y]``.

Synthetic workload recipe: phi is either i.i.d. N(0, 1) per component, or a smooth
Gaussian random field whose Fourier variance is 1 / (m2 + kt * (2 - 2 cos w)
+ (4 - 2 cos kx - 2 cos ky)) (``smooth_field``), the shape of a thermalised
free-boson configuration, optionally shifted by a uniform amplitude along one component
(``ordered_field``).
"""

import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def gaussian_field(seed, L, Nt):
    """phi ~ N(0, 1) i.i.d. per component, library layout [3][Nt][L][L] (float64)."""
    return rng(seed).standard_normal((3, Nt, L, L))


def spectrum(L, Nt, m2, kt):
    """1 / (m2 + kt (2 - 2 cos w) + 4 - 2 cos kx - 2 cos ky) on the [n_tau, m_y, m_x] grid."""
    w = 2 * np.pi * np.arange(Nt) / Nt
    k = 2 * np.pi * np.arange(L) / L
    den = (m2 + kt * (2 - 2 * np.cos(w))[:, None, None]
           + (2 - 2 * np.cos(k))[None, :, None] + (2 - 2 * np.cos(k))[None, None, :])
    return 1.0 / den


def smooth_field(seed, L, Nt, m2, kt):
    """Gaussian random field with variance ``spectrum`` per Fourier mode, library layout."""
    z = rng(seed).standard_normal((3, Nt, L, L))
    zh = np.fft.fftn(z, axes=(1, 2, 3), norm="ortho")
    return np.fft.ifftn(zh * np.sqrt(spectrum(L, Nt, m2, kt))[None], axes=(1, 2, 3),
                        norm="ortho").real


def ordered_field(seed, L, Nt, m2, kt, scale, amp):
    """``scale * smooth_field`` plus the constant ``amp`` on component 3: a uniform (ordered)
    field with Gaussian fluctuations of the ``spectrum`` shape, library layout."""
    f = scale * smooth_field(seed, L, Nt, m2, kt)
    f[2] += amp
    return f


def complex_normal(seed, shape):
    """Standard complex Gaussian: real and imaginary parts N(0, 1/2)."""
    g = rng(seed)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * np.sqrt(0.5)


def fermion_noise(seed, nrhs, L, Nt):
    """nrhs standard complex Gaussian vectors, library layout [nrhs][Nt][L][L][2][2]."""
    return complex_normal(seed, (nrhs, Nt, L, L, 2, 2))


def real_normal(seed, shape):
    return rng(seed).standard_normal(shape)


def uniform(seed):
    return float(rng(seed).random())


# ---- layout permutations -------------------------------------------------------------

def to_paper_boson(a):
    """[3][Nt][y][x] -> [3][Nt][x][y]."""
    return np.ascontiguousarray(np.swapaxes(a, -1, -2))


def from_paper_boson(a):
    """[3][Nt][x][y] -> [3][Nt][y][x]."""
    return np.ascontiguousarray(np.swapaxes(a, -1, -2))


def to_paper_fermion(v):
    """One vector [Nt][y][x][alpha][s] -> [alpha][s][Nt][x][y]."""
    return np.ascontiguousarray(np.transpose(v, (3, 4, 0, 2, 1)))


def from_paper_fermion(v):
    """One vector [alpha][s][Nt][x][y] -> [Nt][y][x][alpha][s]."""
    return np.ascontiguousarray(np.transpose(v, (2, 4, 3, 0, 1)))
