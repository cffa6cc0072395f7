"""Pins for the oracle's boson action, force, metric and leapfrog, each against something
other than the oracle: the Fourier closed form of the quadratic action, central finite
differences, the exact per-mode leapfrog map of a harmonic oscillator, time reversal,
the O(eps^2) energy error of leapfrog and the ensemble identity <exp(-dH)> = 1."""

import numpy as np
import pytest

from oracle.model import Params
from oracle import boson, hmc, fermion

P = Params(L=4, Nt=6, g=1.0, u=1.0)


def rand_phi(p, seed=0, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal((3, p.Nt, p.L, p.L))


def rand_vec(p, seed=1):
    g = np.random.default_rng(seed)
    sh = (2, 2, p.Nt, p.L, p.L)
    return (g.standard_normal(sh) + 1j * g.standard_normal(sh)) * np.sqrt(0.5)


def boson_symbol(p):
    """B(w, k) with S_B = (1/2) sum B |F phi|^2 at u = 0: periodic w = 2 pi n / Nt."""
    w = 2 * np.pi * np.arange(p.Nt) / p.Nt
    k = 2 * np.pi * np.arange(p.L) / p.L
    return p.dtau * (2.0 / (p.c ** 2 * p.dtau ** 2) * (2 - 2 * np.cos(w))[:, None, None]
                     + (2 - 2 * np.cos(k))[None, :, None] + (2 - 2 * np.cos(k))[None, None, :]
                     + p.r)


def test_boson_action_fourier_closed_form():
    p = Params(L=4, Nt=6, u=0.0)
    phi = rand_phi(p, 3)
    ph = np.fft.fftn(phi, axes=(1, 2, 3), norm="ortho")
    ref = 0.5 * np.sum(boson_symbol(p)[None] * np.abs(ph) ** 2)
    assert abs(boson.action(p, phi) - ref) < 1e-12 * ref


def test_boson_action_constant_field():
    # constant phi: only the local terms survive: V dtau [(r/2) phi^2 + (u/4) phi^4]
    p = Params(L=4, Nt=6, r=0.7, u=1.3)
    v = np.array([0.2, -0.5, 0.9])
    phi = np.broadcast_to(v[:, None, None, None], (3, p.Nt, p.L, p.L)).copy()
    q = v @ v
    ref = p.V * p.dtau * (0.5 * p.r * q + 0.25 * p.u * q * q)
    assert abs(boson.action(p, phi) - ref) < 1e-12 * ref


def test_boson_grad_finite_difference():
    phi = rand_phi(P, 4)
    G = boson.grad(P, phi)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in phi.shape)
        e = np.zeros_like(phi)
        e[idx] = h
        fd = (boson.action(P, phi + e) - boson.action(P, phi - e)) / (2 * h)
        assert abs(fd - G[idx]) < 1e-6 * max(1.0, abs(G[idx]))


@pytest.mark.parametrize("nrhs", [1, 2])
def test_force_finite_difference(nrhs):
    phi = rand_phi(P, 5)
    chis = [rand_vec(P, 10 + i) for i in range(nrhs)]
    vps = [hmc.heatbath(P, phi, c) for c in chis]

    def S(f):
        return boson.action(P, f) + hmc.pseudofermion_action(P, f, vps)

    F, s_pf, _ = hmc.force(P, phi, vps)
    assert abs(s_pf - hmc.pseudofermion_action(P, phi, vps)) < 1e-10 * s_pf
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(8):
        idx = tuple(rng.integers(0, s) for s in phi.shape)
        e = np.zeros_like(phi)
        e[idx] = h
        fd = -(S(phi + e) - S(phi - e)) / (2 * h)
        assert abs(fd - F[idx]) < 2e-6 * max(1.0, abs(F[idx])), (idx, fd, F[idx])


def test_fermion_force_vanishes_at_zero_coupling():
    p = Params(L=4, Nt=6, g=0.0)
    phi = rand_phi(p, 6)
    vps = [hmc.heatbath(p, phi, rand_vec(p, 7))]
    F, _, _ = hmc.force(p, phi, vps, include_boson=False)
    assert np.abs(F).max() == 0.0


def test_momentum_kinetic_identities():
    # pi = F^-1(sigma^-1/2 F z) is real and (1/2) sum sigma |F pi|^2 = (1/2)|z|^2 exactly.
    p = Params(L=4, Nt=6)
    sig = np.fft.fftn(rand_phi(p, 1), axes=(1, 2, 3), norm="ortho")
    sig = (sig * np.conj(sig)).real + 0.1          # even in k, positive
    z = rand_phi(p, 2)
    pi = hmc.momentum(sig, z)
    full = np.fft.ifftn(np.fft.fftn(z, axes=(1, 2, 3), norm="ortho") / np.sqrt(sig),
                        axes=(1, 2, 3), norm="ortho")
    assert np.abs(full.imag).max() < 1e-12
    assert abs(hmc.kinetic(sig, pi) - 0.5 * np.sum(z * z)) < 1e-11 * np.sum(z * z)


def test_leapfrog_harmonic_closed_form():
    # Gaussian target (u = 0, no pseudofermions) with the exact metric sigma = 1/B: each
    # Fourier mode is an oscillator H = (1/2) s p^2 + (1/2) b q^2 with s b = 1, and one
    # leapfrog step is the 2x2 map [[1 - e^2/2, e s], [-e b (1 - e^2/4), 1 - e^2/2]].
    p = Params(L=4, Nt=6, u=0.0, g=0.0)
    b = np.broadcast_to(boson_symbol(p)[None], (3, p.Nt, p.L, p.L))
    sig = 1.0 / b
    phi0 = rand_phi(p, 3)
    pi0 = rand_phi(p, 4)
    eps, n = 0.3, 7
    phi1, pi1, _, _ = hmc.leapfrog(p, phi0, pi0, [], sig, eps, n)
    q = np.fft.fftn(phi0, axes=(1, 2, 3), norm="ortho")
    m = np.fft.fftn(pi0, axes=(1, 2, 3), norm="ortho")
    for _ in range(n):
        q, m = ((1 - eps ** 2 / 2) * q + eps * sig * m,
                -eps * b * (1 - eps ** 2 / 4) * q + (1 - eps ** 2 / 2) * m)
    assert np.abs(np.fft.fftn(phi1, axes=(1, 2, 3), norm="ortho") - q).max() < 1e-12
    assert np.abs(np.fft.fftn(pi1, axes=(1, 2, 3), norm="ortho") - m).max() < 1e-10


def test_leapfrog_reversible():
    phi0 = rand_phi(P, 8, 0.5)
    pi0 = rand_phi(P, 9)
    vps = [hmc.heatbath(P, phi0, rand_vec(P, 10))]
    sig = np.ones_like(phi0)
    phi1, pi1, _, _ = hmc.leapfrog(P, phi0, pi0, vps, sig, 0.05, 6)
    phi2, pi2, _, _ = hmc.leapfrog(P, phi1, -pi1, vps, sig, 0.05, 6)
    assert np.abs(phi2 - phi0).max() < 1e-11
    assert np.abs(pi2 + pi0).max() < 1e-10


def test_dH_scales_as_eps_squared():
    p = Params(L=4, Nt=4, g=1.0)
    phi = rand_phi(p, 11, 0.5)
    sig = np.ones_like(phi)
    z = rand_phi(p, 12)
    chi = [rand_vec(p, 13)]
    dh = []
    for n in (4, 8, 16):
        out = hmc.trajectory(p, phi, sig, chi, z, 0.5, 0.4 / n, n)
        dh.append(abs(out["dH"]))
    assert 3.0 < dh[0] / dh[1] < 5.0 and 3.0 < dh[1] / dh[2] < 5.0, dh


def test_trajectory_energy_bookkeeping():
    p = Params(L=4, Nt=4, g=1.0)
    phi = rand_phi(p, 14, 0.5)
    sig = np.ones_like(phi)
    out = hmc.trajectory(p, phi, sig, [rand_vec(p, 15)], rand_phi(p, 16), 0.3, 0.05, 3)
    assert abs(out["H1"] - out["H0"] - out["dH"]) < 1e-12 * abs(out["H0"])
    # the final pseudofermion action is varphi^dag A^-1 varphi at the proposed phi
    vp = hmc.heatbath(p, phi, rand_vec(p, 15))
    assert abs(out["S_PF"][1] - hmc.pseudofermion_action(p, out["phi_proposed"], [vp])) < 1e-10
    assert out["accept"] == (0.3 < np.exp(-out["dH"]))


@pytest.mark.slow
def test_creutz_identity():
    # <exp(-dH)> = 1 for an exact, reversible, volume-preserving integrator (Section HMC).
    p = Params(L=2, Nt=4, g=1.0, u=1.0)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((3, p.Nt, p.L, p.L)) * 0.5
    sig = np.ones_like(phi)
    vals = []
    for t in range(300):
        chi = [rand_vec(p, 1000 + t)]
        out = hmc.trajectory(p, phi, sig, chi, rng.standard_normal(phi.shape), rng.random(),
                             0.12, 4)
        vals.append(np.exp(-out["dH"]))
        phi = out["phi"]
    vals = np.array(vals)
    assert abs(vals.mean() - 1.0) < 4 * vals.std() / np.sqrt(len(vals)) + 1e-3


def test_sigma_estimate_recovers_spectrum():
    # Eq. (covest) on samples of a Gaussian field with known per-mode variance s(k).
    from paper_2204_14241_gb300 import inputs
    L, Nt = 4, 6
    s = inputs.spectrum(L, Nt, 0.5, 2.0)
    samples = [inputs.smooth_field(100 + i, L, Nt, 0.5, 2.0) for i in range(800)]
    est = hmc.sigma_estimate(samples)
    rel = est / s[None]
    assert abs(rel.mean() - 1.0) < 0.02
    assert np.abs(rel - 1).max() < 0.35


def test_sdw_susceptibility_free_field():
    # Gaussian phi with per-mode variance s(k) in each component: chi = 3 s(k) dtau on average
    from oracle import observables
    from paper_2204_14241_gb300 import inputs
    L, Nt, dt = 4, 6, 0.1
    s = inputs.spectrum(L, Nt, 0.5, 2.0)
    samples = [inputs.smooth_field(300 + i, L, Nt, 0.5, 2.0) for i in range(600)]
    chi = observables.sdw_susceptibility(samples, dt)
    rel = chi / (3 * s * dt)
    assert abs(rel.mean() - 1) < 0.02 and np.abs(rel - 1).max() < 0.2


def test_binder_cumulant_limits():
    # B_c = 1 - 3<|Phi|^4>/(5<|Phi|^2>^2): exactly 0.4 for an order parameter of fixed length, 0 on
    # average for a Gaussian one (<|Phi|^4> = 15 s^2 and <|Phi|^2> = 3 s for three N(0, s) components)
    from oracle import observables
    rng = np.random.default_rng(7)
    L, Nt = 4, 6
    fixed = []
    for _ in range(50):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        fixed.append(np.broadcast_to((0.3 * u)[:, None, None, None], (3, Nt, L, L)).copy())
    assert abs(observables.binder_cumulant(fixed) - 0.4) < 1e-12
    gauss = [rng.standard_normal((3, Nt, L, L)) for _ in range(4000)]
    assert abs(observables.binder_cumulant(gauss)) < 0.05


@pytest.mark.parametrize("a", [0.0, 0.5, 0.8])
def test_tau_int_ar1(a):
    # an AR(1) series x_{n+1} = a x_n + sqrt(1 - a^2) e_n has rho(t) = a^t, so
    # tau_int = 1 + 2 sum_t a^t = (1 + a) / (1 - a); the package's FFT estimator agrees with the
    # oracle's lag-by-lag sum on the same series
    from oracle import observables
    from paper_2204_14241_gb300 import observables as gobs
    rng = np.random.default_rng(11)
    n = 100000
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0]
    for i in range(1, n):
        x[i] = a * x[i - 1] + np.sqrt(1 - a * a) * e[i]
    ref = (1 + a) / (1 - a)
    t = observables.tau_int(x)
    assert abs(t - ref) < 0.08 * ref, (t, ref)
    assert abs(gobs.tau_int(x) - t) < 1e-9 * t


def test_presets_follow_the_paper_table():
    from paper_2204_14241_gb300 import presets
    p1, p5 = presets.paper_nesting(1), presets.paper_nesting(5)
    assert p1["t_h"][0] == 1.0 and p1["t_v"][1] == 1.0 and p1["t_v"][0] == 0.45 and p1["t_h"][1] == -0.45
    assert p1["mu"] == (-0.47, 0.47) and p5["t_v"][0] == 0.5085 and p5["mu"] == (-0.44, 0.44)
    assert p1["u"] == 0.0 and p1["c"] == 3.0 and abs(p1["g"] - 0.98995) < 1e-4
