"""Pins for the oracle's fermion matrix and solvers, each against something other than
the oracle itself: closed forms derived from Eq. (D_formula), the antiunitary symmetry the
paper cites for sign-problem freedom, momentum-space block diagonalisation at uniform phi,
numpy's dense solver and eigenvalue routines."""

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle.model import Params
from oracle import fermion, solver, hmc
from paper_2204_14241_gb300 import inputs

P = Params(L=4, Nt=6)


def rand_phi(p, seed=0):
    return np.random.default_rng(seed).standard_normal((3, p.Nt, p.L, p.L))


def rand_vec(p, seed=1):
    g = np.random.default_rng(seed)
    sh = (2, 2, p.Nt, p.L, p.L)
    return g.standard_normal(sh) + 1j * g.standard_normal(sh)


def match_multisets(a, b):
    """Largest distance after optimally pairing two equal-size sets of complex numbers."""
    d = np.abs(a[:, None] - b[None, :])
    i, j = linear_sum_assignment(d)
    return d[i, j].max()


def band_energy(p, a, kx, ky):
    """Fourier transform of band a's hops: a hop of distance d along an axis contributes
    t (e^{i d k} + e^{-i d k}) = 2 t cos(d k) (d = 1: t_h, t_v; d = 2: t2_h, t2_v)."""
    return (2 * p.t_h[a] * np.cos(kx) + 2 * p.t_v[a] * np.cos(ky)
            + 2 * p.t2_h[a] * np.cos(2 * kx) + 2 * p.t2_v[a] * np.cos(2 * ky))


def free_eigs_closed_form(p):
    """Eigenvalues of D at g = 0: e^{i w} - 1 - dtau (mu_a + eps_a(k)), w = (2n+1) pi / Nt
    (antiperiodic), k = 2 pi m / L, each twice (spin)."""
    out = []
    for a in range(2):
        for n in range(p.Nt):
            w = (2 * n + 1) * np.pi / p.Nt
            for mx in range(p.L):
                for my in range(p.L):
                    kx, ky = 2 * np.pi * mx / p.L, 2 * np.pi * my / p.L
                    e = np.exp(1j * w) - 1 - p.dtau * (p.mu[a] + band_energy(p, a, kx, ky))
                    out += [e, e]
    return np.array(out)


# the hops of distance two of the paper's first nesting set, read along each band's weak direction
T2 = dict(t_h=(1.0, 0.0), t_v=(0.0, 1.0), mu=(-0.47, 0.47), t2_h=(0.0, -0.45), t2_v=(0.45, 0.0))


@pytest.mark.parametrize("L,Nt,kw", [(4, 6, {}), (2, 5, {}), (6, 3, {}), (6, 3, T2), (4, 4, T2), (2, 3, T2)])
def test_free_spectrum_closed_form(L, Nt, kw):
    p = Params(L=L, Nt=Nt, g=0.0, **kw)
    D = fermion.dense_D(p, rand_phi(p))
    assert match_multisets(np.linalg.eigvals(D), free_eigs_closed_form(p)) < 1e-12


@pytest.mark.parametrize("kw", [{}, T2])
def test_free_logdet_closed_form(kw):
    # prod over the Nt antiperiodic roots z_n of z^Nt = -1 of (z_n - a) has modulus |1 + a^Nt|
    p = Params(L=6 if kw else 4, Nt=6, g=0.0, **kw)
    D = fermion.dense_D(p, rand_phi(p))
    _, logabs = np.linalg.slogdet(D @ D.conj().T)
    k = 2 * np.pi * np.arange(p.L) / p.L
    ref = 0.0
    for a in range(2):
        eps = band_energy(p, a, k[:, None], k[None, :])
        aa = 1 + p.dtau * (p.mu[a] + eps)
        ref += 2 * 2 * np.sum(np.log(np.abs(1 + aa ** p.Nt)))   # x2 spin, x2 for |det D|^2
    assert abs(logabs - ref) < 1e-10 * abs(ref)


@pytest.mark.parametrize("kw", [{}, T2])
def test_det_real_nonnegative_and_conjugate_pairs(kw):
    # Berg et al. (cited for sign-problem freedom): det D is real and >= 0 for any phi.
    p = Params(L=4, Nt=6, g=1.3, **kw)
    D = fermion.dense_D(p, rand_phi(p, 5))
    sign, _ = np.linalg.slogdet(D)
    assert abs(sign - 1.0) < 1e-10
    ev = np.linalg.eigvals(D)
    assert match_multisets(ev, np.conj(ev)) < 1e-9


@pytest.mark.parametrize("kw", [{}, T2])
def test_antiunitary_symmetry(kw):
    # T = (i sigma^y_spin x sigma^z_band) K with T^2 = -1 commutes with D: U conj(D) U^-1 = D.
    p = Params(L=4, Nt=4, g=0.9, **kw)
    D = fermion.dense_D(p, rand_phi(p, 3))
    isy = np.array([[0, 1], [-1, 0]], dtype=complex)
    sz = np.diag([1.0, -1.0])
    U = np.kron(np.kron(sz, isy), np.eye(p.V))   # (alpha, s, tau, x, y) C-order
    assert np.abs(U @ D.conj() @ np.linalg.inv(U) - D).max() < 1e-13
    assert np.abs(U @ U.conj() + np.eye(p.n)).max() < 1e-13


@pytest.mark.parametrize("kw", [{}, T2])
def test_uniform_phi_block_diagonalisation(kw):
    # Uniform phi: e^{iQ.r} couples k to k+Q, so D splits into 8x8 blocks over
    # (band, spin, {k, k+Q}) per Matsubara frequency; brute-force their eigenvalues.
    p = Params(L=4, Nt=4, g=0.8, **kw)
    ph = np.array([0.3, -0.7, 0.5])
    phi = np.broadcast_to(ph[:, None, None, None], (3, p.Nt, p.L, p.L)).copy()
    D = fermion.dense_D(p, phi)
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    phs = sum(ph[a] * s[a] for a in range(3))
    eigs = []
    for n in range(p.Nt):
        w = (2 * n + 1) * np.pi / p.Nt
        for mx in range(p.L):
            for my in range(p.L):
                ks = [(2 * np.pi * mx / p.L, 2 * np.pi * my / p.L),
                      (2 * np.pi * mx / p.L + np.pi, 2 * np.pi * my / p.L + np.pi)]
                B = np.zeros((8, 8), dtype=complex)   # index (q, alpha, s), q = k or k+Q
                for q, (kx, ky) in enumerate(ks):
                    for a in range(2):
                        e = np.exp(1j * w) - 1 - p.dtau * (p.mu[a] + band_energy(p, a, kx, ky))
                        for sp in range(2):
                            B[q * 4 + a * 2 + sp, q * 4 + a * 2 + sp] = e
                        for sp in range(2):
                            for sq in range(2):
                                B[q * 4 + a * 2 + sp, (1 - q) * 4 + (1 - a) * 2 + sq] = (
                                    p.dtau * p.g * phs[sp, sq])
                eigs.extend(np.linalg.eigvals(B))
    eigs = np.array(eigs)                      # every block appears twice (k and k+Q)
    dense = np.linalg.eigvals(D)
    assert match_multisets(np.concatenate([dense, dense]), eigs) < 1e-11


@pytest.mark.parametrize("L,kw", [(4, {}), (4, T2), (6, T2), (2, T2)])
def test_matrix_free_equals_dense(L, kw):
    p = Params(L=L, Nt=5, g=1.1, **kw)
    phi = rand_phi(p, 7)
    D = fermion.dense_D(p, phi)
    v = rand_vec(p, 8)
    assert np.abs(D @ v.ravel() - fermion.apply_D(p, phi, v).ravel()).max() < 1e-13
    assert np.abs(D.conj().T @ v.ravel() - fermion.apply_Ddag(p, phi, v).ravel()).max() < 1e-13
    A = D @ D.conj().T
    assert np.abs(A @ v.ravel() - fermion.apply_A(p, phi, v).ravel()).max() < 1e-12


def test_heatbath_identity():
    # varphi = D chi  =>  varphi^dag (D D^dag)^{-1} varphi = chi^dag chi (Section HMC).
    phi = rand_phi(P, 2)
    chi = rand_vec(P, 3)
    vp = hmc.heatbath(P, phi, chi)
    s = hmc.pseudofermion_action(P, phi, [vp])
    assert abs(s - np.vdot(chi, chi).real) < 1e-10 * np.vdot(chi, chi).real


@pytest.mark.parametrize("method", ["cg", "pcg"])
def test_cg_matches_dense_solve(method):
    phi = rand_phi(P, 4)
    b = rand_vec(P, 5)
    D = fermion.dense_D(P, phi)
    ref = np.linalg.solve(D @ D.conj().T, b.ravel()).reshape(b.shape)
    f = solver.cg if method == "cg" else solver.pcg
    x, it, res = f(P, phi, b, tol=1e-12)
    assert res < 1e-11
    assert np.abs(x - ref).max() < 1e-9 * np.abs(ref).max()


def test_pcg_exact_at_zero_coupling():
    # g -> 0: P = (D D^dag)^{-1}, so PCG converges in a single iteration (Eq. precon ff.).
    p = Params(L=4, Nt=6, g=0.0)
    x, it, res = solver.pcg(p, rand_phi(p), rand_vec(p), tol=1e-12)
    assert it == 1 and res < 1e-13


def test_twisted_fourier_diagonalises_K():
    # Eq. (Kdiag): K = F~ K-hat F~^*. Apply dense K to twisted plane waves.
    p = Params(L=4, Nt=6, g=0.0)
    K = fermion.dense_D(p, np.zeros((3, p.Nt, p.L, p.L)))
    kh = fermion.free_symbol(p)
    tau = np.arange(p.Nt)[:, None, None]
    x = np.arange(p.L)[None, :, None]
    y = np.arange(p.L)[None, None, :]
    for (a, s, n, mx, my) in [(0, 0, 0, 0, 0), (1, 1, 2, 1, 3), (0, 1, 5, 2, 2), (1, 0, 3, 3, 1)]:
        wave = np.exp(1j * np.pi * (2 * n + 1) * tau / p.Nt + 2j * np.pi * (mx * x + my * y) / p.L)
        v = np.zeros((2, 2, p.Nt, p.L, p.L), dtype=complex)
        v[a, s] = wave
        assert np.abs(K @ v.ravel() - kh[a, n, mx, my] * v.ravel()).max() < 1e-13


@pytest.mark.parametrize("L,kw", [(4, {}), (6, T2)])
def test_precond_is_inverse_of_KKdag(L, kw):
    p = Params(L=L, Nt=6, g=0.7, **kw)
    K = fermion.dense_D(p, np.zeros((3, p.Nt, p.L, p.L)))
    v = rand_vec(p, 9)
    Pv = solver.apply_precond(p, v)
    assert np.abs((K @ K.conj().T) @ Pv.ravel() - v.ravel()).max() < 1e-11 * np.abs(v).max()


def test_precond_quadratic_form_in_frequency_space():
    # <r, P r> = sum P-hat |F~^* r|^2 because F~ = T F is unitary (|T| = 1, F the unitary DFT): the
    # complex64 PCG sums <r, z> this way inside its tau pass instead of re-reading r and z.
    # Also: <r, P r> > 0 (P is positive definite) and the identity fails for a non-unitary F.
    for L, Nt in ((4, 6), (6, 8)):
        p = Params(L=L, Nt=Nt)
        r = rand_vec(p, 30 + L)
        lhs = np.vdot(r, solver.apply_precond(p, r)).real
        T = solver.twist(p)
        rh = np.fft.fftn(np.conj(T) * r, axes=(2, 3, 4), norm="ortho")
        rhs = float(np.sum(solver.precond_symbol(p) * np.abs(rh) ** 2))
        assert lhs > 0 and abs(lhs - rhs) < 1e-12 * lhs
        rh_raw = np.fft.fftn(np.conj(T) * r, axes=(2, 3, 4))   # unnormalised: off by V
        assert abs(float(np.sum(solver.precond_symbol(p) * np.abs(rh_raw) ** 2)) - lhs) > 0.5 * lhs


def test_layout_roundtrip():
    v = inputs.fermion_noise(0, 1, 4, 6)[0]
    assert np.array_equal(inputs.from_paper_fermion(inputs.to_paper_fermion(v)), v)
    f = inputs.gaussian_field(0, 4, 6)
    assert np.array_equal(inputs.from_paper_boson(inputs.to_paper_boson(f)), f)


def test_green_estimator_exact_at_zero_coupling():
    # g = 0: D = K is diagonal in the twisted Fourier basis (Eq. Kdiag), so O = F~^* D^-1 F~ is
    # diagonal with entries 1 / K-hat and v . O v = O_ii for any +-1 vector v.
    from oracle import observables
    p = Params(L=4, Nt=6, g=0.0)
    rng = np.random.default_rng(4)
    probes = [rng.choice([-1.0, 1.0], size=(2, 2, p.Nt, p.L, p.L)) for _ in range(2)]
    est = observables.green_diagonal(p, rand_phi(p), probes)
    kh = fermion.free_symbol(p)[:, None]                    # (alpha, 1, n, m_x, m_y)
    assert np.abs(est - 1.0 / np.broadcast_to(kh, est.shape)).max() < 1e-12


def test_green_estimator_unbiased():
    # E[v . O v] = diag(O): the average over many probes approaches the exact diagonal from a
    # dense inverse (error ~ sqrt(sum_j |O_ij|^2 / S))
    from oracle import observables
    p = Params(L=2, Nt=4, g=0.8)
    phi = rand_phi(p, 6)
    D = fermion.dense_D(p, phi)
    # exact O = F~^* D^-1 F~ as a matrix acting on C-order flattened vectors
    n = p.n
    E = np.eye(n, dtype=complex).reshape((n, 2, 2, p.Nt, p.L, p.L))
    Ft = np.stack([observables.twisted_fourier(p, e, inverse=True).ravel() for e in E], axis=1)
    O = Ft.conj().T @ np.linalg.solve(D, Ft)
    rng = np.random.default_rng(7)
    S = 400
    probes = [rng.choice([-1.0, 1.0], size=(2, 2, p.Nt, p.L, p.L)) for _ in range(S)]
    est = observables.green_diagonal(p, phi, probes).ravel()
    off = np.sqrt((np.abs(O) ** 2).sum(axis=1) - np.abs(np.diag(O)) ** 2)
    assert np.all(np.abs(est - np.diag(O)) < 5 * off / np.sqrt(S) + 1e-12)
