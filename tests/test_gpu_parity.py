"""GPU parity: every step of the hot path, called through the C ABI (libhmc via the ctypes
binding), against the FP64 oracle on the same seeded inputs.

Tolerances (relative to the largest reference entry unless stated):
* FP64 operator applications: 1e-12 (a few hundred roundings of O(1) terms).
* FP32 operator applications: 1e-5 (the bar for the mixed mode; FP32 unit roundoff is 6e-8 and
  each output sums ~20 terms).
* Solves: the oracle's FP64 true residual of the GPU solution is <= 1.5 * tol in both modes.
* Force: 1e-10 relative (the FP64-mode bar), FP64 mode solving to a true residual of 1e-14 and
  the mixed mode to 1e-12. The force is linear in X = A^-1 varphi, so its relative error is at
  most kappa(A) times the relative residual (kappa ~ 40 on the 6 x 6 x 7 case); S_PF
  (variational form, error quadratic in the residual): 1e-10 relative.
* Trajectory: |dH_gpu - dH_oracle| < 1e-8 and phi' within 1e-9.
"""

import numpy as np
import pytest
import torch

from oracle.model import Params
from oracle import fermion, solver, boson, hmc as ohmc
from paper_2204_14241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COUPLINGS = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5, u=1.0, c=3.0)
CASES = [(4, 8), (6, 7), (20, 12), (12, 24)]


def ctx_for(L, Nt, solver_mode="fp64", nrhs=2, tol=1e-12, chains=None, guess=0):
    from paper_2204_14241_gb300.hmc import Context
    return Context(L, Nt, solver=solver_mode, nrhs_max=nrhs, cg_tol=tol, chains=chains, initial_guess=guess,
                   **COUPLINGS)


def oparams(L, Nt, r=None):
    kw = dict(COUPLINGS)
    if r is not None:
        kw["r"] = r
    return Params(L=L, Nt=Nt, **kw)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t.to(dtype) if dtype is not None else t


def to_paper_vecs(t):
    a = t.detach().cpu().numpy().astype(np.complex128)
    return [I.to_paper_fermion(a[k]) for k in range(a.shape[0])]


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("L,Nt", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_D_and_Ddag(L, Nt, prec):
    ctx = ctx_for(L, Nt)
    P = oparams(L, Nt)
    rdt, cdt = (torch.float64, torch.complex128) if prec == "fp64" else (torch.float32, torch.complex64)
    phi = dev(I.gaussian_field(1, L, Nt), rdt)
    x = dev(I.fermion_noise(2, 2, L, Nt), cdt)
    phi_o = I.to_paper_boson(phi.double().cpu().numpy())
    xs = to_paper_vecs(x)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for dagger in (False, True):
        y = ctx.apply_M(phi, x, dagger=dagger)
        ys = to_paper_vecs(y)
        for k in range(2):
            ref = (fermion.apply_Ddag if dagger else fermion.apply_D)(P, phi_o, xs[k])
            assert rel(ys[k], ref) < tol, (dagger, k)


@pytest.mark.parametrize("L,Nt", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_A_fused(L, Nt, prec):
    ctx = ctx_for(L, Nt)
    P = oparams(L, Nt)
    rdt, cdt = (torch.float64, torch.complex128) if prec == "fp64" else (torch.float32, torch.complex64)
    phi = dev(I.gaussian_field(3, L, Nt), rdt)
    x = dev(I.fermion_noise(4, 2, L, Nt), cdt)
    phi_o = I.to_paper_boson(phi.double().cpu().numpy())
    xs = to_paper_vecs(x)
    y, norms = ctx.apply_MdagM(phi, x, norms=True)
    ys = to_paper_vecs(y)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for k in range(2):
        assert rel(ys[k], fermion.apply_A(P, phi_o, xs[k])) < tol
        t = fermion.apply_Ddag(P, phi_o, xs[k])
        n2 = np.vdot(t, t).real
        assert abs(norms[k] - n2) < tol * n2


@pytest.mark.parametrize("L,Nt", [(16, 9), (32, 6), (48, 5)])
def test_apply_A_fp32_strips(L, Nt):
    # L a multiple of 16: the plain FP32 operator runs on full-height strips of 16 columns with
    # TMA staging; one strip wrapping onto itself (L = 16), several strips, time chunks with a
    # ragged last chunk
    ctx = ctx_for(L, Nt, nrhs=3)
    P = oparams(L, Nt)
    phi = dev(I.gaussian_field(30 + L, L, Nt), torch.float32)
    x = dev(I.fermion_noise(31 + L, 3, L, Nt), torch.complex64)
    phi_o = I.to_paper_boson(phi.double().cpu().numpy())
    y, norms = ctx.apply_MdagM(phi, x, norms=True)
    y2 = ctx.apply_MdagM(phi, x)   # without the norm reduction
    for k, xk in enumerate(to_paper_vecs(x)):
        ref = fermion.apply_A(P, phi_o, xk)
        assert rel(to_paper_vecs(y)[k], ref) < 1e-5 and rel(to_paper_vecs(y2)[k], ref) < 1e-5
        t = fermion.apply_Ddag(P, phi_o, xk)
        assert abs(norms[k] - np.vdot(t, t).real) < 1e-5 * norms[k]


@pytest.mark.parametrize("L,Nt", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_preconditioner(L, Nt, prec):
    ctx = ctx_for(L, Nt)
    P = oparams(L, Nt)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    x = dev(I.fermion_noise(5, 2, L, Nt), cdt)
    y = ctx.apply_precond(x)
    xs, ys = to_paper_vecs(x), to_paper_vecs(y)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for k in range(2):
        assert rel(ys[k], solver.apply_precond(P, xs[k])) < tol


@pytest.mark.parametrize("L,Nt", [(16, 8), (24, 6), (40, 4), (80, 4), (20, 160), (12, 80), (16, 48), (16, 96)])
def test_preconditioner_fp32_xy_pass(L, Nt):
    # complex64, L with a compiled (x, y) split: one kernel per band and plane does both axes,
    # leaving the band-major spectrum in digit-permuted order for the in-place tau pass (the same
    # kernels as PCG; N_tau = 160, 80, 48 exercise the tau splits 16 x 10, 10 x 8, 8 x 6, and 96
    # the Stockham tau kernel on that spectrum)
    ctx = ctx_for(L, Nt)
    P = oparams(L, Nt)
    x = dev(I.fermion_noise(50 + L, 2, L, Nt), torch.complex64)
    y = ctx.apply_precond(x)
    for yk, xk in zip(to_paper_vecs(y), to_paper_vecs(x)):
        assert rel(yk, solver.apply_precond(P, xk)) < 1e-5


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_preconditioner_in_place(dtype):
    # y may equal x: the complex64 (x, y) passes keep the band-major spectrum in the context's
    # workspace, so an in-place call gives exactly the out-of-place result
    L, Nt = 16, 8
    ctx = ctx_for(L, Nt)
    x = dev(I.fermion_noise(77, 2, L, Nt), dtype)
    y = ctx.apply_precond(x)
    z = x.clone()
    assert ctx.apply_precond(z, out=z) is z
    assert torch.equal(y, z)
    with pytest.raises(ValueError):
        ctx.apply_precond(x, out=torch.empty_like(x[:1]))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("L,Nt", [(6, 7), (12, 24), (20, 12), (16, 9), (32, 6)])
def test_cg_solve(mode, precond, L, Nt):
    # L = 16, 32 in mixed mode without preconditioner: the complex64 strip operator with the fused
    # x, r, p update (beta ahead of the residual); with it, the strip operator after the p update
    # and the (x, y) preconditioner passes
    tol = 1e-10
    ctx = ctx_for(L, Nt, mode, tol=tol)
    P = oparams(L, Nt)
    phi = dev(I.gaussian_field(6, L, Nt))
    b = dev(I.fermion_noise(7, 2, L, Nt))
    x, st = ctx.cg_solve(phi, b, precond=precond)
    assert st["converged"] and st["true_rel_resid"] <= tol
    phi_o = I.to_paper_boson(phi.cpu().numpy())
    for xk, bk in zip(to_paper_vecs(x), to_paper_vecs(b)):
        res = bk - fermion.apply_A(P, phi_o, xk)
        assert np.linalg.norm(res) <= 1.5 * tol * np.linalg.norm(bk)
    if mode == "mixed":
        assert st["reliable_updates"] >= 1


def test_preconditioner_speedup_point():
    # Supplementary Note 5's claim in miniature: at the study's parameters (nesting v_2, r = 1.26,
    # g = 0.7 sqrt(2), u = 0) the preconditioner cuts the CG iterations several-fold
    from paper_2204_14241_gb300.experiments import precond_point
    pt = precond_point(8, 20, 0.1, n_cfg=1)
    assert pt["pcg_iterations"] > 0 and pt["speedup_iterations"] > 2.0, pt


def test_sdw_zero_mode_series_binder_and_tau():
    # SdwSusceptibility's per-sample chi(0, 0) and |Phi|^2 against the oracle on the same fields,
    # then the Binder cumulant and tau_int of the GPU series against the oracle's
    from oracle import observables as oobs
    from paper_2204_14241_gb300 import observables as gobs
    L, Nt = 6, 8
    ctx = ctx_for(L, Nt)
    est = gobs.SdwSusceptibility(ctx)
    samples = [I.gaussian_field(900 + i, L, Nt) + 0.2 * (i % 3) for i in range(12)]
    for phi in samples:
        est.add(dev(phi))
    V = Nt * L * L
    for phi, m2, chi in zip(samples, est.phi2, est.chi00):
        big = float(np.sum(np.sum(phi, axis=(1, 2, 3)) ** 2))
        assert abs(m2 - big) < 1e-10 * big
        assert abs(chi - COUPLINGS["dtau"] * big / V) < 1e-10 * chi
    b_ref = oobs.binder_cumulant([I.to_paper_boson(p) for p in samples])
    assert abs(gobs.binder_cumulant(est.phi2) - b_ref) < 1e-10
    assert abs(gobs.tau_int(est.chi00) - oobs.tau_int(est.chi00)) < 1e-9


def test_cg_matches_dense_solution():
    L, Nt = 4, 8
    ctx = ctx_for(L, Nt, "mixed", tol=1e-12)
    P = oparams(L, Nt)
    phi = dev(I.gaussian_field(8, L, Nt))
    b = dev(I.fermion_noise(9, 1, L, Nt))
    x, st = ctx.cg_solve(phi, b, precond=True)
    ref = solver.dense_solve(P, I.to_paper_boson(phi.cpu().numpy()), to_paper_vecs(b)[0])
    assert rel(to_paper_vecs(x)[0], ref) < 1e-9


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_force(mode, nrhs):
    L, Nt = 6, 7
    ctx = ctx_for(L, Nt, mode, tol=1e-14 if mode == "fp64" else 1e-12)
    P = oparams(L, Nt)
    phi = dev(I.gaussian_field(10, L, Nt) * 0.7)
    pf = dev(I.fermion_noise(11, nrhs, L, Nt))
    F, spf, sb, st = ctx.force(phi, pf, include_boson=True, precond=True)
    phi_o = I.to_paper_boson(phi.cpu().numpy())
    Fo, spf_o, _ = ohmc.force(P, phi_o, to_paper_vecs(pf), method="dense")
    assert rel(I.to_paper_boson(F.cpu().numpy()), Fo) < 1e-10
    assert abs(spf - spf_o) < 1e-10 * abs(spf_o)
    assert abs(sb - boson.action(P, phi_o)) < 1e-12 * abs(sb)
    Ff, _, _, _ = ctx.force(phi, pf, include_boson=False, precond=False)
    Fo_f, _, _ = ohmc.force(P, phi_o, to_paper_vecs(pf), method="dense", include_boson=False)
    assert rel(I.to_paper_boson(Ff.cpu().numpy()), Fo_f) < 1e-10


@pytest.mark.parametrize("L,Nt", [(4, 8), (6, 7), (20, 12)])
def test_metric_operations(L, Nt):
    ctx = ctx_for(L, Nt)
    w = np.fft.fftn(I.gaussian_field(12, L, Nt), axes=(1, 2, 3), norm="ortho")
    sig_g = (w * np.conj(w)).real + 0.1                       # even in k, positive (library layout)
    z_g = I.gaussian_field(13, L, Nt)
    sig_o, z_o = I.to_paper_boson(sig_g), I.to_paper_boson(z_g)
    sig, z = dev(sig_g), dev(z_g)
    from paper_2204_14241_gb300.hmc import METRIC_MOMENTUM, METRIC_VELOCITY, METRIC_KINETIC, METRIC_ACCUM
    pi = ctx.metric(METRIC_MOMENTUM, sig, z)
    pi_o = ohmc.momentum(sig_o, z_o)
    assert rel(I.to_paper_boson(pi.cpu().numpy()), pi_o) < 1e-12
    v = ctx.metric(METRIC_VELOCITY, sig, pi)
    assert rel(I.to_paper_boson(v.cpu().numpy()), ohmc.velocity(sig_o, pi_o)) < 1e-12
    k = ctx.metric(METRIC_KINETIC, sig, pi)
    assert abs(k - ohmc.kinetic(sig_o, pi_o)) < 1e-12 * abs(k)
    acc = ctx.metric(METRIC_ACCUM, sig, z)
    acc = ctx.metric(METRIC_ACCUM, sig, pi, out=acc)
    ref = ohmc.sigma_estimate([z_o, pi_o]) * 2
    assert rel(I.to_paper_boson(acc.cpu().numpy()), ref) < 1e-12


def test_boson_action_and_force_parity():
    L, Nt = 6, 7
    ctx = ctx_for(L, Nt, nrhs=1)
    P = oparams(L, Nt)
    phi = dev(I.gaussian_field(14, L, Nt))
    pf = dev(np.zeros((1, Nt, L, L, 2, 2), dtype=complex))
    F, spf, sb, _ = ctx.force(phi, pf, include_boson=True, precond=False)
    phi_o = I.to_paper_boson(phi.cpu().numpy())
    assert spf == 0.0
    assert abs(sb - boson.action(P, phi_o)) < 1e-12 * abs(sb)
    assert rel(I.to_paper_boson(F.cpu().numpy()), -boson.grad(P, phi_o)) < 1e-12


@pytest.mark.parametrize("mode,guess", [("fp64", 0), ("mixed", 0), ("mixed", 1), ("mixed", 2), ("mixed", 3), ("mixed", 4),
                                        ("mixed", 5)])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_trajectory_matches_oracle(mode, guess, nrhs):
    # the small configuration: L = 4, Nt = 8, dtau = 0.1, eps = 0.05, n_leap = 10; guess = m starts
    # each force solve from the degree-m extrapolation of the previous solutions (same stopping test)
    L, Nt, eps, n_leap = 4, 8, 0.05, 10
    ctx = ctx_for(L, Nt, mode, nrhs=nrhs, tol=1e-12, guess=guess)
    P = oparams(L, Nt)
    phi0 = I.gaussian_field(20, L, Nt)
    w = np.fft.fftn(I.gaussian_field(21, L, Nt), axes=(1, 2, 3), norm="ortho")
    sig_g = (w * np.conj(w)).real * 0.5 + 0.5
    chi = I.fermion_noise(22, nrhs, L, Nt)
    z = I.gaussian_field(23, L, Nt)
    u = 0.37
    phi = dev(phi0)
    out = ctx.trajectory([phi], [dev(sig_g)], eps, n_leap, nrhs=nrhs, precond=True,
                         chi=[dev(chi)], z=[dev(z)], u=[u])
    ref = ohmc.trajectory(P, I.to_paper_boson(phi0), I.to_paper_boson(sig_g),
                          [I.to_paper_fermion(chi[k]) for k in range(nrhs)], I.to_paper_boson(z), u, eps,
                          n_leap, method="dense")
    assert abs(out["dH"][0] - ref["dH"]) < 1e-8, (out["dH"], ref["dH"])
    assert out["accepted"][0] == ref["accept"]
    e = out["energies"][0]
    assert abs(e[0] - ref["kinetic"][0]) < 1e-10 * abs(e[0])
    assert abs(e[1] - ref["S_B"][0]) < 1e-10 * abs(e[1])
    assert abs(e[2] - ref["S_PF"][0]) < 1e-10 * abs(e[2])
    assert abs(e[5] - ref["S_PF"][1]) < 1e-9 * abs(e[5])
    assert rel(I.to_paper_boson(phi.cpu().numpy()), ref["phi"]) < 1e-9


def test_trajectory_two_chains_uneven():
    chains = [(4, 8, 0.5), (6, 4, 0.8)]
    ctx = ctx_for(4, 8, "mixed", nrhs=1, tol=1e-12, chains=chains)
    phis, sigs, chis, zs, us, refs = [], [], [], [], [], []
    for c, (L, Nt, r) in enumerate(chains):
        phi0 = I.gaussian_field(30 + c, L, Nt) * 0.5
        chi = I.fermion_noise(40 + c, 1, L, Nt)
        z = I.gaussian_field(50 + c, L, Nt)
        sig = np.ones((3, Nt, L, L))
        phis.append(dev(phi0)); sigs.append(dev(sig)); chis.append(dev(chi)); zs.append(dev(z)); us.append(0.5)
        refs.append(ohmc.trajectory(oparams(L, Nt, r), I.to_paper_boson(phi0), I.to_paper_boson(sig),
                                    [I.to_paper_fermion(chi[0])], I.to_paper_boson(z), 0.5, 0.04, 5, method="dense"))
    out = ctx.trajectory(phis, sigs, 0.04, 5, nrhs=1, chi=chis, z=zs, u=us)
    for c in range(2):
        assert abs(out["dH"][c] - refs[c]["dH"]) < 1e-8
        assert rel(I.to_paper_boson(phis[c].cpu().numpy()), refs[c]["phi"]) < 1e-9


def test_philox_known_answers():
    # Random123 known-answer vectors for Philox4x32-10 (Salmon et al., SC'11)
    ctx = ctx_for(4, 8)
    kat = [((0, 0, 0, 0), 0, (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
           ((0xffffffff,) * 4, 0xffffffffffffffff, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
           ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), 0x299f31d0a4093822,
            (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for ctr, key, want in kat:
        got = ctx.philox_raw(key, ctr, 1).cpu().tolist()
        assert tuple(got) == want


def test_philox_normals_statistics():
    ctx = ctx_for(4, 8)
    z = ctx.philox_normal(7, 3, 1_000_000).cpu().numpy()
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1) < 5e-3
    c = ctx.philox_normal(7, 4, 500_000, complex_out=True).cpu().numpy()
    assert abs(np.mean(np.abs(c) ** 2) - 1) < 5e-3 and abs(np.mean(c.real * c.imag)) < 3e-3
    z2 = ctx.philox_normal(7, 3, 1_000_000).cpu().numpy()
    assert np.array_equal(z, z2)


def test_philox_trajectory_reproducible():
    L, Nt = 4, 8
    ctx = ctx_for(L, Nt, "mixed", nrhs=1)
    phi0 = dev(I.gaussian_field(60, L, Nt))
    sig = dev(np.ones((3, Nt, L, L)))
    a, b = phi0.clone(), phi0.clone()
    o1 = ctx.trajectory([a], [sig], 0.05, 4, seed=11, counter=5)
    o2 = ctx.trajectory([b], [sig], 0.05, 4, seed=11, counter=5)
    assert o1["dH"] == o2["dH"] and torch.equal(a, b)


def test_full_size_apply_A_sampled():
    # the largest configuration: L = 80, Nt = 160, 8 right-hand sides, FP32 storage
    L, Nt, K = 80, 160, 8
    ctx = ctx_for(L, Nt, "mixed", nrhs=K)
    P = oparams(L, Nt)
    phi64 = I.smooth_field(70, L, Nt, 0.5, 2.0 / (9 * 0.01)) / np.sqrt(0.1)
    phi = dev(phi64, torch.float32)
    x = dev(I.fermion_noise(71, K, L, Nt), torch.complex64)
    y, norms = ctx.apply_MdagM(phi, x, norms=True)
    phi_o = I.to_paper_boson(phi.double().cpu().numpy())
    xv = x.cpu().numpy().astype(np.complex128)
    yv = y.cpu().numpy().astype(np.complex128)
    for k in (0, K - 1):
        ref = fermion.apply_A(P, phi_o, I.to_paper_fermion(xv[k]))
        assert rel(I.to_paper_fermion(yv[k]), ref) < 1e-5
        t = fermion.apply_Ddag(P, phi_o, I.to_paper_fermion(xv[k]))
        assert abs(norms[k] - np.vdot(t, t).real) < 1e-5 * norms[k]


def test_errors_reported():
    from paper_2204_14241_gb300.hmc import HmcError, HMC_ERR_ARG, HMC_ERR_NOCONV, HMC_ERR_NONFINITE
    L, Nt = 4, 8
    ctx = ctx_for(L, Nt, "mixed", nrhs=1)
    phi = dev(I.gaussian_field(80, L, Nt))
    b = dev(I.fermion_noise(81, 1, L, Nt))
    x, st = ctx.cg_solve(phi, b, maxit=1, precond=False, raise_on_noconv=False)
    assert st["status"] == HMC_ERR_NOCONV and not st["converged"]
    bad = phi.clone()
    bad[0, 0, 0, 0] = float("nan")
    with pytest.raises(HmcError) as e:
        ctx.cg_solve(bad, b)
    assert e.value.code == HMC_ERR_NONFINITE
    with pytest.raises(HmcError) as e:
        ctx._check(ctx.lib.apply_M(ctx.h, 3, 0, None, None, None, 0, 1))
    assert e.value.code == HMC_ERR_ARG
    # the context stays usable after every error
    x, st = ctx.cg_solve(phi, b)
    assert st["converged"]


def test_sdw_susceptibility_matches_oracle():
    from oracle import observables
    from paper_2204_14241_gb300.observables import SdwSusceptibility
    L, Nt = 6, 7
    ctx = ctx_for(L, Nt, nrhs=1)
    est = SdwSusceptibility(ctx)
    samples = [I.gaussian_field(400 + i, L, Nt) for i in range(5)]
    for s in samples:
        est.add(dev(s))
    ref = observables.sdw_susceptibility([I.to_paper_boson(s) for s in samples], 0.1)   # [n, m_x, m_y]
    got = np.swapaxes(est.value().cpu().numpy(), -1, -2)
    assert rel(got, ref) < 1e-12


def test_paper_preset_runs_and_matches_oracle_force():
    from paper_2204_14241_gb300 import presets
    from paper_2204_14241_gb300.hmc import Context
    kw = presets.paper_nesting(2)
    L, Nt = 6, 8
    ctx = Context(L, Nt, solver="mixed", nrhs_max=1, cg_tol=1e-12, **kw)
    phi = dev(I.gaussian_field(410, L, Nt) * 0.5)
    pf = dev(I.fermion_noise(411, 1, L, Nt))
    F, spf, _, _ = ctx.force(phi, pf, include_boson=True, precond=True)
    P = Params(L=L, Nt=Nt, **kw)
    Fo, spf_o, _ = ohmc.force(P, I.to_paper_boson(phi.cpu().numpy()), to_paper_vecs(pf), method="dense")
    assert rel(I.to_paper_boson(F.cpu().numpy()), Fo) < 1e-7 and abs(spf - spf_o) < 1e-10 * abs(spf_o)


def test_warmup_tuner_matches_oracle():
    # Eqs. (acc_ineq) and (ESJD) driven by GPU trajectories against the oracle's tuner on the
    # same explicit noise: identical step-size decisions, acceptance and ESJD estimates.
    from oracle import tuning as otuning
    from paper_2204_14241_gb300.tuning import Tuner
    L, Nt = 4, 8
    ctx = ctx_for(L, Nt, "mixed", nrhs=1, tol=1e-12)
    P = oparams(L, Nt)
    phi0 = I.gaussian_field(500, L, Nt) * 0.5
    sig = np.ones((3, Nt, L, L))

    def raw(t):
        return I.fermion_noise(600 + t, 1, L, Nt), I.gaussian_field(700 + t, L, Nt), I.uniform(800 + t)

    def gpu_noise(t):
        chi, z, u = raw(t)
        return dev(chi), dev(z), u

    def cpu_noise(t):
        chi, z, u = raw(t)
        return [I.to_paper_fermion(chi[0])], I.to_paper_boson(z), u

    gt = Tuner(ctx, dev(phi0), dev(sig), noise=gpu_noise)
    ot = otuning.Tuner(P, I.to_paper_boson(phi0), I.to_paper_boson(sig), cpu_noise)
    e_g, h_g = gt.tune_eps(0.1, rounds=2, window=3)
    e_o, h_o = ot.tune_eps(0.1, rounds=2, window=3)
    assert e_g == e_o
    for a, b in zip(h_g, h_o):
        assert a[0] == b[0] and abs(a[1] - b[1]) < 1e-7 and abs(a[2] - b[2]) < 1e-7
    n_g, es_g = gt.tune_nmax(e_g, [1, 2, 4], per_candidate=2)
    n_o, es_o = ot.tune_nmax(e_o, [1, 2, 4], per_candidate=2)
    assert n_g == n_o
    for n in es_g:
        assert abs(es_g[n] - es_o[n]) < 1e-7 * max(1.0, abs(es_o[n]))
    assert rel(I.to_paper_boson(gt.phi.cpu().numpy()), ot.phi) < 1e-9


def test_mnorm_metric_op():
    from paper_2204_14241_gb300.hmc import METRIC_MNORM
    from oracle import tuning as otuning
    L, Nt = 6, 7
    ctx = ctx_for(L, Nt)
    w = np.fft.fftn(I.gaussian_field(510, L, Nt), axes=(1, 2, 3), norm="ortho")
    sig = (w * np.conj(w)).real + 0.2
    d = I.gaussian_field(511, L, Nt)
    got = ctx.metric(METRIC_MNORM, dev(sig), dev(d))
    ref = otuning.jump_norm2(I.to_paper_boson(sig), I.to_paper_boson(d))
    assert abs(got - ref) < 1e-12 * ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuned_apply_A_parity(prec):
    # autotune = 1 times the tile shapes on the call's buffers; results must not depend on them
    from paper_2204_14241_gb300.hmc import Context
    L, Nt = 20, 12
    ctx = Context(L, Nt, solver="fp64", nrhs_max=2, cg_tol=1e-12, autotune=1, **COUPLINGS)
    P = oparams(L, Nt)
    rdt, cdt = (torch.float64, torch.complex128) if prec == "fp64" else (torch.float32, torch.complex64)
    phi = dev(I.gaussian_field(520, L, Nt), rdt)
    x = dev(I.fermion_noise(521, 2, L, Nt), cdt)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for _ in range(2):   # first call tunes, second reuses the choice
        y, norms = ctx.apply_MdagM(phi, x, norms=True)
        for k, (yk, xk) in enumerate(zip(to_paper_vecs(y), to_paper_vecs(x))):
            phi_o = I.to_paper_boson(phi.double().cpu().numpy())
            assert rel(yk, fermion.apply_A(P, phi_o, xk)) < tol
            t = fermion.apply_Ddag(P, phi_o, xk)
            assert abs(norms[k] - np.vdot(t, t).real) < tol * norms[k]


def test_64_uneven_chains_trajectory():
    # the batched configuration's shape: 64 chains, L in {12, 16, 20, 24}, Nt in {24, 32, 48},
    # r_i ~ U[0.2, 1.0], 2 right-hand sides; one update of every chain, two chains checked
    # against the oracle (PCG to 1e-13 there, 1e-12 here)
    from paper_2204_14241_gb300.hmc import Context
    chains = []
    for i in range(64):
        L = (12, 16, 20, 24)[i % 4]
        Nt = (24, 32, 48)[(i // 4) % 3]
        r = 0.2 + 0.8 * I.uniform(900 + i)
        chains.append((L, Nt, r))
    ctx = Context(12, 24, solver="mixed", nrhs_max=2, cg_tol=1e-12, chains=chains, **{**COUPLINGS})
    phis, sigs, chis, zs, us = [], [], [], [], []
    for i, (L, Nt, r) in enumerate(chains):
        phis.append(dev(I.gaussian_field(1000 + i, L, Nt) * 0.5))
        sigs.append(dev(np.ones((3, Nt, L, L))))
        chis.append(dev(I.fermion_noise(2000 + i, 2, L, Nt)))
        zs.append(dev(I.gaussian_field(3000 + i, L, Nt)))
        us.append(I.uniform(4000 + i))
    phi_in = [p.clone() for p in phis]
    out = ctx.trajectory(phis, sigs, 0.02, 2, nrhs=2, chi=chis, z=zs, u=us)
    assert all(np.isfinite(out["dH"])) and max(out["max_true_resid"]) <= 1e-12
    for i in (0, 1):
        L, Nt, r = chains[i]
        ref = ohmc.trajectory(oparams(L, Nt, r), I.to_paper_boson(phi_in[i].cpu().numpy()),
                              np.ones((3, Nt, L, L)),
                              [I.to_paper_fermion(chis[i].cpu().numpy()[k]) for k in range(2)],
                              I.to_paper_boson(zs[i].cpu().numpy()), us[i], 0.02, 2, method="pcg", tol=1e-13)
        assert abs(out["dH"][i] - ref["dH"]) < 1e-8, (i, out["dH"][i], ref["dH"])
        assert out["accepted"][i] == ref["accept"]
        assert rel(I.to_paper_boson(phis[i].cpu().numpy()), ref["phi"]) < 1e-9


@pytest.mark.parametrize("L,Nt,method", [(6, 7, "dense"), (12, 24, "pcg")])
def test_green_estimator_matches_oracle(L, Nt, method):
    # Section "Fermionic observables": diag(F~^* D^-1 F~) from K Rademacher probes, the K solves
    # as one multi-RHS CG
    from oracle import observables
    K = 3
    ctx = ctx_for(L, Nt, "mixed", nrhs=K, tol=1e-12)
    P = oparams(L, Nt)
    phi0 = I.gaussian_field(530, L, Nt) * 0.7
    rng = np.random.default_rng(531)
    v = rng.choice([-1.0, 1.0], size=(K, Nt, L, L, 2, 2)).astype(np.complex128)
    est, st = ctx.green_estimate(dev(phi0), dev(v))
    assert st["converged"]
    ref = observables.green_diagonal(P, I.to_paper_boson(phi0), [I.to_paper_fermion(v[k]).real for k in range(K)],
                                     method=method, tol=1e-13)
    assert rel(I.to_paper_fermion(est.cpu().numpy()), ref) < 1e-8


def test_green_estimator_free_limit():
    # g = 0: the estimate is 1 / K-hat exactly for any probes (Eq. Kdiag)
    from paper_2204_14241_gb300.hmc import Context
    L, Nt = 8, 12
    kw = dict(COUPLINGS)
    kw["g"] = 0.0
    ctx = Context(L, Nt, solver="mixed", nrhs_max=2, cg_tol=1e-12, **kw)
    P = Params(L=L, Nt=Nt, **kw)
    v = np.random.default_rng(532).choice([-1.0, 1.0], size=(2, Nt, L, L, 2, 2)).astype(np.complex128)
    est, _ = ctx.green_estimate(dev(np.zeros((3, Nt, L, L))), dev(v))
    kh = fermion.free_symbol(P)[:, None]
    ref = 1.0 / np.broadcast_to(kh, (2, 2, Nt, L, L))
    assert rel(I.to_paper_fermion(est.cpu().numpy()), ref) < 1e-9


@pytest.mark.parametrize("precond", [False, True])
def test_trajectory_bench_kernel_set_16x16x16(precond):
    # The benchmark's kernel set on a lattice small enough for the oracle: L = 16 (complex64 strip
    # operator; plain CG with the fused x, r, p update as the benchmark runs it, or PCG with the
    # fused (x, y) preconditioner passes and the in-place tau pass at Nt = 16), 8 right-hand sides,
    # degree-4 chronological start, mixed precision, Yukawa coupling 1, an ordered field (uniform
    # 2.8 along component 3 plus free-boson fluctuations) and the free-boson sigma-hat. Oracle:
    # PCG from a zero start to 1e-13 on every solve.
    L, Nt, K, eps, n_leap = 16, 16, 8, 0.02, 4
    kt = 2.0 / (9 * 0.01)
    ctx = ctx_for(L, Nt, "mixed", nrhs=K, tol=1e-12, guess=4)
    P = oparams(L, Nt)
    phi0 = I.ordered_field(40, L, Nt, 0.5, kt, 1.0 / np.sqrt(0.1), 2.8)
    sig = np.broadcast_to(I.spectrum(L, Nt, 0.5, kt)[None] / 0.1, (3, Nt, L, L)).copy()
    chi = I.fermion_noise(41, K, L, Nt)
    z = I.gaussian_field(42, L, Nt)
    u = 0.45
    phi = dev(phi0)
    out = ctx.trajectory([phi], [dev(sig)], eps, n_leap, nrhs=K, precond=precond, chi=[dev(chi)], z=[dev(z)],
                         u=[u])
    ref = ohmc.trajectory(P, I.to_paper_boson(phi0), I.to_paper_boson(sig),
                          [I.to_paper_fermion(chi[k]) for k in range(K)], I.to_paper_boson(z), u, eps, n_leap,
                          method="pcg", tol=1e-13)
    assert out["status"] == 0 and out["max_true_resid"][0] <= 1e-12
    assert abs(out["dH"][0] - ref["dH"]) < 1e-8, (out["dH"], ref["dH"])
    assert out["accepted"][0] == ref["accept"]
    e = out["energies"][0]
    for got, want in ((e[0], ref["kinetic"][0]), (e[1], ref["S_B"][0]), (e[2], ref["S_PF"][0]),
                      (e[3], ref["kinetic"][1]), (e[4], ref["S_B"][1]), (e[5], ref["S_PF"][1])):
        assert abs(got - want) < 1e-10 * abs(want)
    assert rel(I.to_paper_boson(phi.cpu().numpy()), ref["phi"]) < 1e-9


def test_precision_report_short():
    # The 20 x 20 x 40 single-chain precision report in short (3 trajectories of 4 steps): the
    # mixed solver against the FP64 one on identical noise, per trajectory, at the mixed-mode
    # bars (force and S_PF 1e-5 relative, |dH| 1e-8); and the FP64 mode's force against the
    # oracle at the same field, at the FP64-mode bar 1e-10. Both solvers stop on the same FP64
    # true residual, so their solutions differ by up to the condition number times the tolerance:
    # at 1e-10 the dH difference reaches ~1e-7 (the full report), at 1e-12 it is below 1e-8.
    from paper_2204_14241_gb300.experiments import precision_report
    r = precision_report(n_traj=3, n_leap=4, eps=0.05, tol=1e-12)
    assert all(row["status"] == (0, 0) for row in r["rows"])
    assert r["force_rel_err_max"] < 1e-5 and r["S_pf_rel_err_max"] < 1e-5 and r["dH_err_max"] < 1e-8, r
    L, Nt = 20, 40
    ctx = ctx_for(L, Nt, "fp64", nrhs=1, tol=1e-14)
    P = oparams(L, Nt)
    phi = dev(I.gaussian_field(7, L, Nt))
    pf = dev(I.fermion_noise(8, 1, L, Nt))
    F, spf, _, _ = ctx.force(phi, pf, include_boson=True, precond=True)
    Fo, spf_o, _ = ohmc.force(P, I.to_paper_boson(phi.cpu().numpy()), to_paper_vecs(pf), method="pcg", tol=1e-15)
    assert rel(I.to_paper_boson(F.cpu().numpy()), Fo) < 1e-10
    assert abs(spf - spf_o) < 1e-10 * abs(spf_o)


def test_trajectory_stats_record():
    # the per-trajectory record: one entry per force solve, consistent with the trajectory's
    # totals, and per-phase GPU times that cover the trajectory
    L, Nt, n_leap = 6, 8, 5
    ctx = ctx_for(L, Nt, "mixed", nrhs=2, tol=1e-10, guess=2)
    phi = dev(I.gaussian_field(90, L, Nt) * 0.5)
    sig = dev(np.ones((3, Nt, L, L)))
    out = ctx.trajectory([phi], [sig], 0.05, n_leap, nrhs=2, seed=3, counter=1)
    st = ctx.trajectory_stats(0)
    assert st["n_solves"] == n_leap + 1
    assert sum(st["iterations"]) == out["cg_iterations"][0]
    assert max(st["true_resid"]) == out["max_true_resid"][0]
    assert st["reliable_updates"] >= n_leap + 1
    ph = st["phase_ms"]
    assert all(v >= 0 for v in ph.values()) and ph["solve"] > 0 and ph["metric"] > 0


@pytest.mark.parametrize("centered", [False, True])
def test_sigma_estimate_matches_oracle(centered):
    # Eq. (covest) accumulated by the library over a batch with a nonzero mean, as printed and
    # about the batch mean (tuning.SigmaEstimator), against the oracle's estimates
    from paper_2204_14241_gb300.tuning import SigmaEstimator
    L, Nt = 6, 8
    ctx = ctx_for(L, Nt)
    mu = np.array([0.2, -0.1, 1.5])[:, None, None, None]
    samples = [I.gaussian_field(950 + i, L, Nt) + mu for i in range(6)]
    est = SigmaEstimator(ctx, dev(samples[0]), centered)
    for s in samples:
        est.add(dev(s))
    got = I.to_paper_boson(est.value().cpu().numpy())
    fn = ohmc.sigma_estimate_centered if centered else ohmc.sigma_estimate
    ref = fn([I.to_paper_boson(s) for s in samples])
    assert rel(got, ref) < 1e-12


def test_device_wait_timeout_is_reported():
    # The fused operator's device-side waits are bounded. With test_wait_timeout its first wait
    # targets a barrier that nothing arms: the launch gives up after wait_spin_limit polls, drains
    # its copy in flight and returns, and the call reports HMC_ERR_TIMEOUT; the context stays usable.
    from paper_2204_14241_gb300.hmc import Context, HmcError, HMC_ERR_TIMEOUT
    L, Nt = 16, 8
    ctx = Context(L, Nt, solver="mixed", nrhs_max=1, cg_tol=1e-10, wait_spin_limit=64, test_wait_timeout=1,
                  **COUPLINGS)
    phi = dev(I.gaussian_field(1, L, Nt), torch.float32)
    x = dev(I.fermion_noise(2, 1, L, Nt), torch.complex64)
    with pytest.raises(HmcError) as e:
        ctx.apply_MdagM(phi, x, norms=True)
    assert e.value.code == HMC_ERR_TIMEOUT
    with pytest.raises(HmcError) as e:
        ctx.cg_solve(dev(I.gaussian_field(1, L, Nt)), dev(I.fermion_noise(2, 1, L, Nt)), precond=False)
    assert e.value.code == HMC_ERR_TIMEOUT
    y = ctx.apply_M(phi, x)   # no device-side waits on this path
    P = oparams(L, Nt)
    ref = fermion.apply_D(P, I.to_paper_boson(phi.double().cpu().numpy()), to_paper_vecs(x)[0])
    assert rel(to_paper_vecs(y)[0], ref) < 1e-5
    ok = ctx_for(L, Nt, "mixed", nrhs=1)
    y2, n2 = ok.apply_MdagM(phi, x, norms=True)
    assert rel(to_paper_vecs(y2)[0], fermion.apply_A(P, I.to_paper_boson(phi.double().cpu().numpy()),
                                                       to_paper_vecs(x)[0])) < 1e-5


def _uneven_chains(n=64):
    chains = []
    for i in range(n):
        L = (12, 16, 20, 24)[i % 4]
        Nt = (24, 32, 48)[(i // 4) % 3]
        chains.append((L, Nt, 0.2 + 0.8 * I.uniform(900 + i)))
    return chains


@pytest.mark.parametrize("guess", [0, 3])
def test_64_uneven_chains_batched_trajectory(guess):
    # the batched configuration in its batched form: every force solve of the 64 chains (2 RHS each)
    # is one persistent launch; chains checked against the oracle (PCG to 1e-13 there, 1e-12 here)
    # and every chain against the serial path on the same explicit noise
    from paper_2204_14241_gb300.hmc import Context
    chains = _uneven_chains()
    kw = dict(solver="mixed", nrhs_max=2, cg_tol=1e-12, chains=chains, initial_guess=guess, **COUPLINGS)
    ctx_b = Context(12, 24, batch_chains=1, **kw)
    ctx_s = Context(12, 24, **kw)
    phis, sigs, chis, zs, us = [], [], [], [], []
    for i, (L, Nt, r) in enumerate(chains):
        phis.append(dev(I.gaussian_field(1000 + i, L, Nt) * 0.5))
        sigs.append(dev(np.ones((3, Nt, L, L))))
        chis.append(dev(I.fermion_noise(2000 + i, 2, L, Nt)))
        zs.append(dev(I.gaussian_field(3000 + i, L, Nt)))
        us.append(I.uniform(4000 + i))
    phi_in = [p.clone() for p in phis]
    phis_s = [p.clone() for p in phis]
    out = ctx_b.trajectory(phis, sigs, 0.02, 2, nrhs=2, chi=chis, z=zs, u=us)
    ref_s = ctx_s.trajectory(phis_s, sigs, 0.02, 2, nrhs=2, precond=False, chi=chis, z=zs, u=us)
    assert out["status"] == 0 and max(out["max_true_resid"]) <= 1e-12
    for i in range(64):
        assert abs(out["dH"][i] - ref_s["dH"][i]) < 1e-8, (i, out["dH"][i], ref_s["dH"][i])
        assert out["accepted"][i] == ref_s["accepted"][i]
        assert rel(phis[i].cpu().numpy(), phis_s[i].cpu().numpy()) < 1e-9
    for i in (0, 1, 6):
        L, Nt, r = chains[i]
        ref = ohmc.trajectory(oparams(L, Nt, r), I.to_paper_boson(phi_in[i].cpu().numpy()), np.ones((3, Nt, L, L)),
                              [I.to_paper_fermion(chis[i].cpu().numpy()[k]) for k in range(2)],
                              I.to_paper_boson(zs[i].cpu().numpy()), us[i], 0.02, 2, method="pcg", tol=1e-13)
        assert abs(out["dH"][i] - ref["dH"]) < 1e-8, (i, out["dH"][i], ref["dH"])
        assert out["accepted"][i] == ref["accept"]
        assert rel(I.to_paper_boson(phis[i].cpu().numpy()), ref["phi"]) < 1e-9
    st = ctx_b.trajectory_stats(5)
    assert st["n_solves"] == 3 and sum(st["iterations"]) == out["cg_iterations"][5]


def test_batched_graph_replay_matches_direct_launches():
    # the batched leapfrog as a CUDA graph (captured on the first trajectory, replayed on the
    # next, captured again when eps changes) gives bit for bit the trajectories of the same
    # kernels launched one by one, with the same per-solve statistics
    from paper_2204_14241_gb300.hmc import Context
    chains = _uneven_chains(8)
    kw = dict(solver="mixed", nrhs_max=2, cg_tol=1e-10, chains=chains, initial_guess=2, batch_chains=1, **COUPLINGS)
    ctx_g = Context(12, 24, batch_graph=1, **kw)
    ctx_d = Context(12, 24, batch_graph=0, **kw)
    phis_g = [dev(I.gaussian_field(1200 + i, L, Nt) * 0.5) for i, (L, Nt, _) in enumerate(chains)]
    phis_d = [p.clone() for p in phis_g]
    sigs = [dev(np.ones((3, Nt, L, L))) for (L, Nt, _) in chains]
    for t, eps in enumerate((0.02, 0.02, 0.02, 0.03)):
        og = ctx_g.trajectory(phis_g, sigs, eps, 3, nrhs=2, seed=11, counter=t)
        od = ctx_d.trajectory(phis_d, sigs, eps, 3, nrhs=2, seed=11, counter=t)
        assert og["status"] == 0 and od["status"] == 0
        assert og["dH"] == od["dH"] and og["accepted"] == od["accepted"]
        assert og["cg_iterations"] == od["cg_iterations"]
        assert all(torch.equal(a, b) for a, b in zip(phis_g, phis_d))
        for c in (0, 5):
            sg, sd = ctx_g.trajectory_stats(c), ctx_d.trajectory_stats(c)
            assert sg["n_solves"] == sd["n_solves"] == 4
            assert sg["iterations"] == sd["iterations"] and sg["true_resid"] == sd["true_resid"]
            assert sg["reliable_updates"] == sd["reliable_updates"]


def test_batched_grid_barrier_timeout():
    # the batched solve's grid barriers are bounded: with test_wait_timeout its first barrier
    # waits for one arrival more than there are blocks, gives up after wait_spin_limit
    # microseconds, and the trajectory reports HMC_ERR_TIMEOUT with phi restored
    from paper_2204_14241_gb300.hmc import Context, HMC_ERR_TIMEOUT
    chains = _uneven_chains(4)
    ctx = Context(12, 24, solver="mixed", nrhs_max=1, cg_tol=1e-10, chains=chains, batch_chains=1,
                  test_wait_timeout=1, wait_spin_limit=20000, **COUPLINGS)
    phis = [dev(I.gaussian_field(1100 + i, L, Nt) * 0.5) for i, (L, Nt, _) in enumerate(chains)]
    phi_in = [p.clone() for p in phis]
    sigs = [dev(np.ones((3, Nt, L, L))) for (L, Nt, _) in chains]
    out = ctx.trajectory(phis, sigs, 0.02, 1, nrhs=1, seed=3, counter=0, check=False)
    assert out["status"] == HMC_ERR_TIMEOUT
    assert all(torch.equal(a, b) for a, b in zip(phis, phi_in))
    ok = Context(12, 24, solver="mixed", nrhs_max=1, cg_tol=1e-10, chains=chains, batch_chains=1, **COUPLINGS)
    o2 = ok.trajectory(phis, sigs, 0.02, 1, nrhs=1, seed=3, counter=0)
    assert o2["status"] == 0 and all(np.isfinite(o2["dH"]))
