"""The largest configuration, 80 x 80 x 160 (dtau = 0.1, Yukawa coupling 1), against the FP64
oracle: the force at one field and a two-step trajectory, one pseudofermion right-hand side each,
through the benchmark's kernels (complex64 strip operator, FP64 reliable updates; plain CG with
the fused x, r, p update as the benchmark runs it, and PCG with the fused (x, y) and in-place tau
preconditioner passes; the trajectory with the degree-4 chronological start). The oracle's values are stored in tests/golden/full_size_80x80x160.json, written by
tests/golden/make_full_size.py from the oracle alone (its preconditioned CG takes minutes per
solve at this size); the inputs are regenerated here from the same seeds.

Tolerances: force 1e-7 relative to its largest entry (the mixed-mode bar is 1e-5; both sides
solve to a relative residual of 1e-12), S_PF 1e-10 relative, |dH_gpu - dH_oracle| < 1e-8,
phi' 1e-9 relative to its largest entry."""

import json
import os
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_full_size as G  # noqa: E402


def golden():
    with open(os.path.join(HERE, "golden", "full_size_80x80x160.json")) as f:
        return json.load(f)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def context(guess):
    from paper_2204_14241_gb300.hmc import Context
    return Context(G.L, G.NT, solver="mixed", nrhs_max=1, cg_tol=1e-12, initial_guess=guess, **G.COUPLINGS)


@pytest.mark.parametrize("precond", [True, False])
def test_full_size_force_matches_oracle(precond):
    g = golden()
    phi, sig, pf, chi, z, idx = G.inputs()
    assert list(map(int, idx)) == g["indices"]
    ctx = context(0)
    F, spf, sb, st = ctx.force(dev(phi), dev(pf), include_boson=True, precond=precond)
    assert st["converged"] and st["true_rel_resid"] <= 1e-12
    got = F.cpu().numpy().ravel()[idx]
    want = np.asarray(g["force"]["F_samples"])
    assert np.abs(got - want).max() < 1e-7 * g["force"]["F_max_abs"]
    assert abs(spf - g["force"]["S_pf"]) < 1e-10 * abs(g["force"]["S_pf"])
    ctx.close()


@pytest.mark.parametrize("precond", [True, False])
def test_full_size_trajectory_matches_oracle(precond):
    g = golden()
    t = g["trajectory"]
    phi0, sig, pf, chi, z, idx = G.inputs()
    ctx = context(4)
    phi = dev(phi0)
    out = ctx.trajectory([phi], [dev(sig)], G.EPS, G.NLEAP, nrhs=1, precond=precond, chi=[dev(chi)], z=[dev(z)],
                         u=[G.U])
    assert out["status"] == 0 and out["max_true_resid"][0] <= 1e-12
    assert abs(out["dH"][0] - t["dH"]) < 1e-8, (out["dH"][0], t["dH"])
    assert out["accepted"][0] == t["accept"]
    e = out["energies"][0]
    want = [t["kinetic"][0], t["S_B"][0], t["S_PF"][0], t["kinetic"][1], t["S_B"][1], t["S_PF"][1]]
    for a, b in zip(e, want):
        assert abs(a - b) < 1e-10 * abs(b), (e, want)
    got = phi.cpu().numpy().ravel()[idx]
    if t["accept"]:
        assert np.abs(got - np.asarray(t["phi_samples"])).max() < 1e-9 * t["phi_max_abs"]
    else:
        assert np.array_equal(got, phi0.ravel()[idx])
    ctx.close()
