"""The allocation-free entry point apply_MdagM_static, for callers that must not allocate device
memory after start-up (fixed memory budgets, runtimes that own every allocation, code that
cannot create a context because creating one allocates its workspace).

It must give the same y = D D^dagger x and ||D^dagger x||^2 as the context-based apply_MdagM,
call after call, although its reduction scratch is one fixed device array shared by every
call. Tolerances are those of the operator tests: 1e-12 relative in FP64, 1e-5 in FP32.
This file sorts last so that a run stopping at the first failure has run everything else."""

import numpy as np
import pytest
import torch

from paper_2204_14241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COUPLINGS = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5, u=1.0, c=3.0)


def rel(a, b):
    a, b = a.detach().cpu().numpy(), b.detach().cpu().numpy()
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L,Nt,nrhs", [(12, 24, 2), (20, 12, 3), (6, 7, 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_matches_context_apply(L, Nt, nrhs, prec):
    from paper_2204_14241_gb300.hmc import Context, apply_MdagM_static
    ctx = Context(L, Nt, solver="fp64", nrhs_max=nrhs, **COUPLINGS)
    rdt, cdt = (torch.float64, torch.complex128) if prec == "fp64" else (torch.float32, torch.complex64)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for call in range(2):   # two calls in a row share (and overwrite) the static scratch
        phi = torch.from_numpy(I.gaussian_field(700 + call, L, Nt)).cuda().to(rdt)
        x = torch.from_numpy(I.fermion_noise(710 + call, nrhs, L, Nt)).cuda().to(cdt)
        y_ref, n_ref = ctx.apply_MdagM(phi, x, norms=True)
        y = torch.empty_like(x)
        y, n = apply_MdagM_static(ctx.params, L, Nt, phi, x, y, norms=True)
        assert rel(y, y_ref) < tol
        for a, b in zip(n, n_ref):
            assert abs(a - b) < tol * b
        # without norms the kernel runs without touching the scratch
        y2 = apply_MdagM_static(ctx.params, L, Nt, phi, x, torch.empty_like(x))
        assert rel(y2, y_ref) < tol


def test_static_rejects_oversized_requests():
    # the row-sum scratch holds 64 norms: 65 right-hand sides with norms are refused on the
    # host before anything is launched
    from paper_2204_14241_gb300.hmc import HmcError, HMC_ERR_ARG, Params, apply_MdagM_static
    L, Nt = 4, 8
    p = Params()
    p.dtau, p.g = 0.1, 1.0
    p.t_h[:], p.t_v[:], p.mu[:] = [1.0, 0.5], [0.5, 1.0], [-0.5, -0.5]
    phi = torch.zeros((3, Nt, L, L), dtype=torch.float64, device="cuda")
    x = torch.zeros((65, Nt, L, L, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(HmcError) as e:
        apply_MdagM_static(p, L, Nt, phi, x, torch.empty_like(x), norms=True)
    assert e.value.code == HMC_ERR_ARG and "64" in str(e.value)


def test_static_checks_arguments_before_launch():
    # mismatched precisions, shapes, layouts and devices are refused by the binding before the
    # library is called, so no kernel can read or write outside the tensors
    from paper_2204_14241_gb300.hmc import Params, apply_MdagM_static
    L, Nt = 4, 8
    p = Params()
    p.dtau, p.g = 0.1, 1.0
    phi64 = torch.zeros((3, Nt, L, L), dtype=torch.float64, device="cuda")
    x128 = torch.zeros((2, Nt, L, L, 2, 2), dtype=torch.complex128, device="cuda")
    x64 = x128.to(torch.complex64)
    bad = [
        (phi64.float(), x128, torch.empty_like(x128)),                       # float32 phi, complex128 x
        (phi64, x64, torch.empty_like(x64)),                                 # float64 phi, complex64 x
        (phi64[:, :4].contiguous(), x128, torch.empty_like(x128)),           # phi smaller than (L, Nt)
        (phi64, x128[:, :4].contiguous(), torch.empty_like(x128)),           # x smaller than (L, Nt)
        (phi64, x128, torch.empty_like(x128)[:1]),                           # out smaller than x
        (phi64, x128, torch.empty_like(x64)),                                # out of another dtype
        (phi64, x128.transpose(2, 3), torch.empty_like(x128)),               # x not contiguous
        (phi64.cpu(), x128, torch.empty_like(x128)),                         # phi on the host
    ]
    for phi, x, out in bad:
        with pytest.raises(ValueError):
            apply_MdagM_static(p, L, Nt, phi, x, out, norms=True)


def test_static_partial_sum_limit_message():
    # a 2912 x 2912 x 2 lattice in complex64 has 182 x 182 = 33124 blocks of 16 x 16 sites, so two
    # right-hand sides with norms need 66248 partial sums, past the 65536 static slots; the call
    # is refused before any launch (x and y are left uninitialised) and says so with both factors
    from paper_2204_14241_gb300.hmc import HmcError, HMC_ERR_ARG, Params, apply_MdagM_static
    L, Nt, K = 2912, 2, 2
    p = Params()
    p.dtau, p.g = 0.1, 1.0
    phi = torch.empty((3, Nt, L, L), dtype=torch.float32, device="cuda")
    x = torch.empty((K, Nt, L, L, 2, 2), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(HmcError) as e:
        apply_MdagM_static(p, L, Nt, phi, x, y, norms=True)
    msg = str(e.value)
    assert e.value.code == HMC_ERR_ARG
    assert "66248" in msg and "33124" in msg and "65536" in msg, msg
    del phi, x, y
    torch.cuda.empty_cache()
