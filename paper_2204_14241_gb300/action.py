"""The pseudofermion action S(phi) = sum_k varphi_k^dagger (D D^dagger)^{-1} varphi_k
(Eq. Z with pfs) as a torch.autograd.Function.

forward: one multi-RHS CG solve and the action, through libhmc's `force` entry point
(which also returns the force; only the action is kept).
backward: the force kernel. dS/dphi = -F_PF, where F_PF is the fermion part of the force
(include_boson = 0); the solution X = A^{-1} varphi and Y = D^dagger X are recomputed in
backward, not stored, so memory does not grow with the lattice.
The boson field phi is float64 (3, Nt, L, L); varphi is complex128 (k, Nt, L, L, 2, 2).
Only phi is differentiable: a varphi that requires grad is refused in forward.
"""

import torch


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, phi, phi_pf, hmc_ctx, chain=0, precond=True):
        if fctx.needs_input_grad[1]:
            raise ValueError("PseudofermionAction: only phi is differentiable; pass varphi without requires_grad")
        phi_c = phi.detach().contiguous()
        _, s_pf, _, _ = hmc_ctx.force(phi_c, phi_pf.contiguous(), include_boson=False, precond=precond,
                                      chain=chain)
        fctx.save_for_backward(phi_c, phi_pf)
        fctx.hmc = (hmc_ctx, chain, precond)
        return torch.tensor(s_pf, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(fctx, grad_out):
        phi, phi_pf = fctx.saved_tensors
        hmc_ctx, chain, precond = fctx.hmc
        F, _, _, _ = hmc_ctx.force(phi, phi_pf.contiguous(), include_boson=False, precond=precond, chain=chain)
        return -grad_out * F, None, None, None, None


def pseudofermion_action(phi, phi_pf, hmc_ctx, chain=0, precond=True):
    """S_PF(phi) with gradient -F_PF (see module docstring)."""
    return PseudofermionAction.apply(phi, phi_pf, hmc_ctx, chain, precond)
