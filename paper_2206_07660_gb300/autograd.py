"""torch.autograd.Function wrappers of the two contractions.

The forward passes run the library's kernels (gw_polarization,
gw_selfenergy); the backward passes call the hand-written adjoint chains
(gw_polarization_vjp, gw_selfenergy_vjp).  Gradients follow PyTorch's
convention for complex inputs (dL/dRe + i dL/dIm for a real loss L).  The
context's G (and P~) are re-set from the saved inputs before each backward,
so other calls on the context between forward and backward are harmless.
Setting `gw.adjoint_c64 = True` makes the backward passes run in complex64
arithmetic (gw_polarization_vjp_c64, gw_selfenergy_vjp_c64).
"""
import torch


class Polarization(torch.autograd.Function):
    """P~0(tau) [nq, ntau, naux, naux] from G(tau) [ntau, nk, nao, nao] (Eq. tilde_P0_tau)."""

    @staticmethod
    def forward(ctx, G_tau, gw):
        G_tau = G_tau.detach().contiguous()
        gw.set("G_tau", G_tau)
        gw.polarization()
        out = torch.empty(gw.shape_of("P0_tau"), dtype=torch.complex128, device=G_tau.device)
        gw.get("P0_tau", out=out)
        ctx.gw = gw
        ctx.save_for_backward(G_tau)
        return out

    @staticmethod
    def backward(ctx, Pbar):
        (G_tau,) = ctx.saved_tensors
        ctx.gw.set("G_tau", G_tau)
        return ctx.gw.polarization_vjp(Pbar, c64=getattr(ctx.gw, "adjoint_c64", False)), None


class SelfEnergy(torch.autograd.Function):
    """Sigma~(tau) [ntau, nk, nao, nao] from G(tau) and P~(tau) (Eq. tilde_sigma2).

    The forward also updates the context's stored self-energy (gw_selfenergy
    mixes it with the previous one when damping < 1)."""

    @staticmethod
    def forward(ctx, G_tau, P_tau, gw):
        G_tau = G_tau.detach().contiguous()
        P_tau = P_tau.detach().contiguous()
        gw.set("G_tau", G_tau)
        gw.set("P_tau", P_tau)
        gw.selfenergy()
        out = torch.empty(gw.shape_of("Sigma_tau"), dtype=torch.complex128, device=G_tau.device)
        gw.get("Sigma_tau", out=out)
        ctx.gw = gw
        ctx.save_for_backward(G_tau, P_tau)
        return out

    @staticmethod
    def backward(ctx, Sbar):
        G_tau, P_tau = ctx.saved_tensors
        ctx.gw.set("G_tau", G_tau)
        ctx.gw.set("P_tau", P_tau)
        Gbar, Pbar = ctx.gw.selfenergy_vjp(Sbar, c64=getattr(ctx.gw, "adjoint_c64", False))
        return Gbar, Pbar, None
