"""torch.autograd.Function V_eff -> (rho, U) over the SQ path.

Forward: sq_build_hamiltonian + sq_density + sq_energy.  Backward: sq_density_vjp, the reverse
(adjoint) Chebyshev recursion with checkpoints every `checkpoint_k` steps, including the implicit
change of the Fermi level.  The scale and shift (spectral bounds) are held fixed, so pass explicit
bounds that contain the spectrum for every V_eff you differentiate at.
"""
import torch

from . import sq


class SQDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, veff, cell, precision, bounds, checkpoint_k):
        h = sq.build_for_cell(cell, bounds=bounds, d_veff=veff.detach().contiguous())
        rho = torch.empty_like(veff)
        sq.sq_density(h, cell.K, cell.kT, cell.N_e, precision, 0, rho)
        U, _, _ = sq.sq_energy(h)
        ctx.h = h
        ctx.checkpoint_k = checkpoint_k
        return rho, torch.tensor(U, dtype=torch.float64, device=veff.device)

    @staticmethod
    def backward(ctx, rho_bar, U_bar):
        rb = rho_bar.contiguous()
        ub = float(U_bar) if U_bar is not None else 0.0
        vbar = torch.empty_like(rb)
        sq.sq_density_vjp(ctx.h, rb, ub, ctx.checkpoint_k, vbar)
        ctx.h.close()
        return vbar, None, None, None, None


def sq_density_autograd(veff, cell, bounds, precision=sq.SQ_FP64, checkpoint_k=8):
    """(rho [N_d], U) as differentiable functions of the device tensor veff [N_d] (float64)."""
    return SQDensity.apply(veff, cell, precision, tuple(bounds), checkpoint_k)
