"""torch.autograd functions over the FEWHA operators and the converged reconstruction.

Both run the library's CUDA kernels in forward and backward (no PyTorch arithmetic on the
path): the forward model s = Gamma P phi with its adjoint kernels, and the converged
reconstruction a~ = F W^T M^-1 b(s) whose backward is a second PCG on the symmetric M
(fewha_backward), giving gradients with respect to the slopes, alpha and the layer Cn2
weights; and the fixed-iteration frame a~ = F W^T c_k(s) from a warm start, whose backward
runs the PCG recurrence in reverse (fewha_frame_vjp), giving the gradient with respect to
the slopes of the map the real-time loop runs.
"""

import torch

from .fewha import Reconstructor  # noqa: F401  (type of the `recon` arguments)


class ForwardModel(torch.autograd.Function):
    """s = Gamma P phi (Sec. 2) on the layer values phi; backward P^T Gamma^T."""

    @staticmethod
    def forward(ctx, phi, recon):
        ctx.recon = recon
        return recon.forward(phi.detach().contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.recon.forward_adj(g.detach().contiguous()), None


class ConvergedReconstruction(torch.autograd.Function):
    """a~ = F W^T c*, M(alpha, w) c* = b(s) solved to a tolerance (the MAP estimate).

    slopes: CUDA tensor of the handle's dtype; alpha: 0-d tensor; cn2: 1-d tensor of the
    layer weights (both float64, any device).  Gradients flow to all three.
    """

    @staticmethod
    def forward(ctx, slopes, alpha, cn2, recon, tol, max_iters):
        a = float(alpha)
        w = [float(x) for x in cn2.detach().cpu()]
        if getattr(recon, "_grad_params", None) != (a, tuple(w)):
            recon.update_params(alpha=a, cn2_weights=w)
            recon._grad_params = (a, tuple(w))
        dm, iters, rel = recon.reconstruct_converged(slopes.detach().contiguous(), tol, max_iters)
        ctx.recon = recon
        ctx.meta = (alpha.dtype, alpha.device, cn2.dtype, cn2.device)
        ctx.solve = (iters, rel)
        return dm

    @staticmethod
    def backward(ctx, g):
        gs, ga, gw = ctx.recon.backward(g.detach().contiguous())
        adt, adev, wdt, wdev = ctx.meta
        return (gs, torch.tensor(ga, dtype=adt, device=adev), torch.tensor(gw, dtype=wdt, device=wdev),
                None, None, None)


def reconstruct(recon, slopes, alpha, cn2, tol=None, max_iters=20000):
    """Differentiable converged reconstruction (see ConvergedReconstruction)."""
    return ConvergedReconstruction.apply(slopes, alpha, cn2, recon, tol, max_iters)


def forward_model(recon, phi):
    """Differentiable s = Gamma P phi (see ForwardModel)."""
    return ForwardModel.apply(phi, recon)


class UnrolledFrame(torch.autograd.Function):
    """a~ = F W^T c_k(s): the frame's `iters` PCG iterations from the warm start c0 with the
    explicit initial residual (no control law); backward by reverse mode through the
    recurrence.  Gradients flow to the slopes (c0 is a constant)."""

    @staticmethod
    def forward(ctx, slopes, c0, recon):
        s = slopes.detach().contiguous()
        c = c0.detach().contiguous()
        a, _ = recon.frame_vjp(s, c)
        ctx.recon = recon
        ctx.save_for_backward(s, c)
        return a

    @staticmethod
    def backward(ctx, g):
        s, c = ctx.saved_tensors
        _, gs = ctx.recon.frame_vjp(s, c, g.detach().contiguous())
        return gs, None, None


def frame(recon, slopes, c0):
    """Differentiable fixed-iteration frame (see UnrolledFrame)."""
    return UnrolledFrame.apply(slopes, c0, recon)
