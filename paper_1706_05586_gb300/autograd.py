"""The sampled misfit as a differentiable PyTorch function of the PaLS parameters.

f(p) = ||V^T (C^T A(mu(p))^{-1} B - M) W||_F^2 (Theorem 1, Eq. (EsTResidual)).  The
forward pass runs the block solve of the forward and adjoint columns; the library
keeps both field blocks on the device (checkpointed), so the hand-written backward
is the adjoint-field sensitivity g_mu = -2 Re sum conj(R_s) Z_l U_i followed by the
PaLS chain rule g_p = (dmu/dp)^T g_mu (Eq. (Jacobiancomp), Eq. (UnbiasedGrad)),
without a second solve; for CUDA tensors the gradient is written to device memory
directly (dot_gradient_dev).  With recompute=True the fields are solved again in the
backward pass instead (the state is invalidated after the forward), for callers that
reuse the context for other work in between.

All arithmetic runs in libdot.so; this module only moves p and the results between
PyTorch tensors and the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dot as D


class PalsConstants:
    """mu_in, mu_out, cut-off c, Heaviside half width eps and gamma of Sec. 2."""

    def __init__(self, mu_in, mu_out, c, eps, gamma):
        self.mu_in, self.mu_out, self.c, self.eps, self.gamma = mu_in, mu_out, c, eps, gamma

    def args(self):
        return (self.mu_in, self.mu_out, self.c, self.eps, self.gamma)


def _set_p(handle, p: torch.Tensor, consts: PalsConstants):
    m0 = p.numel() // 5
    if p.is_cuda:
        pc = p.detach().to(torch.float64).contiguous()
        # the context copies pc on its own stream: finish producing it first
        torch.cuda.current_stream(p.device).synchronize()
        D.dot_set_pals_dev(handle, m0, pc.data_ptr(), *consts.args())
        return pc  # kept alive until the evaluation (which synchronizes) has read it
    D.dot_set_pals(handle, p.detach().to(torch.float64).cpu().numpy(), *consts.args())
    return None


# handle -> token of the forward pass whose solve the context currently caches
_cached = {}
_counter = [0]


def _key(handle):
    return getattr(handle, "value", handle)


class DotMisfit(torch.autograd.Function):
    """f(p) with a hand-written backward; see the module docstring."""

    @staticmethod
    def forward(ctx, p, handle, consts, recompute=False):
        keep = _set_p(handle, p, consts)
        f, _ = D.dot_misfit(handle)
        del keep
        _counter[0] += 1
        ctx.token = _counter[0]
        ctx.handle, ctx.consts = handle, consts
        ctx.save_for_backward(p.detach().clone())
        if recompute:
            # drop the cached solve (setting p invalidates it): the backward pass solves again
            D.dot_set_pals(handle, p.detach().to(torch.float64).cpu().numpy(), *consts.args())
            _cached[_key(handle)] = None
        else:
            _cached[_key(handle)] = ctx.token
        return torch.tensor(f, dtype=torch.float64, device=p.device)

    @staticmethod
    def backward(ctx, grad_out):
        (p,) = ctx.saved_tensors
        if _cached.get(_key(ctx.handle)) != ctx.token:
            # the context no longer holds this forward pass's solve (recompute mode, or
            # another forward ran in between): set p again and solve
            keep = _set_p(ctx.handle, p, ctx.consts)
        else:
            keep = None
        if p.is_cuda:
            # the gradient stays on the device: the library writes it there directly
            f_d = torch.empty(1, dtype=torch.float64, device=p.device)
            g_d = torch.empty(p.numel(), dtype=torch.float64, device=p.device)
            D.dot_gradient_dev(ctx.handle, f_d.data_ptr(), g_d.data_ptr())
            g = g_d.to(p.dtype)
        else:
            _, g, _ = D.dot_gradient(ctx.handle, p.numel())
            g = torch.from_numpy(np.asarray(g)).to(dtype=p.dtype)
        del keep
        _cached[_key(ctx.handle)] = ctx.token
        return grad_out * g, None, None, None


def misfit(p: torch.Tensor, handle, consts: PalsConstants, recompute: bool = False) -> torch.Tensor:
    """Differentiable sampled misfit of the context `handle` (grid, D, B, C, M, W, V and
    solver already set) at PaLS parameters p (5 * m0 values, per RBF alpha, beta, chi)."""
    return DotMisfit.apply(p, handle, consts, recompute)
