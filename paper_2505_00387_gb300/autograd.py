"""torch.autograd wrappers of the C ABI.

* ``radon(plan, m)``      d = L m, with backward L^T (aahrt_adjoint) and the
                          adjoint's backward L (aahrt_forward): L is linear, so
                          its vector-Jacobian product is the exact transpose.
* ``radon_adjoint(plan, d)``  m = L^T d, the transpose pair.
* ``fista(plan, d, lam, gamma, iters)``  m^iters of the unrolled sparse solve
                          (Sec. 4, eqs. ISTA and soft, FISTA momentum unless
                          ista=True); backward through aahrt_fista_vjp, which
                          recomputes the iterations from checkpoints.

Everything runs in libaahrt's kernels; these classes only marshal tensors.
Tensors are flat float32 CUDA tensors of the plan's model_len / data_len.
"""
from __future__ import annotations

import torch

from .plan import AahrtPlan


class _Radon(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: AahrtPlan, m: torch.Tensor):
        ctx.plan = plan
        return plan.forward(m.contiguous())

    @staticmethod
    def backward(ctx, g):
        return None, _RadonT.apply(ctx.plan, g.contiguous())


class _RadonT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: AahrtPlan, d: torch.Tensor):
        ctx.plan = plan
        return plan.adjoint(d.contiguous())

    @staticmethod
    def backward(ctx, g):
        return None, _Radon.apply(ctx.plan, g.contiguous())


class _Fista(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: AahrtPlan, d: torch.Tensor, lam: float, gamma: float, iters: int,
                ista: bool, checkpoint: int):
        d = d.contiguous()
        m, _ = plan.sparse_solve(d, lam, iters, ista=ista, gamma=gamma, want_info=False)
        ctx.plan = plan
        ctx.args = (lam, gamma, iters, ista, checkpoint)
        ctx.save_for_backward(d)
        return m

    @staticmethod
    def backward(ctx, m_bar):
        (d,) = ctx.saved_tensors
        lam, gamma, iters, ista, checkpoint = ctx.args
        _, d_bar = ctx.plan.fista_vjp(d, m_bar.contiguous(), lam, gamma, iters, ista=ista,
                                      checkpoint=checkpoint, want_m=False)
        return None, d_bar, None, None, None, None, None


def radon(plan: AahrtPlan, m: torch.Tensor) -> torch.Tensor:
    """d = L m, differentiable in m."""
    return _Radon.apply(plan, m)


def radon_adjoint(plan: AahrtPlan, d: torch.Tensor) -> torch.Tensor:
    """m = L^T d, differentiable in d."""
    return _RadonT.apply(plan, d)


def fista(plan: AahrtPlan, d: torch.Tensor, lam: float, gamma: float, iters: int, *,
          ista: bool = False, checkpoint: int = 10) -> torch.Tensor:
    """m^iters of the unrolled solve from 0, differentiable in d (gamma and
    lambda are constants of the layer)."""
    if not gamma > 0.0:
        raise ValueError("gamma must be > 0 (a fixed step of the layer)")
    return _Fista.apply(plan, d, float(lam), float(gamma), int(iters), bool(ista),
                        int(checkpoint))
