"""torch.autograd adjoint of the triples Jacobian transformation.

``JacobianRight.apply(R1, R2, context, omega)`` returns rho = A R (triples part,
``mlcc3_jacobian_right``); its backward is the transpose transformation
``mlcc3_jacobian_left`` (sigma = L^T A), so no triples amplitudes are stored
between forward and backward: each pass rebuilds them per batch.

The library's adjoint identity <L, A R>_w = <A^T L, R>_w holds under the
unique-element inner product (weight 1/2 on the doubles elements the active-pair
block stores twice).  Autograd works with the plain Euclidean product over the
stored elements, so for an incoming gradient g the backward returns
w * A^T(gbar / w), gbar being g averaged over the two stored copies of an
element; then <g, A R> = <grad, R> for every block-symmetric R.
"""
from __future__ import annotations

import torch


def block_weights(no, nv, NO, NV, device):
    """1/2 where both pairs are active and the element is not diagonal, else 1."""
    w = torch.ones((no, nv, NO, NV), dtype=torch.float64, device=device)
    w[:, :, :no, :nv] = 0.5
    idx_i = torch.arange(no, device=device)[:, None]
    idx_a = torch.arange(nv, device=device)[None, :]
    w[idx_i, idx_a, idx_i, idx_a] = 1.0
    return w


def symmetrize_block(x, no, nv):
    x = x.clone()
    aa = x[..., :no, :nv].clone()
    x[..., :no, :nv] = 0.5 * (aa + aa.permute(*range(aa.dim() - 4), -2, -1, -4, -3))
    return x


class JacobianRight(torch.autograd.Function):
    """rho1, rho2 = A (R1, R2) at frequency omega (one trial vector)."""

    @staticmethod
    def forward(ctx, R1, R2, context, omega):
        NO, NV, no, nv, _ = context.dims
        rho1 = torch.zeros_like(R1)
        rho2 = torch.zeros_like(R2)
        context.jacobian_right([float(omega)], R1.contiguous(), R2.contiguous(), rho1, rho2)
        ctx.context = context
        ctx.omega = float(omega)
        return rho1, rho2

    @staticmethod
    def backward(ctx, g1, g2):
        context = ctx.context
        NO, NV, no, nv, _ = context.dims
        w = block_weights(no, nv, NO, NV, g2.device)
        if g1 is None:
            g1 = torch.zeros((NV, NO), dtype=torch.float64, device=w.device)
        if g2 is None:
            g2 = torch.zeros_like(w)
        L1 = g1.contiguous()
        L2 = (symmetrize_block(g2, no, nv) / w).contiguous()
        s1 = torch.zeros_like(L1)
        s2 = torch.zeros_like(L2)
        context.jacobian_left([ctx.omega], L1, L2, s1, s2)
        return s1, w * s2, None, None


def jacobian_right(context, omega, R1, R2):
    """Differentiable rho = A R (see JacobianRight)."""
    return JacobianRight.apply(R1, R2, context, omega)
