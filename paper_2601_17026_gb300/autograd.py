"""Differentiable optimal-surface energy on float cost volumes.

Forward: each float32 volume is quantised on the device to cq = round_half_even(scale*c)
(inside graph construction) and solved exactly; the output is the optimal energy
E*(c) = min_h E(h) of Eq. 1 in float units (E*_q / scale), and optionally the
structured-hinge loss L = E(h_t) - min_h [E(h) - margin * Hamming(h, h_t)].

Backward (Danskin's theorem; E* is a minimum of functions linear in c): dE*/dc is the
one-hot of the optimal surface, dL/dc = onehot(h_t) - onehot(h_hat) where h_hat solves
the loss-augmented problem. The energy solve, the loss-augmented solve (started from the
energy solve's final state) and the loss value are one library call. Quantisation is treated as the identity in the backward
(the exact gradient of the quantised problem, scaled back to float units). One backward
kernel writes the whole gradient volume.
"""
from __future__ import annotations

import torch

from . import pog

SCALE = 1024.0


def _alpha_q(alpha: float, scale: float) -> int:
    a = alpha * scale
    if a != int(a) or a < 0:
        raise ValueError(f"alpha * scale must be a non-negative integer, got {a}")
    return int(a)


def _solve_all(cost, delta, alpha_q, scale, options, h_aug=None, margin_q=0):
    """All volumes of the batch in one batched solve (quantisation fused into the build)."""
    _, energies, heights = pog.pog_solve_batch_f32(cost, scale, delta, alpha_q, h_aug, margin_q, options)
    return heights, torch.tensor(energies, dtype=torch.int64)


class PogSolve(torch.autograd.Function):
    """(E*, L_hinge, h, h_hat) = PogSolve.apply(cost, delta, alpha, h_target, margin, scale, options).

    cost: float32 CUDA [B, X, Y, Z]. E* and L are float64 [B] (float units); h, h_hat are
    int32 [B, X, Y]. Without h_target, L and h_hat are returned as None.
    """

    @staticmethod
    def forward(ctx, cost, delta, alpha, h_target=None, margin=1.0, scale=SCALE, options=None):
        if cost.dim() != 4 or cost.dtype != torch.float32 or not cost.is_cuda:
            raise ValueError("cost must be a float32 CUDA tensor [B, X, Y, Z]")
        cost = cost.contiguous()
        B, X, Y, Z = cost.shape
        aq = _alpha_q(alpha, scale)
        loss = h_hat = None
        if h_target is None:
            heights, eq = _solve_all(cost, delta, aq, scale, options)
        else:
            # energy solve, loss-augmented solve (warm-started) and the hinge value, in one call
            h_target = h_target.to(device=cost.device, dtype=torch.int32).contiguous()
            r = pog.pog_solve_batch_f32_hinge(cost, scale, h_target, _alpha_q(margin, scale), delta, aq, options)
            heights, h_hat = r["heights"], r["h_hat"]
            eq = torch.tensor(r["energies"], dtype=torch.int64)
            loss = torch.tensor(r["hinge"], dtype=torch.int64).to(torch.float64) / scale
        energy = eq.to(torch.float64) / scale
        ctx.save_for_backward(heights, h_target, h_hat)
        ctx.mark_non_differentiable(heights)
        if h_hat is not None:
            ctx.mark_non_differentiable(h_hat)
        ctx.shape = cost.shape
        return energy.to(cost.device), None if loss is None else loss.to(cost.device), heights, h_hat

    @staticmethod
    def backward(ctx, g_energy, g_loss, _gh, _ghh):
        heights, h_target, h_hat = ctx.saved_tensors
        B, X, Y, Z = ctx.shape
        grad = torch.empty(ctx.shape, dtype=torch.float32, device=heights.device)
        ge = (g_energy if g_energy is not None else torch.zeros(B, device=heights.device)).to(torch.float32).contiguous()
        gl = None
        if h_target is not None and g_loss is not None:
            gl = g_loss.to(torch.float32).contiguous()
        pog.pog_backward(grad, heights, ge, h_target if gl is not None else None,
                         h_hat if gl is not None else None, gl)
        return grad, None, None, None, None, None, None


def pog_energy(cost, delta: int, alpha: float, scale: float = SCALE, options=None):
    """Optimal energy E* [B] (float64, float units) of float32 cost volumes [B, X, Y, Z]."""
    return PogSolve.apply(cost, delta, alpha, None, 1.0, scale, options)[0]


def solve_with_hinge(cost, h_target, delta: int, alpha: float, margin: float = 1.0, scale: float = SCALE,
                     options=None):
    """(E* [B], hinge loss [B], optimal surfaces [B,X,Y], loss-augmented surfaces [B,X,Y])."""
    return PogSolve.apply(cost, delta, alpha, h_target, margin, scale, options)
