"""Differentiable potential energy over path frames (torch.autograd), marshalling only.

PotentialEnergy(X) -> U(X_t) per frame (scps_energy_forces). Its backward
returns g_t * grad U(X_t) through ForceGrad, whose own backward is the
Hessian-vector product H(X_t) v_t (scps_hvp). So second derivatives of path
functionals work, e.g. the gradient of sum_t |grad U(X_t)|^2 (a term of the
Onsager-Machlup action of Eq. (SOM)) is sum_t 2 H(X_t) grad U(X_t).
All arithmetic runs in the CUDA kernels behind the C ABI.
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint as _ckpt


class ForceGrad(torch.autograd.Function):
    """grad U(X_t) for frames X (float32, (T, n, 3), CUDA); backward: H(X_t) v_t."""

    @staticmethod
    def forward(ctx, X, system, topo):
        X = X.contiguous()
        U = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        F = torch.empty_like(X)
        system.energy_forces(topo, X, U, F)
        ctx.save_for_backward(X)
        ctx.system, ctx.topo = system, topo
        return -F

    @staticmethod
    def backward(ctx, v):
        (X,) = ctx.saved_tensors
        HV = torch.empty_like(X)
        ctx.system.hvp(ctx.topo, X, v.contiguous().to(X.dtype), HV)
        return HV, None, None


class PotentialEnergy(torch.autograd.Function):
    """U(X_t) per frame (float64); backward: g_t grad U(X_t), itself differentiable."""

    @staticmethod
    def forward(ctx, X, system, topo):
        X = X.contiguous()
        U = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        system.energy_forces(topo, X, U, None)
        ctx.save_for_backward(X)
        ctx.system, ctx.topo = system, topo
        return U

    @staticmethod
    def backward(ctx, gU):
        (X,) = ctx.saved_tensors
        grad = ForceGrad.apply(X, ctx.system, ctx.topo)
        return gU.to(grad.dtype)[:, None, None] * grad, None, None


def potential_energy(system, X, topo=0):
    return PotentialEnergy.apply(X, system, topo)


def force_norm_action(system, X, topo=0, segment=50):
    """sum_t |grad U(X_t)|^2 over the frames, recomputed per segment of `segment`
    frames in the backward pass (activation checkpointing over path frames)."""

    def seg(xs):
        g = ForceGrad.apply(xs, system, topo)
        return (g.double() ** 2).sum()

    total = X.new_zeros((), dtype=torch.float64)
    for s in range(0, X.shape[0], segment):
        xs = X[s:s + segment]
        total = total + _ckpt.checkpoint(seg, xs, use_reentrant=False)
    return total
