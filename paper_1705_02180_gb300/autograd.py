"""Differentiable potential energy over path frames (torch.autograd), marshalling only.

PotentialEnergy(X) -> U(X_t) per frame (scps_energy_forces). Its backward
returns g_t * grad U(X_t) through ForceGrad, whose own backward is the
Hessian-vector product H(X_t) v_t (scps_hvp). So second derivatives of path
functionals work, e.g. the gradient of sum_t |grad U(X_t)|^2 (a term of the
Onsager-Machlup action of Eq. (SOM)) is sum_t 2 H(X_t) grad U(X_t).
ForceNormSquared computes that action per segment of frames with one force launch
forward and one force + one HVP launch backward (force_norm_action).
All arithmetic runs in the CUDA kernels behind the C ABI.
"""
from __future__ import annotations

import torch


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


class ForceNormSquared(torch.autograd.Function):
    """sum_t |grad U(X_t)|^2 over frames X (float64 scalar). The forces are not kept:
    the backward evaluates them again and returns g * 2 H(X_t) grad U(X_t) (one
    force launch and one HVP launch), which is activation checkpointing over the
    frames without the generic checkpoint machinery. First order only: for further
    derivatives compose ForceGrad instead."""

    @staticmethod
    def forward(ctx, X, system, topo):
        X = X.contiguous()
        U = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        F = torch.empty_like(X)
        system.energy_forces(topo, X, U, F)
        ctx.save_for_backward(X)
        ctx.system, ctx.topo = system, topo
        return (F.double() ** 2).sum()

    @staticmethod
    def backward(ctx, g):
        (X,) = ctx.saved_tensors
        U = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        F = torch.empty_like(X)
        ctx.system.energy_forces(ctx.topo, X, U, F)
        HV = torch.empty_like(X)
        ctx.system.hvp(ctx.topo, X, F.mul_(-2.0), HV)  # v = 2 grad U = -2 F
        return HV * g.to(HV.dtype), None, None


class ForceNormAction(torch.autograd.Function):
    """sum_t |grad U(X_t)|^2 over all frames X (float64 scalar) with activation
    checkpointing over segments of frames: the forward evaluates every frame in one launch
    and keeps only the positions; the backward recomputes the forces of each segment and
    applies 2 H(X_t) grad U(X_t) to it (one force launch and one HVP launch per segment).
    The force launches run in order on one side stream (they share the system's list
    scratch), the HVP launches on another, so that segment k's HVP overlaps segment k+1's
    forces; two segments' forces are live at most. First order only, like ForceNormSquared."""

    @staticmethod
    def forward(ctx, X, system, topo, segment):
        X = X.contiguous()
        U = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        F = torch.empty_like(X)
        system.energy_forces(topo, X, U, F)
        ctx.save_for_backward(X)
        ctx.system, ctx.topo, ctx.segment = system, topo, segment
        return (F.double() ** 2).sum()

    @staticmethod
    def backward(ctx, g):
        (X,) = ctx.saved_tensors
        seg = min(ctx.segment, X.shape[0])
        cur = torch.cuda.current_stream()
        fs, hs = torch.cuda.Stream(), torch.cuda.Stream()  # forces, HVPs
        fs.wait_stream(cur)
        hs.wait_stream(cur)
        U = [torch.empty(seg, dtype=torch.float64, device=X.device) for _ in range(2)]
        F = [torch.empty((seg,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
             for _ in range(2)]
        HV = torch.empty_like(X)
        done_f, done_h = [], []
        for k, s in enumerate(range(0, X.shape[0], seg)):
            n = min(seg, X.shape[0] - s)
            b = k & 1
            if k >= 2:
                fs.wait_event(done_h[k - 2])  # the HVP that read this buffer has finished
            with torch.cuda.stream(fs):
                ctx.system.energy_forces(ctx.topo, X[s:s + n], U[b][:n], F[b][:n])
                F[b][:n].mul_(-2.0)  # v = 2 grad U
                done_f.append(fs.record_event())
            hs.wait_event(done_f[k])
            with torch.cuda.stream(hs):
                ctx.system.hvp(ctx.topo, X[s:s + n], F[b][:n], HV[s:s + n])
                done_h.append(hs.record_event())
        cur.wait_stream(fs)
        cur.wait_stream(hs)
        return HV * g.to(HV.dtype), None, None, None


def force_norm_action(system, X, topo=0, segment=50):
    """sum_t |grad U(X_t)|^2 over the frames; the backward recomputes the forces segment by
    segment of `segment` frames (activation checkpointing over path frames)."""
    return ForceNormAction.apply(X, system, topo, segment)
