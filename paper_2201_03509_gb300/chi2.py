"""Differentiable TOD chi^2 (torch.autograd.Function) over the C ABI.

L(m, g, xi) = sum_q 1/2 sum_{k>=1} [ rhat_k^2 / P_k + ln P_k ],
rhat = C(M(d - g P m)), the correlated-noise-marginalised likelihood of the
gain step.  Forward: tod_project (unit gain) + tod_chi2.  Backward (hand
written): dL/dm = -P^T(g v) through tod_bin (the adjoint of the
projection), dL/dg and dL/d(sigma0, f_knee, alpha) from tod_chi2.  All
arithmetic runs in the library's kernels; this module only marshals.
"""
from __future__ import annotations

import torch

from . import Plan


class TodChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, map_tqu, gain, psd, plan: Plan, d, flags, pix, psi):
        """map_tqu (npix, 3) FP64/FP32, gain (ndetscan,) FP64, psd (ndet, 3)
        FP64; d FP32[N], flags uint32 words, pix int32[N], psi int16[N]
        (decoded pointing).  Returns the scalar chi^2 (FP64)."""
        dev = d.device
        npix = plan.npix
        m4 = torch.zeros((npix, 4), dtype=torch.float32, device=dev)
        m4[:, :3] = map_tqu.detach().to(torch.float32)
        s = torch.empty(plan.N, dtype=torch.float32, device=dev)
        plan.project(m4, pix, psi, None, s)
        g = gain.detach().to(torch.float64).contiguous()
        th = psd.detach().to(torch.float64).contiguous()
        chi2 = torch.empty(plan.nq, dtype=torch.float64, device=dev)
        dg = torch.empty_like(chi2)
        dpsd = torch.empty((plan.nq, 3), dtype=torch.float64, device=dev)
        v = torch.empty(plan.N, dtype=torch.float32, device=dev)
        plan.chi2(d, s, g, flags, th, chi2, dg, dpsd, v)
        ctx.save_for_backward(v, dg, dpsd, g)
        ctx.plan, ctx.flags, ctx.psi, ctx.ndet = plan, flags, psi, psd.shape[0]
        ctx.map_dtype, ctx.psd_dtype = map_tqu.dtype, psd.dtype
        return chi2.sum()

    @staticmethod
    def backward(ctx, grad_out):
        v, dg, dpsd, g = ctx.saved_tensors
        plan = ctx.plan
        dev = v.device
        grad_map = grad_gain = grad_psd = None
        if ctx.needs_input_grad[0]:
            # -P^T(g v): binning of v with unit white-noise weights
            unit = torch.zeros((ctx.ndet, 3), dtype=torch.float64, device=dev)
            unit[:, 0] = 1.0
            unit[:, 1] = 1.0
            unit[:, 2] = -1.0
            zeros = torch.zeros_like(v)
            A = torch.empty((plan.npix, 6), dtype=torch.float64, device=dev)
            b = torch.empty((plan.npix, 3), dtype=torch.float64, device=dev)
            hits = torch.empty(plan.npix, dtype=torch.int32, device=dev)
            plan.bin(ctx.psi, v, zeros, g, ctx.flags, unit, A, b, hits)
            grad_map = (-b * grad_out).to(ctx.map_dtype)
        if ctx.needs_input_grad[1]:
            grad_gain = dg * grad_out
        if ctx.needs_input_grad[2]:
            det = torch.arange(plan.nq, device=dev) % ctx.ndet
            gp = torch.zeros((ctx.ndet, 3), dtype=torch.float64, device=dev)
            gp.index_add_(0, det, dpsd)
            grad_psd = (gp * grad_out).to(ctx.psd_dtype)
        return grad_map, grad_gain, grad_psd, None, None, None, None, None


def tod_chi2(map_tqu, gain, psd, plan, d, flags, pix, psi):
    return TodChi2.apply(map_tqu, gain, psd, plan, d, flags, pix, psi)
