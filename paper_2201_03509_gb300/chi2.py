"""Differentiable TOD chi^2 (torch.autograd.Function) over the C ABI.

L(m, g, xi) = sum_q 1/2 sum_{k>=1} [ rhat_k^2 / P_k + ln P_k ],
rhat = C(M(d - g P m)), the correlated-noise-marginalised likelihood of the
gain step.  Forward: tod_project (tod_project_f64 in FP64) with unit gain,
then tod_chi2 (band total, per-detscan gain derivatives, per-detector PSD
gradients).  Backward (hand written): dL/dm = -P^T(g v) through
tod_project_adjoint.  The pointing is the plan's own decoded pointing, the
one its adjoint bins with.  Every reduction runs in the library's kernels;
this module only marshals tensors and scales by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import Plan


class TodChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, map_tqu, gain, psd, plan: Plan, d, flags, precision):
        """map_tqu (npix, 3), gain (ndetscan,), psd (ndet, 3); d FP32[N],
        flags uint32 words (as int32); precision Plan.PREC_F32 or PREC_F64.
        Returns the scalar chi^2 (FP64)."""
        dev = d.device
        pix, psi = plan.pointing()
        f64 = precision == Plan.PREC_F64
        if f64:
            m3 = map_tqu.detach().to(torch.float64).t().contiguous()
            s = torch.empty(plan.N, dtype=torch.float64, device=dev)
            plan.project_f64(m3, pix, psi, None, s)
        else:
            m4 = torch.zeros((plan.npix, 4), dtype=torch.float32, device=dev)
            m4[:, :3] = map_tqu.detach().to(torch.float32)
            s = torch.empty(plan.N, dtype=torch.float32, device=dev)
            plan.project(m4, pix, psi, None, s)
        g = gain.detach().to(torch.float64).contiguous()
        th = psd.detach().to(torch.float64).contiguous()
        chi2 = torch.empty(plan.nq, dtype=torch.float64, device=dev)
        dg = torch.empty_like(chi2)
        total = torch.empty(1, dtype=torch.float64, device=dev)
        dpsd = torch.empty((plan.ndet, 3), dtype=torch.float64, device=dev)
        v = torch.empty(plan.N, dtype=torch.float64 if f64 else torch.float32, device=dev)
        plan.chi2(d, s, g, flags, th, chi2, dg, total, dpsd, v, precision=precision)
        ctx.save_for_backward(v, dg, dpsd, g)
        ctx.plan, ctx.psi, ctx.precision = plan, psi, precision
        ctx.map_dtype, ctx.psd_dtype = map_tqu.dtype, psd.dtype
        return total[0]

    @staticmethod
    def backward(ctx, grad_out):
        v, dg, dpsd, g = ctx.saved_tensors
        plan = ctx.plan
        grad_map = grad_gain = grad_psd = None
        if ctx.needs_input_grad[0]:
            pt = torch.empty((plan.npix, 3), dtype=torch.float64, device=v.device)
            plan.project_adjoint(ctx.psi, v, g, pt, precision=ctx.precision)     # P^T (g v)
            grad_map = (pt * -grad_out).to(ctx.map_dtype)
        if ctx.needs_input_grad[1]:
            grad_gain = dg * grad_out
        if ctx.needs_input_grad[2]:
            grad_psd = (dpsd * grad_out).to(ctx.psd_dtype)
        return grad_map, grad_gain, grad_psd, None, None, None, None


def tod_chi2(map_tqu, gain, psd, plan, d, flags, precision: int = Plan.PREC_F32):
    return TodChi2.apply(map_tqu, gain, psd, plan, d, flags, precision)
