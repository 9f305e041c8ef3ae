"""Differentiable transforms: torch.autograd.Function wrappers over the C ABI.

The backward pass of synthesis runs the adjoint-synthesis kernel and the
backward pass of analysis the adjoint-analysis kernel (Sect. 4.5), both on
the current CUDA stream; nothing is stored between the passes except the plan
(the Legendre functions are recomputed, not kept).

Gradients follow torch's convention for a real loss L of complex inputs,
grad = dL/dRe + i dL/dIm, with the a_lm stored for m >= 0 only and the
m < 0 coefficients implied by the reality of the maps.  With D = diag(2 - delta_m0):

    synthesis  p = S a:      dL/da = D (Y^H g)      (adjoint synthesis, g = dL/dp;
                                                     Im part of m = 0 entries is 0)
    analysis   a = A p:      dL/dp = W S (D^-1 g)   (adjoint analysis of the
                                                     gradient with m > 0 halved)

where Y^H is the adjoint synthesis (analysis with unit weights) and W S the
adjoint analysis (synthesis times the ring weights).  Both follow from the real
inner product sum Re(conj(x) y) over the stored entries, for which the
synthesis counts every m > 0 coefficient twice (once for -m).  The factors D
and D^-1 are applied inside the library (the SHT_GRADIENT flag of the two
adjoint types); this module only allocates the outputs and passes pointers.

Inputs are CUDA tensors: a_lm as complex128 of shape (narrays, nalm), maps as
float64 of shape (narrays, npix), narrays = ncomp (spin 0) or 2 ncomp (spin:
E, B / Q, U interleaved).
"""
import torch

from . import sht as _sht

__all__ = ["synthesis", "analysis"]


def _rows(t):
    return [t[i] for i in range(t.shape[0])]


def _check(plan, t, dtype, width, what):
    if not t.is_cuda or t.dtype != dtype or t.dim() != 2 or t.shape != (plan.narrays, width):
        raise ValueError(f"{what}: expected a CUDA {dtype} tensor of shape ({plan.narrays}, {width}), "
                         f"got {tuple(t.shape)} {t.dtype} on {t.device}")


class _Synthesis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alm, plan):
        alm = alm.contiguous()
        _check(plan, alm, torch.complex128, plan.alm.size(), "a_lm")
        maps = torch.empty((plan.narrays, plan.geom.npix), dtype=torch.float64, device=alm.device)
        st = torch.cuda.current_stream(alm.device)
        _sht.sht_execute(plan, _sht.SHT_SYNTHESIS, _rows(alm), _rows(maps), 0, st)
        ctx.plan = plan
        return maps

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        g = g.contiguous()
        grad = torch.empty((plan.narrays, plan.alm.size()), dtype=torch.complex128, device=g.device)
        st = torch.cuda.current_stream(g.device)
        _sht.sht_execute(plan, _sht.SHT_ADJOINT_SYNTHESIS, _rows(grad), _rows(g), _sht.SHT_GRADIENT, st)
        return grad, None


class _Analysis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, maps, plan):
        maps = maps.contiguous()
        _check(plan, maps, torch.float64, plan.geom.npix, "maps")
        alm = torch.empty((plan.narrays, plan.alm.size()), dtype=torch.complex128, device=maps.device)
        st = torch.cuda.current_stream(maps.device)
        _sht.sht_execute(plan, _sht.SHT_ANALYSIS, _rows(alm), _rows(maps), 0, st)
        ctx.plan = plan
        return alm

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        g = g.contiguous()
        grad = torch.empty((plan.narrays, plan.geom.npix), dtype=torch.float64, device=g.device)
        st = torch.cuda.current_stream(g.device)
        _sht.sht_execute(plan, _sht.SHT_ADJOINT_ANALYSIS, _rows(g), _rows(grad), _sht.SHT_GRADIENT, st)
        return grad, None


def synthesis(plan, alm):
    """Maps (narrays, npix) float64 from a_lm (narrays, nalm) complex128; differentiable."""
    return _Synthesis.apply(alm, plan)


def analysis(plan, maps):
    """a_lm (narrays, nalm) complex128 from maps (narrays, npix) float64; differentiable."""
    return _Analysis.apply(maps, plan)
