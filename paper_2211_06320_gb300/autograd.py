"""torch.autograd.Function over the FPE path (§7.2: P and P' evaluated by
Algorithm A_p).  Forward: P(z_j) for complex128 points.  Backward, with
g = dL/dP (PyTorch's conjugate Wirtinger convention): dL/dz_j = g_j conj(P'(z_j))
and dL/da_k = sum_j g_j conj(z_j)^k over each point's kept terms
G_p cap [l_j, r_j].  Every step runs in libfpe's kernels; this module only
splits complex tensors into the real and imaginary arrays the C ABI takes.
"""
from __future__ import annotations

import torch

from . import (FPE_WITH_DERIV, Poly, fpe_eval, fpe_grad_coeffs, fpe_grad_points, fpe_precondition,
               fpe_to_complex)


def _parts(z):
    return z.real.contiguous(), z.imag.contiguous()


class PolyEval(torch.autograd.Function):
    """y = P(z) with P preconditioned from the values of `a` (FPE_WITH_DERIV)."""

    @staticmethod
    def forward(ctx, a, z, poly: Poly):
        zr, zi = _parts(z)
        out = fpe_eval(poly, zr, zi)
        re, im = fpe_to_complex(out)
        ctx.poly = poly
        ctx.n_coef = a.shape[0]
        ctx.save_for_backward(zr, zi)
        return torch.complex(re, im)

    @staticmethod
    def backward(ctx, g):
        zr, zi = ctx.saved_tensors
        gr, gi = _parts(g)
        grad_a = grad_z = None
        if ctx.needs_input_grad[1]:
            gz_re, gz_im = fpe_grad_points(ctx.poly, zr, zi, gr, gi)
            grad_z = torch.complex(gz_re, gz_im)
        if ctx.needs_input_grad[0]:
            ga_re = torch.zeros(ctx.n_coef, dtype=torch.float64, device=zr.device)
            ga_im = torch.zeros(ctx.n_coef, dtype=torch.float64, device=zr.device)
            fpe_grad_coeffs(ctx.poly, zr, zi, gr, gi, ga_re, ga_im)
            grad_a = torch.complex(ga_re, ga_im)
        return grad_a, grad_z, None


def precondition_for_grad(a: torch.Tensor, p: int = 53, flags: int = 0) -> Poly:
    """Preconditions the current values of the complex coefficient tensor `a`."""
    ac = a.detach().to("cpu", torch.complex128)
    return fpe_precondition(ac.real.numpy(), ac.imag.numpy(), None, p, flags | FPE_WITH_DERIV)


def poly_eval(a: torch.Tensor, z: torch.Tensor, poly: Poly = None) -> torch.Tensor:
    """Differentiable P(z); `poly` must be preconditioned from a's current values
    (built here when omitted)."""
    if poly is None:
        poly = precondition_for_grad(a)
    return PolyEval.apply(a, z, poly)
