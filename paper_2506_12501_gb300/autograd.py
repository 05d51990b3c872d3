"""torch.autograd front end: integrals as a differentiable function of the
atom centres and the primitive exponents.

The forward pass is ``eri_batch``; the backward pass is the library's
adjoint kernel ``eri_batch_grad`` with W = the incoming gradient, so
``(ERIFunction.apply(...) * W).sum().backward()`` yields
d(sum W (ab|cd)) / d(centres, exponents) with the contraction coefficients
held fixed.
"""
from __future__ import annotations

import torch

from . import binding as _b


class ERIFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, centres, exps, cls, basis, bra_pairs, ket_pairs, quartets):
        out = _b.eri_batch(cls, basis, bra_pairs, ket_pairs, quartets, centres=centres.detach().contiguous(),
                           exps=exps.detach().contiguous())
        ctx.save_for_backward(centres, exps)
        ctx.args = (cls, basis, bra_pairs, ket_pairs, quartets)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        centres, exps = ctx.saved_tensors
        cls, basis, bra, ket, quartets = ctx.args
        gc = torch.zeros_like(centres) if ctx.needs_input_grad[0] else None
        ge = torch.zeros_like(exps) if ctx.needs_input_grad[1] else None
        if gc is not None or ge is not None:
            _b.eri_batch_grad(cls, basis, bra, ket, quartets, grad_out.contiguous(), gc, ge,
                              centres=centres.detach().contiguous(), exps=exps.detach().contiguous())
        return gc, ge, None, None, None, None, None


def eri(centres, exps, cls, basis, bra_pairs, ket_pairs, quartets=None):
    """Differentiable shellsets of class ``cls`` (layout of eri_batch)."""
    return ERIFunction.apply(centres, exps, cls, basis, bra_pairs, ket_pairs, quartets)
