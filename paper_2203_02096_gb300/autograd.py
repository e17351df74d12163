"""Genotype energies as a differentiable torch function.

``score(geno, ctx, grids, lig)`` returns E[B] for genotypes geno[B, G]
(CUDA, FP32).  When geno requires grad, the forward pass runs the fused
energy+gradient kernel (score_grad_batch: one launch computes both) and keeps
dE/dgeno; the backward pass returns grad_output[:, None] * dE/dgeno.  The
analytic gradient is the one the local search uses (translation, quaternion
through its normalisation, torsions).
"""
from __future__ import annotations

import torch

from . import capi


class _Score(torch.autograd.Function):
    @staticmethod
    def forward(fctx, geno, dctx, grids, lig):
        g = geno.detach().contiguous()
        if geno.requires_grad:
            E, dE = capi.score_grad_batch(dctx, grids, lig, g)
            fctx.save_for_backward(dE)
        else:
            E = capi.score_batch(dctx, grids, lig, g)
        return E

    @staticmethod
    def backward(fctx, grad_E):
        (dE,) = fctx.saved_tensors
        return grad_E.unsqueeze(1) * dE, None, None, None


def score(geno: torch.Tensor, dctx: capi.Context, grids: capi.Grids, lig: capi.Ligand) -> torch.Tensor:
    if geno.dim() != 2 or geno.shape[1] != lig.n_genes:
        raise ValueError(f"expected genotypes of shape [B, {lig.n_genes}]")
    if geno.dtype != torch.float32 or not geno.is_cuda:
        raise ValueError("genotypes must be a CUDA float32 tensor")
    return _Score.apply(geno, dctx, grids, lig)
