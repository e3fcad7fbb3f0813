"""Differentiable lattice objective: torch.autograd.Function over the C ABI.

J = w_area * area + w_vol * volume of the resolution-k triangulation
(Section 5 of arXiv 2405.15197) of the lattice with node positions `xyz`
and node radii `node_R`; strut i joins nodes ends[i, 0] and ends[i, 1].
The forward pass builds the meta-mesh (lm_build_metamesh) and evaluates
the objective (lm_objective); the backward pass calls lm_metamesh_backward,
which differentiates with the discrete structure (arcs, segment counts,
stitching order) of the forward pass held fixed.
"""
from __future__ import annotations

import torch

from . import liblm


class LatticeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, node_R, ends, k, w_area=1.0, w_vol=0.0):
        xyz = xyz.detach().contiguous()
        node_R = node_R.detach().contiguous()
        ends = ends.to(torch.int32).contiguous()
        radii = node_R[ends.long()].contiguous()
        mm = liblm.MetaMesh(xyz, ends, radii, stream=torch.cuda.current_stream())
        mm.tri_count(int(k))
        area, vol = mm.objective(int(k))
        ctx.mm = mm
        ctx.k, ctx.w = int(k), (float(w_area), float(w_vol))
        return torch.tensor(ctx.w[0] * area + ctx.w[1] * vol, dtype=torch.float64, device=xyz.device)

    @staticmethod
    def backward(ctx, gJ):
        gx, gr, _, _ = ctx.mm.backward(ctx.k, ctx.w[0], ctx.w[1], stream=torch.cuda.current_stream())
        ctx.mm.close()
        s = gJ.to(gx.dtype)
        return gx * s, gr * s, None, None, None, None


def lattice_objective(xyz, node_R, ends, k, w_area=1.0, w_vol=0.0):
    """w_area * area + w_vol * volume (FP64 scalar tensor), differentiable
    with respect to xyz [N, 3] and node_R [N]."""
    return LatticeObjective.apply(xyz, node_R, ends, k, w_area, w_vol)
