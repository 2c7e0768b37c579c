"""torch.autograd binding: image = PathGraph(sigma_s, g) with a hand-written
backward (pg_propagate_adjoint)."""
from __future__ import annotations

import torch

from . import Vertices, pg_aggregate, pg_build_graph, pg_gather, pg_propagate, pg_propagate_adjoint


class PathGraphFunction(torch.autograd.Function):
    """Forward: graph, aggregation, ``iters`` sweeps, output; backward: the
    adjoint sweep. Differentiable inputs: per-vertex sigma_s and g (caller
    order); everything else in ``ctx_inputs`` is held fixed."""

    @staticmethod
    def forward(ctx, sigma_s, g, tensors: dict, L0, first, bg, spp, width, height, k, iters, wdtype,
                recompute_weights):
        t = dict(tensors)
        t["sigma_s"] = sigma_s.contiguous()
        t["g"] = g.contiguous()
        V = Vertices(t)
        graph = pg_build_graph(V, k)
        _, D = pg_aggregate(graph, V, wdtype)
        L = pg_propagate(graph, L0, iters, keep_history=True)
        img = pg_gather(graph, L, D, first, bg, spp, width, height)
        ctx.graph, ctx.V = graph, V
        ctx.first, ctx.spp, ctx.width, ctx.height = first, spp, width, height
        ctx.recompute = recompute_weights
        return img

    @staticmethod
    def backward(ctx, dI):
        grads = pg_propagate_adjoint(ctx.graph, dI.contiguous(), ctx.first, ctx.spp, ctx.width, ctx.height,
                                     want_sigma_s=ctx.needs_input_grad[0], want_g=ctx.needs_input_grad[1],
                                     recompute_weights=int(ctx.recompute))
        ctx.graph.close()
        return (grads["grad_sigma_s"], grads["grad_g"]) + (None,) * 11


def render(sigma_s, g, tensors, L0, first, bg, spp, width, height, k=16, iters=30, wdtype="f32",
           recompute_weights=False):
    """Differentiable path-graph image w.r.t. per-vertex sigma_s and g."""
    return PathGraphFunction.apply(sigma_s, g, tensors, L0, first, bg, spp, width, height, k, iters, wdtype,
                                   recompute_weights)
