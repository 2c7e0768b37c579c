"""The whole hot path as one call: graph, aggregation, propagation, output
and (optionally) the adjoint of an L2 image loss."""
from __future__ import annotations

import torch

from . import pg_aggregate, pg_build_graph, pg_gather, pg_propagate, pg_propagate_adjoint, Vertices


class Solver:
    """Runs the path-graph hot path on device-resident records.

    k: neighbours per vertex (self included); iters: propagation sweeps;
    wdtype: 'f32' | 'bf16' | 'f16' | 'u16' edge weights; adjoint: also run
    pg_propagate_adjoint for the loss 1/2 |image - target|^2;
    cluster_size: 0 for kNN neighbourhoods, K > 0 for the paper's disjoint
    clusters of expected size K (parts of at most k points); n_vox > 0: the
    adjoint also forms the per-voxel albedo gradient (step() then takes the
    vertices' voxel ids and sigma_t).
    """

    def __init__(self, k: int, iters: int, wdtype: str = "f32", adjoint: bool = True,
                 bbox_lo=(0.0, 0.0, 0.0), bbox_hi=(1.0, 1.0, 1.0), recompute_weights: int = 0,
                 want_g: bool = True, cluster_size: int = 0, cluster_seed: int = 0, n_vox: int = 0):
        self.k, self.iters, self.wdtype, self.adjoint = k, iters, wdtype, adjoint
        self.cluster_size, self.cluster_seed = cluster_size, cluster_seed
        self.bbox_lo, self.bbox_hi = bbox_lo, bbox_hi
        self.recompute_weights = int(recompute_weights)
        self.want_g = want_g
        self.n_vox = int(n_vox)
        self.graph = None
        self.last_image = None
        self.grads = None

    def step(self, V: Vertices, L0, first, bg, spp, width, height, target=None, marks=None, ready=None,
             voxel=None, sigma_t=None):
        """One pass; ``marks`` maps stage names to (start, end) CUDA events.
        ``ready``: a CUDA event the stream waits for after the graph build
        (the build reads only positions; everything else may still be in
        flight until then)."""
        def mark(name, i):
            if marks is not None and name in marks:
                marks[name][i].record(torch.cuda.current_stream())

        if self.graph is not None:
            self.graph.close()
        mark("build", 0)
        self.graph = pg_build_graph(V, self.k, self.bbox_lo, self.bbox_hi, cluster_size=self.cluster_size,
                                    cluster_seed=self.cluster_seed)
        mark("build", 1)
        if ready is not None:
            torch.cuda.current_stream().wait_event(ready)
        mark("aggregate", 0)
        self._c, self.D = pg_aggregate(self.graph, V, self.wdtype)
        mark("aggregate", 1)
        self._L0 = L0
        use_adj = self.adjoint and target is not None
        mark("propagate", 0)
        self.L = pg_propagate(self.graph, L0, self.iters, keep_history=use_adj)
        mark("propagate", 1)
        mark("gather", 0)
        img = pg_gather(self.graph, self.L, self.D, first, bg, spp, width, height)
        mark("gather", 1)
        self.last_image = img
        if use_adj:
            mark("adjoint", 0)
            dI = img - target
            vox = voxel if self.n_vox > 0 else None
            self.grads = pg_propagate_adjoint(self.graph, dI, first, spp, width, height, want_g=self.want_g,
                                              voxel=vox, sigma_t=sigma_t if vox is not None else None,
                                              n_vox=self.n_vox if vox is not None else 0,
                                              recompute_weights=self.recompute_weights)
            mark("adjoint", 1)
        return img

    def time_propagate(self, iters: int, reps: int = 3, keep_history: bool = False, from_idle: bool = False) -> float:
        """Mean device time (ms) of pg_propagate on the current graph. With
        ``from_idle`` each call starts on an idle device, as it does inside a
        step (after the aggregation's synchronisation), so the time includes
        the same wait for the host to issue the call's first work."""
        s = torch.cuda.current_stream()
        L = torch.empty_like(self._L0)
        pg_propagate(self.graph, self._L0, iters, out=L, keep_history=keep_history)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if from_idle:
            tot = 0.0
            for _ in range(reps):
                torch.cuda.synchronize()
                e0.record(s)
                pg_propagate(self.graph, self._L0, iters, out=L, keep_history=keep_history)
                e1.record(s)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            return tot / reps
        e0.record(s)
        for _ in range(reps):
            pg_propagate(self.graph, self._L0, iters, out=L, keep_history=keep_history)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def time_adjoint(self, iters: int, spp: int, width: int, height: int, first, reps: int = 2) -> float:
        """Mean device time (ms) of pg_propagate_adjoint after a forward pass of
        ``iters`` sweeps on the current graph (transposes already built)."""
        s = torch.cuda.current_stream()
        pg_propagate(self.graph, self._L0, iters, keep_history=True)
        dI = torch.ones(width * height, dtype=torch.float32, device="cuda")
        pg_propagate_adjoint(self.graph, dI, first, spp, width, height, want_g=False,
                             recompute_weights=self.recompute_weights)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            pg_propagate_adjoint(self.graph, dI, first, spp, width, height, want_g=False,
                                 recompute_weights=self.recompute_weights)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def solve_host(self, host: dict, host_target, spp, width, height, want_sigma_s: bool = False):
        """End to end from pinned host records to the image on the host,
        through the C ABI's host-buffer entry point (pg_step_host: the
        positions are copied first and the graph built from them while the
        other records are copied on a second stream). The per-voxel albedo
        gradient is formed when the solver has n_vox > 0 and ``host`` holds
        the voxel ids. The image and gradients (``self.host_grads``) live in
        pinned buffers the solver reuses: the next call overwrites them."""
        from . import pg_step_host

        if self.cluster_size or self.recompute_weights:
            raise ValueError("solve_host runs kNN neighbourhoods with the stored transpose")
        nv = self.n_vox if "voxel" in host else 0
        # pinned output buffers, kept between calls
        if getattr(self, "_host_out", None) is None:
            self._host_out = {}
        shapes = {"image": (height, width), "grad_sigma_s": (int(host["px"].numel()),), "grad_albedo": (nv,)}
        for name, shape in shapes.items():
            t = self._host_out.get(name)
            if (t is None or tuple(t.shape) != shape) and (name != "grad_sigma_s" or want_sigma_s) and \
                    (name != "grad_albedo" or nv > 0):
                self._host_out[name] = torch.empty(shape, dtype=torch.float32).pin_memory()
        out = pg_step_host(host, spp, width, height, self.k, self.iters, self.wdtype,
                           target=host_target if self.adjoint else None, n_vox=nv, want_sigma_s=want_sigma_s,
                           bbox_lo=self.bbox_lo, bbox_hi=self.bbox_hi, out=self._host_out)
        self.host_grads = out
        return out["image"]

    def close(self):
        if self.graph is not None:
            self.graph.close()
            self.graph = None
