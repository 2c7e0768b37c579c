"""FP64 CPU oracle of the volumetric path-graph hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product path. It
shares no code with the CUDA library.
"""
from .pathgraph import (  # noqa: F401
    adjoint, aggregate, cluster_graph, dense_fixed_point, extra_direct, final_gather, forward, gather, hg,
    hg_dg, image_loss,
    knn, knn_brute, morton_order, nearest_centre, nearest_centre_brute, path_values, propagate, quantize,
    sample_marginals, splitmix64, sweep, vertex_arrays,
)
