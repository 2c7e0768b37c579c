// Adjoint of aggregation -> propagation -> output (placeholder until the
// reverse sweep lands).
#include "pg_internal.cuh"

extern "C" pg_status pg_propagate_adjoint(pg_graph *g, const float *dI, const int32_t *first, int64_t n_paths,
                                          int32_t spp, int32_t width, int32_t height, float *grad_sigma_s,
                                          float *grad_g, const int32_t *voxel, const float *sigma_t,
                                          float *grad_albedo_vox, int64_t n_vox, int32_t recompute_weights,
                                          pg_stream_t stream) {
    (void)g; (void)dI; (void)first; (void)n_paths; (void)spp; (void)width; (void)height; (void)grad_sigma_s;
    (void)grad_g; (void)voxel; (void)sigma_t; (void)grad_albedo_vox; (void)n_vox; (void)recompute_weights;
    (void)stream;
    return PG_ERR_UNSUPPORTED;
}

extern "C" pg_status pg_graph_release_weights(pg_graph *g) {
    if (!g) return PG_ERR_INVALID_ARG;
    size_t wb = pg_wbytes(g->wdtype);
    pg_free(g, (void **)&g->W, wb * (size_t)g->n * (size_t)g->kp);
    pg_free(g, (void **)&g->t_W, wb * (size_t)g->nnz_t);
    return PG_OK;
}
