// The whole hot path from host buffers: records in, image (and the adjoint's
// sigma_s gradient) out, through the library's own calls. The positions go
// first on the caller's stream, which builds the graph from them while the
// other records are copied on a second stream; the aggregation waits for
// those copies.
#include "pg_internal.cuh"

// dI = image - target
__global__ void loss_grad_kernel(const float *__restrict__ img, const float *__restrict__ tgt, int64_t m,
                                 float *__restrict__ dI) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dI[i] = img[i] - tgt[i];
}

extern "C" pg_status pg_step_host(const pg_vertices *hv, int64_t n, const float *L0, const int32_t *first,
                                  const float *bg, int64_t n_paths, const float *target, const int32_t *voxel,
                                  const pg_step_params *p, float *image, float *grad_sigma_s,
                                  float *grad_albedo_vox, pg_stream_t stream) {
    if (!hv || !p || !image || n < 0 || n_paths < 0) return PG_ERR_INVALID_ARG;
    if (p->spp < 1 || p->width < 1 || p->height < 1 || (int64_t)p->width * p->height * p->spp != n_paths)
        return PG_ERR_INVALID_ARG;
    if (n > 0 && (!L0 || !hv->px || !hv->py || !hv->pz)) return PG_ERR_INVALID_ARG;
    if (n_paths > 0 && (!first || !bg)) return PG_ERR_INVALID_ARG;
    if ((grad_sigma_s || grad_albedo_vox) && !target) return PG_ERR_INVALID_ARG;
    if (grad_albedo_vox && (!voxel || p->n_vox < 1)) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npix = (int64_t)p->width * p->height;
    const size_t nb = (size_t)(n > 0 ? n : 1);
    // device staging: 21 float fields + L0 + successors + the delta flags,
    // then the per-path arrays and the images (each slice 256-byte aligned)
    const float *const *hf[20] = {&hv->px, &hv->py, &hv->pz, &hv->ox, &hv->oy, &hv->oz, &hv->dx,
                                  &hv->dy, &hv->dz, &hv->ex, &hv->ey, &hv->ez, &hv->g, &hv->sigma_s,
                                  &hv->sigma_t, &hv->w_prop, &hv->Le, &hv->pe_e, &hv->Lph, &hv->pe_ph};
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t fsz = al(4 * nb), psz = al(4 * (size_t)(n_paths > 0 ? n_paths : 1)), isz = al(4 * (size_t)npix);
    const bool vox = grad_albedo_vox != nullptr;
    const size_t vsz = vox ? al(4 * (size_t)p->n_vox) : 0;
    const size_t total = 22 * fsz + al(nb) + 2 * psz + 3 * isz + (vox ? fsz + vsz : 0);
    unsigned char *buf = nullptr;
    PG_TRY(pg_alloc(nullptr, (void **)&buf, total, s));
    float *dfield[20];
    for (int i = 0; i < 20; i++) dfield[i] = (float *)(buf + i * fsz);
    float *dL0 = (float *)(buf + 20 * fsz);
    int32_t *dsucc = (int32_t *)(buf + 21 * fsz);
    uint8_t *ddelta = buf + 22 * fsz;
    unsigned char *q = buf + 22 * fsz + al(nb);
    int32_t *dfirst = (int32_t *)q;
    float *dbg = (float *)(q + psz);
    float *dimg = (float *)(q + 2 * psz), *dtgt = (float *)(q + 2 * psz + isz), *dI = (float *)(q + 2 * psz + 2 * isz);
    int32_t *dvox = vox ? (int32_t *)(q + 2 * psz + 3 * isz) : nullptr;
    float *dga = vox ? (float *)(q + 2 * psz + 3 * isz + fsz) : nullptr;
    float *dL = nullptr, *dD = nullptr, *dgs = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t copied = nullptr;
    pg_graph *g = nullptr;
    pg_status st = PG_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes, cudaStream_t on) {
        if (st == PG_OK && bytes && src && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, on) != cudaSuccess)
            st = PG_ERR_CUDA;
    };
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) != cudaSuccess)
        st = PG_ERR_CUDA;
    // the side stream starts after the caller's earlier work on `stream`
    if (st == PG_OK && (cudaEventRecord(copied, s) != cudaSuccess || cudaStreamWaitEvent(side, copied, 0) != cudaSuccess))
        st = PG_ERR_CUDA;
    for (int i = 0; i < 3; i++) cp(dfield[i], *hf[i], 4 * (size_t)n, s);
    for (int i = 3; i < 20; i++) cp(dfield[i], *hf[i], 4 * (size_t)n, side);
    cp(dL0, L0, 4 * (size_t)n, side);
    cp(dsucc, hv->succ, 4 * (size_t)n, side);
    cp(ddelta, hv->e_delta, (size_t)n, side);
    cp(dfirst, first, 4 * (size_t)n_paths, side);
    cp(dbg, bg, 4 * (size_t)n_paths, side);
    if (target) cp(dtgt, target, 4 * (size_t)npix, side);
    if (vox) cp(dvox, voxel, 4 * (size_t)n, side);
    if (st == PG_OK && cudaEventRecord(copied, side) != cudaSuccess) st = PG_ERR_CUDA;
    pg_vertices dv = {};
    dv.px = dfield[0], dv.py = dfield[1], dv.pz = dfield[2], dv.ox = dfield[3], dv.oy = dfield[4], dv.oz = dfield[5];
    dv.dx = dfield[6], dv.dy = dfield[7], dv.dz = dfield[8], dv.ex = dfield[9], dv.ey = dfield[10], dv.ez = dfield[11];
    dv.g = dfield[12], dv.sigma_s = dfield[13], dv.sigma_t = dfield[14], dv.w_prop = dfield[15];
    dv.Le = dfield[16], dv.pe_e = dfield[17], dv.Lph = dfield[18], dv.pe_ph = dfield[19];
    dv.e_delta = ddelta, dv.succ = dsucc;
    pg_build_params bp = {};
    bp.k = p->k;
    for (int a = 0; a < 3; a++) bp.bbox_lo[a] = p->bbox_lo[a], bp.bbox_hi[a] = p->bbox_hi[a];
    bp.r2_max = -1;
    if (st == PG_OK) st = pg_build_graph(&dv, n, &bp, stream, &g);
    if (st == PG_OK && cudaStreamWaitEvent(s, copied, 0) != cudaSuccess) st = PG_ERR_CUDA;
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&dL, 4 * nb, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&dD, 4 * nb, s);
    if (st == PG_OK) st = pg_aggregate(g, &dv, p->wdtype, nullptr, dD, stream);
    const bool adj = target != nullptr && p->adjoint;
    if (st == PG_OK) st = pg_propagate(g, nullptr, dL0, p->iters, 0.0, adj ? 1 : 0, dL, nullptr, nullptr, stream);
    if (st == PG_OK)
        st = pg_gather(g, dL, dD, dfirst, dbg, n_paths, p->spp, p->width, p->height, dimg, stream);
    if (st == PG_OK && adj) {
        loss_grad_kernel<<<pg_blocks(npix, 256), 256, 0, s>>>(dimg, dtgt, npix, dI);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        if (st == PG_OK) st = pg_alloc(nullptr, (void **)&dgs, 4 * nb, s);
        if (st == PG_OK)
            st = pg_propagate_adjoint(g, dI, dfirst, n_paths, p->spp, p->width, p->height, dgs, nullptr, dvox,
                                      vox ? dfield[14] : nullptr, dga, vox ? p->n_vox : 0, 0, stream);
    }
    if (st == PG_OK && cudaMemcpyAsync(image, dimg, 4 * (size_t)npix, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = PG_ERR_CUDA;
    if (st == PG_OK && grad_sigma_s && adj && n > 0 &&
        cudaMemcpyAsync(grad_sigma_s, dgs, 4 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = PG_ERR_CUDA;
    if (st == PG_OK && vox && adj &&
        cudaMemcpyAsync(grad_albedo_vox, dga, 4 * (size_t)p->n_vox, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = PG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess && st == PG_OK) st = PG_ERR_CUDA;
    if (side) { // its copies may still be in flight after an early error
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
    }
    if (g) pg_graph_destroy(g);
    for (void *x : {(void *)dL, (void *)dD, (void *)dgs, (void *)buf})
        if (x) cudaFreeAsync(x, s);
    if (copied) cudaEventDestroy(copied);
    (void)cudaGetLastError();
    return st;
}
