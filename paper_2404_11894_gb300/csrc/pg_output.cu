// Per-path output into pixels (Section 4, "Final output"): the radiance a
// path's first vertex f sends along its continuation edge into the camera,
//   val_p = bg_p + (tau/p_t)_f * ( sum_j A_{f,j} L_j + Dir_p ),
// averaged over the spp paths of a pixel. Options: the direct term from
// extra emitter samples recorded at f (Section 4, "Handling direct light"),
// and a final gather, one more aggregation at the first vertices over their
// own k nearest vertices (the optional final gather of the Fig. 2 caption).
#include <algorithm>

#include "pg_internal.cuh"

// ------------------------------------------------------------------ gather over N(f)
// One thread per pixel; its spp paths in order. Row f of the propagation
// matrix already holds (tau/p_t)_f A+_{f,j}.
template <typename WT>
__global__ void gather_kernel(const int32_t *__restrict__ first, const float *__restrict__ bg,
                              const float *__restrict__ L, const float *__restrict__ D,
                              const float *__restrict__ Dp, const int32_t *__restrict__ c2m,
                              const int32_t *__restrict__ m2c, const int32_t *__restrict__ m2r,
                              const int32_t *__restrict__ nbr, const WT *__restrict__ W,
                              const float *__restrict__ rscale, const float4 *__restrict__ LV, int kp, int spp,
                              int64_t npix, int64_t n, float *__restrict__ image) {
    int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float acc = 0.0f;
    for (int sidx = 0; sidx < spp; sidx++) {
        int64_t p = pix * spp + sidx;
        float val = bg[p];
        int32_t f = first[p];
        if (f >= 0 && f < n) { // out-of-range entries are treated as -1
            int32_t m = c2m[f];
            int64_t r = m2r[m];
            float sc = WTraits<WT>::id == PG_W_F32 ? 1.0f : rscale[r];
            float sum = 0.0f;
            for (int i = 0; i < kp; i++) {
                int32_t j = nbr[(int64_t)m * kp + i];
                if (j >= 0) sum = fmaf(WTraits<WT>::dec(W[r * kp + i]), L[m2c[j]], sum);
            }
            val += fmaf(sum, sc, LV[m].w * (Dp ? Dp[p] : D[f]));
        }
        acc += val;
    }
    image[pix] = acc / (float)spp;
}

// ------------------------------------------------------------------ extra direct samples
// D^x_f per path: the M extra emitter samples and the path's own phase
// sample at f, balance heuristic with M emitter samples and one phase
// sample; a delta-light sample is averaged (weight 1/M).
__global__ void extra_direct_kernel(const int32_t *__restrict__ first, int64_t n_paths, int64_t n,
                                    const int32_t *__restrict__ c2m, const float4 *__restrict__ OG,
                                    const float4 *__restrict__ DP, const float4 *__restrict__ LV, int M,
                                    const float *__restrict__ ex, const float *__restrict__ ey,
                                    const float *__restrict__ ez, const float *__restrict__ Le,
                                    const float *__restrict__ pe, const uint8_t *__restrict__ delta,
                                    float *__restrict__ Dp, int32_t *__restrict__ flags) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_paths) return;
    const int32_t f = first[p];
    if (f < 0 || f >= n) {
        Dp[p] = 0.0f;
        return;
    }
    const int32_t m = c2m[f];
    const float4 og = OG[m], dp = DP[m], lv = LV[m];
    const HGc h = hg_consts(og.w);
    const float eo = unit_err(og.x, og.y, og.z);
    const float Mf = (float)M;
    float acc = 0.0f;
    int bad = 0;
    for (int i = 0; i < M; i++) {
        const int64_t q = p * M + i;
        const float x = ex[q], y = ey[q], z = ez[q], le = Le[q], pq = pe[q];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(le) || !isfinite(pq)) {
            bad |= PG_FLAG_NONFINITE;
            continue;
        }
        if (le < 0.0f || pq < 0.0f) bad |= PG_FLAG_BAD_RANGE;
        const float rho = hg_eval(h, one_plus_dot_u(og.x, og.y, og.z, eo, x, y, z, unit_err(x, y, z)));
        acc += delta[q] ? rho * le / Mf : rho * le / fmaf(Mf, pq, rho);
    }
    const float rd = hg_eval(h, one_plus_dot_u(og.x, og.y, og.z, eo, dp.x, dp.y, dp.z, unit_err(dp.x, dp.y, dp.z)));
    acc += rd * lv.y / fmaf(Mf, dp.w, rd);
    Dp[p] = lv.z * acc;
    if (bad) atomicOr(flags, bad);
}

// ------------------------------------------------------------------ final gather
__global__ void first_to_morton_kernel(const int32_t *__restrict__ first, int64_t n_paths, int64_t n,
                                       const int32_t *__restrict__ c2m, int32_t *__restrict__ qm) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_paths) return;
    const int32_t f = first[p];
    qm[p] = (f >= 0 && f < n) ? c2m[f] : -1;
}

// kNN graph without a radius limit: its rows hold self, then the others in
// (distance, caller index) order, so the kfg nearest are a row's prefix
__global__ void fg_prefix_kernel(const int32_t *__restrict__ qm, int64_t n_paths, const int32_t *__restrict__ nbr,
                                 int kp, int kfg, int kpf, int32_t *__restrict__ fgn) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_paths * kpf) return;
    const int64_t p = e >> (__ffs(kpf) - 1); // kpf is a power of two
    const int i = (int)(e & (kpf - 1));
    const int32_t m = qm[p];
    fgn[e] = (m >= 0 && i < kfg) ? nbr[(int64_t)m * kp + i] : -1;
}

// Groups of KPF lanes per path, lane j holding entry j of N_fg(f) (slot 0 =
// f). Each lane forms its sample's marginal over the group's strategies
// (their (o, g) passed round the group by shuffles, summed in slot order),
// then the receiver's balance-heuristic weight; the group sums its terms.
template <int KPF>
__global__ void __launch_bounds__(256) fg_values_kernel(
    const int32_t *__restrict__ first, const float *__restrict__ bg, int64_t n_paths, int64_t n,
    const int32_t *__restrict__ fgn, const int32_t *__restrict__ m2c, const float4 *__restrict__ OG,
    const float4 *__restrict__ DP, const float4 *__restrict__ LV, const float *__restrict__ L,
    const float *__restrict__ D, const float *__restrict__ Dp, float *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (KPF - 1);
    const int src = lane & ~(KPF - 1);
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / KPF;
    const bool ok = p < n_paths;
    const int32_t f = ok ? first[p] : -1;
    const bool has = f >= 0 && f < n;
    const int32_t nj = has ? fgn[p * KPF + j] : -1;
    const bool valid = nj >= 0;
    float4 og = make_float4(0.f, 0.f, 1.f, 0.f), dp = make_float4(0.f, 0.f, 1.f, 0.f),
           lv = make_float4(0.f, 0.f, 0.f, 0.f);
    float Lj = 0.0f;
    if (valid) {
        og = OG[nj];
        dp = DP[nj];
        Lj = L[m2c[nj]];
        if (j == 0) lv = LV[nj];
    }
    const HGc hl = hg_consts(og.w);
    const float eo = unit_err(og.x, og.y, og.z);
    const float ed = unit_err(dp.x, dp.y, dp.z);
    float pm = 0.0f;
#pragma unroll 4
    for (int l = 0; l < KPF; l++) {
        const int s = src + l;
        HGc h;
        h.C = __shfl_sync(0xffffffffu, hl.C, s);
        h.a = __shfl_sync(0xffffffffu, hl.a, s);
        h.b2 = __shfl_sync(0xffffffffu, hl.b2, s);
        const float ox = __shfl_sync(0xffffffffu, og.x, s), oy = __shfl_sync(0xffffffffu, og.y, s),
                    oz = __shfl_sync(0xffffffffu, og.z, s), el = __shfl_sync(0xffffffffu, eo, s);
        const int vl = __shfl_sync(0xffffffffu, (int)valid, s);
        if (vl) pm += hg_eval(h, one_plus_dot_u(ox, oy, oz, el, dp.x, dp.y, dp.z, ed));
    }
    HGc hf;
    hf.C = __shfl_sync(0xffffffffu, hl.C, src);
    hf.a = __shfl_sync(0xffffffffu, hl.a, src);
    hf.b2 = __shfl_sync(0xffffffffu, hl.b2, src);
    const float fx = __shfl_sync(0xffffffffu, og.x, src), fy = __shfl_sync(0xffffffffu, og.y, src),
                fz = __shfl_sync(0xffffffffu, og.z, src), ef = __shfl_sync(0xffffffffu, eo, src);
    const float sig = __shfl_sync(0xffffffffu, lv.z, src), w = __shfl_sync(0xffffffffu, lv.w, src);
    const float rf = hg_eval(hf, one_plus_dot_u(fx, fy, fz, ef, dp.x, dp.y, dp.z, ed));
    float t = valid ? sig * rf / pm * Lj : 0.0f;
#pragma unroll
    for (int o = KPF / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (ok && j == 0) vals[p] = has ? bg[p] + w * (t + (Dp ? Dp[p] : D[f])) : bg[p];
}

__global__ void pixel_mean_kernel(const float *__restrict__ vals, int spp, int64_t npix, float *__restrict__ image) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float acc = 0.0f;
    for (int s = 0; s < spp; s++) acc += vals[pix * spp + s];
    image[pix] = acc / (float)spp;
}

__global__ void fg_nbr_out_kernel(const int32_t *__restrict__ fgn, int kpf, int k, int64_t n_paths,
                                  const int32_t *__restrict__ m2c, int32_t *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_paths * k) return;
    const int64_t p = e / k;
    const int i = (int)(e - p * k);
    const int32_t j = fgn[p * kpf + i];
    out[e] = j >= 0 ? m2c[j] : -1;
}

// ------------------------------------------------------------------ entry points
template <typename WT>
static void launch_gather(const pg_graph *g, const float *L, const float *D, const float *Dp, const int32_t *first,
                          const float *bg, int spp, int64_t npix, float *image, cudaStream_t s) {
    gather_kernel<WT><<<pg_blocks(npix, 128), 128, 0, s>>>(first, bg, L, D, Dp, g->c2m, g->m2c, g->m2r, g->nbr,
                                                           (const WT *)g->W, g->rscale, g->LV, g->kp, spp, npix,
                                                           g->n, image);
    pg_count_launches(1);
}

template <int KPF>
static void launch_fg_values(const pg_graph *g, const int32_t *first, const float *bg, int64_t n_paths,
                             const int32_t *fgn, const float *L, const float *D, const float *Dp, float *vals,
                             cudaStream_t s) {
    fg_values_kernel<KPF><<<pg_blocks(n_paths * KPF, 256), 256, 0, s>>>(first, bg, n_paths, g->n, fgn, g->m2c, g->OG,
                                                                        g->DP, g->LV, L, D, Dp, vals);
    pg_count_launches(1);
}

extern "C" pg_status pg_gather_ex(const pg_graph *g, const float *L, const float *D, const int32_t *first,
                                  const float *bg, int64_t n_paths, int32_t spp, int32_t width, int32_t height,
                                  const pg_output_params *params, float *image, pg_stream_t stream) {
    if (!g || spp <= 0 || width < 0 || height < 0) return PG_ERR_INVALID_ARG;
    if (n_paths != (int64_t)width * height * spp) return PG_ERR_INVALID_ARG;
    if (!g->aggregated || !g->W) return PG_ERR_STATE;
    const int kfg = params ? params->final_gather_k : 0;
    const pg_extra_samples *x = params ? params->extra : nullptr;
    if (kfg < 0) return PG_ERR_INVALID_ARG;
    if (kfg > PG_MAX_K) return PG_ERR_UNSUPPORTED;
    const int64_t npix = (int64_t)width * height;
    if (npix == 0) return PG_OK;
    if (!first || !bg || !image) return PG_ERR_INVALID_ARG;
    if (g->n > 0 && (!L || (!x && !D))) return PG_ERR_INVALID_ARG;
    if (x && (x->m < 1 || !x->ex || !x->ey || !x->ez || !x->Le || !x->pe_e || !x->e_delta))
        return PG_ERR_INVALID_ARG;
    if (x && n_paths > INT64_MAX / x->m) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    pg_status st = PG_OK;
    float *Dp = nullptr, *vals = nullptr;
    int32_t *flags = nullptr, *qm = nullptr, *fgn = nullptr;
    const int kpf = kfg > 0 ? pg_row_width(kfg) : 0;
    if (x) {
        st = pg_alloc(nullptr, (void **)&flags, 16, s);
        if (st == PG_OK) st = pg_alloc(nullptr, (void **)&Dp, 4 * (size_t)n_paths, s);
        if (st == PG_OK && cudaMemsetAsync(flags, 0, 4, s) != cudaSuccess) st = PG_ERR_CUDA;
        if (st == PG_OK) {
            extra_direct_kernel<<<pg_blocks(n_paths, 256), 256, 0, s>>>(first, n_paths, g->n, g->c2m, g->OG, g->DP,
                                                                        g->LV, x->m, x->ex, x->ey, x->ez, x->Le,
                                                                        x->pe_e, x->e_delta, Dp, flags);
            pg_count_launches(1);
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
    }
    if (st == PG_OK && kfg > 0) {
        st = pg_alloc(nullptr, (void **)&qm, 4 * (size_t)n_paths, s);
        if (st == PG_OK) st = pg_alloc(nullptr, (void **)&fgn, 4 * (size_t)n_paths * kpf, s);
        if (st == PG_OK) st = pg_alloc(nullptr, (void **)&vals, 4 * (size_t)n_paths, s);
        if (st == PG_OK) {
            first_to_morton_kernel<<<pg_blocks(n_paths, 256), 256, 0, s>>>(first, n_paths, g->n, g->c2m, qm);
            pg_count_launches(1);
            if (g->clusters == 0 && g->r2_max < 0 && kfg <= g->k) {
                fg_prefix_kernel<<<pg_blocks(n_paths * kpf, 256), 256, 0, s>>>(qm, n_paths, g->nbr, g->kp, kfg, kpf,
                                                                               fgn);
                pg_count_launches(1);
            } else {
                st = pg_launch_knn_queries(g, qm, n_paths, kfg, fgn, s);
            }
        }
        if (st == PG_OK) {
            switch (kpf) {
                case 4: launch_fg_values<4>(g, first, bg, n_paths, fgn, L, D, Dp, vals, s); break;
                case 8: launch_fg_values<8>(g, first, bg, n_paths, fgn, L, D, Dp, vals, s); break;
                case 16: launch_fg_values<16>(g, first, bg, n_paths, fgn, L, D, Dp, vals, s); break;
                default: launch_fg_values<32>(g, first, bg, n_paths, fgn, L, D, Dp, vals, s); break;
            }
            pixel_mean_kernel<<<pg_blocks(npix, 256), 256, 0, s>>>(vals, spp, npix, image);
            pg_count_launches(1);
            if (params->fg_nbr) {
                fg_nbr_out_kernel<<<pg_blocks(n_paths * kfg, 256), 256, 0, s>>>(fgn, kpf, kfg, n_paths, g->m2c,
                                                                                params->fg_nbr);
                pg_count_launches(1);
            }
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
    } else if (st == PG_OK) {
        switch (g->wdtype) {
            case PG_W_F32: launch_gather<float>(g, L, D, Dp, first, bg, spp, npix, image, s); break;
            case PG_W_BF16: launch_gather<__nv_bfloat16>(g, L, D, Dp, first, bg, spp, npix, image, s); break;
            case PG_W_F16: launch_gather<__half>(g, L, D, Dp, first, bg, spp, npix, image, s); break;
            case PG_W_U16: launch_gather<pg_unorm16>(g, L, D, Dp, first, bg, spp, npix, image, s); break;
        }
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    int32_t hflags = 0;
    if (st == PG_OK && x) {
        if (cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = PG_ERR_CUDA;
    }
    for (void *ptr : {(void *)Dp, (void *)vals, (void *)flags, (void *)qm, (void *)fgn})
        if (ptr) cudaFreeAsync(ptr, s);
    if (st != PG_OK) {
        (void)cudaGetLastError();
        return st;
    }
    if (hflags & PG_FLAG_NONFINITE) return PG_ERR_NONFINITE;
    if (hflags & PG_FLAG_BAD_RANGE) return PG_ERR_INVALID_ARG;
    return PG_OK;
}

extern "C" pg_status pg_gather(const pg_graph *g, const float *L, const float *D, const int32_t *first,
                               const float *bg, int64_t n_paths, int32_t spp, int32_t width, int32_t height,
                               float *image, pg_stream_t stream) {
    return pg_gather_ex(g, L, D, first, bg, n_paths, spp, width, height, nullptr, image, stream);
}
