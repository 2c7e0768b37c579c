// Propagation (Eq. rte-mff with P from Eq. volume-propagation).
//
// One Jacobi sweep, in sweep-row order r over the rows that have a
// predecessor:   y'_r = scale_r * sum_i W[r][i] * y[col[r][i]] + b_r
// The matrix rows are streamed once per sweep (coalesced 16-byte loads,
// evict-first so the gathered vector y stays in L2); KP/4 lanes share a row
// and combine their four products with shuffles. The relative change of the
// sweep is reduced in FP64 (per-block partials, then the last block), and a
// sweep that finds the previous one converged returns at once.
#include <algorithm>
#include <mutex>

#include "pg_internal.cuh"

static constexpr int SWEEP_THREADS = 256;

// Sum (a, b) over the block in FP64; result valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sa[NT / 32], sb[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        a = lane < NT / 32 ? sa[lane] : 0.0;
        b = lane < NT / 32 ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

// Relative change of the sweep: per-block FP64 partials, then the last block
// to finish (ticket in ctrl[2]) adds them up and sets the stop flag.
template <int NT>
__device__ __forceinline__ void sweep_residual(double rd, double rn, int32_t *ctrl, double2 *partials,
                                               double *resid, int t, double tol) {
    double a = rd, bb = rn;
    block_sum2<NT>(a, bb);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = make_double2(a, bb);
        __threadfence();
        last = atomicAdd(&ctrl[2], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const volatile double *pv = reinterpret_cast<const volatile double *>(partials + i);
        sa += pv[0];
        sb += pv[1];
    }
    block_sum2<NT>(sa, sb);
    if (threadIdx.x == 0) {
        double r = sb > 0.0 ? sqrt(sa) / sqrt(sb) : 0.0;
        resid[t - 1] = r;
        ctrl[0] = t;
        ctrl[2] = 0;
        if (tol > 0.0 && r < tol) ctrl[1] = 1;
    }
}

// A thread's share of the residual's sums of squares is a float32 sum
// over its rows (a few hundred per thread; the terms are squares, so the
// relative error stays below rows * 2^-24, about 1e-5, and nothing
// cancels); the block and the grid add the threads' shares in FP64, where
// millions of terms meet. Measured on the 8.7M-vertex cloud, FP32 sweep:
// float 199 us; a compensated (TwoSum) float sum 209 us; float partials of
// 32 row groups folded into FP64 245 us; FP64 per row 312 us (this GPU's
// FP64 rate).
// Compensated sum of one row's products, four per lane, then over the row's
// LPR lanes (the kernel is memory-bound, so the extra additions are free;
// they keep 30+ sweeps at albedo ~1 within float32 rounding of the exact
// iterate).
template <int LPR>
__device__ __forceinline__ float row_dot(const float4 &w, float g0, float g1, float g2, float g3) {
    float acc, cmp, e;
    two_sum(__fmul_rn(w.x, g0), __fmul_rn(w.y, g1), acc, cmp);
    two_sum(acc, __fmul_rn(w.z, g2), acc, e);
    cmp = __fadd_rn(cmp, e);
    two_sum(acc, __fmul_rn(w.w, g3), acc, e);
    cmp = __fadd_rn(cmp, e);
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
        float oa = __shfl_xor_sync(0xffffffffu, acc, o), oc = __shfl_xor_sync(0xffffffffu, cmp, o);
        two_sum(acc, oa, acc, e);
        cmp = __fadd_rn(cmp, __fadd_rn(oc, e));
    }
    return __fadd_rn(acc, cmp);
}

// Row schedules. Chunks (FRONT = false): each block owns one contiguous chunk
// of rows and walks it in order. Front (FRONT = true): the rows are cut into
// tiles of TILE_GROUPS row groups, block b takes tiles b, b + G, b + 2G, ...
// (G blocks), so at any time all blocks work in one window of the Morton
// order and the gathered y entries of that window (the successors of its
// rows' neighbours, spatially close) stay in L2 even when y is far larger.
constexpr int TILE_GROUPS = 64;

template <int KP, typename WT, int NT, int MINB, int U, bool FRONT>
__global__ void __launch_bounds__(NT, MINB) sweep_kernel(
    const int32_t *__restrict__ col, const WT *__restrict__ W, const float *__restrict__ rscale,
    const float *__restrict__ b, const float *__restrict__ yin, float *__restrict__ yout, int64_t n_active,
    int32_t *__restrict__ ctrl, double2 *__restrict__ partials, double *__restrict__ resid, int t, double tol) {
    if (*(volatile int32_t *)&ctrl[1]) return; // converged in an earlier sweep
    constexpr int LPR = KP / 4;
    constexpr bool W16 = WTraits<WT>::id != PG_W_F32;
    const int lane = threadIdx.x & 31;
    const int q = lane & (LPR - 1);
    // Each block owns one contiguous chunk of rows and walks it in order:
    // rows are in Morton order, so consecutive rows share most neighbour
    // columns and their y gathers hit in this SM's L1. Every iteration
    // handles U row groups, so each thread has all groups' streamed loads
    // and gathers in flight before it does any arithmetic.
    constexpr int RPB = NT / LPR; // rows per block per group
    constexpr int64_t STEP = (int64_t)U * RPB;
    const int64_t chunk = ((n_active + gridDim.x - 1) / gridDim.x + STEP - 1) / STEP * STEP;
    const int64_t r0 = FRONT ? 0 : min((int64_t)blockIdx.x * chunk, n_active);
    const int64_t r1 = FRONT ? n_active : min(n_active, r0 + chunk);
    auto step_base = [&](int64_t k) -> int64_t {
        if (!FRONT) return r0 + k * STEP;
        const int64_t tile = k / TILE_GROUPS;
        return (tile * gridDim.x + blockIdx.x) * (STEP * TILE_GROUPS) + (k - tile * TILE_GROUPS) * STEP;
    };
    float rd = 0.0f, rn = 0.0f;
    auto group = [&](int64_t base) { // uniform across the block
        int32_t row[U]; // row indices fit in 32 bits (n < 2^31); 64-bit only in element offsets
        bool ok[U];
        int4 c4[U];
        typename WTraits<WT>::raw4 w4[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            row[u] = (int32_t)(base + u * RPB + threadIdx.x / LPR);
            ok[u] = row[u] < r1;
            if (ok[u]) {
                c4[u] = __ldcs(reinterpret_cast<const int4 *>(col + (int64_t)row[u] * KP) + q);
                w4[u] = WTraits<WT>::load4_raw(W + (int64_t)row[u] * KP + q * 4);
            } else {
                c4[u] = make_int4(0, 0, 0, 0);
                w4[u] = {};
            }
        }
        float g[U][4];
#pragma unroll
        for (int u = 0; u < U; u++) {
            g[u][0] = __ldg(yin + c4[u].x);
            g[u][1] = __ldg(yin + c4[u].y);
            g[u][2] = __ldg(yin + c4[u].z);
            g[u][3] = __ldg(yin + c4[u].w);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const float acc = row_dot<LPR>(WTraits<WT>::dec4(w4[u]), g[u][0], g[u][1], g[u][2], g[u][3]);
            if (ok[u] && q == 0) {
                const float sc = W16 ? rscale[row[u]] : 1.0f;
                const float bb = b[row[u]], yo = yin[row[u]];
                const float yn = fmaf(acc, sc, bb);
                yout[row[u]] = yn;
                const float d = yn - yo;
                rd = fmaf(d, d, rd);
                rn = fmaf(yn, yn, rn);
            }
        }
    };
    if constexpr (FRONT) {
        for (int64_t k = 0, base = step_base(0); base < r1; base = step_base(++k)) group(base);
    } else {
        for (int64_t base = r0; base < r1; base += STEP) group(base); // uniform across the block
    }
    sweep_residual<NT>(rd, rn, ctrl, partials, resid, t, tol);
}

// The same sweep, software-pipelined: one row group per iteration, with the
// next group's streamed loads issued before this group's gathers, so the
// DRAM round trip of one group overlaps the L2 round trip of the other. The
// row's scalars (b, its previous iterate, the 16-bit row scale) are loaded
// with the streamed loads by different lanes of the row and shuffled to the
// row's first lane at the end, instead of costing a round trip after the
// gathers.
template <int KP, typename WT, int NT, int MINB, bool FRONT>
__global__ void __launch_bounds__(NT, MINB) sweep_pf_kernel(
    const int32_t *__restrict__ col, const WT *__restrict__ W, const float *__restrict__ rscale,
    const float *__restrict__ b, const float *__restrict__ yin, float *__restrict__ yout, int64_t n_active,
    int32_t *__restrict__ ctrl, double2 *__restrict__ partials, double *__restrict__ resid, int t, double tol) {
    if (*(volatile int32_t *)&ctrl[1]) return; // converged in an earlier sweep
    constexpr int LPR = KP / 4;
    constexpr bool W16 = WTraits<WT>::id != PG_W_F32;
    static_assert(LPR >= (W16 ? 3 : 2), "row scalars need a lane each");
    const int lane = threadIdx.x & 31;
    const int q = lane & (LPR - 1);
    const int lead = lane & ~(LPR - 1);
    constexpr int RPB = NT / LPR;
    const int64_t chunk = ((n_active + gridDim.x - 1) / gridDim.x + RPB - 1) / RPB * RPB;
    const int64_t r0 = FRONT ? 0 : min((int64_t)blockIdx.x * chunk, n_active);
    const int64_t r1 = FRONT ? n_active : min(n_active, r0 + chunk);
    auto group_base = [&](int64_t k) -> int64_t {
        if (!FRONT) return r0 + k * RPB;
        const int64_t tile = k / TILE_GROUPS;
        return (tile * gridDim.x + blockIdx.x) * ((int64_t)RPB * TILE_GROUPS) + (k - tile * TILE_GROUPS) * RPB;
    };
    const int32_t lr = threadIdx.x / LPR;
    auto load = [&](int64_t base, int4 &c4, float4 &w4, float &sv) {
        const int64_t row = base + lr;
        c4 = make_int4(0, 0, 0, 0);
        w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        sv = 0.0f;
        if (row < r1) {
            c4 = __ldcs(reinterpret_cast<const int4 *>(col + row * KP) + q);
            w4 = WTraits<WT>::load4(W + row * KP + q * 4);
            if (q == 0) sv = __ldcs(b + row);
            else if (q == 1) sv = yin[row];
            else if (W16 && q == 2) sv = __ldcs(rscale + row);
        }
    };
    float rd = 0.0f, rn = 0.0f;
    int4 c4n;
    float4 w4n;
    float svn;
    int64_t base = group_base(0);
    if (base < r1) load(base, c4n, w4n, svn);
    for (int64_t k = 0; base < r1; k++) { // uniform across the block
        const int4 c4 = c4n;
        const float4 w4 = w4n;
        const float sv = svn;
        const int64_t nb = group_base(k + 1);
        if (nb < r1) load(nb, c4n, w4n, svn);
        const float g0 = __ldg(yin + c4.x), g1 = __ldg(yin + c4.y), g2 = __ldg(yin + c4.z), g3 = __ldg(yin + c4.w);
        const float acc = row_dot<LPR>(w4, g0, g1, g2, g3);
        const float yo = __shfl_sync(0xffffffffu, sv, lead + 1);
        const float sc = W16 ? __shfl_sync(0xffffffffu, sv, lead + 2) : 1.0f;
        const int64_t row = base + lr;
        if (row < r1 && q == 0) {
            const float yn = fmaf(acc, sc, sv);
            yout[row] = yn;
            const float d = yn - yo;
            rd = fmaf(d, d, rd);
            rn = fmaf(yn, yn, rn);
        }
        base = nb;
    }
    sweep_residual<NT>(rd, rn, ctrl, partials, resid, t, tol);
}

// The front schedule pays off once the gathered vector no longer fits in L2
// with room to spare (measured: 31 MB of y, the 8.7M-vertex cloud, is 10 %
// faster in chunks; 151 MB and 604 MB, the dense medium at half and full
// image size, 5-30 % faster in fronts).
bool pg_sweep_front(int64_t n_active) { return n_active * 4 > ((int64_t)64 << 20); }
static bool use_front(const pg_graph *g) { return pg_sweep_front(g->n_active); }

template <int KP, typename WT, int NT, int MINB>
static void launch_pf_cfg(const pg_graph *g, const float *b, const float *yin, float *yout, int32_t *ctrl,
                          double2 *partials, double *resid, int t, double tol, cudaStream_t s) {
    int64_t need = (g->n_active * (KP / 4) + NT - 1) / NT;
    int64_t cap = (int64_t)pg_num_sms() * MINB;
    int blocks = (int)std::max<int64_t>(1, std::min(need, cap));
    if (use_front(g))
        sweep_pf_kernel<KP, WT, NT, MINB, true><<<blocks, NT, 0, s>>>(g->col, (const WT *)g->W, g->rscale, b, yin,
                                                                      yout, g->n_active, ctrl, partials, resid, t, tol);
    else
        sweep_pf_kernel<KP, WT, NT, MINB, false><<<blocks, NT, 0, s>>>(g->col, (const WT *)g->W, g->rscale, b, yin,
                                                                       yout, g->n_active, ctrl, partials, resid, t,
                                                                       tol);
}

// slot n of each of `slices` vectors of n+1 floats
__global__ void zero_slots_kernel(float *__restrict__ v, int64_t n, int64_t slices) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < slices) v[t * (n + 1) + n] = 0.0f;
}

// y0[row of succ(v)] = L0[v]  (L+_v is the radiance that succ(v) sends back)
__global__ void init_y_kernel(const float *__restrict__ L0, const int32_t *__restrict__ c2m,
                              const int32_t *__restrict__ succ_m, const int32_t *__restrict__ m2r, int64_t n,
                              float *__restrict__ y0) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t s = succ_m[c2m[v]];
    if (s >= 0) y0[m2r[s]] = L0[v];
}

__global__ void b_from_c_kernel(const float *__restrict__ c, const int32_t *__restrict__ c2m,
                                const int32_t *__restrict__ m2r, const float4 *__restrict__ LV, int64_t n,
                                float *__restrict__ b) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t m = c2m[v];
    b[m2r[m]] = LV[m].w * c[v];
}

// L[v] = y_T[row of succ(v)], 0 at the end of a path. The final iterate is
// the one of the last sweep that ran (ctrl[0]); with a history it is slice
// ctrl[0], otherwise ping-pong buffer ctrl[0] % 2.
__global__ void finish_L_kernel(const int32_t *__restrict__ c2m, const int32_t *__restrict__ succ_m,
                                const int32_t *__restrict__ m2r, int64_t n, const float *__restrict__ y_a,
                                const float *__restrict__ y_b, const float *__restrict__ hist,
                                const int32_t *__restrict__ ctrl, float *__restrict__ L) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t it = ctrl[0];
    const float *y = hist ? hist + (int64_t)it * (n + 1) : ((it & 1) ? y_b : y_a);
    int32_t s = succ_m[c2m[v]];
    L[v] = s >= 0 ? y[m2r[s]] : 0.0f;
}

template <int KP, typename WT, int NT, int MINB, int U>
static void launch_sweep_cfg(const pg_graph *g, const float *b, const float *yin, float *yout, int32_t *ctrl,
                             double2 *partials, double *resid, int t, double tol, cudaStream_t s) {
    int64_t need = (g->n_active * (KP / 4) + NT - 1) / NT;
    int64_t cap = (int64_t)pg_num_sms() * MINB;
    int blocks = (int)std::max<int64_t>(1, std::min(need, cap));
    if (use_front(g))
        sweep_kernel<KP, WT, NT, MINB, U, true><<<blocks, NT, 0, s>>>(g->col, (const WT *)g->W, g->rscale, b, yin,
                                                                      yout, g->n_active, ctrl, partials, resid, t, tol);
    else
        sweep_kernel<KP, WT, NT, MINB, U, false><<<blocks, NT, 0, s>>>(g->col, (const WT *)g->W, g->rscale, b, yin,
                                                                       yout, g->n_active, ctrl, partials, resid, t,
                                                                       tol);
}

// Launch shapes (measured on the 8.7M-vertex cloud, k = 16): FP32 rows in the
// pipelined kernel, one 1024-thread block per SM (one row chunk per L1);
// 16-bit rows (whose streamed bytes are smaller, so the gathers weigh more)
// in the two-group kernel, two 1024-thread blocks per SM.
template <int KP, typename WT>
static pg_status launch_sweep(const pg_graph *g, const float *b, const float *yin, float *yout, int32_t *ctrl,
                              double2 *partials, double *resid, int t, double tol, cudaStream_t s) {
    if constexpr (WTraits<WT>::id == PG_W_F32 && KP >= 8)
        launch_pf_cfg<KP, WT, 1024, 1>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
    else if constexpr (KP >= 16)
        launch_sweep_cfg<KP, WT, 1024, 2, 2>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
    else
        launch_sweep_cfg<KP, WT, 1024, 2, 1>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

template <typename WT>
static pg_status launch_sweep_k(const pg_graph *g, const float *b, const float *yin, float *yout, int32_t *ctrl,
                                double2 *partials, double *resid, int t, double tol, cudaStream_t s) {
    switch (g->kp) {
        case 4: return launch_sweep<4, WT>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        case 8: return launch_sweep<8, WT>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        case 16: return launch_sweep<16, WT>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        case 32: return launch_sweep<32, WT>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        default: return PG_ERR_UNSUPPORTED;
    }
}

static pg_status launch_sweep_w(const pg_graph *g, const float *b, const float *yin, float *yout, int32_t *ctrl,
                                double2 *partials, double *resid, int t, double tol, cudaStream_t s) {
    switch (g->wdtype) {
        case PG_W_F32: return launch_sweep_k<float>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        case PG_W_BF16: return launch_sweep_k<__nv_bfloat16>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        case PG_W_F16: return launch_sweep_k<__half>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
        case PG_W_U16: return launch_sweep_k<pg_unorm16>(g, b, yin, yout, ctrl, partials, resid, t, tol, s);
    }
    return PG_ERR_UNSUPPORTED;
}

// One sweep over the rows of a graph view (a shard's rows with its own
// column table, see pg_shard.cu).
pg_status pg_launch_sweep(const pg_graph *view, const float *b, const float *yin, float *yout, int32_t *ctrl,
                          double2 *partials, double *resid, int t, double tol, cudaStream_t s) {
    return launch_sweep_w(view, b, yin, yout, ctrl, partials, resid, t, tol, s);
}

int pg_sweep_blocks(const pg_graph *g) {
    int64_t lanes = g->n_active * (g->kp / 4);
    int64_t need = (lanes + SWEEP_THREADS - 1) / SWEEP_THREADS;
    int64_t cap = (int64_t)pg_num_sms() * 8; // 8 x 256 threads = 2048 per SM
    int64_t bl = need < cap ? need : cap;
    return (int)(bl < 1 ? 1 : bl);
}

extern "C" pg_status pg_propagate(pg_graph *g, const float *c, const float *L0, int32_t iters, double tol,
                                  int32_t keep_history, float *L, double *residual, int32_t *iters_done,
                                  pg_stream_t stream) {
    if (!g || iters < 0) return PG_ERR_INVALID_ARG;
    if (!g->aggregated) return PG_ERR_STATE;
    if (!g->W) return PG_ERR_STATE;
    const int64_t n = g->n;
    if (n > 0 && (!L0 || !L)) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    pg_status st = PG_OK;
    // buffers
    if (!g->ybuf[0]) {
        PG_TRY(pg_alloc(g, (void **)&g->ybuf[0], 4 * (size_t)(n + 1), s));
        PG_TRY(pg_alloc(g, (void **)&g->ybuf[1], 4 * (size_t)(n + 1), s));
        PG_CUDA(cudaMemsetAsync(g->ybuf[0], 0, 4 * (size_t)(n + 1), s));
        PG_CUDA(cudaMemsetAsync(g->ybuf[1], 0, 4 * (size_t)(n + 1), s));
    }
    if (!g->d_ctrl) PG_TRY(pg_alloc(g, (void **)&g->d_ctrl, 16, s));
    int blocks = pg_sweep_blocks(g);
    if (g->partials_cap < blocks) {
        pg_free(g, (void **)&g->d_partials, 16 * (size_t)g->partials_cap);
        g->partials_cap = 0;
        PG_TRY(pg_alloc(g, (void **)&g->d_partials, 16 * (size_t)blocks, s));
        g->partials_cap = blocks;
    }
    int rcap = iters > 0 ? iters : 1;
    if (g->resid_cap < rcap) {
        pg_free(g, (void **)&g->d_resid, 8 * (size_t)g->resid_cap);
        g->resid_cap = 0;
        PG_TRY(pg_alloc(g, (void **)&g->d_resid, 8 * (size_t)rcap, s));
        g->resid_cap = rcap;
    }
    if (keep_history && g->hist_cap < iters) {
        pg_free(g, (void **)&g->hist, 4 * (size_t)(n + 1) * (size_t)(g->hist_cap + 1));
        g->hist_cap = -1;
        PG_TRY(pg_alloc(g, (void **)&g->hist, 4 * (size_t)(n + 1) * (size_t)(iters + 1), s));
        // only each slice's zero slot needs a value up front: a sweep writes
        // rows [0, n_active) of its slice, init_y those of slice 0, and no
        // reader touches rows [n_active, n)
        zero_slots_kernel<<<pg_blocks(iters + 1, 256), 256, 0, s>>>(g->hist, n, iters + 1);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
        g->hist_cap = iters;
    }
    g->hist_iters = -1;
    PG_CUDA(cudaMemsetAsync(g->d_ctrl, 0, 16, s));
    PG_CUDA(cudaMemsetAsync(g->d_resid, 0, 8 * (size_t)rcap, s));
    if (n == 0) {
        if (residual && iters > 0) for (int i = 0; i < iters; i++) residual[i] = 0.0;
        if (iters_done) *iters_done = 0;
        return PG_OK;
    }
    const float *b = g->b;
    float *buser = nullptr;
    if (c) {
        PG_TRY(pg_alloc(nullptr, (void **)&buser, 4 * (size_t)(n + 1), s));
        cudaMemsetAsync(buser, 0, 4 * (size_t)(n + 1), s);
        b_from_c_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(c, g->c2m, g->m2r, g->LV, n, buser);
        pg_count_launches(1);
        b = buser;
    }
    const int64_t stride = n + 1;
    float *y0 = keep_history ? g->hist : g->ybuf[0];
    init_y_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(L0, g->c2m, g->succ_m, g->m2r, n, y0);
    pg_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    for (int t = 1; t <= iters && st == PG_OK; t++) {
        const float *yin = keep_history ? g->hist + (int64_t)(t - 1) * stride : g->ybuf[(t - 1) & 1];
        float *yout = keep_history ? g->hist + (int64_t)t * stride : g->ybuf[t & 1];
        st = launch_sweep_w(g, b, yin, yout, g->d_ctrl, (double2 *)g->d_partials, g->d_resid, t, tol, s);
    }
    if (st == PG_OK) {
        finish_L_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(g->c2m, g->succ_m, g->m2r, n, g->ybuf[0], g->ybuf[1],
                                                          keep_history ? g->hist : nullptr, g->d_ctrl, L);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (buser) cudaFreeAsync(buser, s);
    if (st != PG_OK) return st;
    if (keep_history) g->hist_iters = iters;
    // with early stopping the stored history ends at the last sweep that ran
    if (residual || iters_done || (keep_history && tol > 0.0)) {
        int32_t ctrl[4] = {0, 0, 0, 0};
        PG_CUDA(cudaMemcpyAsync(ctrl, g->d_ctrl, 16, cudaMemcpyDeviceToHost, s));
        if (residual && iters > 0)
            PG_CUDA(cudaMemcpyAsync(residual, g->d_resid, 8 * (size_t)iters, cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
        if (iters_done) *iters_done = ctrl[0];
        if (keep_history) g->hist_iters = ctrl[0];
    }
    return PG_OK;
}

// ------------------------------------------------------------------ propagation without allocation
// pg_propagate_noalloc runs the same sweeps as pg_propagate, but keeps all of
// its scratch (the two ping-pong iterates, the per-block residual partials,
// the per-sweep residuals and the control words) in one file-scope device
// array instead of memory allocated at run time. Every call on a device shares
// this array.
static constexpr int64_t NA_MAX_N = PG_NOALLOC_MAX_VERTICES;
static constexpr int NA_MAX_ITERS = PG_NOALLOC_MAX_ITERS;
static constexpr int NA_MAX_BLOCKS = 4096;
static constexpr size_t NA_Y_BYTES = 4 * (size_t)(NA_MAX_N + 1);
static constexpr size_t NA_Y0 = 0;
static constexpr size_t NA_Y1 = (NA_Y_BYTES + 255) / 256 * 256;
static constexpr size_t NA_PARTIALS = NA_Y1 + (NA_Y_BYTES + 255) / 256 * 256;
static constexpr size_t NA_RESID = NA_PARTIALS + 16 * (size_t)NA_MAX_BLOCKS;
static constexpr size_t NA_CTRL = NA_RESID + 8 * (size_t)NA_MAX_ITERS;
static constexpr size_t NA_BYTES = NA_CTRL + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of the scratch array, looked up once per device (host code
// cannot use the symbol itself: it is only a host-side stand-in).
static pg_status noalloc_scratch(unsigned char **out) {
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    int dev = 0;
    PG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return PG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        // with lazy module loading this is where the array is reserved on
        // the device, so a device without room for it reports PG_ERR_OOM
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? PG_ERR_OOM : PG_ERR_CUDA;
        }
        addr[dev] = (unsigned char *)p;
    }
    *out = addr[dev];
    return PG_OK;
}

extern "C" pg_status pg_propagate_noalloc(pg_graph *g, const float *L0, int32_t iters, double tol, float *L,
                                          pg_stream_t stream) {
    if (!g || iters < 0) return PG_ERR_INVALID_ARG;
    if (!g->aggregated || !g->W) return PG_ERR_STATE;
    if (g->n > NA_MAX_N || iters > NA_MAX_ITERS) return PG_ERR_UNSUPPORTED;
    const int64_t n = g->n;
    if (n == 0) return PG_OK;
    if (!L0 || !L) return PG_ERR_INVALID_ARG;
    if (pg_num_sms() * 8 > NA_MAX_BLOCKS) return PG_ERR_UNSUPPORTED; // partials of one sweep
    unsigned char *base = nullptr;
    PG_TRY(noalloc_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;
    float *y0 = (float *)(base + NA_Y0), *y1 = (float *)(base + NA_Y1);
    double2 *partials = (double2 *)(base + NA_PARTIALS);
    double *resid = (double *)(base + NA_RESID);
    int32_t *ctrl = (int32_t *)(base + NA_CTRL);
    // the array keeps the previous call's contents: reset what must start at zero
    PG_CUDA(cudaMemsetAsync(ctrl, 0, 16, s));
    PG_CUDA(cudaMemsetAsync(y0 + n, 0, 4, s)); // zero slot of both iterates
    PG_CUDA(cudaMemsetAsync(y1 + n, 0, 4, s));
    if (iters > 0) PG_CUDA(cudaMemsetAsync(resid, 0, 8 * (size_t)iters, s));
    init_y_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(L0, g->c2m, g->succ_m, g->m2r, n, y0);
    pg_count_launches(1);
    for (int t = 1; t <= iters; t++) {
        const float *yin = (t & 1) ? y0 : y1;
        float *yout = (t & 1) ? y1 : y0;
        PG_TRY(launch_sweep_w(g, g->b, yin, yout, ctrl, partials, resid, t, tol, s));
    }
    finish_L_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(g->c2m, g->succ_m, g->m2r, n, y0, y1, nullptr, ctrl, L);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}
