// Aggregation (Section 3.5): the MIS edge weights A+ of Eq. ag-indirect, the
// direct term A°L° of Eq. ag-direct, and the non-aggregated direct light D
// used at output (Section 4, "Handling direct light"). A sample's marginal
// density is summed over the rows that aggregate it, so that its balance
// weights over those rows sum to one (as within one of the paper's clusters)
// and the sweep matrix's column sums stay below the albedo.
//
// Layout produced for the propagation sweep (Eq. rte-mff, L+ = P A+ L+ + P c):
// the sweep works on y_s = (tau/p_t)_s (A+ L+ + c)_s, the radiance that s
// sends to its predecessor, so L+_v = y_{succ(v)} and
//   y_s <- sum_{j in N(s)} W_{s,j} y_{succ(j)} + b_s,
//   W_{s,j} = (tau/p_t)_s A+_{s,j},  b_s = (tau/p_t)_s c_s.
// Rows are stored in "sweep order" r: vertices that have a predecessor first
// (in Morton order), then the paths' first vertices, whose y is never read
// by a sweep. Column ids are sweep rows of succ(j); j at the end of its path
// (or a missing neighbour) points at the zero slot n.
#include "pg_internal.cuh"

// One vertex's records, 64 bytes: (o, g), (d, p_ph), (e, p_e or -1 for a
// delta light), (Le, Lph, sigma_s, w).
struct alignas(16) vrec64 {
    float4 og, dp, ep, lv;
};

// Pass 1, caller order i: read and check the vertex's records (coalesced)
// and write them as one 64-byte record, still in caller order, with the
// Morton index of the vertex's successor. Writing the four Morton-ordered
// arrays from here would scatter 16-byte pieces of 32-byte sectors; the
// second pass gathers whole 64-byte records instead and writes in order.
__global__ void pack_kernel(pg_vertices v, int64_t n, const int32_t *__restrict__ c2m, vrec64 *__restrict__ rec,
                            int32_t *__restrict__ succ_c, int32_t *__restrict__ predcnt,
                            int32_t *__restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float ox = v.ox[i], oy = v.oy[i], oz = v.oz[i], g = v.g[i];
    float dx = v.dx[i], dy = v.dy[i], dz = v.dz[i], pph = v.pe_ph[i];
    float ex = v.ex[i], ey = v.ey[i], ez = v.ez[i], pe = v.pe_e[i];
    float Le = v.Le[i], Lph = v.Lph[i], ss = v.sigma_s[i], w = v.w_prop[i];
    int delta = v.e_delta[i] != 0;
    int32_t sc = v.succ[i];
    bool fin = isfinite(ox) && isfinite(oy) && isfinite(oz) && isfinite(g) && isfinite(dx) && isfinite(dy) &&
               isfinite(dz) && isfinite(pph) && isfinite(ex) && isfinite(ey) && isfinite(ez) && isfinite(pe) &&
               isfinite(Le) && isfinite(Lph) && isfinite(ss) && isfinite(w);
    int f = 0;
    if (!fin) f |= PG_FLAG_NONFINITE;
    if (!(fabsf(g) < 1.0f) || ss < 0.0f || w < 0.0f || pph < 0.0f || (!delta && pe < 0.0f)) f |= PG_FLAG_BAD_RANGE;
    int32_t sm = -1;
    if (sc >= 0) {
        if (sc >= n || sc == i) {
            f |= PG_FLAG_BAD_INDEX;
        } else {
            sm = c2m[sc];
            atomicAdd(&predcnt[sm], 1); // a second predecessor is flagged by active_flag_kernel
        }
    } else if (sc != -1) {
        f |= PG_FLAG_BAD_INDEX;
    }
    if (f) atomicOr(flags, f);
    vrec64 r;
    r.og = make_float4(ox, oy, oz, g);
    r.dp = make_float4(dx, dy, dz, pph);
    r.ep = make_float4(ex, ey, ez, delta ? -1.0f : pe);
    r.lv = make_float4(Le, Lph, ss, w);
    rec[i] = r;
    succ_c[i] = sm;
}

// Pass 2, Morton order m: the four record arrays and the successor.
__global__ void permute_records_kernel(const vrec64 *__restrict__ rec, const int32_t *__restrict__ succ_c,
                                       const int32_t *__restrict__ m2c, int64_t n, float4 *__restrict__ OG,
                                       float4 *__restrict__ DP, float4 *__restrict__ EP, float4 *__restrict__ LV,
                                       int32_t *__restrict__ succ_m) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int32_t i = m2c[m];
    const vrec64 r = rec[i];
    OG[m] = r.og;
    DP[m] = r.dp;
    EP[m] = r.ep;
    LV[m] = r.lv;
    succ_m[m] = succ_c[i];
}

__global__ void active_flag_kernel(const int32_t *__restrict__ predcnt, int64_t n, int32_t *__restrict__ act,
                                   int32_t *__restrict__ flags) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int32_t pc = predcnt[m];
    act[m] = pc > 0 ? 1 : 0;
    if (pc > 1) atomicOr(flags, PG_FLAG_TWO_PREDS);
}

// sweep row of each vertex's successor, or the zero slot n at a path end
__global__ void succ_row_kernel(const int32_t *__restrict__ succ_m, const int32_t *__restrict__ m2r, int64_t n,
                                int32_t *__restrict__ sr) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int32_t s = succ_m[m];
    sr[m] = s >= 0 ? m2r[s] : (int32_t)n;
}

// act holds the exclusive prefix of the active flags; predcnt the flags' source
__global__ void row_order_kernel(const int32_t *__restrict__ predcnt, const int32_t *__restrict__ act_prefix,
                                 const int32_t *__restrict__ d_n_active, int64_t n, int32_t *__restrict__ m2r,
                                 int32_t *__restrict__ r2m) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int32_t pre = act_prefix[m];
    int32_t r = predcnt[m] > 0 ? pre : (*d_n_active + (int32_t)(m - pre));
    m2r[m] = r;
    r2m[r] = (int32_t)m;
}

// Pass 1: the marginal densities of every sample over the rows that use it
// (Eq. indirect-weight read on a neighbour graph: sample j is combined by the
// strategies of R(j) = {r : j in N(r)}, so pm_d[j] = sum_{r in R(j)}
// rho_r(o_r, d_j), pm_e[j] likewise for e_j, and kin[j] = |R(j)|). One group
// of KP lanes per row r; lane i adds row r's two phase-function values for
// its sample nbr[r][i] with exact fixed-point atomics.
template <int KP>
__global__ void __launch_bounds__(256) marginal_kernel(const int32_t *__restrict__ nbr,
                                                       const float4 *__restrict__ OG,
                                                       const float4 *__restrict__ DP,
                                                       const float4 *__restrict__ EP, int64_t n,
                                                       unsigned long long *__restrict__ pmd,
                                                       unsigned long long *__restrict__ pme,
                                                       uint32_t *__restrict__ kin) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = t / KP;
    if (m >= n) return;
    const int32_t nj = nbr[t];
    if (nj < 0) return;
    const float4 og = OG[m], dp = DP[nj], ep = EP[nj];
    const HGc h = hg_consts(og.w);
    const float eo = unit_err(og.x, og.y, og.z);
    const float rd = hg_eval(h, one_plus_dot_u(og.x, og.y, og.z, eo, dp.x, dp.y, dp.z, unit_err(dp.x, dp.y, dp.z)));
    const float re = hg_eval(h, one_plus_dot_u(og.x, og.y, og.z, eo, ep.x, ep.y, ep.z, unit_err(ep.x, ep.y, ep.z)));
    atomicAdd(pmd + nj, pg_pm_fix(rd));
    atomicAdd(pme + nj, pg_pm_fix(re));
    atomicAdd(kin + nj, 1u);
}

// Pass 2: one group of KP lanes per row s (Morton order m); lane j owns
// neighbour slot j of N(s) and forms that sample's weights from the
// receiver's phase function and the sample's marginals. Blocks stride over
// the rows (a fixed grid), so the count of swept entries costs one atomic
// per block.
template <int KP, typename WT>
__global__ void __launch_bounds__(256) aggregate_kernel(
    const int32_t *__restrict__ nbr, const float4 *__restrict__ OG, const float4 *__restrict__ DP,
    const float4 *__restrict__ EP, const float4 *__restrict__ LV, const int32_t *__restrict__ sr,
    const unsigned long long *__restrict__ pmd, const unsigned long long *__restrict__ pme,
    const uint32_t *__restrict__ kin, const int32_t *__restrict__ m2r, const int32_t *__restrict__ m2c, int64_t n,
    int64_t n_active, WT *__restrict__ W, float *__restrict__ rscale, int32_t *__restrict__ col,
    float *__restrict__ b, float *__restrict__ c_m, float *__restrict__ D_m, float *__restrict__ c_out,
    float *__restrict__ D_out, unsigned long long *__restrict__ nnz_counter) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (KP - 1);
    const int src = lane & ~(KP - 1); // lane of slot 0 (the receiver itself)
    constexpr int RPB = 256 / KP;     // rows per block per iteration
    unsigned long long counted_total = 0;
    for (int64_t base = (int64_t)blockIdx.x * RPB; base < n; base += (int64_t)gridDim.x * RPB) {
        const int64_t m = base + threadIdx.x / KP;
        const bool row_ok = m < n;
        const int32_t nj = row_ok ? nbr[m * KP + j] : -1;
        const bool valid = nj >= 0;
        const float4 os = row_ok ? OG[m] : make_float4(0.f, 0.f, 1.f, 0.f);
        float4 dp = make_float4(0.f, 0.f, 1.f, 0.f), ep = make_float4(0.f, 0.f, 1.f, 0.f),
               lv = make_float4(0.f, 0.f, 0.f, 0.f);
        int32_t cl = (int32_t)n; // sweep row of succ(j), or the zero slot
        float pm_d = 1.0f, pm_e = 1.0f, kj = 1.0f;
        if (valid) {
            dp = DP[nj];
            ep = EP[nj];
            lv = LV[nj];
            cl = sr[nj];
            pm_d = pg_pm_float(pmd[nj]);
            pm_e = pg_pm_float(pme[nj]);
            kj = (float)kin[nj];
        }
        const unsigned gmask = (KP == 32) ? 0xffffffffu : (((1u << KP) - 1u) << src);
        const float Ks = (float)__popc(__ballot_sync(0xffffffffu, valid) & gmask); // |N(s)|
        const HGc hs = hg_consts(os.w);
        const float es = unit_err(os.x, os.y, os.z);
        const float rho_sd = hg_eval(hs, one_plus_dot_u(os.x, os.y, os.z, es, dp.x, dp.y, dp.z, unit_err(dp.x, dp.y, dp.z)));
        const float rho_se = hg_eval(hs, one_plus_dot_u(os.x, os.y, os.z, es, ep.x, ep.y, ep.z, unit_err(ep.x, ep.y, ep.z)));
        const float sig_s = __shfl_sync(0xffffffffu, lv.z, src);
        const float w_s = __shfl_sync(0xffffffffu, lv.w, src);
        const bool delta = ep.w < 0.0f;
        float A = 0.0f, term = 0.0f;
        if (valid) {
            A = sig_s * rho_sd / pm_d;
            const float Ae = delta ? sig_s * rho_se / Ks : sig_s * rho_se / fmaf(kj, ep.w, pm_e);
            const float Aph = sig_s * rho_sd / fmaf(kj, dp.w, pm_d);
            term = fmaf(Ae, lv.x, Aph * lv.y);
        }
        // c_s: sum over the group's lanes (fixed butterfly order)
        float c = term;
    #pragma unroll
        for (int o = KP / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        // D_s from slot 0's own samples (K = 1)
        float Dterm = 0.0f;
        if (j == 0 && valid) {
            const float De = delta ? rho_se * lv.x : rho_se * lv.x / (rho_se + ep.w);
            const float Dp = rho_sd * lv.y / (rho_sd + dp.w);
            Dterm = sig_s * (De + Dp);
        }
        const float Wt = w_s * A;
        const int32_t r = row_ok ? m2r[m] : 0;
        float mx = 1.0f;
        if (WTraits<WT>::id != PG_W_F32) {
            mx = Wt;
    #pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            mx = mx > 0.0f ? mx : 1.0f;
        }
        // 16-bit payload: the row's weights relative to its largest one, rounded
        // to nearest (error diffusion along the row was measured to be worse:
        // the gathered radiance of a row's columns is far from uniform)
        const WT wq = WTraits<WT>::enc(Wt, mx);
        const float scale = WTraits<WT>::scale(mx);
        if (row_ok) {
            W[(int64_t)r * KP + j] = wq;
            col[(int64_t)r * KP + j] = cl;
            if (j == 0) {
                b[r] = w_s * c;
                if (WTraits<WT>::id != PG_W_F32) rscale[r] = scale;
                c_m[m] = c;
                D_m[m] = Dterm;
                const int32_t ci = m2c[m];
                if (c_out) c_out[ci] = c;
                if (D_out) D_out[ci] = Dterm;
            }
        }
        // edge updates per sweep: real entries of rows that have a predecessor
        const bool counted = row_ok && valid && cl < n && r < n_active;
        counted_total += __popc(__ballot_sync(0xffffffffu, counted));
    }
    __shared__ unsigned long long s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    if (lane == 0 && counted_total) atomicAdd(&s_cnt, counted_total);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(nnz_counter, s_cnt);
}

template <int KP, typename WT>
static pg_status launch_agg(pg_graph *g, float *c_out, float *D_out, unsigned long long *cnt, cudaStream_t s) {
    int64_t threads = g->n * KP;
    PG_CUDA(cudaMemsetAsync(g->pmd, 0, 8 * (size_t)g->n, s));
    PG_CUDA(cudaMemsetAsync(g->pme, 0, 8 * (size_t)g->n, s));
    PG_CUDA(cudaMemsetAsync(g->kin, 0, 4 * (size_t)g->n, s));
    int32_t *sr = nullptr;
    PG_TRY(pg_alloc(nullptr, (void **)&sr, 4 * (size_t)g->n, s));
    marginal_kernel<KP><<<pg_blocks(threads, 256), 256, 0, s>>>(g->nbr, g->OG, g->DP, g->EP, g->n, g->pmd, g->pme,
                                                                g->kin);
    succ_row_kernel<<<pg_blocks(g->n, 256), 256, 0, s>>>(g->succ_m, g->m2r, g->n, sr);
    // a fixed grid of exactly the resident blocks: every block strides over
    // the same share of rows, so a grid larger than one wave would leave a
    // second, nearly empty wave
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, aggregate_kernel<KP, WT>, 256, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            b = 1;
        }
        return b < 1 ? 1 : b;
    }();
    int64_t need = (g->n * KP + 255) / 256;
    int64_t cap = (int64_t)pg_num_sms() * per_sm;
    aggregate_kernel<KP, WT><<<(int)(need < cap ? need : cap), 256, 0, s>>>(
        g->nbr, g->OG, g->DP, g->EP, g->LV, sr, g->pmd, g->pme, g->kin, g->m2r, g->m2c, g->n, g->n_active,
        (WT *)g->W, g->rscale, g->col, g->b, g->c_m, g->D_m, c_out, D_out, cnt);
    pg_count_launches(3);
    cudaFreeAsync(sr, s);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

template <typename WT>
static pg_status launch_agg_k(pg_graph *g, float *c_out, float *D_out, unsigned long long *cnt, cudaStream_t s) {
    switch (g->kp) {
        case 4: return launch_agg<4, WT>(g, c_out, D_out, cnt, s);
        case 8: return launch_agg<8, WT>(g, c_out, D_out, cnt, s);
        case 16: return launch_agg<16, WT>(g, c_out, D_out, cnt, s);
        case 32: return launch_agg<32, WT>(g, c_out, D_out, cnt, s);
        default: return PG_ERR_UNSUPPORTED;
    }
}

static bool verts_ok(const pg_vertices *v) {
    return v->ox && v->oy && v->oz && v->dx && v->dy && v->dz && v->ex && v->ey && v->ez && v->g && v->sigma_s &&
           v->w_prop && v->Le && v->pe_e && v->Lph && v->pe_ph && v->e_delta && v->succ;
}

extern "C" pg_status pg_aggregate(pg_graph *g, const pg_vertices *v, pg_wdtype wdtype, float *c, float *D,
                                  pg_stream_t stream) {
    if (!g) return PG_ERR_INVALID_ARG;
    if (wdtype != PG_W_F32 && wdtype != PG_W_BF16 && wdtype != PG_W_F16 && wdtype != PG_W_U16)
        return PG_ERR_INVALID_ARG;
    if (g->n > 0 && (!v || !verts_ok(v))) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    const int64_t n = g->n;
    const size_t kp = (size_t)g->kp;
    // (re)allocate the aggregation buffers
    size_t wb_old = pg_wbytes(g->wdtype);
    pg_free(g, (void **)&g->W, wb_old * n * kp);
    pg_free_transposes(g);
    g->aggregated = 0;
    g->hist_iters = -1;
    g->wdtype = wdtype;
    pg_status st = PG_OK;
#define A(ptr, bytes) \
    if (st == PG_OK && !(ptr)) st = pg_alloc(g, (void **)&(ptr), (bytes), s)
    A(g->m2r, 4 * (size_t)n);
    A(g->r2m, 4 * (size_t)n);
    A(g->OG, 16 * (size_t)n);
    A(g->DP, 16 * (size_t)n);
    A(g->EP, 16 * (size_t)n);
    A(g->LV, 16 * (size_t)n);
    A(g->succ_m, 4 * (size_t)n);
    A(g->W, pg_wbytes(wdtype) * n * kp);
    A(g->rscale, 4 * (size_t)n);
    A(g->col, 4 * n * kp);
    A(g->b, 4 * (size_t)(n + 1));
    A(g->c_m, 4 * (size_t)n);
    A(g->D_m, 4 * (size_t)n);
    A(g->pmd, 8 * (size_t)n);
    A(g->pme, 8 * (size_t)n);
    A(g->kin, 4 * (size_t)n);
#undef A
    if (st != PG_OK) return st;
    if (n == 0) {
        g->aggregated = 1;
        g->n_active = 0;
        g->nnz_swept = 0;
        return PG_OK;
    }
    int32_t *predcnt = nullptr, *act = nullptr, *d_nact = nullptr;
    unsigned long long *d_cnt = nullptr;
    // The caller-order records live in the entry-column array until the
    // weight pass writes it (4 kp bytes per vertex, enough from kp = 16),
    // else in a temporary; the successors' Morton indices live in act,
    // which the active-row flags overwrite after the permutation.
    vrec64 *rec = nullptr, *rec_tmp = nullptr;
    st = pg_alloc(nullptr, (void **)&predcnt, 4 * (size_t)n, s);
    if (st == PG_OK) {
        if ((size_t)4 * kp >= sizeof(vrec64))
            rec = reinterpret_cast<vrec64 *>(g->col);
        else if ((st = pg_alloc(nullptr, (void **)&rec_tmp, sizeof(vrec64) * (size_t)n, s)) == PG_OK)
            rec = rec_tmp;
    }
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&act, 4 * (size_t)n, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&d_nact, 16, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&d_cnt, 16, s);
    if (st == PG_OK && (cudaMemsetAsync(predcnt, 0, 4 * (size_t)n, s) != cudaSuccess ||
                        cudaMemsetAsync(d_cnt, 0, 16, s) != cudaSuccess ||
                        cudaMemsetAsync(g->flags, 0, 16, s) != cudaSuccess))
        st = PG_ERR_CUDA;
    if (st == PG_OK) {
        pack_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(*v, n, g->c2m, rec, act, predcnt, g->flags);
        permute_records_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(rec, act, g->m2c, n, g->OG, g->DP, g->EP, g->LV,
                                                                 g->succ_m);
        pg_count_launches(2);
        active_flag_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(predcnt, n, act, g->flags);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK) st = pg_scan_exclusive(g, act, n, d_nact, s);
    int32_t h_nact = 0;
    if (st == PG_OK) {
        row_order_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(predcnt, act, d_nact, n, g->m2r, g->r2m);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    int32_t hflags = 0;
    if (st == PG_OK && (cudaMemcpyAsync(&h_nact, d_nact, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaMemcpyAsync(&hflags, g->flags, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    if (st == PG_OK && (hflags & PG_FLAG_NONFINITE)) st = PG_ERR_NONFINITE;
    if (st == PG_OK && hflags) st = PG_ERR_INVALID_ARG;
    if (st == PG_OK) {
        g->n_active = h_nact;
        if (cudaMemsetAsync(g->b + n, 0, 4, s) != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK) {
        switch (wdtype) {
            case PG_W_F32: st = launch_agg_k<float>(g, c, D, d_cnt, s); break;
            case PG_W_BF16: st = launch_agg_k<__nv_bfloat16>(g, c, D, d_cnt, s); break;
            case PG_W_F16: st = launch_agg_k<__half>(g, c, D, d_cnt, s); break;
            case PG_W_U16: st = launch_agg_k<pg_unorm16>(g, c, D, d_cnt, s); break;
        }
    }
    unsigned long long h_cnt = 0;
    if (st == PG_OK && (cudaMemcpyAsync(&h_cnt, d_cnt, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    if (predcnt) cudaFreeAsync(predcnt, s);
    if (rec_tmp) cudaFreeAsync(rec_tmp, s);
    if (act) cudaFreeAsync(act, s);
    if (d_nact) cudaFreeAsync(d_nact, s);
    if (d_cnt) cudaFreeAsync(d_cnt, s);
    if (st != PG_OK) {
        (void)cudaGetLastError();
        return st;
    }
    g->nnz_swept = (int64_t)h_cnt;
    g->aggregated = 1;
    return PG_OK;
}
