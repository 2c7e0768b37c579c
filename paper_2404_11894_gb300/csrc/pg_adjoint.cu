// Adjoint of aggregation -> propagation -> output for a fixed graph.
//
// The forward pass in sweep rows r (see pg_aggregate.cu) is
//   y_t[r] = sum_i W~[r][i] y_{t-1}[col[r][i]] + b[r],  t = 1..T, r active,
//   val_p  = bg_p + sum_i W~[f][i] y_T[col[f][i]] + (tau/p_t)_f D_f
// with W~ = (tau/p_t)_s A+ (times the row scale for 16-bit weights) and
// b = (tau/p_t)_s c_s. For dLoss/dImage = dI, each path's first vertex f gets
// nu_f = dI[pixel]/spp, and the reverse sweeps are
//   mu_T = W~^T nu,   mu_{t-1} = W~^T mu_t   (t = T..2).
// Every weight of row s is sigma_s(s) times a factor, so
//   dLoss/dsigma_s(s) = ( sum_t mu_t[s] y_t[s] + nu_s (val_s - bg) ) / sigma_s(s).
// For g the per-edge adjoints Gamma[s][i] = sum_t mu_t[s] y_{t-1}[col] (+ the
// output term nu_s y_T[col]) are formed from the kept iterates y_t and the
// reverse iterates mu_t, and with beta_s = sum_t mu_t[s] pushed through the
// derivatives of the MIS weights (numerators and marginal densities).
//
// W~^T is applied either from a transposed copy of the stored weights
// (columns sorted by row: deterministic), or, with recompute_weights, by
// re-evaluating each row's weights from the vertex records and scattering
// with atomic adds (no weight memory).
#include "pg_internal.cuh"

__global__ void scale_rows_kernel(const float *__restrict__ mu, const float *__restrict__ rs, int64_t na,
                                  float *__restrict__ us) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < na) us[r] = mu[r] * rs[r];
}

// ------------------------------------------------------------------ transpose build
__global__ void tcount_kernel(const int32_t *__restrict__ col, int64_t r0, int64_t r1, int kp, int64_t ncols,
                              int64_t *__restrict__ cnt) {
    int64_t e = r0 * kp + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= r1 * kp) return;
    int32_t c = col[e];
    if (c < ncols) atomicAdd(reinterpret_cast<unsigned long long *>(cnt + c), 1ull);
}

// Four entries of one row per thread: their column offsets, slot atomics and
// scattered writes are independent, so a thread keeps four of these chains
// in flight instead of waiting on one (the pass is bound by their latency).
template <typename WT>
__global__ void tfill_kernel(const int32_t *__restrict__ col, const WT *__restrict__ W, int64_t r0, int64_t r1,
                             int kp, int64_t ncols, const int64_t *__restrict__ tptr, int32_t *__restrict__ fill,
                             int2 *__restrict__ tent) {
    const int64_t q = r0 * (kp / 4) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; // kp is a power of two >= 4
    if (q >= r1 * (kp / 4)) return;
    const int4 c4 = reinterpret_cast<const int4 *>(col)[q];
    const int32_t c[4] = {c4.x, c4.y, c4.z, c4.w};
    const int64_t e = 4 * q;
    const int32_t row = (int32_t)(e >> (__ffs(kp) - 1));
    int64_t at[4];
    int32_t wb[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        at[i] = c[i] < ncols ? tptr[c[i]] : 0;
        wb[i] = WTraits<WT>::bits(W[e + i]);
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
        if (c[i] < ncols) at[i] += atomicAdd(&fill[c[i]], 1);
#pragma unroll
    for (int i = 0; i < 4; i++)
        if (c[i] < ncols) tent[at[i]] = make_int2(row, wb[i]);
}

// The active rows' column lengths from the aggregation's counts: sample j's
// column is the sweep row of its successor, and |R(j)| counts every row that
// uses j, so the active rows' share is |R(j)| less the first-vertex rows'
// count of the same column (already in cntF, before rounding).
__global__ void tcount_active_kernel(const uint32_t *__restrict__ kin, const int32_t *__restrict__ succ_m,
                                     const int32_t *__restrict__ m2r, int64_t n, int64_t ncols,
                                     const int64_t *__restrict__ cntF, int64_t *__restrict__ cntA) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t sj = succ_m[j];
    if (sj < 0) return;
    const int32_t c = m2r[sj];
    if (c >= ncols) return;
    cntA[c] = (int64_t)kin[j] - cntF[c];
}

// Column lengths rounded up to even, so that every column starts on a
// 16-byte boundary and the reverse sweep loads its entries in pairs.
__global__ void tround_kernel(int64_t *__restrict__ cnt, int64_t ncols) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncols) cnt[c] = (cnt[c] + 1) & ~(int64_t)1;
}

// Batcher's odd-even merge sort by the row key: 191 compare-exchanges for
// 32 entries against a bitonic network's 240 (2 % less transpose build).
// The comparator pairs are listed at compile time so that the unrolled
// network indexes registers only.
template <int N>
struct OddEvenNet {
    static constexpr int count() {
        int c = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k; i++)
                        if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) c++;
        return c;
    }
    static constexpr int C = count();
    int a[C], b[C];
    constexpr OddEvenNet() : a(), b() {
        int c = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k; i++)
                        if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                            a[c] = i + j;
                            b[c] = i + j + k;
                            c++;
                        }
    }
};
template <int N>
__device__ __forceinline__ void oddeven_rows(int2 (&kv)[N]) {
    constexpr OddEvenNet<N> net;
#pragma unroll
    for (int c = 0; c < OddEvenNet<N>::C; c++) {
        const int x = net.a[c], y = net.b[c];
        if (kv[x].x > kv[y].x) {
            const int2 t = kv[x];
            kv[x] = kv[y];
            kv[y] = t;
        }
    }
}

// A column starts at an even entry (lengths are rounded up to even), so its
// entries move in 16-byte pairs; an odd column's last pair ends in its pad
// entry, which is read as a sentinel and not written back.
template <int N>
__device__ __forceinline__ void sort_column(int2 *__restrict__ tent, int64_t a, int32_t len) {
    int2 kv[N];
    const int4 *src = reinterpret_cast<const int4 *>(tent + a);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        int4 u = make_int4(INT32_MAX, 0, INT32_MAX, 0);
        if (i < len) u = src[i / 2];
        kv[i] = make_int2(u.x, u.y);
        kv[i + 1] = i + 1 < len ? make_int2(u.z, u.w) : make_int2(INT32_MAX, 0);
    }
    oddeven_rows<N>(kv);
    int4 *dst = reinterpret_cast<int4 *>(tent + a);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        if (i + 1 < len)
            dst[i / 2] = make_int4(kv[i].x, kv[i].y, kv[i + 1].x, kv[i + 1].y);
        else if (i < len)
            tent[a + i] = kv[i];
    }
}

// Order each column's entries by source row (a row appears once per column),
// which makes the reverse sweep's summation order deterministic, and write
// the column's pad entry (source row pad_row < 0, skipped by the sweep) when
// its length was rounded up. Columns of up to 32 entries (all of them for
// k <= 16 in practice) are sorted in registers by one 32-entry sorting
// network (a 16-entry one for the shorter columns made nearly every warp
// run both, as 30 % of a kNN graph's columns hold more than 16); longer
// ones by insertion sort in memory.
__global__ void __launch_bounds__(128) tsort_kernel(const int64_t *__restrict__ tptr,
                                                    const int32_t *__restrict__ fill, int64_t ncols,
                                                    int32_t pad_row, int2 *__restrict__ tent) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int64_t a = tptr[c];
    const int32_t len = fill[c];
    if (a + len < tptr[c + 1]) tent[a + len] = make_int2(pad_row, 0);
    if (len <= 1) return;
    if (len <= 32) {
        sort_column<32>(tent, a, len);
        return;
    }
    for (int64_t i = a + 1; i < a + len; i++) {
        const int2 v = tent[i];
        int64_t j = i - 1;
        while (j >= a && tent[j].x > v.x) {
            tent[j + 1] = tent[j];
            j--;
        }
        tent[j + 1] = v;
    }
}

// ------------------------------------------------------------------ seeds
// nu on first-vertex rows; us = nu * row scale (what W^T multiplies)
__global__ void seed_kernel(const int32_t *__restrict__ first, const float *__restrict__ dI, int64_t n_paths,
                            int spp, int64_t n, const int32_t *__restrict__ c2m, const int32_t *__restrict__ m2r,
                            const float *__restrict__ rscale, float *__restrict__ nu, float *__restrict__ us) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_paths) return;
    int32_t f = first[p];
    if (f < 0 || f >= n) return;
    int32_t r = m2r[c2m[f]];
    float v = dI[p / spp] / (float)spp;
    nu[r] = v; // a vertex starts at most one path
    us[r] = rscale ? v * rscale[r] : v;
}

// ------------------------------------------------------------------ reverse sweep (stored transpose)
// Four lanes per column c: mu_out[c] = sum_e tW[e] us_in[trow[e]] over the
// column's entries (rows ascending), two entries per 16-byte load, each block
// walking its columns in order (neighbouring columns draw on neighbouring
// rows). When y_t is given it also accumulates
// G[c] += mu_in[c] y_t[c] (and B[c] += mu_in[c] when B is given); those
// column scalars are loaded up front, one per lane, so they travel with the
// entry loads. us_out (the next input, mu times the 16-bit row scale) is
// written only when it differs from mu_out.
static constexpr int TS_THREADS = 256;

// The sweep is software-pipelined: the first pass of entries
// (2 LPC PAIRS of them) of the next column group is loaded before this
// group's gathers, with the column extents two groups ahead, so a column's
// DRAM round trip overlaps the previous one's L2 round trip. Longer columns
// take their remaining passes unpipelined.
// Column schedules as in the forward sweep: contiguous chunks per block, or
// (FRONT) tiles of TS_TILE_GROUPS column groups dealt round-robin to the
// blocks, so all blocks work in one window of the column order and the
// gathered reverse iterates of that window stay in L2.
static constexpr int TS_TILE_GROUPS = 64;

template <typename WT, int NT, int MINB, bool FRONT, int LPC, int PAIRS>
__global__ void __launch_bounds__(NT, MINB) tsweep_pf_kernel(
    const int64_t *__restrict__ tptr, const int2 *__restrict__ tent,
    const float *__restrict__ us_in, const float *__restrict__ mu_in, const float *__restrict__ y_t,
    const float *__restrict__ rscale, int64_t ncols, int write_out, float *__restrict__ mu_out,
    float *__restrict__ us_out, float *__restrict__ G, float *__restrict__ B) {
    static_assert(LPC == 2 || LPC == 4, "two or four lanes per column");
    constexpr int CPB = NT / LPC;
    const int lane = threadIdx.x & 31;
    const int q = lane & (LPC - 1);
    const int lead = lane & ~(LPC - 1);
    const bool acc_g = y_t != nullptr;
    const int64_t chunk = ((ncols + gridDim.x - 1) / gridDim.x + CPB - 1) / CPB * CPB;
    const int64_t c0 = FRONT ? 0 : (int64_t)blockIdx.x * chunk;
    const int64_t c1 = FRONT ? ncols : min(ncols, c0 + chunk);
    auto gbase = [&](int64_t k) -> int64_t {
        if (!FRONT) return c0 + k * CPB;
        const int64_t tile = k / TS_TILE_GROUPS;
        return (tile * gridDim.x + blockIdx.x) * ((int64_t)CPB * TS_TILE_GROUPS) + (k - tile * TS_TILE_GROUPS) * CPB;
    };
    const int cl = threadIdx.x / LPC;
    auto extent = [&](int64_t c, int64_t &a, int64_t &b) {
        a = b = 0;
        if (write_out && c < c1) {
            a = tptr[c];
            b = tptr[c + 1];
        }
    };
    auto first_pass = [&](int64_t a, int64_t b, int4 (&ent)[PAIRS]) {
#pragma unroll
        for (int u = 0; u < PAIRS; u++) {
            const int64_t e = a + 2 * q + 2 * LPC * u;
            ent[u] = e < b ? __ldcs(reinterpret_cast<const int4 *>(tent + e)) : make_int4(-1, 0, -1, 0);
        }
    };
    int64_t a1, b1, a2, b2; // extents of the next group and the one after
    int4 en[PAIRS];         // first pass of the next group
    {
        int64_t a0, b0;
        extent(gbase(0) + cl, a0, b0);
        first_pass(a0, b0, en);
        extent(gbase(1) + cl, a1, b1);
        // the current group's extent travels with its entries
        a2 = a0;
        b2 = b0;
    }
    for (int64_t k = 0, base = gbase(0); base < c1; base = gbase(++k)) {
        const int64_t c = base + cl;
        const bool ok = c < c1;
        const int64_t ca = a2, cb = b2; // this group's extent
        int4 ent[PAIRS];
#pragma unroll
        for (int u = 0; u < PAIRS; u++) ent[u] = en[u];
        // next group's first pass, and the extent of the group after it
        first_pass(a1, b1, en);
        a2 = a1;
        b2 = b1;
        extent(gbase(k + 2) + cl, a1, b1);
        // column scalars: four lanes hold mu_in, y_t, G, B; two lanes hold
        // (mu_in, G) and (y_t, B)
        float sv = 0.0f, sv2 = 0.0f, rs = 1.0f;
        if (ok && acc_g) {
            if (q == 0) sv = mu_in[c];
            else if (q == 1) sv = __ldcs(y_t + c);
            else if (q == 2) sv = G[c];
            else if (B) sv = B[c];
            if constexpr (LPC == 2) {
                if (q == 0) sv2 = G[c];
                else if (B) sv2 = B[c];
            }
        }
        if (ok && rscale && write_out && q == 0) rs = __ldcs(rscale + c);
        float acc = 0.0f;
        if (ok && write_out) {
#pragma unroll
            for (int u = 0; u < PAIRS; u++) {
                if (ent[u].x >= 0) acc = fmaf(WTraits<WT>::from_bits(ent[u].y), __ldg(us_in + ent[u].x), acc);
                if (ent[u].z >= 0) acc = fmaf(WTraits<WT>::from_bits(ent[u].w), __ldg(us_in + ent[u].z), acc);
            }
            for (int64_t a = ca + 2 * LPC * PAIRS; a < cb; a += 2 * LPC * PAIRS) {
                int4 more[PAIRS];
                first_pass(a, cb, more);
#pragma unroll
                for (int u = 0; u < PAIRS; u++) {
                    if (more[u].x >= 0) acc = fmaf(WTraits<WT>::from_bits(more[u].y), __ldg(us_in + more[u].x), acc);
                    if (more[u].z >= 0) acc = fmaf(WTraits<WT>::from_bits(more[u].w), __ldg(us_in + more[u].z), acc);
                }
            }
        }
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const float m = __shfl_sync(0xffffffffu, sv, lead);
        const float yv = __shfl_sync(0xffffffffu, sv, lead + 1);
        if (ok) {
            if (q == 0 && write_out) {
                mu_out[c] = acc;
                if (us_out) us_out[c] = acc * rs;
            }
            if (acc_g) {
                if constexpr (LPC == 4) {
                    if (q == 2) G[c] = fmaf(m, yv, sv);
                    if (q == 3 && B) B[c] = sv + m;
                } else {
                    if (q == 0) G[c] = fmaf(m, yv, sv2);
                    if (q == 1 && B) B[c] = sv2 + m;
                }
            }
        }
    }
}

// output term of first-vertex rows: G[f] = nu_f (val_f - bg) with
// val_f - bg = sum_i W~[f][i] y_T[col] + (tau/p_t)_f D_f
template <typename WT>
__global__ void first_rows_kernel(const int32_t *__restrict__ first, int64_t n_paths, int64_t n,
                                  const int32_t *__restrict__ c2m, const int32_t *__restrict__ m2r,
                                  const int32_t *__restrict__ col, const WT *__restrict__ W,
                                  const float *__restrict__ rscale, const float *__restrict__ yT,
                                  const float4 *__restrict__ LV, const float *__restrict__ D_m,
                                  const float *__restrict__ nu, int kp, float *__restrict__ G) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_paths) return;
    int32_t f = first[p];
    if (f < 0 || f >= n) return;
    int32_t m = c2m[f];
    int64_t r = m2r[m];
    float sum = 0.0f;
    for (int i = 0; i < kp; i++) sum = fmaf(WTraits<WT>::dec(W[r * kp + i]), yT[col[r * kp + i]], sum);
    if (rscale) sum *= rscale[r];
    G[r] += nu[r] * (sum + LV[m].w * D_m[m]);
}

// ------------------------------------------------------------------ reverse sweep (stored rows, scatter)
// Rows [r0, r1) in the forward layout: out[col[r][i]] += W[r][i] * us_in[r]
// with float atomics (no transposed copy), KP/4 lanes per row and 16-byte
// loads like the forward sweep. Accumulates G[r] += mu_in[r] y_t[r] and
// B[r] += mu_in[r] when y_t is given.
template <int KP, typename WT>
__global__ void __launch_bounds__(256) scatter_sweep_kernel(
    const int32_t *__restrict__ col, const WT *__restrict__ W, int64_t r0, int64_t r1, int64_t n,
    const float *__restrict__ us_in, const float *__restrict__ mu_in, const float *__restrict__ y_t, int write_out,
    float *__restrict__ out, float *__restrict__ G, float *__restrict__ B) {
    constexpr int LPR = KP / 4;
    const int lane = threadIdx.x & 31;
    const int q = lane & (LPR - 1);
    const int64_t row = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    if (row >= r1) return;
    const float u = us_in[row];
    if (write_out && u != 0.0f) {
        const int4 c4 = __ldcs(reinterpret_cast<const int4 *>(col + row * KP) + q);
        const float4 w4 = WTraits<WT>::load4(W + row * KP + q * 4);
        if (c4.x < n) atomicAdd(out + c4.x, w4.x * u);
        if (c4.y < n) atomicAdd(out + c4.y, w4.y * u);
        if (c4.z < n) atomicAdd(out + c4.z, w4.z * u);
        if (c4.w < n) atomicAdd(out + c4.w, w4.w * u);
    }
    if (y_t && q == 0) {
        const float m = mu_in[row];
        G[row] = fmaf(m, y_t[row], G[row]);
        if (B) B[row] += m;
    }
}

// ------------------------------------------------------------------ recompute mode
// Row s (Morton m) re-evaluates its weights W~[s][j] = w_s sigma_s rho_s(o_s,d_j)
// / pm_d[j] from the vertex records and the stored sample marginals, and
// scatters u[r] W~ into out[col] with atomics. Also accumulates G/B (y_t
// given) for the rows.
__device__ __forceinline__ float recompute_weight(const float4 &os, const float4 &dp, float w_s, float sig_s,
                                                  float pm_d) {
    const HGc hs = hg_consts(os.w);
    const float rho = hg_eval(hs, one_plus_dot_u(os.x, os.y, os.z, unit_err(os.x, os.y, os.z), dp.x, dp.y, dp.z,
                                                  unit_err(dp.x, dp.y, dp.z)));
    return w_s * (sig_s * rho / pm_d);
}

template <int KP>
__global__ void __launch_bounds__(256) recompute_scatter_kernel(
    const int32_t *__restrict__ nbr, const float4 *__restrict__ OG, const float4 *__restrict__ DP,
    const float4 *__restrict__ LV, const int32_t *__restrict__ succ_m, const unsigned long long *__restrict__ pmd,
    const int32_t *__restrict__ m2r, const int32_t *__restrict__ r2m, int64_t r0, int64_t r1,
    const float *__restrict__ u, const float *__restrict__ y_t, int write_out, float *__restrict__ out,
    float *__restrict__ G, float *__restrict__ B) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (KP - 1);
    const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / KP;
    if (r >= r1) return; // whole groups leave together (r is uniform over a group)
    const int32_t m = r2m[r];
    const float ur = u[r];
    if (write_out && ur != 0.0f) {
        const int32_t nj = nbr[(int64_t)m * KP + j];
        if (nj >= 0) {
            const int32_t sj = succ_m[nj];
            if (sj >= 0) {
                const float4 lvs = LV[m];
                const float Wt = recompute_weight(OG[m], DP[nj], lvs.w, lvs.z, pg_pm_float(pmd[nj]));
                atomicAdd(out + m2r[sj], ur * Wt);
            }
        }
    }
    if (j == 0 && y_t) {
        G[r] = fmaf(ur, y_t[r], G[r]);
        if (B) B[r] += ur;
    }
}

// first-vertex rows in recompute mode: G[f] = nu_f (val_f - bg)
template <int KP>
__global__ void __launch_bounds__(256) recompute_first_kernel(
    const int32_t *__restrict__ nbr, const float4 *__restrict__ OG, const float4 *__restrict__ DP,
    const float4 *__restrict__ LV, const int32_t *__restrict__ succ_m, const unsigned long long *__restrict__ pmd,
    const int32_t *__restrict__ m2r, const int32_t *__restrict__ r2m, int64_t r0, int64_t r1,
    const float *__restrict__ nu, const float *__restrict__ yT, const float *__restrict__ D_m,
    float *__restrict__ G) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (KP - 1);
    const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / KP;
    const bool row_ok = r < r1;
    const int32_t m = row_ok ? r2m[r] : 0;
    const int32_t nj = row_ok ? nbr[(int64_t)m * KP + j] : -1;
    const float4 lvs = row_ok ? LV[m] : make_float4(0.f, 0.f, 0.f, 0.f);
    float term = 0.0f;
    if (nj >= 0) {
        const int32_t sj = succ_m[nj];
        if (sj >= 0) term = recompute_weight(OG[m], DP[nj], lvs.w, lvs.z, pg_pm_float(pmd[nj])) * yT[m2r[sj]];
    }
#pragma unroll
    for (int o = KP / 2; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
    if (row_ok && j == 0) G[r] += nu[r] * (term + lvs.w * D_m[m]);
}

// ------------------------------------------------------------------ outputs
__global__ void grad_sigma_kernel(const float *__restrict__ G, const int32_t *__restrict__ c2m,
                                  const int32_t *__restrict__ m2r, const float4 *__restrict__ LV, int64_t n,
                                  float *__restrict__ gs_out, const int32_t *__restrict__ voxel,
                                  const float *__restrict__ sigma_t, float *__restrict__ ga, int64_t n_vox) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t m = c2m[v];
    float ss = LV[m].z;
    float gsv = ss > 0.0f ? G[m2r[m]] / ss : 0.0f;
    if (gs_out) gs_out[v] = gsv;
    if (ga) {
        int32_t x = voxel[v];
        if (x >= 0 && x < n_vox) atomicAdd(ga + x, sigma_t[v] * gsv);
    }
}

// d/dg through the aggregation, given the edge adjoints Gamma (dLoss/dW~),
// beta (dLoss/db) and nu (dLoss/d(w D)). Per entry (s, j), j in N(s):
//   A_sj = sig_s rho_s(d_j)/pm_d[j], Ae_sj = sig_s rho_s(e_j)/me[j] (delta:
//   /|N(s)|), Aph_sj = sig_s rho_s(d_j)/mph[j], me = pm_e + K_j pe_e,
//   mph = pm_d + K_j pe_ph, and pm_d[j] = sum over the rows r using j of
//   rho_r(o_r, d_j) (pm_e likewise), so g_s enters row s's numerators and the
//   marginals of every sample s uses. Pass 1 forms each entry's numerator
//   factors and adds its share of dLoss/dpm_d[j], dLoss/dpm_e[j] (atomics);
//   pass 2 takes drho_s/dg_s times (numerator factor + marginal adjoint) over
//   the row's entries, plus the non-aggregated direct term.
template <int KP>
__global__ void __launch_bounds__(256) grad_g_marg_kernel(
    const int32_t *__restrict__ nbr, const float4 *__restrict__ OG, const float4 *__restrict__ DP,
    const float4 *__restrict__ EP, const float4 *__restrict__ LV, const int32_t *__restrict__ m2r, int64_t n,
    int64_t n_active, const int32_t *__restrict__ col, const float *__restrict__ yhist,
    const float *__restrict__ muhist, int T, const float *__restrict__ B, const float *__restrict__ nu,
    const unsigned long long *__restrict__ pmd, const unsigned long long *__restrict__ pme,
    const uint32_t *__restrict__ kin, float *__restrict__ gpm_d, float *__restrict__ gpm_e,
    float2 *__restrict__ num) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (KP - 1);
    const int src = lane & ~(KP - 1);
    const int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / KP;
    const bool row_ok = m < n;
    const int32_t nj = row_ok ? nbr[m * KP + j] : -1;
    const bool valid = nj >= 0;
    const unsigned gmask = (KP == 32) ? 0xffffffffu : (((1u << KP) - 1u) << src);
    const float Ks = (float)__popc(__ballot_sync(0xffffffffu, valid) & gmask);
    const float4 lvs = row_ok ? LV[m] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (!valid) {
        if (row_ok) num[m * KP + j] = make_float2(0.f, 0.f);
        return;
    }
    const float4 os = OG[m], dp = DP[nj], ep = EP[nj], lv = LV[nj];
    const float sig = lvs.z, w_s = lvs.w;
    const int64_t r = m2r[m];
    // edge adjoint Gamma = dLoss/dW~ of this entry: sum over the sweeps that
    // used it (mu_t of the row times the iterate it multiplied), or the output
    // term nu y_T for a path's first vertex
    float Gam = 0.0f;
    const int32_t cl = col[r * KP + j];
    const int64_t stride = n + 1;
    if (r < n_active) {
        for (int t = 1; t <= T; t++) Gam = fmaf(muhist[t * stride + r], yhist[(t - 1) * stride + cl], Gam);
    } else {
        Gam = nu[r] * yhist[(int64_t)T * stride + cl];
    }
    const float gA = w_s * Gam;      // dLoss/dA+ of this entry
    const float gc = w_s * B[r];     // dLoss/dc of the row
    const HGc hs = hg_consts(os.w);
    const float es = unit_err(os.x, os.y, os.z);
    const float rho_sd = hg_eval(hs, one_plus_dot_u(os.x, os.y, os.z, es, dp.x, dp.y, dp.z, unit_err(dp.x, dp.y, dp.z)));
    const float rho_se = hg_eval(hs, one_plus_dot_u(os.x, os.y, os.z, es, ep.x, ep.y, ep.z, unit_err(ep.x, ep.y, ep.z)));
    const float pm_d = pg_pm_float(pmd[nj]), pm_e = pg_pm_float(pme[nj]), kj = (float)kin[nj];
    const bool delta = ep.w < 0.0f;
    const float me = fmaf(kj, ep.w, pm_e), mph = fmaf(kj, dp.w, pm_d);
    const float cd = -sig * rho_sd * (gA / (pm_d * pm_d) + gc * lv.y / (mph * mph));
    const float ce = delta ? 0.0f : -sig * rho_se * gc * lv.x / (me * me);
    if (cd != 0.0f) atomicAdd(gpm_d + nj, cd);
    if (ce != 0.0f) atomicAdd(gpm_e + nj, ce);
    const float nd = sig * (gA / pm_d + gc * lv.y / mph);
    const float ne = sig * gc * lv.x / (delta ? Ks : me);
    num[m * KP + j] = make_float2(nd, ne);
}

template <int KP>
__global__ void __launch_bounds__(256) grad_g_kernel(
    const int32_t *__restrict__ nbr, const float4 *__restrict__ OG, const float4 *__restrict__ DP,
    const float4 *__restrict__ EP, const float4 *__restrict__ LV, const int32_t *__restrict__ m2r, int64_t n,
    const float *__restrict__ nu, const float *__restrict__ gpm_d, const float *__restrict__ gpm_e,
    const float2 *__restrict__ num, float *__restrict__ gg) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (KP - 1);
    const int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / KP;
    const bool row_ok = m < n;
    const int32_t nj = row_ok ? nbr[m * KP + j] : -1;
    float acc = 0.0f;
    if (nj >= 0) {
        const float4 os = OG[m], dp = DP[nj], ep = EP[nj];
        const float es = unit_err(os.x, os.y, os.z);
        float rho_sd, rho_se;
        const float drho_sd =
            hg_eval_dg(os.w, one_plus_dot_u(os.x, os.y, os.z, es, dp.x, dp.y, dp.z, unit_err(dp.x, dp.y, dp.z)), &rho_sd);
        const float drho_se =
            hg_eval_dg(os.w, one_plus_dot_u(os.x, os.y, os.z, es, ep.x, ep.y, ep.z, unit_err(ep.x, ep.y, ep.z)), &rho_se);
        const float2 nde = num[m * KP + j];
        acc = drho_sd * (nde.x + gpm_d[nj]) + drho_se * (nde.y + gpm_e[nj]);
        if (j == 0) {
            // D_s = sigma_s (De + Dp) with K = 1, own samples (slot 0 = s)
            const float4 lv = LV[m];
            const float gD = lv.w * nu[m2r[m]];
            const bool delta = ep.w < 0.0f;
            const float dDe = delta ? drho_se * lv.x : drho_se * lv.x * ep.w / ((rho_se + ep.w) * (rho_se + ep.w));
            const float dDp = drho_sd * lv.y * dp.w / ((rho_sd + dp.w) * (rho_sd + dp.w));
            acc += gD * lv.z * (dDe + dDp);
        }
    }
#pragma unroll
    for (int o = KP / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (row_ok && j == 0) gg[m] = acc;
}

__global__ void permute_m2c_kernel(const float *__restrict__ in_m, const int32_t *__restrict__ c2m, int64_t n,
                                   float *__restrict__ out_c) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    out_c[v] = in_m[c2m[v]];
}

// ------------------------------------------------------------------ host
// Two transposes of the stored weights: the active rows' (applied in every
// reverse sweep) and the first-vertex rows' (applied once, to the output
// adjoint nu), so the reverse sweeps never stream the first rows' entries.
template <typename WT>
static pg_status build_transpose(pg_graph *g, cudaStream_t s) {
    const int64_t n = g->n, na = g->n_active;
    const int kp = g->kp;
    pg_tcsr *ts[2] = {&g->tA, &g->tF};
    const int64_t r0[2] = {0, na}, r1[2] = {na, n};
    int32_t *fill = nullptr;
    int64_t *d_total = nullptr;
    pg_status st = PG_OK;
    for (int i = 0; i < 2 && st == PG_OK; i++) st = pg_alloc(g, (void **)&ts[i]->ptr, 8 * (size_t)(na + 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&fill, 4 * (size_t)(na + 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&d_total, 16, s);
    if (st != PG_OK) {
        if (fill) cudaFreeAsync(fill, s);
        return st;
    }
    // Column lengths: the first-vertex rows' by counting their entries, the
    // active rows' (nine in ten entries) from |R(j)| less those.
    for (int i = 0; i < 2; i++) PG_CUDA(cudaMemsetAsync(ts[i]->ptr, 0, 8 * (size_t)(na + 1), s));
    if (n > na) {
        tcount_kernel<<<pg_blocks((n - na) * kp, 256), 256, 0, s>>>(g->col, na, n, kp, na, g->tF.ptr);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
    }
    if (na > 0) {
        tcount_active_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(g->kin, g->succ_m, g->m2r, n, na, g->tF.ptr,
                                                                g->tA.ptr);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
    }
    for (int i = 0; i < 2; i++) {
        if (r1[i] > r0[i]) {
            tround_kernel<<<pg_blocks(na, 256), 256, 0, s>>>(ts[i]->ptr, na);
            pg_count_launches(1);
            PG_LAUNCH_CHECK();
        }
        PG_TRY(pg_scan_exclusive64(g, ts[i]->ptr, na + 1, d_total + i, s));
    }
    // No host round trip for the totals: each transpose gets room for every
    // entry its rows can hold plus one pad per column (at most 1 + 1/k of the
    // live entries), so the build can be queued behind other work.
    for (int i = 0; i < 2; i++) {
        ts[i]->nnz = (r1[i] - r0[i]) * kp + na + 1;
        PG_TRY(pg_alloc(g, (void **)&ts[i]->ent, 8 * (size_t)ts[i]->nnz, s));
        if (r1[i] == r0[i]) continue;
        PG_CUDA(cudaMemsetAsync(fill, 0, 4 * (size_t)(na + 1), s));
        tfill_kernel<WT><<<pg_blocks((r1[i] - r0[i]) * (kp / 4), 256), 256, 0, s>>>(
            g->col, (const WT *)g->W, r0[i], r1[i], kp, na, ts[i]->ptr, fill, ts[i]->ent);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
        tsort_kernel<<<pg_blocks(na, 128), 128, 0, s>>>(ts[i]->ptr, fill, na, -1, ts[i]->ent);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
    }
    cudaFreeAsync(fill, s);
    cudaFreeAsync(d_total, s);
    return PG_OK;
}

void pg_free_transposes(pg_graph *g) {
    for (pg_tcsr *t : {&g->tA, &g->tF}) {
        pg_free(g, (void **)&t->ent, 8 * (size_t)t->nnz);
        pg_free(g, (void **)&t->ptr, 8 * (size_t)(g->n_active + 1));
        t->nnz = 0;
    }
}

template <typename WT>
static pg_status adjoint_store(pg_graph *g, float *us0, float *mu_a, float *mu_b, float *us_a, float *us_b,
                               float *G, float *B, float *muhist, cudaStream_t s) {
    const int64_t n = g->n, na = g->n_active;
    const int T = g->hist_iters;
    const int64_t stride = n + 1;
    const float *rs = g->wdtype == PG_W_F32 ? nullptr : g->rscale;
    if (!g->tA.ptr) PG_TRY(build_transpose<WT>(g, s));
    // four lanes per column with a first pass of 24 entries (8 more than the
    // typical column of k = 16, so only ~0.2 % of the columns of a kNN graph
    // take a second pass, and fewer registers than a 32-entry pass: 15 %
    // faster on the 151 M-column dense medium, 2 % on the cloud),
    // software-pipelined (next group's first pass in flight during this
    // group's gathers); at most 64 registers, 4 blocks of 256 per SM
    // round-robin tiles: four 256-thread blocks per SM; contiguous chunks: one
    // 1024-thread block per SM, so each SM's L1 serves one chunk of columns
    // (3 % faster on the cloud, 1 % slower in tiles on the dense medium)
    const bool front = pg_sweep_front(na);
    const int nt = front ? TS_THREADS : 1024;
    int64_t need = (na * 4 + nt - 1) / nt;
    int64_t cap = (int64_t)pg_num_sms() * (front ? 4 : 1);
    const int tb = (int)(need < cap ? (need > 0 ? need : 1) : cap);
    auto tsweep = [&](const pg_tcsr &t, const float *us_in, const float *mu_in, const float *y_t, int wo,
                      float *mu_out, float *us_out) {
        if (front)
            tsweep_pf_kernel<WT, TS_THREADS, 4, true, 4, 3><<<tb, TS_THREADS, 0, s>>>(
                t.ptr, t.ent, us_in, mu_in, y_t, rs, na, wo, mu_out, us_out, G, B);
        else
            tsweep_pf_kernel<WT, 1024, 1, false, 4, 3><<<tb, 1024, 0, s>>>(t.ptr, t.ent, us_in, mu_in, y_t, rs, na, wo,
                                                                         mu_out, us_out, G, B);
    };
    // mu_t lives in slice t of the history when one is kept, else ping-pong
    auto mu_slot = [&](int t) { return muhist ? muhist + (int64_t)t * stride : ((t & 1) ? mu_b : mu_a); };
    // with FP32 weights us = mu, so the reverse iterate itself is the next input
    float *us_cur = rs ? us_a : mu_slot(T), *us_nxt = us_b;
    // mu_T = W^T nu (nu lives on the first-vertex rows)
    tsweep(g->tF, us0, nullptr, nullptr, 1, mu_slot(T), rs ? us_cur : nullptr);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    for (int t = T; t >= 1; t--) {
        const float *y_t = g->hist + (int64_t)t * stride;
        float *out_us = rs ? us_nxt : nullptr;
        tsweep(g->tA, us_cur, mu_slot(t), y_t, t > 1 ? 1 : 0, mu_slot(t - 1), out_us);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
        if (rs) {
            float *tu = us_cur;
            us_cur = us_nxt;
            us_nxt = tu;
        } else {
            us_cur = mu_slot(t - 1);
        }
    }
    return PG_OK;
}

template <int KP, typename WT>
static pg_status adjoint_scatter(pg_graph *g, float *us0, float *mu_a, float *mu_b, float *us_a, float *us_b,
                                 float *G, float *B, float *muhist, cudaStream_t s) {
    const int64_t n = g->n, na = g->n_active;
    const int T = g->hist_iters;
    const int64_t stride = n + 1;
    const float *rs = g->wdtype == PG_W_F32 ? nullptr : g->rscale;
    auto mu_slot = [&](int t) { return muhist ? muhist + (int64_t)t * stride : ((t & 1) ? mu_b : mu_a); };
    // mu_T = W^T nu: scatter from the first-vertex rows [na, n)
    PG_CUDA(cudaMemsetAsync(mu_slot(T), 0, 4 * (size_t)stride, s));
    scatter_sweep_kernel<KP, WT><<<pg_blocks((n - na) * (KP / 4), 256), 256, 0, s>>>(
        g->col, (const WT *)g->W, na, n, n, us0, nullptr, nullptr, 1, mu_slot(T), G, B);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    float *us_cur = us_a;
    for (int t = T; t >= 1; t--) {
        // us = mu_t * row scale (the 16-bit payload multiplies it)
        const float *mu_t = mu_slot(t);
        const float *us_in = mu_t;
        if (rs) {
            scale_rows_kernel<<<pg_blocks(na, 256), 256, 0, s>>>(mu_t, rs, na, us_cur);
            pg_count_launches(1);
            us_in = us_cur;
        }
        if (t > 1) PG_CUDA(cudaMemsetAsync(mu_slot(t - 1), 0, 4 * (size_t)stride, s));
        scatter_sweep_kernel<KP, WT><<<pg_blocks(na * (KP / 4), 256), 256, 0, s>>>(
            g->col, (const WT *)g->W, 0, na, n, us_in, mu_t, g->hist + (int64_t)t * stride, t > 1 ? 1 : 0,
            mu_slot(t - 1), G, B);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
    }
    (void)us_b;
    return PG_OK;
}

template <typename WT>
static pg_status adjoint_scatter_k(pg_graph *g, float *us0, float *mu_a, float *mu_b, float *us_a, float *us_b,
                                   float *G, float *B, float *muhist, cudaStream_t s) {
    switch (g->kp) {
        case 4: return adjoint_scatter<4, WT>(g, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, s);
        case 8: return adjoint_scatter<8, WT>(g, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, s);
        case 16: return adjoint_scatter<16, WT>(g, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, s);
        case 32: return adjoint_scatter<32, WT>(g, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, s);
        default: return PG_ERR_UNSUPPORTED;
    }
}

template <int KP>
static pg_status adjoint_recompute(pg_graph *g, float *nu, float *mu_a, float *mu_b, float *G, float *B,
                                   float *muhist, cudaStream_t s) {
    const int64_t n = g->n, na = g->n_active;
    const int T = g->hist_iters;
    const int64_t stride = n + 1;
    auto mu_slot = [&](int t) { return muhist ? muhist + (int64_t)t * stride : ((t & 1) ? mu_b : mu_a); };
    // mu_T = W^T nu from the first-vertex rows [na, n)
    PG_CUDA(cudaMemsetAsync(mu_slot(T), 0, 4 * (size_t)(n + 1), s));
    const float *yT = g->hist + (int64_t)T * stride;
    recompute_scatter_kernel<KP><<<pg_blocks((n - na) * KP, 256), 256, 0, s>>>(
        g->nbr, g->OG, g->DP, g->LV, g->succ_m, g->pmd, g->m2r, g->r2m, na, n, nu, nullptr, 1, mu_slot(T), G, B);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    for (int t = T; t >= 1; t--) {
        if (t > 1) PG_CUDA(cudaMemsetAsync(mu_slot(t - 1), 0, 4 * (size_t)(n + 1), s));
        const float *y_t = g->hist + (int64_t)t * stride;
        recompute_scatter_kernel<KP><<<pg_blocks(na * KP, 256), 256, 0, s>>>(
            g->nbr, g->OG, g->DP, g->LV, g->succ_m, g->pmd, g->m2r, g->r2m, 0, na, mu_slot(t), y_t, t > 1 ? 1 : 0,
            mu_slot(t - 1), G, B);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
    }
    // output term of first-vertex rows
    recompute_first_kernel<KP><<<pg_blocks((n - na) * KP, 256), 256, 0, s>>>(
        g->nbr, g->OG, g->DP, g->LV, g->succ_m, g->pmd, g->m2r, g->r2m, na, n, nu, yT, g->D_m, G);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

template <int KP>
static pg_status launch_grad_g(pg_graph *g, const float *muhist, const float *B, const float *nu, float *gg_m,
                               cudaStream_t s) {
    const int64_t n = g->n;
    float *gpm = nullptr;
    float2 *num = nullptr;
    PG_TRY(pg_alloc(nullptr, (void **)&gpm, 8 * (size_t)n, s));
    pg_status st = pg_alloc(nullptr, (void **)&num, 8 * (size_t)n * KP, s);
    if (st == PG_OK && cudaMemsetAsync(gpm, 0, 8 * (size_t)n, s) != cudaSuccess) st = PG_ERR_CUDA;
    if (st == PG_OK) {
        grad_g_marg_kernel<KP><<<pg_blocks(n * KP, 256), 256, 0, s>>>(
            g->nbr, g->OG, g->DP, g->EP, g->LV, g->m2r, n, g->n_active, g->col, g->hist, muhist, g->hist_iters, B,
            nu, g->pmd, g->pme, g->kin, gpm, gpm + n, num);
        grad_g_kernel<KP><<<pg_blocks(n * KP, 256), 256, 0, s>>>(g->nbr, g->OG, g->DP, g->EP, g->LV, g->m2r, n, nu,
                                                                 gpm, gpm + n, num, gg_m);
        pg_count_launches(2);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (gpm) cudaFreeAsync(gpm, s);
    if (num) cudaFreeAsync(num, s);
    return st;
}

extern "C" pg_status pg_prepare_adjoint(pg_graph *g, pg_stream_t stream) {
    if (!g) return PG_ERR_INVALID_ARG;
    if (!g->aggregated || !g->W) return PG_ERR_STATE;
    if (g->tA.ptr || g->n == 0) return PG_OK; // built for the current weights, or nothing to build
    cudaStream_t s = (cudaStream_t)stream;
    return pg_dispatch_w(g->wdtype, [&](auto tag) { return build_transpose<typename decltype(tag)::type>(g, s); });
}

extern "C" pg_status pg_propagate_adjoint(pg_graph *g, const float *dI, const int32_t *first, int64_t n_paths,
                                          int32_t spp, int32_t width, int32_t height, float *grad_sigma_s,
                                          float *grad_g, const int32_t *voxel, const float *sigma_t,
                                          float *grad_albedo_vox, int64_t n_vox, int32_t recompute_weights,
                                          pg_stream_t stream) {
    if (!g || spp <= 0 || width < 0 || height < 0) return PG_ERR_INVALID_ARG;
    if (n_paths != (int64_t)width * height * spp) return PG_ERR_INVALID_ARG;
    if (!g->aggregated || g->hist_iters < 0 || !g->hist) return PG_ERR_STATE;
    if (recompute_weights < 0 || recompute_weights > 2) return PG_ERR_INVALID_ARG;
    if (recompute_weights != 1 && !g->W) return PG_ERR_STATE;
    if (grad_albedo_vox && (!voxel || !sigma_t || n_vox < 0)) return PG_ERR_INVALID_ARG;
    if (n_paths > 0 && (!dI || !first)) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    const int64_t n = g->n;
    if (grad_albedo_vox && n_vox > 0) PG_CUDA(cudaMemsetAsync(grad_albedo_vox, 0, 4 * (size_t)n_vox, s));
    if (n == 0) return PG_OK;
    const bool want_g = grad_g != nullptr;
    float *nu = nullptr, *us0 = nullptr, *mu_a = nullptr, *mu_b = nullptr, *us_a = nullptr, *us_b = nullptr;
    float *G = nullptr, *B = nullptr, *muhist = nullptr, *gg_m = nullptr;
    const size_t vb = 4 * (size_t)(n + 1);
    pg_status st = PG_OK;
#define T_ALLOC(p, bytes) \
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&(p), (bytes), s)
    T_ALLOC(nu, vb);
    T_ALLOC(us0, vb);
    T_ALLOC(mu_a, vb);
    T_ALLOC(mu_b, vb);
    T_ALLOC(us_a, vb);
    T_ALLOC(us_b, vb);
    T_ALLOC(G, vb);
    if (want_g) {
        T_ALLOC(B, vb); // sum of the reverse iterates: only the g gradient uses it
        T_ALLOC(muhist, vb * (size_t)(g->hist_iters + 1)); // mu_t per reverse sweep
        T_ALLOC(gg_m, vb);
    }
#undef T_ALLOC
    if (st == PG_OK) {
        cudaMemsetAsync(nu, 0, vb, s);
        cudaMemsetAsync(us0, 0, vb, s);
        cudaMemsetAsync(G, 0, vb, s);
        if (B) cudaMemsetAsync(B, 0, vb, s);
        cudaMemsetAsync(mu_a, 0, vb, s);
        cudaMemsetAsync(mu_b, 0, vb, s);
        cudaMemsetAsync(us_a, 0, vb, s); // rows past n_active must read as zero
        cudaMemsetAsync(us_b, 0, vb, s);
        if (want_g) {
            cudaMemsetAsync(muhist, 0, vb * (size_t)(g->hist_iters + 1), s);
            cudaMemsetAsync(gg_m, 0, vb, s);
        }
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK && n_paths > 0) {
        const float *rs = g->wdtype == PG_W_F32 ? nullptr : g->rscale;
        seed_kernel<<<pg_blocks(n_paths, 256), 256, 0, s>>>(first, dI, n_paths, spp, n, g->c2m, g->m2r,
                                                             recompute_weights == 1 ? nullptr : rs, nu, us0);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK) {
        if (recompute_weights == 2) {
            st = pg_dispatch_w(g->wdtype, [&](auto tag) {
                return adjoint_scatter_k<typename decltype(tag)::type>(g, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, s);
            });
        } else if (recompute_weights) {
            switch (g->kp) {
                case 4: st = adjoint_recompute<4>(g, nu, mu_a, mu_b, G, B, muhist, s); break;
                case 8: st = adjoint_recompute<8>(g, nu, mu_a, mu_b, G, B, muhist, s); break;
                case 16: st = adjoint_recompute<16>(g, nu, mu_a, mu_b, G, B, muhist, s); break;
                case 32: st = adjoint_recompute<32>(g, nu, mu_a, mu_b, G, B, muhist, s); break;
                default: st = PG_ERR_UNSUPPORTED;
            }
        } else {
            st = pg_dispatch_w(g->wdtype, [&](auto tag) {
                return adjoint_store<typename decltype(tag)::type>(g, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, s);
            });
        }
        // output term of the first-vertex rows from the stored weights
        if (st == PG_OK && recompute_weights != 1 && n_paths > 0) {
            const float *rs = g->wdtype == PG_W_F32 ? nullptr : g->rscale;
            const float *yT = g->hist + (int64_t)g->hist_iters * (n + 1);
            st = pg_dispatch_w(g->wdtype, [&](auto tag) {
                using WT = typename decltype(tag)::type;
                first_rows_kernel<WT><<<pg_blocks(n_paths, 256), 256, 0, s>>>(
                    first, n_paths, n, g->c2m, g->m2r, g->col, (const WT *)g->W, rs, yT, g->LV, g->D_m, nu, g->kp, G);
                pg_count_launches(1);
                return PG_OK;
            });
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
    }
    if (st == PG_OK && (grad_sigma_s || grad_albedo_vox)) {
        grad_sigma_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(G, g->c2m, g->m2r, g->LV, n, grad_sigma_s, voxel, sigma_t,
                                                            grad_albedo_vox, n_vox);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK && want_g) {
        switch (g->kp) {
            case 4: st = launch_grad_g<4>(g, muhist, B, nu, gg_m, s); break;
            case 8: st = launch_grad_g<8>(g, muhist, B, nu, gg_m, s); break;
            case 16: st = launch_grad_g<16>(g, muhist, B, nu, gg_m, s); break;
            case 32: st = launch_grad_g<32>(g, muhist, B, nu, gg_m, s); break;
            default: st = PG_ERR_UNSUPPORTED;
        }
        if (st == PG_OK) {
            permute_m2c_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(gg_m, g->c2m, n, grad_g);
            pg_count_launches(1);
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
            }
    }
    float *bufs[] = {nu, us0, mu_a, mu_b, us_a, us_b, G, B, muhist, gg_m};
    for (float *p : bufs)
        if (p) cudaFreeAsync(p, s);
    return st;
}

extern "C" pg_status pg_graph_release_weights(pg_graph *g) {
    if (!g) return PG_ERR_INVALID_ARG;
    size_t wb = pg_wbytes(g->wdtype);
    pg_free(g, (void **)&g->W, wb * (size_t)g->n * (size_t)g->kp);
    pg_free_transposes(g);
    return PG_OK;
}
