// Internal definitions shared by the libpg translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pg.h"

#define PG_QBITS 21
#define PG_QMASK ((1u << PG_QBITS) - 1u)
#define PG_MAX_K 32

// Bit flags raised by validation kernels (read back at synchronising calls).
enum : int {
    PG_FLAG_NONFINITE = 1,
    PG_FLAG_BAD_INDEX = 2,
    PG_FLAG_TWO_PREDS = 4,
    PG_FLAG_BAD_RANGE = 8,
};

// Transposed weights by column (sweep row of the column's vertex), entries
// sorted by source row: ptr[n_active + 1] (64-bit: a large graph holds more
// than 2^31 entries), ent[nnz] = (source row, weight bits).
struct pg_tcsr {
    int64_t *ptr = nullptr;
    int2 *ent = nullptr;
    int64_t nnz = 0; // entries allocated (the live ones are [ptr[0], ptr[ncols]))
};

struct pg_graph {
    int64_t n = 0;
    int32_t k = 0;
    int32_t kp = 0;        // stored row width: 4, 8, 16 or 32
    int32_t level = 0;     // hash-grid level L: 2^L cells per axis
    float lo[3] = {0, 0, 0};
    float scale = 0;       // 2^21 / max extent, float32
    int64_t r2_max = -1;
    cudaStream_t stream = nullptr; // stream of the most recent call (frees go here)
    int64_t bytes = 0;

    // ---- graph build (Morton order m) ----
    int32_t *m2c = nullptr;        // m -> caller index
    int32_t *c2m = nullptr;        // caller -> m
    uint64_t *qpos = nullptr;      // quantised position qx | qy << 21 | qz << 42, m order
    int2 *cell_se = nullptr;       // (start, count) per cell, index x + G (y + G z)
    int32_t *nbr = nullptr;        // [n][kp], m-space neighbour ids, -1 padded; slot 0 = self
    int64_t knn_exact = 0;         // queries resolved by the exact neighbour kernel
    int64_t clusters = 0;          // cluster mode: number of parts (neighbourhoods)

    // ---- aggregation ----
    int aggregated = 0;
    pg_wdtype wdtype = PG_W_F32;
    int64_t n_active = 0;          // rows with a predecessor: sweep rows [0, n_active)
    int64_t nnz_swept = 0;
    int32_t *m2r = nullptr;        // m -> sweep row r
    int32_t *r2m = nullptr;        // r -> m
    float4 *OG = nullptr;          // (o, g)           m order
    float4 *DP = nullptr;          // (d, pe_ph)       m order
    float4 *EP = nullptr;          // (e, pe_e or -1 for a delta light) m order
    float4 *LV = nullptr;          // (Le, Lph, sigma_s, w_prop) m order
    int32_t *succ_m = nullptr;     // m-space successor or -1
    void *W = nullptr;             // [n][kp] weights (tau/p_t)_s * A+_{s,j}, sweep-row order
    float *rscale = nullptr;       // [n] per-row scale (16-bit weights)
    int32_t *col = nullptr;        // [n][kp] sweep-row index of succ(j); n = zero slot
    float *b = nullptr;            // [n] (tau/p_t)_s * c_s, sweep-row order
    unsigned long long *pmd = nullptr; // [n] marginal pm_d of sample m over the rows that use it (fixed point)
    unsigned long long *pme = nullptr; // [n] the same for the emitter sample e_m
    uint32_t *kin = nullptr;       // [n] number of rows that use sample m, |R(m)|
    float *c_m = nullptr;          // [n] c_s, m order
    float *D_m = nullptr;          // [n] D_s, m order

    // ---- propagation ----
    float *ybuf[2] = {nullptr, nullptr}; // (n+1) floats each; [n] stays 0
    float *hist = nullptr;               // (hist_iters+1) x (n+1), sweep-row order
    int32_t hist_iters = -1;
    int32_t hist_cap = -1;
    double *d_resid = nullptr;           // residual per sweep
    int32_t resid_cap = 0;
    int32_t *d_ctrl = nullptr;           // [0] iters_done, [1] stop flag, [2] block counter
    double *d_partials = nullptr;        // per-block residual partials
    int32_t partials_cap = 0;

    // ---- adjoint (lazily built) ----
    pg_tcsr tA;                   // transpose of the active rows [0, n_active)
    pg_tcsr tF;                   // transpose of the first-vertex rows [n_active, n)
    int32_t *flags = nullptr;     // validation flags (device)
};

// ------------------------------------------------------------------ helpers
#define PG_TRY(expr)                                   \
    do {                                               \
        pg_status _s = (expr);                         \
        if (_s != PG_OK) return _s;                    \
    } while (0)

#define PG_CUDA(expr)                                  \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) {                       \
            (void)cudaGetLastError();                  \
            return _e == cudaErrorMemoryAllocation ? PG_ERR_OOM : PG_ERR_CUDA; \
        }                                              \
    } while (0)

#define PG_LAUNCH_CHECK() PG_CUDA(cudaGetLastError())

static inline int pg_blocks(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)(b < 1 ? 1 : b);
}

pg_status pg_alloc(pg_graph *g, void **p, size_t bytes, cudaStream_t s);
void pg_free(pg_graph *g, void **p, size_t bytes);
int pg_num_sms();
void pg_count_launches(int k); // diagnostic count of kernel launches

// Stable LSD radix sort of (key, value) pairs by key bits [0, nbits).
pg_status pg_radix_sort(pg_graph *g, uint32_t *keys, int32_t *vals, int64_t n, int nbits, cudaStream_t s);
// Exclusive prefix sum of n int32 counts (in place); total written to *d_total if non-NULL.
pg_status pg_scan_exclusive(pg_graph *g, int32_t *data, int64_t n, int32_t *d_total, cudaStream_t s);
// 64-bit offsets (totals past 2^31, e.g. the transposed weights of 150M+ vertices)
pg_status pg_scan_exclusive64(pg_graph *g, int64_t *data, int64_t n, int64_t *d_total, cudaStream_t s);

// ------------------------------------------------------------------ device math
// 1 + a.b for unit vectors, with the rounding errors of the three products
// and two sums carried along (error-free transformations: TwoProduct by FMA,
// TwoSum by Knuth's six-operation form). Near the forward peak of a
// phase function 1 + a.b is tiny and a plain float32 dot product would lose
// most of its digits. Explicit _rn intrinsics keep the compiler from fusing
// the sums into FMAs, which would break the error-free transformations.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
__device__ __forceinline__ float one_plus_dot(float ax, float ay, float az, float bx, float by, float bz) {
    float p = __fmul_rn(ax, bx);
    float err = __fmaf_rn(ax, bx, -p);
    float h = __fmul_rn(ay, by);
    float f = __fmaf_rn(ay, by, -h);
    float s, q;
    two_sum(p, h, s, q);
    err = __fadd_rn(err, __fadd_rn(f, q));
    h = __fmul_rn(az, bz);
    f = __fmaf_rn(az, bz, -h);
    two_sum(s, h, p, q);
    err = __fadd_rn(err, __fadd_rn(f, q));
    two_sum(1.0f, p, s, q);
    return __fadd_rn(s, __fadd_rn(q, err));
}
// |v|^2 - 1 of a (nearly) unit vector, accurate to a few ulps of the result
// (error-free products and sums; evaluated once per vector)
__device__ __forceinline__ float unit_err(float x, float y, float z) {
    const float p1 = __fmul_rn(x, x), p2 = __fmul_rn(y, y), p3 = __fmul_rn(z, z);
    const float e1 = __fmaf_rn(x, x, -p1), e2 = __fmaf_rn(y, y, -p2), e3 = __fmaf_rn(z, z, -p3);
    float s1, q1, s2, q2;
    two_sum(p1, p2, s1, q1);
    two_sum(s1, p3, s2, q2);
    const float s3 = __fsub_rn(s2, 1.0f); // exact: s2 is close to 1
    return __fadd_rn(s3, __fadd_rn(__fadd_rn(q1, q2), __fadd_rn(e1, __fadd_rn(e2, e3))));
}
// 1 + a.b from the vectors and their unit_err: 1 + a.b = (|a+b|^2 - ea - eb) / 2.
// Near the forward peak a ~ -b, |a+b| is small and computed to full relative
// precision, so this is as accurate as one_plus_dot at a third of the cost.
__device__ __forceinline__ float one_plus_dot_u(float ax, float ay, float az, float ea, float bx, float by, float bz,
                                                float eb) {
    const float sx = ax + bx, sy = ay + by, sz = az + bz;
    const float s2 = fmaf(sz, sz, fmaf(sy, sy, sx * sx));
    return 0.5f * (s2 - (ea + eb));
}

// rsqrt refined by one Newton step (the hardware estimate alone is ~2 ulp)
__device__ __forceinline__ float rsqrt_nr(float x) {
    float r = rsqrtf(x);
    return r * fmaf(-0.5f * x, r * r, 1.5f);
}

// Henyey-Greenstein rho(o, d) with mu = -o.d, written as
//   (1-g^2)/(4 pi) * den^(-3/2),  den = (1-g)^2 + 2 g (1 + o.d)
// (equal to 1 + g^2 - 2 g mu). hgc holds (C = (1-g^2)/(4 pi), (1-g)^2, 2g)
// for the strategy; opd is 1 + o.d from one_plus_dot.
struct HGc {
    float C, a, b2;
};
__device__ __forceinline__ HGc hg_consts(float g) {
    const float inv4pi = 0.0795774715459476679f;
    HGc h;
    h.C = (1.0f - g * g) * inv4pi;
    float omg = 1.0f - g;
    h.a = omg * omg;
    h.b2 = 2.0f * g;
    return h;
}
__device__ __forceinline__ float hg_eval(const HGc &h, float opd) {
    float den = fmaf(h.b2, opd, h.a);
    float r = rsqrt_nr(den);
    return h.C * (r * r * r);
}
// d rho / d g = -2g/(4 pi) den^-3/2 - 3 (1-g^2)/(4 pi) (g + o.d) den^-5/2
__device__ __forceinline__ float hg_eval_dg(float g, float opd, float *rho_out) {
    const float inv4pi = 0.0795774715459476679f;
    float omg = 1.0f - g;
    float den = fmaf(2.0f * g, opd, omg * omg);
    float r = rsqrt_nr(den);
    float r3 = r * r * r;
    float C = (1.0f - g * g) * inv4pi;
    *rho_out = C * r3;
    return -2.0f * g * inv4pi * r3 - 3.0f * C * ((g - 1.0f) + opd) * (r3 * r * r);
}

// quantised position packed as qx | qy << 21 | qz << 42
__device__ __forceinline__ int3 pg_qpos_unpack(uint64_t c) {
    return make_int3((int32_t)(c & PG_QMASK), (int32_t)((c >> 21) & PG_QMASK), (int32_t)(c >> 42));
}

__device__ __forceinline__ uint32_t part1by2(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return part1by2(x) | (part1by2(y) << 1) | (part1by2(z) << 2);
}

// ------------------------------------------------------------------ edge-weight storage
// The sweep matrix stores W~ = (tau/p_t)_s A+_{s,j} as FP32, or per row as an
// FP32 scale times a 16-bit payload: BF16 and FP16 hold each weight relative
// to the row's largest one (payload w / max, scale max); U16 holds it as
// 16-bit unsigned fixed point, q = round(65535 w / max), scale max / 65535
// (the weights are non-negative and the scale carries the range, so all 16
// bits resolve the weight: absolute error at most max / 131070). Every
// reader forms weight = dec(payload) * scale.
struct pg_unorm16 {
    uint16_t q;
};

// exact float value of a 16-bit unsigned field of x: its bits placed in the
// mantissa of 2^23 (one byte permute), minus 2^23
__device__ __forceinline__ float u16_lo(uint32_t x) {
    return __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7410)) - 8388608.0f;
}
__device__ __forceinline__ float u16_hi(uint32_t x) {
    return __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7432)) - 8388608.0f;
}

template <typename T>
struct WTraits;
template <>
struct WTraits<float> {
    static constexpr pg_wdtype id = PG_W_F32;
    __device__ static float enc(float w, float) { return w; }
    __device__ static float scale(float) { return 1.0f; }
    __device__ static float dec(float w) { return w; }
    __device__ static int32_t bits(float w) { return __float_as_int(w); }
    __device__ static float from_bits(int32_t b) { return __int_as_float(b); }
    // four consecutive weights, streamed (evict-first)
    __device__ static float4 load4(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
    // the same as raw bits, decoded later (fewer registers held across the gathers)
    using raw4 = float4;
    __device__ static raw4 load4_raw(const float *p) { return load4(p); }
    __device__ static float4 dec4(raw4 r) { return r; }
};
template <>
struct WTraits<__nv_bfloat16> {
    static constexpr pg_wdtype id = PG_W_BF16;
    __device__ static __nv_bfloat16 enc(float w, float mx) { return __float2bfloat16_rn(w / mx); }
    __device__ static float scale(float mx) { return mx; }
    __device__ static float dec(__nv_bfloat16 w) { return __bfloat162float(w); }
    __device__ static int32_t bits(__nv_bfloat16 w) { return (int32_t)__bfloat16_as_ushort(w); }
    __device__ static float from_bits(int32_t b) { return __bfloat162float(__ushort_as_bfloat16((unsigned short)b)); }
    __device__ static float4 load4(const __nv_bfloat16 *p) { return dec4(load4_raw(p)); }
    using raw4 = uint2;
    __device__ static raw4 load4_raw(const __nv_bfloat16 *p) { return __ldcs(reinterpret_cast<const uint2 *>(p)); }
    __device__ static float4 dec4(uint2 u) {
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <>
struct WTraits<__half> {
    static constexpr pg_wdtype id = PG_W_F16;
    __device__ static __half enc(float w, float mx) { return __float2half_rn(w / mx); }
    __device__ static float scale(float mx) { return mx; }
    __device__ static float dec(__half w) { return __half2float(w); }
    __device__ static int32_t bits(__half w) { return (int32_t)__half_as_ushort(w); }
    __device__ static float from_bits(int32_t b) { return __half2float(__ushort_as_half((unsigned short)b)); }
    __device__ static float4 load4(const __half *p) { return dec4(load4_raw(p)); }
    using raw4 = uint2;
    __device__ static raw4 load4_raw(const __half *p) { return __ldcs(reinterpret_cast<const uint2 *>(p)); }
    __device__ static float4 dec4(uint2 u) {
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <>
struct WTraits<pg_unorm16> {
    static constexpr pg_wdtype id = PG_W_U16;
    __device__ static pg_unorm16 enc(float w, float mx) {
        pg_unorm16 r;
        r.q = (uint16_t)__float2uint_rn(fminf(w / mx, 1.0f) * 65535.0f);
        return r;
    }
    __device__ static float scale(float mx) { return mx / 65535.0f; }
    __device__ static float dec(pg_unorm16 w) { return u16_lo(w.q); }
    __device__ static int32_t bits(pg_unorm16 w) { return (int32_t)w.q; }
    __device__ static float from_bits(int32_t b) { return u16_lo((uint32_t)b); }
    __device__ static float4 load4(const pg_unorm16 *p) { return dec4(load4_raw(p)); }
    using raw4 = uint2;
    __device__ static raw4 load4_raw(const pg_unorm16 *p) { return __ldcs(reinterpret_cast<const uint2 *>(p)); }
    __device__ static float4 dec4(uint2 u) { return make_float4(u16_lo(u.x), u16_hi(u.x), u16_lo(u.y), u16_hi(u.y)); }
};

template <typename T>
struct pg_type_tag {
    using type = T;
};
// f(pg_type_tag<WT>{}) for the storage type of weight format t
template <typename F>
static pg_status pg_dispatch_w(pg_wdtype t, F &&f) {
    switch (t) {
        case PG_W_F32: return f(pg_type_tag<float>{});
        case PG_W_BF16: return f(pg_type_tag<__nv_bfloat16>{});
        case PG_W_F16: return f(pg_type_tag<__half>{});
        case PG_W_U16: return f(pg_type_tag<pg_unorm16>{});
    }
    return PG_ERR_UNSUPPORTED;
}

// Sample marginals are summed as unsigned 64-bit fixed point with 34
// fraction bits: integer additions are exact, so the sums (and every weight
// formed from them) do not depend on the order the atomics land in. A term is
// a float phase-function value rounded to a multiple of 2^-34 (absolute error
// at most 2^-35, below 1e-5 relative for any |g| <= 0.999); sums stay below
// 2^30 (2^64 / 2^34) for any realistic number of rows per sample.
#define PG_PM_FRAC_BITS 34
__device__ __forceinline__ unsigned long long pg_pm_fix(float x) {
    return __float2ull_rn(x * 17179869184.0f); // x * 2^34, exact scaling
}
__device__ __forceinline__ float pg_pm_float(unsigned long long a) {
    return __ull2float_rn(a) * 5.820766091346740722656e-11f; // rounded to float, then * 2^-34 (exact)
}

static inline size_t pg_wbytes(pg_wdtype t) { return t == PG_W_F32 ? 4 : 2; }
// stored row width for k entries: 4, 8, 16 or 32 (128-bit aligned rows)
static inline int pg_row_width(int k) { return k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32; }

// Launchers implemented in the per-stage translation units.
pg_status pg_launch_knn(pg_graph *g, cudaStream_t s);
// exact k nearest vertices (self first) of nq query points qm[t] (Morton
// index or -1) among all the graph's vertices, no radius limit: out row t
// (row width pg_row_width(k), Morton ids, -1 padded; all -1 for qm[t] < 0)
pg_status pg_launch_knn_queries(const pg_graph *g, const int32_t *qm, int64_t nq, int k, int32_t *out,
                                cudaStream_t s);
// cluster neighbourhoods (keys: the vertices' sorted Morton cell keys)
pg_status pg_launch_clusters(pg_graph *g, const uint32_t *keys, int32_t K, uint64_t seed, cudaStream_t s);
void pg_free_transposes(pg_graph *g); // releases both transposes (weights changed)
// whether the sweeps deal their rows / columns to the blocks in round-robin
// tiles (a window of the Morton order at a time) rather than in chunks
bool pg_sweep_front(int64_t n_active);
pg_status pg_launch_aggregate(pg_graph *g, float *c_out, float *D_out, cudaStream_t s);
// one propagation sweep over the rows [0, view->n_active) of a graph view:
// yout[r] = sum_i W[r][i] yin[col[r][i]] (* rscale[r]) + b[r]
pg_status pg_launch_sweep(const pg_graph *view, const float *b, const float *yin, float *yout, int32_t *ctrl,
                          double2 *partials, double *resid, int t, double tol, cudaStream_t s);
// grid size of one sweep launch (residual partials needed per sweep)
int pg_sweep_blocks(const pg_graph *g);
