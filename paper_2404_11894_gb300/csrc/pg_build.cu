// Graph build: neighbour edges E_N of the path graph (Section 3.1).
//
// Vertices are quantised to 21-bit integer coordinates, bucketed into a
// uniform grid of 2^L cells per axis whose cells are numbered in Morton
// order, and stably sorted by cell (so a cell is a contiguous range of the
// sorted "Morton order" m, and spatially close vertices are close in m). A
// table indexed by the cell's (x, y, z) gives each cell's (start, count).
// Each query then scans rings of cells around its own and keeps its k-1
// nearest others in registers, ordered by (squared integer distance, caller
// index), until the k-1-th distance is provably below any unscanned cell.
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <type_traits>

#include "pg_internal.cuh"

__global__ void quantize_kernel(const float *__restrict__ px, const float *__restrict__ py,
                                const float *__restrict__ pz, int64_t n, float lo0, float lo1, float lo2,
                                float scale, int level, uint32_t *__restrict__ cellkey, int32_t *__restrict__ idx,
                                uint64_t *__restrict__ qpos_c, int32_t *__restrict__ flags) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    float p[3] = {px[v], py[v], pz[v]};
    float lo[3] = {lo0, lo1, lo2};
    uint32_t q[3];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        finite &= isfinite(p[a]);
        // float32 round-to-nearest steps, never contracted into an FMA
        float t = __fmul_rn(__fsub_rn(p[a], lo[a]), scale);
        float f = floorf(t);
        int32_t qi;
        if (!(f > 0.0f)) qi = 0;                       // negative, zero or NaN
        else if (f >= (float)PG_QMASK) qi = (int32_t)PG_QMASK;
        else qi = (int32_t)f;
        q[a] = (uint32_t)qi;
    }
    if (!finite) atomicOr(flags, PG_FLAG_NONFINITE);
    int sh = PG_QBITS - level;
    cellkey[v] = morton3(q[0] >> sh, q[1] >> sh, q[2] >> sh);
    idx[v] = (int32_t)v;
    qpos_c[v] = (uint64_t)q[0] | ((uint64_t)q[1] << 21) | ((uint64_t)q[2] << 42);
}

__global__ void permute_build_kernel(const int32_t *__restrict__ m2c, const uint64_t *__restrict__ qpos_c, int64_t n,
                                     uint64_t *__restrict__ qpos, int32_t *__restrict__ c2m) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int32_t c = m2c[m];
    qpos[m] = qpos_c[c];
    c2m[c] = (int32_t)m;
}

// (start, count) of every cell, indexed x + G (y + G z), from the Morton-
// indexed exclusive prefix of the cell counts
__device__ __forceinline__ uint32_t compact1by2(uint32_t x) {
    x &= 0x09249249u;
    x = (x ^ (x >> 2)) & 0x030C30C3u;
    x = (x ^ (x >> 4)) & 0x0300F00Fu;
    x = (x ^ (x >> 8)) & 0x030000FFu;
    x = (x ^ (x >> 16)) & 0x000003FFu;
    return x;
}
__global__ void cell_table_kernel(const int32_t *__restrict__ cell_start, int64_t ncells, int level,
                                  int2 *__restrict__ cell_se) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    uint32_t x = compact1by2((uint32_t)c), y = compact1by2((uint32_t)c >> 1), z = compact1by2((uint32_t)c >> 2);
    int64_t lin = (int64_t)x + ((int64_t)y << level) + ((int64_t)z << (2 * level));
    int32_t a = cell_start[c];
    cell_se[lin] = make_int2(a, cell_start[c + 1] - a);
}

__global__ void cell_count_kernel(const uint32_t *__restrict__ sorted_keys, int64_t n, int32_t *__restrict__ counts) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    atomicAdd(&counts[sorted_keys[m]], 1);
}

// The 26 neighbours of a cell, packed (dx+1) | (dy+1) << 2 | (dz+1) << 4 and
// ordered by the number of non-zero offsets: faces, then edges, then corners.
__constant__ int c_ring1[26];
// the 98 cells of ring 2 (the shell of the 5x5x5 block), packed
// (dx + 2) | (dy + 2) << 3 | (dz + 2) << 6, nearest classes first (by the
// number of axes at distance 2, then the sum of |d|)
__constant__ int c_ring2[98];

static void ring1_table(int out[26]) {
    int n = 0;
    for (int cls = 1; cls <= 3; cls++)
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++)
                    if ((dx != 0) + (dy != 0) + (dz != 0) == cls) out[n++] = (dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4);
}

static void ring2_table(int out[98]) {
    int n = 0;
    for (int far = 1; far <= 3; far++)
        for (int sum = 2; sum <= 6; sum++)
            for (int dz = -2; dz <= 2; dz++)
                for (int dy = -2; dy <= 2; dy++)
                    for (int dx = -2; dx <= 2; dx++) {
                        const int f = (abs(dx) == 2) + (abs(dy) == 2) + (abs(dz) == 2);
                        if (f == far && abs(dx) + abs(dy) + abs(dz) == sum)
                            out[n++] = (dx + 2) | ((dy + 2) << 3) | ((dz + 2) << 6);
                    }
}

// (d2, id) lexicographic order
__device__ __forceinline__ bool knn_less(int64_t da, int32_t ia, int64_t db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

// A first-ring list entry is one 64-bit key (d2 << 31) | caller id, which
// orders like (d2, id) while d2 < KNN_SAT.
static constexpr uint64_t KNN_SAT = (1ull << 33) - 1;

// Marker in a queued query's saved list: no list was kept, the exact kernel
// starts from the query's own cell.
static constexpr uint64_t KNN_FRESH = UINT64_MAX - 1;

// First ring: one thread per query over its own cell and the 26 around it,
// with a threshold from the local density; queries that need more rings go
// to the exact kernel. With one thread per query and the candidates of a
// warp's queries met in step, some lane wanted an insertion into its sorted
// list at almost every candidate, so the warp ran the insertion network for
// nearly all of them (about 60 % of this kernel's time went to insertions).
// Here each query
//   1. reads the vertex counts N of its 27 cells from the cell table and
//      takes the radius that would hold k - 1 of them at uniform density,
//      r^2 = (81 cs^3 (k - 1) / (4 pi (N - 1)))^(2/3), times 1.5625 (1.25
//      in radius) as its threshold T (any T gives the same list; this one
//      buffers about 29 candidates per query on the cloud, and 0.2 % of the
//      queries fall outside 15..48; 1.2 in radius left 0.8 % with fewer
//      than 15 and was 0.6 % slower, 1.1 in radius 37 % slower),
//   2. scans the cells that have a point closer than T and appends the
//      candidates with d2 < T to a shared-memory buffer (no insertion),
//   3. inserts the buffered candidates into its sorted register list; the
//      lanes of a warp now insert together, about as often as the largest
//      buffer holds.
// With at least k - 1 candidates below T the list is the k - 1 smallest
// (d2, id) of the 27 cells, as inserting every candidate gives; a query with
// fewer (and T below its radius limit) or with an overflowing buffer is
// queued for the exact kernel, which starts from its own cell.
// D32: 32-bit squared distances (grid level >= 7: cells of at most 2^14
// units, so d2 < 3 * (2 cs)^2 <= 3 * 2^30 inside the block); otherwise
// 64-bit, and a buffered candidate at d2 >= 2^33 - 1 (whose key would
// saturate) sends the query to the exact kernel.
template <int KP>
constexpr int ke_threads() { return KP <= 16 ? 128 : 64; } // the buffer is 3 KP entries a thread

template <int KP, bool QUERY, bool D32>
__global__ void __launch_bounds__(ke_threads<KP>(), 4) knn_est_kernel(
    const uint64_t *__restrict__ qpos, const int32_t *__restrict__ m2c, const int2 *__restrict__ cell_se, int64_t n, int k, int level, int64_t r2_max,
    const int32_t *__restrict__ c2m, int32_t *__restrict__ nbr, int32_t *__restrict__ redo,
    int32_t *__restrict__ redo_count, uint64_t *__restrict__ redo_keys, int64_t redo_cap,
    const int32_t *__restrict__ qlist = nullptr) {
    constexpr int M = KP - 1;
    constexpr int CAP = 3 * KP;
    constexpr int NT = ke_threads<KP>();
    using DT = typename std::conditional<D32, uint32_t, uint64_t>::type;
    constexpr DT DT_MAX = (DT)~(DT)0;
    __shared__ int32_t buf[CAP][NT];
    const int tx = threadIdx.x;
    const int64_t t = (int64_t)blockIdx.x * NT + tx;
    if (t >= n) return; // no block-wide barrier below
    const int64_t m = QUERY ? (int64_t)qlist[t] : t;
    if (QUERY && m < 0) {
        for (int i = 0; i < KP; i++) nbr[t * KP + i] = -1;
        return;
    }
    const uint64_t qp = qpos[m];
    const int32_t qx = (int32_t)(qp & PG_QMASK), qy = (int32_t)((qp >> 21) & PG_QMASK), qz = (int32_t)(qp >> 42);
    const int sh = PG_QBITS - level;
    const int G = 1 << level;
    const DT cs = (DT)1 << sh;
    const int cx = qx >> sh, cy = qy >> sh, cz = qz >> sh;
    const int km1 = k - 1;
    const int pad = M - km1;
    DT glo[3], ghi[3];
    {
        const int32_t q3[3] = {qx, qy, qz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const DT o = (DT)q3[a] & (cs - 1);
            glo[a] = (o + 1) * (o + 1);
            ghi[a] = (cs - o) * (cs - o);
        }
    }
    uint64_t bk[M > 0 ? M : 1];
#pragma unroll
    for (int i = 0; i < M; i++) bk[i] = i < pad ? 0ull : UINT64_MAX;
    int found = 0;
    bool fresh = false;
    if (km1 > 0) {
        // 1. the threshold from the 27 cells' counts
        int64_t nb = 0;
        for (int ci = 0; ci < 27; ci++) {
            const int x = cx + ci % 3 - 1, y = cy + (ci / 3) % 3 - 1, z = cz + ci / 9 - 1;
            if (x < 0 || x >= G || y < 0 || y >= G || z < 0 || z >= G) continue;
            nb += cell_se[(int64_t)x + ((int64_t)y << level) + ((int64_t)z << (2 * level))].y;
        }
        DT T = DT_MAX;
        if (nb - 1 > km1) {
            const float c3 = (float)cs * (float)cs * (float)cs;
            const float r2 = cbrtf(81.0f * c3 * (float)km1 / (12.566370614359172f * (float)(nb - 1)));
            const float tf = 1.5625f * r2 * r2;
            if (tf < (D32 ? 3.3e9f : 1.0e19f)) T = (DT)tf;
        }
        // a radius limit caps the threshold; below the cap the list is exact
        // whatever the count
        bool capped = false;
        if (r2_max >= 0 && (uint64_t)T > (uint64_t)r2_max) {
            T = (DT)(r2_max + 1);
            capped = true;
        }
        if (T == DT_MAX) capped = true; // every candidate of the block is buffered
        // 2. buffer the candidates closer than T
        int cnt = 0;
        bool sat = false;
        for (int ci = 0; ci < 27; ci++) {
            int dx = 0, dy = 0, dz = 0;
            if (ci > 0) {
                const int o = c_ring1[ci - 1];
                dx = (o & 3) - 1;
                dy = ((o >> 2) & 3) - 1;
                dz = ((o >> 4) & 3) - 1;
            }
            const int x = cx + dx, y = cy + dy, z = cz + dz;
            if (x < 0 || x >= G || y < 0 || y >= G || z < 0 || z >= G) continue;
            if (ci > 0) {
                const DT lb = (dx < 0 ? glo[0] : (dx > 0 ? ghi[0] : (DT)0)) +
                              (dy < 0 ? glo[1] : (dy > 0 ? ghi[1] : (DT)0)) +
                              (dz < 0 ? glo[2] : (dz > 0 ? ghi[2] : (DT)0));
                if (lb >= T) continue; // no point of the cell is closer than T
            }
            const int2 se = cell_se[(int64_t)x + ((int64_t)y << level) + ((int64_t)z << (2 * level))];
            const int32_t p1 = se.x + se.y;
            auto visit = [&](int32_t p, uint64_t c) {
                if (p == m) return;
                const int32_t ex = (int32_t)(c & PG_QMASK) - qx, ey = (int32_t)((c >> 21) & PG_QMASK) - qy,
                              ez = (int32_t)(c >> 42) - qz;
                DT d2;
                if (D32) {
                    d2 = (DT)((uint32_t)(ex * ex) + (uint32_t)(ey * ey) + (uint32_t)(ez * ez));
                } else {
                    d2 = (DT)((int64_t)ex * ex + (int64_t)ey * ey + (int64_t)ez * ez);
                    sat |= d2 < T && (uint64_t)d2 >= KNN_SAT;
                }
                if (d2 >= T) return;
                if (cnt < CAP) buf[cnt][tx] = p;
                cnt++;
            };
            // two positions per 16-byte load
            int32_t p = se.x;
            if ((p & 1) && p < p1) {
                visit(p, qpos[p]);
                p++;
            }
            for (; p + 1 < p1; p += 2) {
                const ulonglong2 two = __ldg(reinterpret_cast<const ulonglong2 *>(qpos + p));
                visit(p, two.x);
                visit(p + 1, two.y);
            }
            if (p < p1) visit(p, qpos[p]);
        }
        // 3. select: the buffered candidates into the sorted list
        fresh = sat || cnt > CAP || (cnt < km1 && !capped);
        found = fresh ? 0 : cnt;
        for (int i = 0; i < found; i++) {
            const int32_t p = buf[i][tx];
            const uint64_t c = qpos[p];
            const int32_t ex = (int32_t)(c & PG_QMASK) - qx, ey = (int32_t)((c >> 21) & PG_QMASK) - qy,
                          ez = (int32_t)(c >> 42) - qz;
            const uint64_t d2 = D32 ? (uint64_t)((uint32_t)(ex * ex) + (uint32_t)(ey * ey) + (uint32_t)(ez * ez))
                                    : (uint64_t)((int64_t)ex * ex + (int64_t)ey * ey + (int64_t)ez * ez);
            const uint64_t key = (d2 << 31) | (uint64_t)(uint32_t)m2c[p]; // caller id breaks ties
#pragma unroll
            for (int j = M - 1; j > 0; --j) {
                const uint64_t prev = bk[j - 1];
                if (key < bk[j]) bk[j] = key < prev ? prev : key;
            }
            if (key < bk[0]) bk[0] = key;
        }
        // done iff the (k-1)-th entry is closer than anything outside the block
        int64_t bnd = INT64_MAX;
        {
            const int cc[3] = {cx, cy, cz};
            const int32_t q[3] = {qx, qy, qz};
#pragma unroll
            for (int a2 = 0; a2 < 3; a2++) {
                if (cc[a2] - 1 > 0) {
                    const int64_t dlo = (int64_t)q[a2] - (int64_t)(cc[a2] - 1) * (int64_t)cs + 1;
                    bnd = dlo < bnd ? dlo : bnd;
                }
                if (cc[a2] + 1 < G - 1) {
                    const int64_t dhi = (int64_t)(cc[a2] + 2) * (int64_t)cs - q[a2];
                    bnd = dhi < bnd ? dhi : bnd;
                }
            }
        }
        bool done = bnd == INT64_MAX; // whole grid scanned
        if (!done) {
            const int64_t bnd2 = bnd * bnd;
            const uint64_t worst = bk[M - 1];
            const int64_t worst_d = worst == UINT64_MAX ? INT64_MAX : (int64_t)(worst >> 31);
            done = (found >= km1 && worst_d < bnd2) || (r2_max >= 0 && bnd2 > r2_max);
        }
        // queue the query for the exact kernel; one counter atomic per
        // converged group of lanes, not one per query (a single hot address)
        const bool need = fresh || !done;
        const unsigned am = __activemask();
        const unsigned need_mask = __ballot_sync(am, need);
        if (need) {
            const int lane = tx & 31;
            const int leader = __ffs(need_mask) - 1;
            int32_t base = 0;
            if (lane == leader) base = atomicAdd(redo_count, __popc(need_mask));
            base = __shfl_sync(need_mask, base, leader);
            const int32_t slot = base + __popc(need_mask & ((1u << lane) - 1u));
            redo[slot] = (int32_t)t;
            // the list holds the true k-1 nearest of the 27 cells: the exact
            // kernel resumes from it at ring 2 (from ring 0 for a fresh query)
            if (slot < redo_cap) {
                if (fresh) {
                    redo_keys[(int64_t)slot * M] = KNN_FRESH;
                } else {
#pragma unroll
                    for (int i = 0; i < M; i++) redo_keys[(int64_t)slot * M + i] = bk[i];
                }
            }
            return;
        }
    }
    int32_t *row = nbr + t * KP;
    row[0] = (int32_t)m;
#pragma unroll
    for (int i = 0; i < M; i++) {
        const int pos = i - pad; // rank among the k-1 others
        if (pos >= 0) row[1 + pos] = bk[i] != UINT64_MAX ? c2m[(int32_t)(bk[i] & 0x7fffffffu)] : -1;
    }
    for (int pos = km1; pos < M; pos++) row[1 + pos] = -1;
}

// Exact path for queued queries, one warp per query: entries (int64 d2,
// caller id) compared lexicographically, held one per lane (lane i = slot i
// of the ascending list; lanes below `pad` hold a sentinel that precedes
// every entry, so the (k-1)-th real entry is always lane M-1). The lanes
// scan a ring's cells in parallel, one cell each, and every candidate that
// beats the current (k-1)-th entry is inserted by all lanes together: a lane
// whose entry is larger takes its left neighbour's entry, or the candidate
// where the neighbour's is smaller (the register list's insertion, spread
// over the warp). The few queries that get here need long ring scans; one
// thread per query left most lanes of a warp idle behind the longest one.
// QUERY = false: the build's redo list (*d_count entries), row m of nbr.
// QUERY = true without qlist: nq query points list[t] (Morton index, or -1
// for none), row t of nbr; with qlist: the first-ring kernel's queued query
// slots list[t] (*d_count entries), slot u asking for vertex qlist[u], row
// u of nbr. With saved_keys, query t resumes at ring 2 from the first-ring
// kernel's list (entry t of the queue).
template <int KP, bool QUERY>
__global__ void __launch_bounds__(128) knn_exact_kernel(const uint64_t *__restrict__ qpos,
                                                        const int32_t *__restrict__ m2c,
                                                        const int2 *__restrict__ cell_se,
                                                        const int32_t *__restrict__ c2m, const int32_t *__restrict__ list,
                                                        const int32_t *__restrict__ d_count, int64_t nq, int k,
                                                        int level, int64_t r2_max, int32_t *__restrict__ nbr,
                                                        const uint64_t *__restrict__ saved_keys, int64_t saved_cap,
                                                        const int32_t *__restrict__ qlist = nullptr) {
    constexpr int M = KP - 1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; // one query per warp
    if (t >= ((QUERY && !qlist) ? nq : (int64_t)*d_count)) return;        // uniform over the warp
    const int64_t slot = !QUERY ? (int64_t)list[t] : (qlist ? (int64_t)list[t] : t);
    const int64_t m = !QUERY ? slot : (qlist ? (int64_t)qlist[slot] : (int64_t)list[t]);
    int32_t *row = nbr + slot * KP;
    if (QUERY && m < 0) {
        if (lane < KP) row[lane] = -1;
        return;
    }
    const uint64_t qp = qpos[m];
    const int32_t qx = (int32_t)(qp & PG_QMASK), qy = (int32_t)((qp >> 21) & PG_QMASK), qz = (int32_t)(qp >> 42);
    const int sh = PG_QBITS - level;
    const int G = 1 << level;
    const int64_t cs = (int64_t)1 << sh;
    const int cx = qx >> sh, cy = qy >> sh, cz = qz >> sh;
    const int32_t q3o[3] = {qx & (int32_t)(cs - 1), qy & (int32_t)(cs - 1), qz & (int32_t)(cs - 1)};
    const int km1 = k - 1;
    const int pad = M - km1;
    int64_t bd = lane < pad ? (int64_t)-1 : INT64_MAX;
    int32_t bi = lane < pad ? -1 : INT32_MAX;
    int found = 0;
    int r_start = 0;
    if (saved_keys && t < saved_cap && saved_keys[t * M] != KNN_FRESH) {
        // resume from the first-ring kernel's list of rings 0 and 1
        bool real = false;
        if (lane >= pad && lane < M) {
            const uint64_t key = saved_keys[t * M + lane];
            if (key != UINT64_MAX) {
                bd = (int64_t)(key >> 31);
                bi = (int32_t)(key & 0x7fffffffu);
                real = true;
            }
        }
        found = __popc(__ballot_sync(FULL, real));
        r_start = 2;
    }
    int64_t worst_d = __shfl_sync(FULL, bd, M - 1);
    int32_t worst_i = __shfl_sync(FULL, bi, M - 1);

    if (km1 > 0) {
        for (int r = r_start;; r++) {
            // ring r: the shell of the (2r+1)^3 block of cells around the own
            // (ring 2, where most queued queries end, from a table: no
            // divisions, no interior cells)
            const int span = 2 * r + 1;
            const bool tab = r == 2;
            const int ncell = tab ? 98 : span * span * span;
            for (int c0 = 0; c0 < ncell; c0 += 32) {
                int32_t p = 0, p1 = 0; // this lane's cell
                const int ci = c0 + lane;
                if (ci < ncell) {
                    int dx, dy, dz;
                    if (tab) {
                        const int o = c_ring2[ci];
                        dx = (o & 7) - 2;
                        dy = ((o >> 3) & 7) - 2;
                        dz = ((o >> 6) & 7) - 2;
                    } else {
                        dx = ci % span - r;
                        dy = (ci / span) % span - r;
                        dz = ci / (span * span) - r;
                    }
                    const int x = cx + dx, y = cy + dy, z = cz + dz;
                    bool use = (tab || abs(dx) == r || abs(dy) == r || abs(dz) == r) && x >= 0 && x < G && y >= 0 &&
                               y < G && z >= 0 && z < G;
                    if (use && worst_d != INT64_MAX) {
                        // a cell whose nearest point is farther than the
                        // (k-1)-th entry cannot contribute
                        const int d3[3] = {dx, dy, dz};
                        int64_t lb = 0;
#pragma unroll
                        for (int a = 0; a < 3; a++) {
                            const int64_t o = q3o[a];
                            const int64_t gap = d3[a] < 0 ? o + 1 + (int64_t)(-d3[a] - 1) * cs
                                                          : (d3[a] > 0 ? cs - o + (int64_t)(d3[a] - 1) * cs : 0);
                            lb += gap * gap;
                        }
                        use = lb <= worst_d;
                    }
                    if (use) {
                        const int2 se = cell_se[(int64_t)x + ((int64_t)y << level) + ((int64_t)z << (2 * level))];
                        p = se.x;
                        p1 = se.x + se.y;
                    }
                }
                // the lanes walk their cells together, one candidate each per step
                while (__any_sync(FULL, p < p1)) {
                    int64_t d2 = INT64_MAX;
                    int32_t id = INT32_MAX;
                    bool cand = false;
                    if (p < p1) {
                        if (p != m) {
                            const uint64_t cq = qpos[p];
                            const int64_t ex = (int64_t)(cq & PG_QMASK) - qx, ey = (int64_t)((cq >> 21) & PG_QMASK) - qy,
                                          ez = (int64_t)(cq >> 42) - qz;
                            d2 = ex * ex + ey * ey + ez * ez;
                            cand = d2 <= worst_d && (r2_max < 0 || d2 <= r2_max);
                            if (cand) { // the caller id breaks ties
                                id = m2c[p];
                                cand = knn_less(d2, id, worst_d, worst_i);
                            }
                        }
                        p++;
                    }
                    unsigned ins = __ballot_sync(FULL, cand);
                    while (ins) {
                        const int src = __ffs(ins) - 1;
                        ins &= ins - 1;
                        const int64_t cd = __shfl_sync(FULL, d2, src);
                        const int32_t cid = __shfl_sync(FULL, id, src);
                        if (!knn_less(cd, cid, worst_d, worst_i)) continue; // the list moved on
                        const int64_t ud = __shfl_up_sync(FULL, bd, 1);
                        const int32_t ui = __shfl_up_sync(FULL, bi, 1);
                        if (lane < M && knn_less(cd, cid, bd, bi)) {
                            if (lane > 0 && knn_less(cd, cid, ud, ui)) {
                                bd = ud;
                                bi = ui;
                            } else {
                                bd = cd;
                                bi = cid;
                            }
                        }
                        found++;
                        worst_d = __shfl_sync(FULL, bd, M - 1);
                        worst_i = __shfl_sync(FULL, bi, M - 1);
                    }
                }
            }
            // lower bound on the distance to any vertex outside the scanned
            // block of cells [c - r, c + r]^3
            int64_t bnd = INT64_MAX;
            {
                const int c[3] = {cx, cy, cz};
                const int32_t q[3] = {qx, qy, qz};
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const int lo_c = c[a] - r, hi_c = c[a] + r;
                    if (lo_c > 0) {
                        const int64_t dlo = (int64_t)q[a] - (int64_t)lo_c * cs + 1;
                        bnd = dlo < bnd ? dlo : bnd;
                    }
                    if (hi_c < G - 1) {
                        const int64_t dhi = (int64_t)(hi_c + 1) * cs - q[a];
                        bnd = dhi < bnd ? dhi : bnd;
                    }
                }
            }
            if (bnd == INT64_MAX) break;                       // whole grid scanned
            const int64_t bnd2 = bnd * bnd;
            if (found >= km1 && worst_d < bnd2) break;          // nothing outside can enter
            if (r2_max >= 0 && bnd2 > r2_max) break;            // nothing outside is in range
        }
    }
    if (lane == 0) row[0] = (int32_t)m;
    if (lane < M) {
        const int pos = lane - pad; // rank among the k-1 others
        if (pos >= 0) row[1 + pos] = bi != INT32_MAX ? c2m[bi] : -1;
        if (lane >= km1) row[1 + lane] = -1;
    }
}

template <int KP>
static pg_status launch_knn_t(pg_graph *g, cudaStream_t s) {
    const int64_t n = g->n;
    int32_t *redo = nullptr, *cnt = nullptr;
    uint64_t *redo_keys = nullptr;
    // lists saved for the first redo_cap queued queries (usually all of them)
    const int64_t redo_cap = n / 8 + 1024;
    PG_TRY(pg_alloc(nullptr, (void **)&redo, 4 * (size_t)(n > 0 ? n : 1), s));
    pg_status st = pg_alloc(nullptr, (void **)&cnt, 16, s);
    if (st == PG_OK && redo_cap > 0)
        st = pg_alloc(nullptr, (void **)&redo_keys, 8 * (size_t)redo_cap * (KP - 1 > 0 ? KP - 1 : 1), s);
    if (st == PG_OK && cudaMemsetAsync(cnt, 0, 4, s) != cudaSuccess) st = PG_ERR_CUDA;
    if (st == PG_OK) {
        constexpr int NT = ke_threads<KP>();
        if (g->level >= 7)
            knn_est_kernel<KP, false, true><<<pg_blocks(n, NT), NT, 0, s>>>(
                g->qpos, g->m2c, g->cell_se, n, g->k, g->level, g->r2_max, g->c2m, g->nbr, redo, cnt, redo_keys, redo_cap);
        else
            knn_est_kernel<KP, false, false><<<pg_blocks(n, NT), NT, 0, s>>>(
                g->qpos, g->m2c, g->cell_se, n, g->k, g->level, g->r2_max, g->c2m, g->nbr, redo, cnt, redo_keys, redo_cap);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    int32_t h_cnt = 0;
    if (st == PG_OK && (cudaMemcpyAsync(&h_cnt, cnt, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    g->knn_exact = h_cnt;
    if (st == PG_OK && h_cnt > 0) {
        knn_exact_kernel<KP, false><<<pg_blocks(32 * (int64_t)h_cnt, 128), 128, 0, s>>>(g->qpos, g->m2c, g->cell_se, g->c2m, redo, cnt, 0,
                                                                         g->k, g->level, g->r2_max, g->nbr, redo_keys,
                                                                         redo_cap);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    cudaFreeAsync(redo, s);
    cudaFreeAsync(cnt, s);
    if (redo_keys) cudaFreeAsync(redo_keys, s);
    return st;
}

static pg_status upload_ring1(cudaStream_t s) {
    static std::once_flag once;
    static int ring[26], ring2[98];
    std::call_once(once, [] {
        ring1_table(ring);
        ring2_table(ring2);
    });
    // the constants live per device: copy them before every launch
    PG_CUDA(cudaMemcpyToSymbolAsync(c_ring1, ring, sizeof(ring), 0, cudaMemcpyHostToDevice, s));
    PG_CUDA(cudaMemcpyToSymbolAsync(c_ring2, ring2, sizeof(ring2), 0, cudaMemcpyHostToDevice, s));
    return PG_OK;
}

pg_status pg_launch_knn_queries(const pg_graph *g, const int32_t *qm, int64_t nq, int k, int32_t *out,
                                cudaStream_t s) {
    if (nq <= 0) return PG_OK;
    PG_TRY(upload_ring1(s));
    const int kp = pg_row_width(k);
    // first ring for every query; the queued ones resume from their saved
    // lists at ring 2 (the exact kernel reads the queue length on the device)
    int32_t *redo = nullptr, *cnt = nullptr;
    uint64_t *keys = nullptr;
    pg_status st = pg_alloc(nullptr, (void **)&redo, 4 * (size_t)nq, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&cnt, 16, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&keys, 8 * (size_t)nq * (kp - 1 > 0 ? kp - 1 : 1), s);
    if (st == PG_OK && cudaMemsetAsync(cnt, 0, 4, s) != cudaSuccess) st = PG_ERR_CUDA;
    if (st == PG_OK) {
#define Q(KP)                                                                                                    \
    if (g->level >= 7)                                                                                           \
        knn_est_kernel<KP, true, true><<<pg_blocks(nq, ke_threads<KP>()), ke_threads<KP>(), 0, s>>>(             \
            g->qpos, g->m2c, g->cell_se, nq, k, g->level, -1, g->c2m, out, redo, cnt, keys, nq, qm);             \
    else                                                                                                         \
        knn_est_kernel<KP, true, false><<<pg_blocks(nq, ke_threads<KP>()), ke_threads<KP>(), 0, s>>>(            \
            g->qpos, g->m2c, g->cell_se, nq, k, g->level, -1, g->c2m, out, redo, cnt, keys, nq, qm);             \
    knn_exact_kernel<KP, true><<<pg_blocks(32 * nq, 128), 128, 0, s>>>(g->qpos, g->m2c, g->cell_se, g->c2m, redo, cnt, nq, k, \
                                                                 g->level, -1, out, keys, nq, qm)
        switch (kp) {
            case 4: Q(4); break;
            case 8: Q(8); break;
            case 16: Q(16); break;
            case 32: Q(32); break;
            default: st = PG_ERR_UNSUPPORTED;
        }
#undef Q
        pg_count_launches(2);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (redo) cudaFreeAsync(redo, s);
    if (cnt) cudaFreeAsync(cnt, s);
    if (keys) cudaFreeAsync(keys, s);
    return st;
}

pg_status pg_launch_knn(pg_graph *g, cudaStream_t s) {
    PG_TRY(upload_ring1(s));
    switch (g->kp) {
        case 4: return launch_knn_t<4>(g, s);
        case 8: return launch_knn_t<8>(g, s);
        case 16: return launch_knn_t<16>(g, s);
        case 32: return launch_knn_t<32>(g, s);
        default: return PG_ERR_UNSUPPORTED;
    }
}

static int auto_level(int64_t n, int k) {
    // about four vertices per cell over the whole box
    double cells = (double)n * 4.0 / (double)(k > 0 ? k : 1);
    int L = (int)(log2(cells > 1.0 ? cells : 1.0) / 3.0 + 0.5);
    if (L < 1) L = 1;
    if (L > 10) L = 10;
    return L;
}

static pg_status graph_free_all(pg_graph *g);

extern "C" pg_status pg_build_graph(const pg_vertices *v, int64_t n, const pg_build_params *p, pg_stream_t stream,
                                    pg_graph **out) {
    if (!out || !p) return PG_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || n >= INT32_MAX) return PG_ERR_INVALID_ARG;
    if (p->k < 1 || p->k > PG_MAX_K) return PG_ERR_UNSUPPORTED;
    if (p->grid_level < 0 || p->grid_level > 10) return PG_ERR_UNSUPPORTED;
    if (p->cluster_size < 0) return PG_ERR_INVALID_ARG;
    if (n > 0 && (!v || !v->px || !v->py || !v->pz)) return PG_ERR_INVALID_ARG;
    float span = 0.0f;
    for (int a = 0; a < 3; a++) {
        if (!isfinite(p->bbox_lo[a]) || !isfinite(p->bbox_hi[a])) return PG_ERR_INVALID_ARG;
        float e = p->bbox_hi[a] - p->bbox_lo[a];
        if (!(e > 0.0f)) return PG_ERR_INVALID_ARG;
        span = e > span ? e : span;
    }
    cudaStream_t s = (cudaStream_t)stream;
    pg_graph *g = new pg_graph();
    g->stream = s;
    g->n = n;
    g->k = p->k;
    g->kp = pg_row_width(p->k);
    g->level = p->grid_level ? p->grid_level : auto_level(n, p->k);
    for (int a = 0; a < 3; a++) g->lo[a] = p->bbox_lo[a];
    {
        volatile float two21 = (float)(1u << PG_QBITS);
        volatile float sp = span;
        g->scale = two21 / sp; // float32 division, as the quantisation step defines it
    }
    g->r2_max = p->r2_max;

    pg_status st = PG_OK;
    int64_t ncells = (int64_t)1 << (3 * g->level);
    uint32_t *keys = nullptr;
    uint64_t *qpos_c = nullptr;
    int32_t *cell_start = nullptr;
#define A(ptr, bytes) \
    if (st == PG_OK) st = pg_alloc(g, (void **)&(ptr), (bytes), s)
    A(g->flags, sizeof(int32_t) * 4);
    A(g->m2c, sizeof(int32_t) * n);
    A(g->c2m, sizeof(int32_t) * n);
    A(g->qpos, sizeof(uint64_t) * n);
    A(g->cell_se, sizeof(int2) * ncells);
    A(g->nbr, sizeof(int32_t) * n * g->kp);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&keys, sizeof(uint32_t) * (n > 0 ? n : 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&qpos_c, sizeof(uint64_t) * (n > 0 ? n : 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&cell_start, sizeof(int32_t) * (ncells + 1), s);
#undef A
    if (st == PG_OK) {
        if (cudaMemsetAsync(g->flags, 0, sizeof(int32_t) * 4, s) != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK && n > 0) {
        quantize_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(v->px, v->py, v->pz, n, g->lo[0], g->lo[1], g->lo[2],
                                                          g->scale, g->level, keys, g->m2c, qpos_c, g->flags);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        if (st == PG_OK) st = pg_radix_sort(g, keys, g->m2c, n, 3 * g->level, s);
        if (st == PG_OK) {
            permute_build_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(g->m2c, qpos_c, n, g->qpos, g->c2m);
            pg_count_launches(1);
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
        if (st == PG_OK && cudaMemsetAsync(cell_start, 0, sizeof(int32_t) * (ncells + 1), s) != cudaSuccess)
            st = PG_ERR_CUDA;
        if (st == PG_OK) {
            cell_count_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(keys, n, cell_start);
            pg_count_launches(1);
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
        if (st == PG_OK) st = pg_scan_exclusive(g, cell_start, ncells + 1, nullptr, s);
        if (st == PG_OK) {
            cell_table_kernel<<<pg_blocks(ncells, 256), 256, 0, s>>>(cell_start, ncells, g->level, g->cell_se);
            pg_count_launches(1);
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
        if (st == PG_OK)
            st = p->cluster_size > 0 ? pg_launch_clusters(g, keys, p->cluster_size, p->cluster_seed, s)
                                     : pg_launch_knn(g, s);
    }
    if (keys) cudaFreeAsync(keys, s);
    if (qpos_c) cudaFreeAsync(qpos_c, s);
    if (cell_start) cudaFreeAsync(cell_start, s);
    int32_t hflags = 0;
    if (st == PG_OK) {
        if (cudaMemcpyAsync(&hflags, g->flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = PG_ERR_CUDA;
    }
    if (st == PG_OK && (hflags & PG_FLAG_NONFINITE)) st = PG_ERR_NONFINITE;
    if (st != PG_OK) {
        (void)cudaGetLastError();
        graph_free_all(g);
        delete g;
        return st;
    }
    *out = g;
    return PG_OK;
}

__global__ void neighbors_out_kernel(const int32_t *__restrict__ nbr, const int32_t *__restrict__ m2c, int64_t n,
                                     int kp, int k, int32_t *__restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * k) return;
    int64_t m = t / k;
    int i = (int)(t - m * k);
    int32_t j = nbr[m * kp + i];
    out[(int64_t)m2c[m] * k + i] = j >= 0 ? m2c[j] : -1;
}

extern "C" pg_status pg_graph_neighbors(const pg_graph *g, int32_t *nbr, pg_stream_t stream) {
    if (!g || (!nbr && g->n > 0)) return PG_ERR_INVALID_ARG;
    if (g->n == 0) return PG_OK;
    neighbors_out_kernel<<<pg_blocks(g->n * g->k, 256), 256, 0, (cudaStream_t)stream>>>(g->nbr, g->m2c, g->n, g->kp,
                                                                                         g->k, nbr);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

extern "C" pg_status pg_graph_get_info(const pg_graph *g, pg_graph_info *info) {
    if (!g || !info) return PG_ERR_INVALID_ARG;
    info->n = g->n;
    info->k = g->k;
    info->row_width = g->kp;
    info->grid_level = g->level;
    info->aggregated = g->aggregated;
    info->n_active = g->n_active;
    info->nnz_swept = g->nnz_swept;
    info->device_bytes = g->bytes;
    info->weight_dtype = (int32_t)g->wdtype;
    info->history_iters = g->hist_iters;
    info->knn_exact = g->knn_exact;
    info->clusters = g->clusters;
    return PG_OK;
}

static pg_status graph_free_all(pg_graph *g) {
    size_t n = (size_t)g->n, kp = (size_t)g->kp;
    size_t ncells = ((size_t)1 << (3 * g->level)) + 1;
    size_t wb = pg_wbytes(g->wdtype);
    pg_free(g, (void **)&g->flags, sizeof(int32_t) * 4);
    pg_free(g, (void **)&g->m2c, 4 * n);
    pg_free(g, (void **)&g->c2m, 4 * n);
    pg_free(g, (void **)&g->qpos, 8 * n);
    pg_free(g, (void **)&g->cell_se, 8 * (ncells - 1));
    pg_free(g, (void **)&g->nbr, 4 * n * kp);
    pg_free(g, (void **)&g->m2r, 4 * n);
    pg_free(g, (void **)&g->r2m, 4 * n);
    pg_free(g, (void **)&g->OG, 16 * n);
    pg_free(g, (void **)&g->DP, 16 * n);
    pg_free(g, (void **)&g->EP, 16 * n);
    pg_free(g, (void **)&g->LV, 16 * n);
    pg_free(g, (void **)&g->succ_m, 4 * n);
    pg_free(g, (void **)&g->W, wb * n * kp);
    pg_free(g, (void **)&g->rscale, 4 * n);
    pg_free(g, (void **)&g->col, 4 * n * kp);
    pg_free(g, (void **)&g->b, 4 * (n + 1));
    pg_free(g, (void **)&g->c_m, 4 * n);
    pg_free(g, (void **)&g->D_m, 4 * n);
    pg_free(g, (void **)&g->ybuf[0], 4 * (n + 1));
    pg_free(g, (void **)&g->ybuf[1], 4 * (n + 1));
    pg_free(g, (void **)&g->hist, 4 * (n + 1) * (size_t)(g->hist_cap + 1));
    pg_free(g, (void **)&g->d_resid, 8 * (size_t)g->resid_cap);
    pg_free(g, (void **)&g->d_ctrl, 16);
    pg_free(g, (void **)&g->d_partials, 16 * (size_t)g->partials_cap);
    pg_free(g, (void **)&g->pmd, 8 * n);
    pg_free(g, (void **)&g->pme, 8 * n);
    pg_free(g, (void **)&g->kin, 4 * n);
    pg_free_transposes(g);
    return PG_OK;
}

extern "C" void pg_graph_destroy(pg_graph *g) {
    if (!g) return;
    graph_free_all(g); // stream-ordered frees: no synchronisation needed
    (void)cudaGetLastError();
    delete g;
}

extern "C" const char *pg_status_string(pg_status s) {
    switch (s) {
        case PG_OK: return "ok";
        case PG_ERR_INVALID_ARG: return "invalid argument";
        case PG_ERR_OOM: return "out of device memory";
        case PG_ERR_CUDA: return "CUDA error";
        case PG_ERR_NONFINITE: return "non-finite input";
        case PG_ERR_TIMEOUT: return "device wait timed out";
        case PG_ERR_UNSUPPORTED: return "unsupported parameter";
        case PG_ERR_STATE: return "invalid call order";
        default: return "unknown status";
    }
}
