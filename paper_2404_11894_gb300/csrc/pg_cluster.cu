// Cluster neighbourhoods (Section 3.1: about N/K cluster centres, every point
// joins its nearest centre, large clusters are split until the sizes are
// even; Section 4 "Path graph solver": centres drawn at random, the nearest
// centre found by searching neighbouring bins of the hash grid).
//
// On the Morton-sorted vertices of the graph build:
//   1. vertex v is a centre iff splitmix64(seed, v) < floor((2^64 - 1) / K)
//      (caller index v; with none drawn, caller vertex 0 is the centre);
//   2. each vertex's nearest centre (exact integer squared distance, ties by
//      the smaller caller index), by rings of cells of a grid of the centres;
//   3. members grouped by centre with a stable sort, so each cluster lists
//      its members in Morton order; a cluster of S > k members is cut into
//      P = ceil(S / k) parts, the i-th member going to part floor(i P / S);
//   4. N(s) = s, then the other members of s's part in Morton order.
#include "pg_internal.cuh"

// Output i of the SplitMix64 generator started from `seed` (the published
// increment and finaliser).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void centre_flag_kernel(const int32_t *__restrict__ m2c, int64_t n, uint64_t seed, uint64_t thr,
                                   int32_t *__restrict__ flag) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    flag[m] = splitmix64_at(seed, (uint64_t)(uint32_t)m2c[m]) < thr ? 1 : 0; // by caller index
}

__global__ void set_one_kernel(int32_t *__restrict__ flag, const int32_t *__restrict__ c2m) { flag[c2m[0]] = 1; }

// centres in Morton order, with their cell keys
__global__ void centre_list_kernel(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int64_t n,
                                   const uint32_t *__restrict__ keys, int32_t *__restrict__ cent,
                                   uint32_t *__restrict__ ckeys) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n || !flag[m]) return;
    cent[pos[m]] = (int32_t)m;
    ckeys[pos[m]] = keys[m];
}

__device__ __forceinline__ bool centre_less(int64_t da, int32_t ia, int64_t db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

// Nearest centre of every vertex: rings of cells around the vertex's own,
// until the best distance is below the distance to any unscanned cell.
__global__ void __launch_bounds__(128) nearest_centre_kernel(const uint64_t *__restrict__ qpos,
                                                             const int32_t *__restrict__ m2c,
                                                             const int32_t *__restrict__ cent,
                                                             const int2 *__restrict__ c_se, int level, int64_t n,
                                                             int32_t *__restrict__ owner) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int3 qr = pg_qpos_unpack(qpos[m]);
    const int sh = PG_QBITS - level;
    const int G = 1 << level;
    const int64_t cs = (int64_t)1 << sh;
    const int cx = qr.x >> sh, cy = qr.y >> sh, cz = qr.z >> sh;
    int64_t best_d = INT64_MAX;
    int32_t best_id = INT32_MAX, best = -1;
    for (int r = 0;; r++) {
        const int span = 2 * r + 1;
        const int64_t ncell = (int64_t)span * span * span;
        for (int64_t t = 0; t < ncell; t++) {
            const int dx = (int)(t % span) - r, dy = (int)((t / span) % span) - r, dz = (int)(t / ((int64_t)span * span)) - r;
            if (r > 0 && abs(dx) != r && abs(dy) != r && abs(dz) != r) continue; // interior: scanned already
            const int x = cx + dx, y = cy + dy, z = cz + dz;
            if (x < 0 || x >= G || y < 0 || y >= G || z < 0 || z >= G) continue;
            const int2 se = c_se[(int64_t)x + ((int64_t)y << level) + ((int64_t)z << (2 * level))];
            for (int32_t i = se.x; i < se.x + se.y; i++) {
                const int32_t cm = cent[i];
                const int3 cq = pg_qpos_unpack(qpos[cm]);
                const int64_t ex = cq.x - qr.x, ey = cq.y - qr.y, ez = cq.z - qr.z;
                const int64_t d2 = ex * ex + ey * ey + ez * ez;
                if (d2 <= best_d) { // the caller index breaks ties
                    const int32_t cid = m2c[cm];
                    if (centre_less(d2, cid, best_d, best_id)) {
                        best_d = d2;
                        best_id = cid;
                        best = i;
                    }
                }
            }
        }
        // lower bound on the distance to any centre outside [c - r, c + r]^3
        int64_t bnd = INT64_MAX;
        const int c[3] = {cx, cy, cz};
        const int32_t q[3] = {qr.x, qr.y, qr.z};
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
        if (bnd == INT64_MAX) break;                     // whole grid scanned
        if (best >= 0 && best_d < bnd * bnd) break;      // nothing outside can tie or win
    }
    owner[m] = best;
}

// per-cell centre counts (Morton-indexed) and the (start, count) table indexed
// by the cell's position, as for the vertices themselves
__global__ void centre_cell_count_kernel(const uint32_t *__restrict__ ckeys, int64_t nc,
                                         int32_t *__restrict__ counts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) atomicAdd(&counts[ckeys[i]], 1);
}

__device__ __forceinline__ uint32_t cl_compact1by2(uint32_t x) {
    x &= 0x09249249u;
    x = (x ^ (x >> 2)) & 0x030C30C3u;
    x = (x ^ (x >> 4)) & 0x0300F00Fu;
    x = (x ^ (x >> 8)) & 0x030000FFu;
    x = (x ^ (x >> 16)) & 0x000003FFu;
    return x;
}

__global__ void centre_cell_table_kernel(const int32_t *__restrict__ cell_start, int64_t ncells, int level,
                                         int2 *__restrict__ c_se) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    uint32_t x = cl_compact1by2((uint32_t)c), y = cl_compact1by2((uint32_t)c >> 1), z = cl_compact1by2((uint32_t)c >> 2);
    int64_t lin = (int64_t)x + ((int64_t)y << level) + ((int64_t)z << (2 * level));
    int32_t a = cell_start[c];
    c_se[lin] = make_int2(a, cell_start[c + 1] - a);
}

__global__ void identity_kernel(int32_t *__restrict__ v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

// 1 where a new cluster starts in the sorted order
__global__ void head_kernel(const uint32_t *__restrict__ owner_s, int64_t n, int32_t *__restrict__ head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) head[i] = (i == 0 || owner_s[i] != owner_s[i - 1]) ? 1 : 0;
}

// cstart[cluster] = first sorted position; head holds the exclusive prefix of
// the start flags, owner_s the sorted keys
__global__ void cluster_start_kernel(const uint32_t *__restrict__ owner_s, const int32_t *__restrict__ hpre,
                                     int64_t n, int32_t *__restrict__ cstart) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || owner_s[i] != owner_s[i - 1]) cstart[hpre[i]] = (int32_t)i;
}

// one thread per sorted position: write the member's neighbourhood (its part)
__global__ void cluster_rows_kernel(const int32_t *__restrict__ sorted_m, const uint32_t *__restrict__ owner_s,
                                    const int32_t *__restrict__ hpre, const int32_t *__restrict__ cstart,
                                    int32_t nclusters, int64_t n, int k, int kp, int32_t *__restrict__ nbr,
                                    unsigned long long *__restrict__ parts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool head = i == 0 || owner_s[i] != owner_s[i - 1];
    const int32_t c = hpre[i] + (head ? 1 : 0) - 1; // cluster of position i
    const int64_t a = cstart[c];
    const int64_t b = c + 1 < nclusters ? cstart[c + 1] : n;
    const int64_t S = b - a, loc = i - a;
    const int64_t P = (S + k - 1) / k;
    const int64_t part = loc * P / S;
    const int64_t ps = (part * S + P - 1) / P, pe = ((part + 1) * S + P - 1) / P;
    // count the parts: one per part's first member, one atomic per warp
    const unsigned first = __ballot_sync(__activemask(), loc == ps);
    if (first && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicAdd(parts, (unsigned long long)__popc(first));
    const int32_t v = sorted_m[i];
    int32_t *row = nbr + (int64_t)v * kp;
    row[0] = v;
    int slot = 1;
    for (int64_t u = ps; u < pe; u++) {
        const int32_t w = sorted_m[a + u];
        if (w != v) row[slot++] = w;
    }
    for (; slot < kp; slot++) row[slot] = -1;
}

pg_status pg_launch_clusters(pg_graph *g, const uint32_t *keys, int32_t K, uint64_t seed, cudaStream_t s) {
    const int64_t n = g->n;
    const int level = g->level;
    const int64_t ncells = (int64_t)1 << (3 * level);
    int32_t *flag = nullptr, *pos = nullptr, *cent = nullptr, *cstart_cells = nullptr, *owner = nullptr,
            *sorted_m = nullptr, *hpre = nullptr, *cstart = nullptr, *d_tot = nullptr;
    uint32_t *ckeys = nullptr;
    int2 *c_se = nullptr;
    pg_status st = PG_OK;
#define T_ALLOC(p, bytes) \
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&(p), (bytes), s)
    T_ALLOC(flag, 4 * (size_t)n);
    T_ALLOC(pos, 4 * (size_t)n);
    T_ALLOC(cent, 4 * (size_t)n);
    T_ALLOC(ckeys, 4 * (size_t)n);
    T_ALLOC(cstart_cells, 4 * (size_t)(ncells + 1));
    T_ALLOC(c_se, 8 * (size_t)ncells);
    T_ALLOC(owner, 4 * (size_t)n);
    T_ALLOC(sorted_m, 4 * (size_t)n);
    T_ALLOC(hpre, 4 * (size_t)n);
    T_ALLOC(cstart, 4 * (size_t)n);
    T_ALLOC(d_tot, 16);
#undef T_ALLOC
    const uint64_t thr = 0xFFFFFFFFFFFFFFFFull / (uint64_t)K;
    int32_t h_tot = 0;
    if (st == PG_OK) {
        centre_flag_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(g->m2c, n, seed, thr, flag);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
        if (cudaMemcpyAsync(pos, flag, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK) st = pg_scan_exclusive(g, pos, n, d_tot, s);
    if (st == PG_OK && (cudaMemcpyAsync(&h_tot, d_tot, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    if (st == PG_OK && h_tot == 0) { // no centre drawn: caller vertex 0 is the one centre
        set_one_kernel<<<1, 1, 0, s>>>(flag, g->c2m);
        pg_count_launches(1);
        if (cudaMemcpyAsync(pos, flag, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = PG_ERR_CUDA;
        if (st == PG_OK) st = pg_scan_exclusive(g, pos, n, nullptr, s);
        h_tot = 1;
    }
    const int64_t nc = h_tot;
    if (st == PG_OK) {
        centre_list_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(flag, pos, n, keys, cent, ckeys);
        pg_count_launches(1);
        if (cudaMemsetAsync(cstart_cells, 0, 4 * (size_t)(ncells + 1), s) != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (st == PG_OK) {
        centre_cell_count_kernel<<<pg_blocks(nc, 256), 256, 0, s>>>(ckeys, nc, cstart_cells);
        pg_count_launches(1);
        st = pg_scan_exclusive(g, cstart_cells, ncells + 1, nullptr, s);
    }
    if (st == PG_OK) {
        centre_cell_table_kernel<<<pg_blocks(ncells, 256), 256, 0, s>>>(cstart_cells, ncells, level, c_se);
        nearest_centre_kernel<<<pg_blocks(n, 128), 128, 0, s>>>(g->qpos, g->m2c, cent, c_se, level, n, owner);
        identity_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(sorted_m, n);
        pg_count_launches(3);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    // stable sort by centre: members of a cluster stay in Morton order
    int nbits = 0;
    while (((int64_t)1 << nbits) < nc) nbits++;
    if (st == PG_OK) st = pg_radix_sort(g, reinterpret_cast<uint32_t *>(owner), sorted_m, n, nbits, s);
    int32_t h_ncl = 0;
    if (st == PG_OK) {
        head_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(reinterpret_cast<const uint32_t *>(owner), n, hpre);
        pg_count_launches(1);
        st = pg_scan_exclusive(g, hpre, n, d_tot, s);
    }
    if (st == PG_OK && (cudaMemcpyAsync(&h_ncl, d_tot, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    if (st == PG_OK) {
        cluster_start_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(reinterpret_cast<const uint32_t *>(owner), hpre, n,
                                                               cstart);
        if (cudaMemsetAsync(d_tot, 0, 8, s) != cudaSuccess) st = PG_ERR_CUDA;
        cluster_rows_kernel<<<pg_blocks(n, 256), 256, 0, s>>>(sorted_m, reinterpret_cast<const uint32_t *>(owner),
                                                              hpre, cstart, h_ncl, n, g->k, g->kp, g->nbr,
                                                              reinterpret_cast<unsigned long long *>(d_tot));
        pg_count_launches(2);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    unsigned long long h_parts = 0;
    if (st == PG_OK && (cudaMemcpyAsync(&h_parts, d_tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    g->knn_exact = 0;
    g->clusters = (int64_t)h_parts;
    void *bufs[] = {flag, pos, cent, ckeys, cstart_cells, c_se, owner, sorted_m, hpre, cstart, d_tot};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, s);
    return st;
}
