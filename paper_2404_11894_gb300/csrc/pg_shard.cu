// Sharded propagation sweeps (one shard per GPU).
//
// The Jacobi sweep of Eq. rte-mff updates every swept row from the previous
// iterate only, so its rows split into independent parts. The rows are in
// Morton order, so a contiguous range of rows is a spatial slab of the
// medium and most of the columns its rows read are its own rows. Shard p
// owns rows [R_p, R_p+1), cut so that every shard holds nearly the same
// number of live entries, and keeps a local iterate
//     z_p = [ own rows | halo | zero slot ]
// where the halo holds, in ascending global order, the columns its rows read
// but another shard owns (neighbours across the slab boundary and
// continuation edges that leave the slab). Because the halo is sorted and
// the ranges are contiguous, the values each peer q supplies form one
// contiguous segment of the halo; q sends them from its own rows in the
// same order. One sweep is then: every shard packs what each peer needs,
// the packs are exchanged, each shard copies what it received into its
// halo segments and sweeps its rows with the ordinary sweep kernel on a
// column table re-indexed into z_p. Each row's sum runs in the same order
// as in pg_propagate, so the result is bitwise the same.
#include <algorithm>
#include <vector>

#include "pg_internal.cuh"

struct pg_shard {
    int32_t n_shards = 0, shard = 0, kp = 0;
    int64_t n_rows = 0;                 // swept rows of the whole graph
    int64_t zero_slot = 0;              // global zero column
    std::vector<int64_t> row_begin;     // n_shards + 1
    std::vector<int32_t> halo;          // global columns read but owned by peers, ascending
    std::vector<int64_t> recv_begin;    // n_shards + 1: halo segment owned by each shard
    std::vector<int32_t> send_idx;      // own local rows each peer reads, grouped by peer
    std::vector<int64_t> send_begin;    // n_shards + 1
    std::vector<int32_t> local_col;     // own rows x kp, indices into z_p
    // device side (shards made from a graph)
    const pg_graph *g = nullptr;
    int32_t *d_col = nullptr;
    int32_t *d_send = nullptr;
    int32_t *d_halo = nullptr;
    int32_t *d_ctrl = nullptr;
    double *d_partials = nullptr;
    double *d_resid = nullptr;
    int32_t partials_cap = 0;
};

static int64_t own_rows(const pg_shard *p) { return p->row_begin[p->shard + 1] - p->row_begin[p->shard]; }
static int64_t local_len(const pg_shard *p) { return own_rows(p) + (int64_t)p->halo.size() + 1; }

// Host plan from the column table of all swept rows (row r's entries at
// col[r * kp + i]; zero_slot marks an empty entry).
static pg_status plan(pg_shard *p, const int32_t *col, int64_t n_rows, int32_t kp, int64_t zero_slot,
                      int32_t n_shards, int32_t shard) {
    p->n_shards = n_shards;
    p->shard = shard;
    p->kp = kp;
    p->n_rows = n_rows;
    p->zero_slot = zero_slot;
    for (int64_t e = 0; e < n_rows * kp; e++)
        if (col[e] != zero_slot && (col[e] < 0 || col[e] >= n_rows)) return PG_ERR_INVALID_ARG;
    // contiguous row ranges of nearly equal live-entry counts
    std::vector<int64_t> pre(n_rows + 1, 0);
    for (int64_t r = 0; r < n_rows; r++) {
        int64_t c = 0;
        for (int i = 0; i < kp; i++) c += col[r * kp + i] != zero_slot;
        pre[r + 1] = pre[r] + c;
    }
    p->row_begin.assign(n_shards + 1, n_rows);
    p->row_begin[0] = 0;
    for (int q = 1; q < n_shards; q++) {
        const int64_t target = (pre[n_rows] * q + n_shards / 2) / n_shards;
        p->row_begin[q] = std::lower_bound(pre.begin(), pre.end(), target) - pre.begin();
        p->row_begin[q] = std::max(p->row_begin[q], p->row_begin[q - 1]);
    }
    const int64_t r0 = p->row_begin[shard], r1 = p->row_begin[shard + 1];
    // halo: columns outside the own range, ascending, grouped by owner
    std::vector<uint8_t> mark(n_rows, 0);
    for (int64_t e = r0 * kp; e < r1 * kp; e++) {
        const int64_t c = col[e];
        if (c != zero_slot && (c < r0 || c >= r1)) mark[c] = 1;
    }
    p->halo.clear();
    for (int64_t c = 0; c < n_rows; c++)
        if (mark[c]) p->halo.push_back((int32_t)c);
    p->recv_begin.assign(n_shards + 1, 0);
    for (int q = 0; q <= n_shards; q++)
        p->recv_begin[q] = std::lower_bound(p->halo.begin(), p->halo.end(), (int32_t)std::min<int64_t>(
                                                p->row_begin[q], INT32_MAX)) - p->halo.begin();
    p->recv_begin[n_shards] = (int64_t)p->halo.size();
    // the own rows' table re-indexed into z_p
    const int64_t rows = r1 - r0, zl = rows + (int64_t)p->halo.size();
    p->local_col.resize(rows * kp);
    for (int64_t e = r0 * kp; e < r1 * kp; e++) {
        const int64_t c = col[e];
        int64_t l;
        if (c == zero_slot) l = zl;
        else if (c >= r0 && c < r1) l = c - r0;
        else l = rows + (std::lower_bound(p->halo.begin(), p->halo.end(), (int32_t)c) - p->halo.begin());
        p->local_col[e - r0 * kp] = (int32_t)l;
    }
    // what each peer reads from the own rows, ascending (its halo segment order)
    p->send_idx.clear();
    p->send_begin.assign(n_shards + 1, 0);
    std::vector<uint8_t> need(rows, 0);
    for (int q = 0; q < n_shards; q++) {
        p->send_begin[q] = (int64_t)p->send_idx.size();
        if (q == shard) continue;
        std::fill(need.begin(), need.end(), 0);
        for (int64_t e = p->row_begin[q] * kp; e < p->row_begin[q + 1] * kp; e++) {
            const int64_t c = col[e];
            if (c != zero_slot && c >= r0 && c < r1) need[c - r0] = 1;
        }
        for (int64_t i = 0; i < rows; i++)
            if (need[i]) p->send_idx.push_back((int32_t)i);
    }
    p->send_begin[n_shards] = (int64_t)p->send_idx.size();
    return PG_OK;
}

extern "C" pg_status pg_shard_create_host(const int32_t *col, int64_t n_rows, int32_t row_width, int64_t zero_slot,
                                          int32_t n_shards, int32_t shard, pg_shard **out) {
    if (!out) return PG_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rows < 0 || (n_rows > 0 && !col) || row_width < 1 || n_shards < 1 || shard < 0 || shard >= n_shards ||
        n_rows >= INT32_MAX || zero_slot < n_rows || zero_slot >= INT32_MAX)
        return PG_ERR_INVALID_ARG;
    pg_shard *p = new pg_shard();
    pg_status st = plan(p, col, n_rows, row_width, zero_slot, n_shards, shard);
    if (st != PG_OK) {
        delete p;
        return st;
    }
    *out = p;
    return PG_OK;
}

extern "C" pg_status pg_shard_get_info(const pg_shard *p, pg_shard_info *info) {
    if (!p || !info) return PG_ERR_INVALID_ARG;
    info->n_shards = p->n_shards;
    info->shard = p->shard;
    info->row_width = p->kp;
    info->row_begin = p->row_begin[p->shard];
    info->row_end = p->row_begin[p->shard + 1];
    info->n_halo = (int64_t)p->halo.size();
    info->local_len = local_len(p);
    info->n_send = (int64_t)p->send_idx.size();
    return PG_OK;
}

extern "C" pg_status pg_shard_get_lists(const pg_shard *p, int64_t *row_begin, int64_t *recv_begin,
                                        int64_t *send_begin, int32_t *halo, int32_t *send_idx, int32_t *local_col) {
    if (!p) return PG_ERR_INVALID_ARG;
    if (row_begin) std::copy(p->row_begin.begin(), p->row_begin.end(), row_begin);
    if (recv_begin) std::copy(p->recv_begin.begin(), p->recv_begin.end(), recv_begin);
    if (send_begin) std::copy(p->send_begin.begin(), p->send_begin.end(), send_begin);
    if (halo) std::copy(p->halo.begin(), p->halo.end(), halo);
    if (send_idx) std::copy(p->send_idx.begin(), p->send_idx.end(), send_idx);
    if (local_col) std::copy(p->local_col.begin(), p->local_col.end(), local_col);
    return PG_OK;
}

// ------------------------------------------------------------------ device side
// out[i] = z[idx[i]]
__global__ void shard_pack_kernel(const float *__restrict__ z, const int32_t *__restrict__ idx, int64_t m,
                                  float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = z[idx[i]];
}

extern "C" pg_status pg_shard_create(const pg_graph *g, int32_t n_shards, int32_t shard, pg_stream_t stream,
                                     pg_shard **out) {
    if (!g || !out) return PG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g->aggregated || !g->W) return PG_ERR_STATE;
    if (n_shards < 1 || shard < 0 || shard >= n_shards) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t na = g->n_active, kp = g->kp;
    std::vector<int32_t> col((size_t)(na * kp));
    if (na > 0) {
        PG_CUDA(cudaMemcpyAsync(col.data(), g->col, 4 * (size_t)(na * kp), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
    }
    pg_shard *p = nullptr;
    PG_TRY(pg_shard_create_host(col.data(), na, (int32_t)kp, g->n, n_shards, shard, &p));
    p->g = g;
    pg_status st = PG_OK;
    const int64_t rows = own_rows(p);
    pg_graph view = {};
    view.n_active = rows;
    view.kp = g->kp;
    p->partials_cap = pg_sweep_blocks(&view);
    st = pg_alloc(nullptr, (void **)&p->d_col, 4 * (size_t)std::max<int64_t>(rows * kp, 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&p->d_send, 4 * std::max<size_t>(p->send_idx.size(), 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&p->d_halo, 4 * std::max<size_t>(p->halo.size(), 1), s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&p->d_ctrl, 16, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&p->d_partials, 16 * (size_t)p->partials_cap, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&p->d_resid, 8, s);
    if (st == PG_OK && rows > 0 &&
        cudaMemcpyAsync(p->d_col, p->local_col.data(), 4 * (size_t)(rows * kp), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        st = PG_ERR_CUDA;
    if (st == PG_OK && !p->send_idx.empty() &&
        cudaMemcpyAsync(p->d_send, p->send_idx.data(), 4 * p->send_idx.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        st = PG_ERR_CUDA;
    if (st == PG_OK && !p->halo.empty() &&
        cudaMemcpyAsync(p->d_halo, p->halo.data(), 4 * p->halo.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = PG_ERR_CUDA;
    if (st == PG_OK && cudaStreamSynchronize(s) != cudaSuccess) st = PG_ERR_CUDA;
    if (st != PG_OK) {
        (void)cudaGetLastError();
        pg_shard_destroy(p);
        return st;
    }
    *out = p;
    return PG_OK;
}

extern "C" pg_status pg_shard_load(const pg_shard *p, const float *y, float *z, pg_stream_t stream) {
    if (!p || !p->g) return PG_ERR_STATE;
    if (!y || !z) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t rows = own_rows(p), nh = (int64_t)p->halo.size();
    if (rows > 0)
        PG_CUDA(cudaMemcpyAsync(z, y + p->row_begin[p->shard], 4 * (size_t)rows, cudaMemcpyDeviceToDevice, s));
    if (nh > 0) {
        shard_pack_kernel<<<pg_blocks(nh, 256), 256, 0, s>>>(y, p->d_halo, nh, z + rows);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
    }
    PG_CUDA(cudaMemsetAsync(z + rows + nh, 0, 4, s));
    return PG_OK;
}

extern "C" pg_status pg_shard_pack(const pg_shard *p, const float *z, float *send, pg_stream_t stream) {
    if (!p || !p->g) return PG_ERR_STATE;
    const int64_t m = (int64_t)p->send_idx.size();
    if (m == 0) return PG_OK;
    if (!z || !send) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    shard_pack_kernel<<<pg_blocks(m, 256), 256, 0, s>>>(z, p->d_send, m, send);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

extern "C" pg_status pg_shard_sweep(pg_shard *p, const float *z_in, float *z_out, pg_stream_t stream) {
    if (!p || !p->g) return PG_ERR_STATE;
    const pg_graph *g = p->g;
    if (!g->aggregated || !g->W) return PG_ERR_STATE;
    const int64_t rows = own_rows(p);
    if (rows == 0) return PG_OK;
    if (!z_in || !z_out || z_in == z_out) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t r0 = p->row_begin[p->shard];
    // a view of the graph holding only the own rows, with the local table
    pg_graph view = {};
    view.n = g->n;
    view.kp = g->kp;
    view.wdtype = g->wdtype;
    view.n_active = rows;
    view.col = p->d_col;
    view.W = (char *)g->W + (size_t)r0 * g->kp * pg_wbytes(g->wdtype);
    view.rscale = g->rscale ? g->rscale + r0 : nullptr;
    PG_CUDA(cudaMemsetAsync(p->d_ctrl, 0, 16, s));
    return pg_launch_sweep(&view, g->b + r0, z_in, z_out, p->d_ctrl, (double2 *)p->d_partials, p->d_resid, 1, 0.0,
                           s);
}

extern "C" void pg_shard_destroy(pg_shard *p) {
    if (!p) return;
    for (void *q : {(void *)p->d_col, (void *)p->d_send, (void *)p->d_halo, (void *)p->d_ctrl,
                    (void *)p->d_partials, (void *)p->d_resid})
        if (q) cudaFree(q);
    (void)cudaGetLastError();
    delete p;
}

// ------------------------------------------------------------------ the sweep vector and L+
// y[row of succ(v)] = L[v]; every other entry (first-vertex rows, zero slot) 0
__global__ void y_from_L_kernel(const float *__restrict__ L, const int32_t *__restrict__ c2m,
                                const int32_t *__restrict__ succ_m, const int32_t *__restrict__ m2r, int64_t n,
                                float *__restrict__ y) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t s = succ_m[c2m[v]];
    if (s >= 0) y[m2r[s]] = L[v];
}

// L[v] = y[row of succ(v)], 0 at the end of a path
__global__ void L_from_y_kernel(const float *__restrict__ y, const int32_t *__restrict__ c2m,
                                const int32_t *__restrict__ succ_m, const int32_t *__restrict__ m2r, int64_t n,
                                float *__restrict__ L) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t s = succ_m[c2m[v]];
    L[v] = s >= 0 ? y[m2r[s]] : 0.0f;
}

extern "C" pg_status pg_graph_y_from_L(const pg_graph *g, const float *L, float *y, pg_stream_t stream) {
    if (!g || !g->aggregated) return PG_ERR_STATE;
    if (g->n > 0 && (!L || !y)) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    PG_CUDA(cudaMemsetAsync(y, 0, 4 * (size_t)(g->n + 1), s));
    if (g->n == 0) return PG_OK;
    y_from_L_kernel<<<pg_blocks(g->n, 256), 256, 0, s>>>(L, g->c2m, g->succ_m, g->m2r, g->n, y);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

extern "C" pg_status pg_graph_L_from_y(const pg_graph *g, const float *y, float *L, pg_stream_t stream) {
    if (!g || !g->aggregated) return PG_ERR_STATE;
    if (g->n == 0) return PG_OK;
    if (!L || !y) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    L_from_y_kernel<<<pg_blocks(g->n, 256), 256, 0, s>>>(y, g->c2m, g->succ_m, g->m2r, g->n, L);
    pg_count_launches(1);
    PG_LAUNCH_CHECK();
    return PG_OK;
}
