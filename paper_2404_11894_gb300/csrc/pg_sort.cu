// Device primitives: stream-ordered allocation, exclusive scan, and a stable
// LSD radix sort of (uint32 key, int32 value) pairs.
#include <atomic>
#include <mutex>

#include "pg_internal.cuh"

static std::atomic<long long> g_launches{0};
void pg_count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
extern "C" int64_t pg_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

// The library's own stream-ordered memory pool on each device. Freed blocks
// stay in it (release threshold: never) instead of going back to the driver
// at every synchronisation, so a graph rebuilt every frame reuses its memory.
// Being private, it leaves the device's default pool, which other code in the
// process may share, exactly as the caller configured it.
static cudaMemPool_t lib_pool(int dev) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        (void)cudaGetLastError();
        pools[dev] = pool;
    }
    return pools[dev];
}

pg_status pg_alloc(pg_graph *g, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return PG_ERR_CUDA;
    }
    cudaMemPool_t pool = lib_pool(dev);
    if (!pool) return PG_ERR_CUDA;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? PG_ERR_OOM : PG_ERR_CUDA;
    }
    if (g) g->bytes += (int64_t)bytes;
    return PG_OK;
}

void pg_free(pg_graph *g, void **p, size_t bytes) {
    if (*p) {
        cudaFreeAsync(*p, g ? g->stream : nullptr);
        if (g) g->bytes -= (int64_t)(bytes == 0 ? 16 : bytes);
    }
    *p = nullptr;
}

int pg_num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------------ scan
// Three-phase exclusive scan: per-block sums, a scan of the block sums
// (recursively), then per-block scans offset by the scanned block sums.
static constexpr int SCAN_THREADS = 512;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total) {
    __shared__ T warp_sums[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    T off = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return off + x - v;
}

template <typename T>
__global__ void scan_block_sums(const T *__restrict__ data, int64_t n, T *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T acc = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) acc += data[idx];
    }
    T total;
    (void)block_exclusive_scan<T>(acc, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename T>
__global__ void scan_block_apply(T *__restrict__ data, int64_t n, const T *__restrict__ offs, T *__restrict__ d_total,
                                 int64_t nblocks) {
    // each thread owns SCAN_ITEMS consecutive elements
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? data[idx] : 0;
        s += v[i];
    }
    T total;
    T ex = block_exclusive_scan<T>(s, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        if (idx < n) data[idx] = ex;
        ex += v[i];
    }
    if (d_total && blockIdx.x == nblocks - 1 && threadIdx.x == SCAN_THREADS - 1) *d_total = ex;
}

template <typename T>
static pg_status scan_exclusive(pg_graph *g, T *data, int64_t n, T *d_total, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) PG_CUDA(cudaMemsetAsync(d_total, 0, sizeof(T), s));
        return PG_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        scan_block_apply<T><<<1, SCAN_THREADS, 0, s>>>(data, n, nullptr, d_total, 1);
        pg_count_launches(1);
        PG_LAUNCH_CHECK();
        return PG_OK;
    }
    T *sums = nullptr;
    PG_TRY(pg_alloc(nullptr, (void **)&sums, sizeof(T) * nb, s));
    scan_block_sums<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(data, n, sums);
    pg_count_launches(1);
    pg_status st = PG_OK;
    if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    if (st == PG_OK) st = scan_exclusive<T>(g, sums, nb, nullptr, s);
    if (st == PG_OK) {
        scan_block_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(data, n, sums, d_total, nb);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    cudaFreeAsync(sums, s);
    return st;
}

pg_status pg_scan_exclusive(pg_graph *g, int32_t *data, int64_t n, int32_t *d_total, cudaStream_t s) {
    return scan_exclusive<int32_t>(g, data, n, d_total, s);
}

pg_status pg_scan_exclusive64(pg_graph *g, int64_t *data, int64_t n, int64_t *d_total, cudaStream_t s) {
    return scan_exclusive<int64_t>(g, data, n, d_total, s);
}

// ------------------------------------------------------------------ radix sort
// One 8-bit digit per pass over tiles of SORT_TILE pairs: (1) per-tile digit
// histograms, (2) an exclusive scan of the digit-major histogram table gives
// every (digit, tile) its output offset, (3) each tile scatters its pairs in
// input order (warp match + per-warp prefix), which keeps the sort stable.
static constexpr int SORT_THREADS = 256;
static constexpr int SORT_ROUNDS = 16;
static constexpr int SORT_TILE = SORT_THREADS * SORT_ROUNDS;

__global__ void radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
                           int64_t ntiles) {
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; r++) {
        int64_t idx = base + (int64_t)r * SORT_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void radix_scatter(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                              uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int shift,
                              const int32_t *__restrict__ offs, int64_t ntiles) {
    __shared__ int32_t run[256];
    __shared__ int32_t wcnt[SORT_THREADS / 32][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; r++) {
        for (int w = 0; w < SORT_THREADS / 32; w++) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t idx = base + (int64_t)r * SORT_THREADS + threadIdx.x;
        bool valid = idx < n;
        uint32_t key = valid ? kin[idx] : 0u;
        int32_t val = valid ? vin[idx] : 0;
        uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & lt_mask);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[wid][digit] = __popc(peers);
        __syncthreads();
        {
            int d = threadIdx.x;
            int32_t acc = run[d];
            for (int w = 0; w < SORT_THREADS / 32; w++) {
                int32_t t = wcnt[w][d];
                wcnt[w][d] = acc;
                acc += t;
            }
            run[d] = acc;
        }
        __syncthreads();
        if (valid) {
            int32_t pos = wcnt[wid][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

pg_status pg_radix_sort(pg_graph *g, uint32_t *keys, int32_t *vals, int64_t n, int nbits, cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return PG_OK;
    int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    uint32_t *k2 = nullptr;
    int32_t *v2 = nullptr, *hist = nullptr;
    pg_status st = pg_alloc(nullptr, (void **)&k2, sizeof(uint32_t) * n, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&v2, sizeof(int32_t) * n, s);
    if (st == PG_OK) st = pg_alloc(nullptr, (void **)&hist, sizeof(int32_t) * 256 * ntiles, s);
    uint32_t *kin = keys, *kout = k2;
    int32_t *vin = vals, *vout = v2;
    int passes = (nbits + 7) / 8;
    for (int p = 0; p < passes && st == PG_OK; p++) {
        int shift = 8 * p;
        radix_hist<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(kin, n, shift, hist, ntiles);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        if (st == PG_OK) st = pg_scan_exclusive(g, hist, 256 * ntiles, nullptr, s);
        if (st == PG_OK) {
            radix_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
            pg_count_launches(1);
            if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
        }
        uint32_t *tk = kin; kin = kout; kout = tk;
        int32_t *tv = vin; vin = vout; vout = tv;
    }
    if (st == PG_OK && kin != keys) {
        cudaMemcpyAsync(keys, kin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vin, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    if (k2) cudaFreeAsync(k2, s);
    if (v2) cudaFreeAsync(v2, s);
    if (hist) cudaFreeAsync(hist, s);
    return st;
}
