// Single-pass prefix scans with decoupled look-back (Merrill & Garland, 2016):
//  * k_compact  - ordered stream compaction of the indices i < n with pred(i),
//                 by warp ballots, a shared-memory scan of the per-warp counts
//                 and a look-back across tiles.  Used for the push frontier
//                 F = {v : |r_v| > h_v}, row-block starts and graph ingest.
//  * k_scan     - exclusive prefix sum of int64 values from a loader functor.
// Tiles take their id from an atomic counter, so a tile only ever waits on
// tiles that were already running; every wait is bounded by kSpinLimit.
#pragma once

#include "fj_common.cuh"

namespace fj {

constexpr unsigned long long kStFlagShift = 62;
constexpr unsigned long long kStAgg = 1ULL << kStFlagShift;
constexpr unsigned long long kStPrefix = 2ULL << kStFlagShift;
constexpr unsigned long long kStValMask = (1ULL << kStFlagShift) - 1;

__device__ __forceinline__ void st_publish(unsigned long long *st, unsigned long long word)
{
    __threadfence();
    atomicExch(st, word);
}

__device__ __forceinline__ unsigned long long st_read(const unsigned long long *st)
{
    unsigned long long w = *reinterpret_cast<const volatile unsigned long long *>(st);
    __threadfence();
    return w;
}

// Polls a tile's status word until the tile has published it (flag bits
// set), at most `limit` times; false when it gave up.
__device__ __forceinline__ bool wait_published(const unsigned long long *st, long long limit, unsigned long long &w)
{
    for (long long spins = 0;; ++spins) {
        w = st_read(st);
        if (w >> kStFlagShift) return true;
        if (spins >= limit) return false;
        __nanosleep(32);
    }
}

// Called by one thread per tile.  Publishes the tile aggregate, walks back to
// the nearest inclusive prefix and returns this tile's exclusive prefix.
static __device__ __noinline__ long long lookback_prefix(unsigned long long *status, int tile, long long agg,
                                                  int *err)
{
    if (tile == 0) {
        st_publish(&status[0], kStPrefix | (unsigned long long)agg);
        return 0;
    }
    st_publish(&status[tile], kStAgg | (unsigned long long)agg);
    long long excl = 0;
    int p = tile - 1;
    while (p >= 0) {
        unsigned long long w;
        if (!wait_published(&status[p], kSpinLimit, w)) {
            dev_error(err, DEV_SPIN_TIMEOUT);
            w = kStPrefix;  // give up: treat as a zero prefix
        }
        excl += (long long)(w & kStValMask);
        if ((w >> kStFlagShift) == 2) break;
        --p;
    }
    st_publish(&status[tile], kStPrefix | (unsigned long long)(excl + agg));
    return excl;
}

// Scratch needed by one k_compact / k_scan launch over n items.
inline int64_t scan_tiles(int64_t n, int items_per_tile) { return ceil_div(n > 0 ? n : 1, items_per_tile); }

// ---------------------------------------------------------------- compaction

template <int THREADS, int ITEMS, typename Pred>
__global__ void __launch_bounds__(THREADS)
k_compact(int64_t n, Pred pred, int32_t *__restrict__ out, long long *count_out,
          unsigned long long *status, unsigned int *tile_ctr, int *err)
{
    constexpr int NW = THREADS / 32;
    constexpr int TOT = ITEMS * NW;
    constexpr int E = (TOT + 31) / 32;
    __shared__ int s_tile;
    __shared__ int s_cnt[TOT];
    __shared__ long long s_base;
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * (THREADS * ITEMS);
    unsigned masks[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * THREADS + threadIdx.x;
        bool f = idx < n && pred(idx);
        masks[i] = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_cnt[i * NW + wid] = __popc(masks[i]);
    }
    __syncthreads();
    if (wid == 0) {
        int loc[E];
        int sum = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int j = lane * E + e;
            int v = j < TOT ? s_cnt[j] : 0;
            loc[e] = sum;
            sum += v;
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int excl = incl - sum;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int j = lane * E + e;
            if (j < TOT) s_cnt[j] = excl + loc[e];
        }
        int total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 0) {
            s_total = total;
            s_base = lookback_prefix(status, tile, total, err);
        }
    }
    __syncthreads();
    const long long b = s_base;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if ((masks[i] >> lane) & 1u) {
            int64_t idx = base + (int64_t)i * THREADS + threadIdx.x;
            out[b + s_cnt[i * NW + wid] + __popc(masks[i] & lt)] = (int32_t)idx;
        }
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0 && count_out) *count_out = b + s_total;
}

// Host launcher.  status must hold scan_tiles(n, THREADS*ITEMS) words and
// tile_ctr one word; both are cleared here on `stream`.
template <int THREADS = 256, int ITEMS = 8, typename Pred>
cudaError_t compact(int64_t n, Pred pred, int32_t *out, long long *count_out,
                    unsigned long long *status, unsigned int *tile_ctr, int *err, cudaStream_t stream)
{
    int64_t tiles = scan_tiles(n, THREADS * ITEMS);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * tiles, stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    k_compact<THREADS, ITEMS, Pred><<<(unsigned)tiles, THREADS, 0, stream>>>(n, pred, out, count_out,
                                                                            status, tile_ctr, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- generic scan

// out[i] = sum_{j < i} load(j) for i < n (int64); *total_out = sum of all.
template <int THREADS, int ITEMS, typename Load>
__global__ void __launch_bounds__(THREADS)
k_scan(int64_t n, Load load, long long *__restrict__ out, long long *total_out,
       unsigned long long *status, unsigned int *tile_ctr, int *err)
{
    constexpr int NW = THREADS / 32;
    __shared__ long long s_val[THREADS * ITEMS];
    __shared__ long long s_warp[NW];
    __shared__ int s_tile;
    __shared__ long long s_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * (THREADS * ITEMS);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * THREADS + threadIdx.x;
        s_val[i * THREADS + threadIdx.x] = idx < n ? (long long)load(idx) : 0LL;
    }
    __syncthreads();
    long long loc[ITEMS];
    long long sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        long long v = s_val[threadIdx.x * ITEMS + i];
        loc[i] = sum;
        sum += v;
    }
    long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long wv = lane < NW ? s_warp[lane] : 0LL;
        long long wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) s_warp[lane] = wi - wv;
        long long total = __shfl_sync(0xffffffffu, wi, 31);
        if (lane == 0) {
            s_base = lookback_prefix(status, tile, total, err);
            if (tile == (int)gridDim.x - 1 && total_out) *total_out = s_base + total;
        }
    }
    __syncthreads();
    const long long pre = s_base + s_warp[wid] + (incl - sum);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) s_val[threadIdx.x * ITEMS + i] = pre + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * THREADS + threadIdx.x;
        if (idx < n) out[idx] = s_val[i * THREADS + threadIdx.x];
    }
}

template <int THREADS = 256, int ITEMS = 8, typename Load>
cudaError_t scan(int64_t n, Load load, long long *out, long long *total_out, unsigned long long *status,
                 unsigned int *tile_ctr, int *err, cudaStream_t stream)
{
    int64_t tiles = scan_tiles(n, THREADS * ITEMS);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * tiles, stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    k_scan<THREADS, ITEMS, Load><<<(unsigned)tiles, THREADS, 0, stream>>>(n, load, out, total_out, status,
                                                                         tile_ctr, err);
    return cudaGetLastError();
}

}  // namespace fj
