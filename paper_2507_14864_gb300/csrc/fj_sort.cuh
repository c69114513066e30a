// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits.
// Per pass: per-tile digit histograms -> one exclusive scan over the
// digit-major histogram table -> a stable scatter in which each key's rank
// inside its tile comes from __match_any_sync peer groups and per-warp
// running digit counts.  Stability makes the transpose of a row-ordered CSR
// come out with ascending row ids in every column, and makes repeated arcs
// keep their input order.
#pragma once

#include "fj_scan.cuh"

namespace fj {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

static __global__ void __launch_bounds__(kSortThreads)
k_radix_hist(int64_t n, const uint32_t *__restrict__ keys, int shift, unsigned *__restrict__ hist,
             int64_t ntiles)
{
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kSortThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

static __global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(int64_t n, const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int shift,
                const long long *__restrict__ offs, int64_t ntiles)
{
    constexpr int NW = kSortThreads / 32;
    __shared__ unsigned whist[NW][256];
    __shared__ long long woff[NW][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NW * 256; i += kSortThreads) whist[i / 256][i % 256] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + (int64_t)wid * 32 * kSortItems;
    const unsigned lt = lanemask_lt();
    uint32_t k[kSortItems], v[kSortItems];
    unsigned rk[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = wbase + (int64_t)i * 32 + lane;
        bool valid = idx < n;
        k[i] = valid ? kin[idx] : 0u;
        v[i] = valid ? vin[idx] : 0u;
        unsigned vm = __ballot_sync(0xffffffffu, valid);
        unsigned d = (k[i] >> shift) & 255u;
        unsigned peers = 0, rank = 0;
        if (valid) {
            peers = __match_any_sync(vm, d);
            rank = __popc(peers & lt);
            rk[i] = whist[wid][d] + rank;
        }
        __syncwarp();
        if (valid && rank == 0) whist[wid][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        long long run = offs[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < NW; ++w) {
            woff[w][d] = run;
            run += whist[w][d];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = wbase + (int64_t)i * 32 + lane;
        if (idx < n) {
            unsigned d = (k[i] >> shift) & 255u;
            long long dst = woff[wid][d] + rk[i];
            kout[dst] = k[i];
            vout[dst] = v[i];
        }
    }
}

struct HistLoad {
    const unsigned *h;
    __device__ long long operator()(int64_t i) const { return (long long)h[i]; }
};

// Scratch for sort_pairs(n): two key/value buffers are the caller's; this is
// the histogram table plus scan state.
struct SortScratch {
    unsigned *hist = nullptr;             // 256 * ntiles
    long long *offs = nullptr;            // 256 * ntiles
    unsigned long long *status = nullptr; // scan tiles of 256 * ntiles
    unsigned int *tile_ctr = nullptr;
    int64_t cap_tiles = 0;
};

inline int64_t sort_tiles(int64_t n) { return ceil_div(n > 0 ? n : 1, kSortTile); }

inline cudaError_t sort_scratch_alloc(SortScratch &s, int64_t n)
{
    int64_t t = sort_tiles(n);
    if (t <= s.cap_tiles) return cudaSuccess;
    cudaFree(s.hist);
    cudaFree(s.offs);
    cudaFree(s.status);
    cudaFree(s.tile_ctr);
    s = SortScratch();
    cudaError_t e;
    if ((e = dev_malloc(&s.hist, sizeof(unsigned) * 256 * t)) != cudaSuccess) return e;
    if ((e = dev_malloc(&s.offs, sizeof(long long) * 256 * t)) != cudaSuccess) return e;
    if ((e = dev_malloc(&s.status, sizeof(unsigned long long) * scan_tiles(256 * t, 256 * 8))) != cudaSuccess)
        return e;
    if ((e = dev_malloc(&s.tile_ctr, sizeof(unsigned int))) != cudaSuccess) return e;
    s.cap_tiles = t;
    return cudaSuccess;
}

inline void sort_scratch_free(SortScratch &s)
{
    cudaFree(s.hist);
    cudaFree(s.offs);
    cudaFree(s.status);
    cudaFree(s.tile_ctr);
    s = SortScratch();
}

// Sorts (k0, v0) by the low `key_bits` bits of the keys, stably; the result
// ends in (k0, v0) or (k1, v1): *result_in_1 tells which.
inline cudaError_t sort_pairs(int64_t n, int key_bits, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                              SortScratch &s, int *err, cudaStream_t stream, bool *result_in_1)
{
    *result_in_1 = false;
    if (n <= 1) return cudaSuccess;
    cudaError_t e = sort_scratch_alloc(s, n);
    if (e != cudaSuccess) return e;
    int64_t t = sort_tiles(n);
    int passes = (key_bits + 7) / 8;
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int p = 0; p < passes; ++p) {
        k_radix_hist<<<(unsigned)t, kSortThreads, 0, stream>>>(n, ki, 8 * p, s.hist, t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = scan<256, 8>(256 * t, HistLoad{s.hist}, s.offs, nullptr, s.status, s.tile_ctr, err, stream)) !=
            cudaSuccess)
            return e;
        k_radix_scatter<<<(unsigned)t, kSortThreads, 0, stream>>>(n, ki, vi, ko, vo, 8 * p, s.offs, t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t *tk = ki, *tv = vi;
        ki = ko; vi = vo; ko = tk; vo = tv;
        *result_in_1 = !*result_in_1;
    }
    return cudaSuccess;
}

inline int bits_for(int64_t max_value)
{
    int b = 1;
    while (b < 32 && (int64_t(1) << b) <= max_value) ++b;
    return b;
}

}  // namespace fj
