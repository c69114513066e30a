// Warp walk of a tile of the warp-tile item plan for k right-hand sides
// (node-major [n][k] vectors), shared by the batch sweep, the batch
// certificate and the batch measures.
#pragma once
#include <type_traits>

#include "fj_internal.cuh"

#ifndef FJ_IDX_OK
#error "define FJ_IDX_OK (a bounds check with its translation unit's record) before including fj_tile.cuh"
#endif

namespace fj {

// Walk of one warp tile for k right-hand sides.  Lane j owns vectors j and
// j + 32.  Columns and weights are read 32 nonzeros at a time (one coalesced
// load per lane) and broadcast by shuffles; D gathers of the neighbours'
// k-vectors (contiguous in the node-major layout) are issued before any is
// consumed.  Rows are finished as the walk passes their ends, so short rows
// share load batches.  begin(x) is called when row x becomes current (to
// start its own loads early); src(c) gives the k-vector read for column c;
// add(acc, a, v) accumulates a * v, or add(acc, a, v, h) does, told the half
// h (0: vector lane, 1: vector lane + 32); apply(x, acc1, acc2) receives row
// x's sums.  A chunk of a long row (chunk = true) sums [k0, k1) of row r0 and
// calls apply once.
template <typename Acc, typename V, bool W, int D, typename Begin, typename Src, typename Add, typename Apply>
__device__ __forceinline__ void warp_tile_k(int64_t r0, int64_t r1, int64_t k0, int64_t k1, bool chunk,
                                            const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                            const float *__restrict__ w, Begin begin, Src src, Add add, Apply apply,
                                            int lane, bool has1, bool has2, int64_t n_rows)
{
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(32 % D == 0, "gather depth divides the load batch");
    // row ends of the tile (at most kWarpRows = 64 rows): lane i holds the ends of rows r0+i and r0+32+i
    int64_t e_lo = k1, e_hi = k1;
    if (!chunk) {
        if (r0 + lane < r1) e_lo = rp[r0 + lane + 1];
        if (r0 + 32 + lane < r1) e_hi = rp[r0 + 33 + lane];
    } else {
        r1 = r0 + 1;
    }
    int64_t x = r0;
    auto row_end = [&](int64_t xx) -> int64_t {
        const int i = (int)(xx - r0);
        return __shfl_sync(FULL, i < 32 ? e_lo : e_hi, i & 31);
    };
    int64_t xe = x < r1 ? row_end(x) : k1;
    if (x < r1) begin(x);
    Acc a1{}, a2{};
    auto flush_until = [&](int64_t pos) {
        while (x < r1 && xe <= pos) {
            apply(x, a1, a2);
            a1 = Acc{};
            a2 = Acc{};
            ++x;
            if (x < r1) {
                xe = row_end(x);
                begin(x);
            }
        }
    };
    for (int64_t base = k0; base < k1; base += 32) {
        const int64_t kk = base + lane;
        int32_t cl = 0;
        float al = 0.f;
        if (kk < k1) {
            cl = __ldg(col + kk);
            al = W ? __ldg(w + kk) : 1.f;
            if (!FJ_IDX_OK(15, cl, n_rows)) {
                cl = 0;
                al = 0.f;
            }
        }
        const int m = (int)(k1 - base < 32 ? k1 - base : 32);
        for (int t = 0; t < m; t += D) {
            V v1[D], v2[D];
            float aa[D];
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int32_t c = __shfl_sync(FULL, cl, (t + u) & 31);
                aa[u] = __shfl_sync(FULL, al, (t + u) & 31);
                const V *p = src(c);
                const bool in = t + u < m;
                v1[u] = (in && has1) ? __ldg(p + lane) : V(0);
                v2[u] = (in && has2) ? __ldg(p + lane + 32) : V(0);
            }
#pragma unroll
            for (int u = 0; u < D; ++u) {
                if (t + u < m) {
                    flush_until(base + t + u);
                    if constexpr (std::is_invocable_v<Add, Acc &, float, V, int>) {
                        add(a1, aa[u], v1[u], 0);
                        add(a2, aa[u], v2[u], 1);
                    } else {
                        add(a1, aa[u], v1[u]);
                        add(a2, aa[u], v2[u]);
                    }
                }
            }
        }
    }
    flush_until(k1);
}

}  // namespace fj
