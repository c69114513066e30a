// Learned warm start: a three-layer message-passing network predicting z0,
// from which the push solver starts (a push from any start reaches the same
// certificate, Lemmas 3 and 5).  The network has no counterpart in the paper.
//
//   x_v = [s_v, log(1 + d_v), log(1 + din_v), m_v],  m_v = sum_j a_vj s_j / d_v
//   h^l_v = relu(Ws^l^T h^{l-1}_v + Wn^l^T g^{l-1}_v + b^l),
//   g^{l-1}_v = sum_j a_vj h^{l-1}_j / d_v,  h^0 = x,  width 64,  l = 1, 2, 3
//   z0_v = b_v + w_o . h^3_v + b_o,  b_v = (s_v + d_v m_v) / (1 + d_v) (one
//   Jacobi step from s);   loss = mean_v (z0_v - z_v)^2
//
// Every dense product runs on the tensor cores (tcgen05.mma kind::f16, BF16
// operands, FP32 accumulation in tensor memory), one CTA per 128-row tile:
//   forward   D[128 nodes][64]   = [h | g] (K = 2 F_in, padded to 16) x W^T
//   backward  D[128 nodes][128]  = dq (K = 64) x [Ws | Wn]^T   (dh_self, dg)
//             D[128 feat][64]   += X^T dq over chunks of 128 nodes  (dW)
// with dq = bf16(dh * [h > 0]).  The aggregations (m, g and the adjoint of g)
// run over the graph's warp-tile plan (tiles of at most 64 rows and 512
// nonzeros, longer rows cut into 512-nonzero chunks), so a hub with 10^5
// neighbours is spread over many warps instead of serialising one; sums are
// FP32 (FP64 for m).  Parameters are FP32 (Adam state too); the GEMMs read
// BF16 copies packed once per update into the exact shared-memory image of
// their B operand.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fj_internal.cuh"
#include "fj_tc.cuh"

namespace fj {

constexpr int kHid = 64;
constexpr int kFin0 = 4;
constexpr int kTile = 128;  // rows per CTA tile (M of the MMA)
constexpr uint32_t kWaitLimit = 1u << 22;
// Dynamic shared memory of each GEMM kernel: its tiles, or more, so that the
// CTAs resident on one SM never hold more than the 512 tensor-memory columns
// (64 columns: at most 7 CTAs per SM; 128 columns: at most 4).
constexpr int kSmemFwd4 = 30 * 1024;   // tiles 6 KB, 64 columns
constexpr int kSmemFwd64 = 49 * 1024;  // tiles 48 KB, 64 columns
constexpr int kSmemDx = 57 * 1024;     // tiles 32 KB, 128 columns
constexpr int kSmemDw = 49 * 1024;     // tiles 48 KB, 64 columns

// Offsets of one layer's parameters in the flat FP32 vector.
struct LayerOff {
    int fin, ws, wn, b;
};

__host__ __device__ constexpr int layer_size(int fin) { return 2 * fin * kHid + kHid; }

static LayerOff layer_off(int l)
{
    int at = 0;
    for (int i = 0; i < l; ++i) at += layer_size(i == 0 ? kFin0 : kHid);
    const int fin = l == 0 ? kFin0 : kHid;
    return LayerOff{fin, at, at + fin * kHid, at + 2 * fin * kHid};
}

static int head_off() { return layer_size(kFin0) + 2 * layer_size(kHid); }
static int param_count() { return head_off() + kHid + 1; }

__device__ __forceinline__ float bf(__nv_bfloat16 x) { return __bfloat162float(x); }

// ---------------------------------------------------------------- packing

// B operand images in the K-major no-swizzle layout (fj_tc.cuh):
//   forward  [64 hidden][Kp] with element (n, k) = Ws[k][n] (k < F),
//            Wn[k - F][n] (F <= k < 2F), 0 beyond
//   backward [2F features][64] with element (f, h) = [Ws; Wn][f][h]
__global__ void k_pack_fwd(const float *__restrict__ theta, int ws, int wn, int fin, int kp,
                           __nv_bfloat16 *__restrict__ img)
{
    const int total = kHid * kp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int n = i / kp, k = i - n * kp;
        float v = 0.f;
        if (k < fin) v = theta[ws + k * kHid + n];
        else if (k < 2 * fin) v = theta[wn + (k - fin) * kHid + n];
        img[tc::kmajor_offset(n, k, kp) / 2] = __float2bfloat16_rn(v);
    }
}

__global__ void k_pack_bwd(const float *__restrict__ theta, int ws, int fin, __nv_bfloat16 *__restrict__ img)
{
    const int total = 2 * fin * kHid;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int f = i / kHid, h = i - f * kHid;
        // [Ws; Wn] is contiguous in theta: row f of the stacked matrix
        img[tc::kmajor_offset(f, h, kHid) / 2] = __float2bfloat16_rn(theta[ws + f * kHid + h]);
    }
}

// ---------------------------------------------------------------- aggregation over the warp-tile plan

constexpr int kShortAgg = 8;  // rows of at most this many nonzeros are summed by one lane

// m_v = sum_j a_vj s_j / d_v (FP64; 0 when d_v = 0).  Short rows one lane
// each, longer rows the whole warp; a chunk of a long row leaves its partial
// sum in part[] and the last chunk to finish completes the row.
__global__ void __launch_bounds__(256)
k_agg_s(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
        const int32_t *__restrict__ col, const float *__restrict__ w, const double *__restrict__ deg,
        const double *__restrict__ s, double *__restrict__ m, double *part, int32_t *cnt,
        const int32_t *__restrict__ slot_first, const int32_t *__restrict__ slot_nchunk, int64_t n, int *err)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto term = [&](int64_t k) -> double {
        const int32_t j = col[k];
        if (j < 0 || j >= n) {
            dev_error(err, DEV_BAD_COL);
            return 0.0;
        }
        return (w ? (double)w[k] : 1.0) * s[j];
    };
    auto finish = [&](int64_t x, double acc) {
        const float d = (float)deg[x];  // FP32 scale: m is rounded to bfloat16 / FP32 downstream
        m[x] = d > 0.f ? (double)((float)acc * __frcp_rn(d)) : 0.0;
    };
    for (int64_t ii = warp; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (r0 < 0 || r1 > n || r0 >= r1) continue;
        if (it.slot < 0) {
            for (int half = 0; half < 2; ++half) {
                const int64_t x = r0 + lane + 32 * half;
                const bool mine = x < r1;
                int64_t a = 0, e = 0;
                if (mine) {
                    a = rp[x];
                    e = rp[x + 1];
                }
                const bool shortrow = mine && e - a <= kShortAgg;
                if (shortrow) {
                    double acc = 0.0;
                    for (int64_t k = a; k < e; ++k) acc += term(k);
                    finish(x, acc);
                }
                unsigned longs = __ballot_sync(FULL, mine && !shortrow);
                while (longs) {
                    const int src = __ffs(longs) - 1;
                    longs &= longs - 1;
                    const int64_t al = __shfl_sync(FULL, a, src), el = __shfl_sync(FULL, e, src);
                    double acc = 0.0;
                    for (int64_t k = al + lane; k < el; k += 32) acc += term(k);
                    acc = warp_sum(acc);
                    if (lane == 0) finish(r0 + src + 32 * half, acc);
                }
            }
        } else {
            double acc = 0.0;
            for (int64_t k = it.k0 + lane; k < it.k1; k += 32) acc += term(k);
            acc = warp_sum(acc);
            const int slot = it.slot, first = slot_first[slot], nch = slot_nchunk[slot];
            const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
            if (lane == 0) {
                part[first + ci] = acc;
                __threadfence();
                if (atomicAdd(&cnt[slot], 1) == nch - 1) {
                    __threadfence();
                    double t = 0.0;
                    for (int c = 0; c < nch; ++c) t += __ldcg(part + first + c);
                    cnt[slot] = 0;
                    finish(r0, t);
                }
            }
        }
    }
}

// x_v in BF16 (4 per node) from s, the degrees and m; the base term b_v (FP32).
__global__ void k_features(int64_t n, const double *__restrict__ deg, const int32_t *__restrict__ indeg,
                           const double *__restrict__ s, const double *__restrict__ m, __nv_bfloat16 *__restrict__ x,
                           float *__restrict__ base)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const float d = (float)deg[v], sv = (float)s[v], mv = (float)m[v];
        base[v] = (sv + d * mv) * __frcp_rn(1.f + d);
        x[4 * v + 0] = __float2bfloat16_rn(sv);
        x[4 * v + 1] = __float2bfloat16_rn(log1pf(d));
        x[4 * v + 2] = __float2bfloat16_rn(log1pf((float)indeg[v]));
        x[4 * v + 3] = __float2bfloat16_rn(mv);
    }
}

// g_v = sum_j a_vj x_j / d_v for 4-wide BF16 rows (FP32 sums), layout as k_agg_s.
__global__ void __launch_bounds__(256)
k_agg4(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
       const int32_t *__restrict__ col, const float *__restrict__ w, const double *__restrict__ deg,
       const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ g, float *part, int32_t *cnt,
       const int32_t *__restrict__ slot_first, const int32_t *__restrict__ slot_nchunk, int64_t n, int *err)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto add = [&](int64_t k, float (&acc)[4]) {
        const int32_t j = col[k];
        if (j < 0 || j >= n) {
            dev_error(err, DEV_BAD_COL);
            return;
        }
        const float a = w ? w[k] : 1.f;
        const uint2 raw = *reinterpret_cast<const uint2 *>(x + 4 * (int64_t)j);
        const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
        const float2 q = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
        acc[0] += a * p.x;
        acc[1] += a * p.y;
        acc[2] += a * q.x;
        acc[3] += a * q.y;
    };
    auto finish = [&](int64_t v, const float (&acc)[4]) {
        const float d = (float)deg[v];
        const float inv = d > 0.f ? __frcp_rn(d) : 0.f;
        __nv_bfloat162 lo = __floats2bfloat162_rn(acc[0] * inv, acc[1] * inv);
        __nv_bfloat162 hi = __floats2bfloat162_rn(acc[2] * inv, acc[3] * inv);
        uint2 raw;
        raw.x = *reinterpret_cast<unsigned *>(&lo);
        raw.y = *reinterpret_cast<unsigned *>(&hi);
        *reinterpret_cast<uint2 *>(g + 4 * v) = raw;
    };
    for (int64_t ii = warp; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (r0 < 0 || r1 > n || r0 >= r1) continue;
        if (it.slot < 0) {
            for (int half = 0; half < 2; ++half) {
                const int64_t xr = r0 + lane + 32 * half;
                const bool mine = xr < r1;
                int64_t a = 0, e = 0;
                if (mine) {
                    a = rp[xr];
                    e = rp[xr + 1];
                }
                const bool shortrow = mine && e - a <= kShortAgg;
                if (shortrow) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int64_t k = a; k < e; ++k) add(k, acc);
                    finish(xr, acc);
                }
                unsigned longs = __ballot_sync(FULL, mine && !shortrow);
                while (longs) {
                    const int src = __ffs(longs) - 1;
                    longs &= longs - 1;
                    const int64_t al = __shfl_sync(FULL, a, src), el = __shfl_sync(FULL, e, src);
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int64_t k = al + lane; k < el; k += 32) add(k, acc);
#pragma unroll
                    for (int f = 0; f < 4; ++f) acc[f] = warp_sum(acc[f]);
                    if (lane == 0) finish(r0 + src + 32 * half, acc);
                }
            }
        } else {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int64_t k = it.k0 + lane; k < it.k1; k += 32) add(k, acc);
#pragma unroll
            for (int f = 0; f < 4; ++f) acc[f] = warp_sum(acc[f]);
            const int slot = it.slot, first = slot_first[slot], nch = slot_nchunk[slot];
            const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
            if (lane == 0) {
                for (int f = 0; f < 4; ++f) part[(int64_t)(first + ci) * 4 + f] = acc[f];
                __threadfence();
                if (atomicAdd(&cnt[slot], 1) == nch - 1) {
                    __threadfence();
                    float t[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int c = 0; c < nch; ++c)
                        for (int f = 0; f < 4; ++f) t[f] += __ldcg(part + (int64_t)(first + c) * 4 + f);
                    cnt[slot] = 0;
                    finish(r0, t);
                }
            }
        }
    }
}

// g_v = sum_j a_vj h_j / d_v for 64-wide BF16 rows: one warp per tile, rows in
// turn.  The warp is four slots of eight lanes; lane (slot, sub) loads the
// 16-byte part `sub` (features 8 sub .. 8 sub + 7) of neighbour row slot,
// slot + 4, ..., so one load instruction gathers four rows and four
// instructions (sixteen rows) are in flight.  The slots' FP32 sums are added
// by shuffles at the row's end.  A chunk of a long row leaves 64 FP32 partials.
__global__ void __launch_bounds__(256)
k_agg64(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
        const int32_t *__restrict__ col, const float *__restrict__ w, const double *__restrict__ deg,
        const __nv_bfloat16 *__restrict__ h, __nv_bfloat16 *__restrict__ g, float *part, int32_t *cnt,
        const int32_t *__restrict__ slot_first, const int32_t *__restrict__ slot_nchunk, int64_t n, int *err)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int U = 4;  // load instructions in flight per lane
    const int lane = threadIdx.x & 31, slot = lane >> 3, sub = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint4 *h4 = reinterpret_cast<const uint4 *>(h);  // 8 uint4 per row
    auto add8 = [](float (&acc)[8], uint4 v, float a) {
        const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(p[i]);
            acc[2 * i] += a * f.x;
            acc[2 * i + 1] += a * f.y;
        }
    };
    auto store8 = [](uint4 *dst, const float (&acc)[8], float scale) {
        uint4 o;
        __nv_bfloat162 *q = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = __floats2bfloat162_rn(acc[2 * i] * scale, acc[2 * i + 1] * scale);
        *dst = o;
    };
    for (int64_t ii = warp; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0;
        const bool chunk = it.slot >= 0;
        const int64_t r1 = chunk ? r0 + 1 : it.r1;
        if (r0 < 0 || r1 > n || r0 >= r1 || (!chunk && r1 - r0 > kWarpRows)) continue;
        for (int64_t x = r0; x < r1; ++x) {
            const int64_t a = chunk ? it.k0 : rp[x], e = chunk ? it.k1 : rp[x + 1];
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int64_t base = a; base < e; base += 32) {
                const int64_t kk = base + lane;
                int32_t cl = 0;
                float al = 0.f;
                if (kk < e) {
                    cl = col[kk];
                    al = w ? w[kk] : 1.f;
                    if (cl < 0 || cl >= n) {
                        dev_error(err, DEV_BAD_COL);
                        cl = 0;
                        al = 0.f;
                    }
                }
                const int m = (int)(e - base < 32 ? e - base : 32);
                for (int t = 0; t < m; t += 4 * U) {
                    uint4 v[U];
                    float aa[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int idx = t + 4 * u + slot;
                        const int32_t c = __shfl_sync(FULL, cl, idx & 31);
                        aa[u] = __shfl_sync(FULL, al, idx & 31);
                        v[u] = idx < m ? h4[(int64_t)c * 8 + sub] : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (t + 4 * u + slot < m) add8(acc, v[u], aa[u]);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[i] += __shfl_xor_sync(FULL, acc[i], 8);
                acc[i] += __shfl_xor_sync(FULL, acc[i], 16);
            }
            if (chunk) {
                const int slt = it.slot, first = slot_first[slt];
                const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
                if (slot == 0) {
                    float4 *pp = reinterpret_cast<float4 *>(part + (int64_t)(first + ci) * 64 + 8 * sub);
                    pp[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                    pp[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
                }
            } else if (slot == 0) {
                const float d = (float)deg[x];
                store8(reinterpret_cast<uint4 *>(g + x * 64) + sub, acc, d > 0.f ? __frcp_rn(d) : 0.f);
            }
        }
        if (chunk) {
            __threadfence();
            __syncwarp();
            const int slt = it.slot, first = slot_first[slt], nch = slot_nchunk[slt];
            int last = 0;
            if (lane == 0) last = atomicAdd(&cnt[slt], 1) == nch - 1;
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
                float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (slot == 0)
                    for (int c = 0; c < nch; ++c) {
                        const float4 *pp = reinterpret_cast<const float4 *>(part + (int64_t)(first + c) * 64 + 8 * sub);
                        const float4 p0 = __ldcg(pp), p1 = __ldcg(pp + 1);
                        acc[0] += p0.x; acc[1] += p0.y; acc[2] += p0.z; acc[3] += p0.w;
                        acc[4] += p1.x; acc[5] += p1.y; acc[6] += p1.z; acc[7] += p1.w;
                    }
                if (lane == 0) cnt[slt] = 0;
                if (slot == 0) {
                    const float d = (float)deg[r0];
                    store8(reinterpret_cast<uint4 *>(g + r0 * 64) + sub, acc, d > 0.f ? __frcp_rn(d) : 0.f);
                }
            }
        }
    }
}

// Adjoint of the 64-wide aggregation: dh[j] += (a_vj / d_v) dg[v] for every
// arc v -> j, scattered along the same tiles (atomic float2 adds).
__global__ void __launch_bounds__(256)
k_scatter64(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
            const int32_t *__restrict__ col, const float *__restrict__ w, const double *__restrict__ deg,
            const float *__restrict__ dg, float *__restrict__ dh, int64_t n, int *err)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ii = warp; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.slot >= 0 ? it.r0 + 1 : it.r1;
        if (r0 < 0 || r1 > n || r0 >= r1) continue;
        for (int64_t v = r0; v < r1; ++v) {
            const float d = (float)deg[v];
            if (!(d > 0.f)) continue;
            const float inv = __frcp_rn(d);
            float2 gv = reinterpret_cast<const float2 *>(dg + v * 64)[lane];
            gv.x *= inv;
            gv.y *= inv;
            const int64_t a = it.slot >= 0 ? it.k0 : rp[v], e = it.slot >= 0 ? it.k1 : rp[v + 1];
            for (int64_t base = a; base < e; base += 32) {
                const int64_t kk = base + lane;
                int32_t cl = -1;
                float al = 0.f;
                if (kk < e) {
                    cl = col[kk];
                    al = w ? w[kk] : 1.f;
                    if (cl < 0 || cl >= n) {
                        dev_error(err, DEV_BAD_COL);
                        cl = -1;
                    }
                }
                const int mm = (int)(e - base < 32 ? e - base : 32);
                for (int t = 0; t < mm; ++t) {
                    const int32_t c = __shfl_sync(FULL, cl, t);
                    const float aj = __shfl_sync(FULL, al, t);
                    if (c >= 0) atomicAdd(reinterpret_cast<float2 *>(dh + (int64_t)c * 64) + lane,
                                          make_float2(aj * gv.x, aj * gv.y));
                }
            }
        }
    }
}

// ---------------------------------------------------------------- common GEMM epilogue plumbing

// Allocates ncols tensor-memory columns (warp 0), initialises the mbarrier.
__device__ __forceinline__ void gemm_setup(uint32_t *tslot, uint64_t *bar, uint32_t ncols)
{
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tslot, ncols);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) tc::mbar_init(bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ __forceinline__ void gemm_teardown(uint32_t taddr, uint32_t ncols)
{
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(taddr, ncols);
}

// Thread 0 issues K / 16 MMAs over A (rows x K) and B (N x K) tiles at
// a_s / b_s and commits to bar; everyone waits (bounded) for that phase.
__device__ __forceinline__ bool gemm_run(uint32_t taddr, uint32_t a_s, uint32_t b_s, int K, uint32_t idesc,
                                         bool accumulate, uint64_t *bar, uint32_t parity)
{
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = tc::smem_desc(a_s + 256u * s, 128u, sbo);
            const uint64_t bd = tc::smem_desc(b_s + 256u * s, 128u, sbo);
            tc::mma_bf16(taddr, ad, bd, idesc, accumulate || s > 0);
        }
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait_bounded(bar, parity, kWaitLimit);
    tc::fence_after_sync();
    return ok;
}

// ---------------------------------------------------------------- forward layer

// One layer on a tile of 128 nodes: stage [h_v | g_v] (BF16, g from the
// aggregation pass) and the packed weights, one MMA chain, epilogue
// relu(D + b) -> h_out (BF16); the last layer also writes
// z0 = base + w_o . h + b_o.
template <int FIN, bool LAST>
__global__ void __launch_bounds__(128)
k_layer_fwd(int64_t n, const __nv_bfloat16 *__restrict__ h_in, const __nv_bfloat16 *__restrict__ g_in,
            const __nv_bfloat16 *__restrict__ img, const float *__restrict__ bias, const float *__restrict__ head,
            const float *__restrict__ base, __nv_bfloat16 *__restrict__ h_out, float *__restrict__ z0, int *err)
{
    constexpr int KP = FIN == kFin0 ? 16 : 2 * FIN;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sa = smem;                        // 128 x KP
    unsigned char *sb = smem + kTile * KP * 2;       // 64 x KP
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kTile;
    gemm_setup(&tslot, &bar, 64);
    const uint32_t taddr = tslot;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(img);
        uint4 *dst = reinterpret_cast<uint4 *>(sb);
        for (int i = threadIdx.x; i < kHid * KP * 2 / 16; i += 128) dst[i] = src[i];
    }
    if constexpr (FIN == kFin0) {
        // row t: [x (8 bytes) | g (8 bytes)] in K group 0, zeros in K group 1
        const int64_t v = r0 + threadIdx.x;
        uint4 row = make_uint4(0, 0, 0, 0);
        if (v < n) {
            const uint2 xs = *reinterpret_cast<const uint2 *>(h_in + 4 * v);
            const uint2 gs = *reinterpret_cast<const uint2 *>(g_in + 4 * v);
            row = make_uint4(xs.x, xs.y, gs.x, gs.y);
        }
        *reinterpret_cast<uint4 *>(sa + tc::kmajor_offset(threadIdx.x, 0, KP)) = row;
        *reinterpret_cast<uint4 *>(sa + tc::kmajor_offset(threadIdx.x, 8, KP)) = make_uint4(0, 0, 0, 0);
    } else {
        // warp per row, lane l: features 2l, 2l + 1 of h and of g
        for (int rr = wid; rr < kTile; rr += 4) {
            const int64_t v = r0 + rr;
            __nv_bfloat162 self2 = __floats2bfloat162_rn(0.f, 0.f), agg2 = self2;
            if (v < n) {
                self2 = reinterpret_cast<const __nv_bfloat162 *>(h_in + v * FIN)[lane];
                agg2 = reinterpret_cast<const __nv_bfloat162 *>(g_in + v * FIN)[lane];
            }
            *reinterpret_cast<__nv_bfloat162 *>(sa + tc::kmajor_offset(rr, 2 * lane, KP)) = self2;
            *reinterpret_cast<__nv_bfloat162 *>(sa + tc::kmajor_offset(rr, FIN + 2 * lane, KP)) = agg2;
        }
    }
    const bool ok = gemm_run(taddr, tc::smem_addr(sa), tc::smem_addr(sb), KP, tc::idesc_bf16_f32(kTile, kHid), false,
                             &bar, 0);
    if (!ok && threadIdx.x == 0) dev_error(err, DEV_SPIN_TIMEOUT);
    // epilogue: thread t of warp w holds row 32 w + t
    const int64_t v = r0 + threadIdx.x;
    float zacc = 0.f;
#pragma unroll
    for (int c0 = 0; c0 < kHid; c0 += 16) {
        float acc[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * wid) << 16) + (uint32_t)c0, acc);
        tc::tmem_wait_ld();
        __align__(16) __nv_bfloat16 hb[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float pre = acc[i] + bias[c0 + i];
            hb[i] = __float2bfloat16_rn(pre > 0.f ? pre : 0.f);
            if (LAST) zacc += head[c0 + i] * bf(hb[i]);
        }
        if (v < n && ok) {
            uint4 *dst = reinterpret_cast<uint4 *>(h_out + v * kHid + c0);
            dst[0] = reinterpret_cast<const uint4 *>(hb)[0];
            dst[1] = reinterpret_cast<const uint4 *>(hb)[1];
        }
    }
    if (LAST && v < n) z0[v] = base[v] + zacc + head[kHid];
    gemm_teardown(taddr, 64);
}

// ---------------------------------------------------------------- loss and head gradient

// dz_v = 2 (z0_v - z_v) / n;  dh3_v = dz_v w_o (FP32);  grad w_o += dz_v h3_v;
// grad b_o += dz_v;  loss += (z0_v - z_v)^2 / n.  Warp per node, lanes over
// features.
__global__ void __launch_bounds__(256)
k_loss_head(int64_t n, const float *__restrict__ z0, const double *__restrict__ z, const __nv_bfloat16 *__restrict__ h3,
            const float *__restrict__ wo, float *__restrict__ dh, float *__restrict__ gwo, double *__restrict__ loss)
{
    __shared__ float sw[8][kHid + 1];
    __shared__ double sl[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float g0 = 0.f, g1 = 0.f, gb = 0.f;
    double l = 0.0;
    const float w0 = wo[2 * lane], w1 = wo[2 * lane + 1];
    for (int64_t v = warp; v < n; v += nwarps) {
        const double diff = (double)z0[v] - z[v];
        const float dz = (float)(2.0 * diff / (double)n);
        const float2 hv = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(h3 + v * kHid)[lane]);
        reinterpret_cast<float2 *>(dh + v * kHid)[lane] = make_float2(dz * w0, dz * w1);
        g0 += dz * hv.x;
        g1 += dz * hv.y;
        if (lane == 0) {
            gb += dz;
            l += diff * diff / (double)n;
        }
    }
    sw[wid][2 * lane] = g0;
    sw[wid][2 * lane + 1] = g1;
    if (lane == 0) {
        sw[wid][kHid] = gb;
        sl[wid] = l;
    }
    __syncthreads();
    if (threadIdx.x <= kHid) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += sw[i][threadIdx.x];
        atomicAdd(&gwo[threadIdx.x], t);
    }
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sl[i];
        atomicAdd(loss, t);
    }
}

// ---------------------------------------------------------------- backward: dX = dq [Ws | Wn]^T

// Tile of 128 nodes: dq = bf16(dh * [h > 0]) (K = 64) times the backward image
// (N = 128); columns 0..63 (the gradient through h_v itself) overwrite the
// tile's rows of dh in place (each tile reads its rows before the MMA), columns
// 64..127 (the gradient of g) go to dg.
__global__ void __launch_bounds__(128)
k_layer_dx(int64_t n, float *dh, const __nv_bfloat16 *__restrict__ h, const __nv_bfloat16 *__restrict__ img,
           float *__restrict__ dg, int *err)
{
    constexpr int K = kHid, N = 2 * kHid;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sa = smem;                  // 128 x 64
    unsigned char *sb = smem + kTile * K * 2;  // 128 x 64
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kTile;
    gemm_setup(&tslot, &bar, 128);
    const uint32_t taddr = tslot;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(img);
        uint4 *dst = reinterpret_cast<uint4 *>(sb);
        for (int i = threadIdx.x; i < N * K * 2 / 16; i += 128) dst[i] = src[i];
    }
    for (int rr = wid; rr < kTile; rr += 4) {
        const int64_t v = r0 + rr;
        __nv_bfloat162 q = __floats2bfloat162_rn(0.f, 0.f);
        if (v < n) {
            const float2 g = reinterpret_cast<const float2 *>(dh + v * kHid)[lane];
            const float2 hv = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(h + v * kHid)[lane]);
            q = __floats2bfloat162_rn(hv.x > 0.f ? g.x : 0.f, hv.y > 0.f ? g.y : 0.f);
        }
        *reinterpret_cast<__nv_bfloat162 *>(sa + tc::kmajor_offset(rr, 2 * lane, K)) = q;
    }
    const bool ok = gemm_run(taddr, tc::smem_addr(sa), tc::smem_addr(sb), K, tc::idesc_bf16_f32(kTile, N), false,
                             &bar, 0);
    if (!ok && threadIdx.x == 0) dev_error(err, DEV_SPIN_TIMEOUT);
    const int64_t v = r0 + threadIdx.x;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float acc[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * wid) << 16) + (uint32_t)c0, acc);
        tc::tmem_wait_ld();
        if (v < n && ok) {
            float *dst = c0 < kHid ? dh + v * kHid + c0 : dg + v * kHid + (c0 - kHid);
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4 *>(dst + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
        }
    }
    gemm_teardown(taddr, 128);
}

// ---------------------------------------------------------------- backward: dW = X^T dq, db

// Chunks of 128 nodes, grid-strided: A = X^T (128 feature rows, rows >= 2F
// zero; K = the chunk's nodes), B = dq^T (64 hidden rows; K = nodes), the
// product accumulating in tensor memory across the CTA's chunks; then one
// atomic per element into grad [Ws; Wn].  db = sum of the FP32 dpre.
template <int FIN>
__global__ void __launch_bounds__(128)
k_layer_dw(int64_t n, const __nv_bfloat16 *__restrict__ h_in, const __nv_bfloat16 *__restrict__ g_in,
           const float *__restrict__ dh, const __nv_bfloat16 *__restrict__ h, float *__restrict__ gw,
           float *__restrict__ gb, int *err)
{
    constexpr int KC = kTile;  // nodes per chunk
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float sdb[kHid];
    unsigned char *sa = smem;                   // 128 features x KC
    unsigned char *sb = smem + kTile * KC * 2;  // 64 hidden x KC
    const int64_t nchunks = (n + KC - 1) / KC;
    if ((int64_t)blockIdx.x >= nchunks) return;
    gemm_setup(&tslot, &bar, 64);
    const uint32_t taddr = tslot;
    const int t = threadIdx.x, wid = t >> 5;
    if (t < kHid) sdb[t] = 0.f;
    // rows 2F..127 of A stay zero for every chunk
    for (int i = t; i < kTile * KC * 2 / 16; i += 128) reinterpret_cast<uint4 *>(sa)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    float db[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i) db[i] = 0.f;
    uint32_t parity = 0;
    bool ok = true, first = true;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t v = c * KC + t;  // this thread's node (column t of both operands)
        const bool in = v < n;
        // A column t: features of node v
#pragma unroll 4
        for (int f = 0; f < FIN; ++f) {
            const __nv_bfloat16 a = in ? h_in[v * FIN + f] : __float2bfloat16_rn(0.f);
            const __nv_bfloat16 b = in ? g_in[v * FIN + f] : __float2bfloat16_rn(0.f);
            *reinterpret_cast<__nv_bfloat16 *>(sa + tc::kmajor_offset(f, t, KC)) = a;
            *reinterpret_cast<__nv_bfloat16 *>(sa + tc::kmajor_offset(FIN + f, t, KC)) = b;
        }
        // B column t: dq of node v
#pragma unroll 8
        for (int hh = 0; hh < kHid; ++hh) {
            float d = 0.f;
            if (in && bf(h[v * kHid + hh]) > 0.f) d = dh[v * kHid + hh];
            db[hh] += d;
            *reinterpret_cast<__nv_bfloat16 *>(sb + tc::kmajor_offset(hh, t, KC)) = __float2bfloat16_rn(d);
        }
        const bool run_ok = gemm_run(taddr, tc::smem_addr(sa), tc::smem_addr(sb), KC, tc::idesc_bf16_f32(kTile, kHid),
                                     !first, &bar, parity);
        ok = __syncthreads_and(run_ok && ok) != 0;  // uniform across the CTA
        parity ^= 1u;
        first = false;
        if (!ok) break;
    }
    if (!ok && t == 0) dev_error(err, DEV_SPIN_TIMEOUT);
    // db: reduce over the CTA's threads
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        float x = db[i];
        x = warp_sum(x);
        if ((t & 31) == 0) atomicAdd(&sdb[i], x);
    }
    // D row r = feature r (thread t holds row t): rows < 2F go to grad [Ws; Wn]
#pragma unroll
    for (int c0 = 0; c0 < kHid; c0 += 16) {
        float acc[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * wid) << 16) + (uint32_t)c0, acc);
        tc::tmem_wait_ld();
        if (ok && t < 2 * FIN)
#pragma unroll
            for (int i = 0; i < 16; ++i) atomicAdd(&gw[t * kHid + c0 + i], acc[i]);
    }
    __syncthreads();
    if (t < kHid) atomicAdd(&gb[t], sdb[t]);
    gemm_teardown(taddr, 64);
}

// ---------------------------------------------------------------- Adam, clamp

__global__ void k_adam(int np, float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// z0 (FP32) -> FP64 output: clamped to [min s, max s] (the range comes from the
// order keys reduced by k_range), except that a node that listens to nobody
// (d_v = 0) takes its own opinion, its exact equilibrium value.
__device__ __forceinline__ unsigned long long okey(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double okey_inv(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
    return __longlong_as_double((long long)b);
}

__global__ void k_range(int64_t n, const double *__restrict__ s, unsigned long long *mm)
{
    unsigned long long lo = ~0ULL, hi = 0ULL;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = okey(s[v]);
        lo = k < lo ? k : lo;
        hi = k > hi ? k : hi;
    }
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
}

__global__ void k_clamp_out(int64_t n, const float *__restrict__ z0, const unsigned long long *__restrict__ mm,
                            const double *__restrict__ deg, const double *__restrict__ s, double *__restrict__ out)
{
    const double lo = okey_inv(mm[0]), hi = okey_inv(mm[1]);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)z0[v];
        out[v] = deg[v] > 0.0 ? (x < lo ? lo : (x > hi ? hi : x)) : s[v];
    }
}

}  // namespace fj

using namespace fj;

// ---------------------------------------------------------------- handle

struct fj_mpnn {
    int device = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *img_fwd[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *img_bwd[3] = {nullptr, nullptr, nullptr};
    int64_t step = 0;
    bool have_grad = false;
    // activations, grown on demand
    int64_t cap = 0;
    __nv_bfloat16 *x = nullptr, *g0 = nullptr;          // n x 4
    __nv_bfloat16 *h[3] = {nullptr, nullptr, nullptr};  // n x 64
    __nv_bfloat16 *g[2] = {nullptr, nullptr};           // n x 64 (inputs of layers 2, 3)
    float *z0 = nullptr;
    double *mv = nullptr;                               // n: m_v
    float *base = nullptr;                              // n: one Jacobi step from s
    int64_t cap_part = 0;
    float *part = nullptr;                              // per long-row chunk: 64 partial sums
    int64_t cap_bwd = 0;
    float *dh = nullptr, *dg = nullptr;                 // n x 64
    double *sin = nullptr, *zin = nullptr, *zout = nullptr;  // host staging
    int64_t cap_stage = 0;
    double *loss = nullptr;
    unsigned long long *mm = nullptr;
    int *err = nullptr;
};

namespace {

fj_status mpnn_check(fj_mpnn *m, cudaStream_t st)
{
    int h = 0;
    FJ_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    if (h) {
        FJ_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), st));
        set_error("network kernel reported device error %d", h);
        return h == DEV_SPIN_TIMEOUT ? FJ_ERR_TIMEOUT : FJ_ERR_INVALID_ARG;
    }
    return FJ_OK;
}

fj_status pack_all(fj_mpnn *m, cudaStream_t st)
{
    for (int l = 0; l < 3; ++l) {
        const LayerOff o = layer_off(l);
        const int kp = o.fin == kFin0 ? 16 : 2 * o.fin;
        k_pack_fwd<<<grid_for(kHid * kp, 256), 256, 0, st>>>(m->theta, o.ws, o.wn, o.fin, kp, m->img_fwd[l]);
        if (l > 0) k_pack_bwd<<<grid_for(2 * o.fin * kHid, 256), 256, 0, st>>>(m->theta, o.ws, o.fin, m->img_bwd[l]);
    }
    FJ_CUDA(cudaGetLastError());
    return FJ_OK;
}

template <typename T>
fj_status grow(T **p, int64_t count)
{
    dev_free(*p);
    *p = nullptr;
    FJ_CUDA(dev_malloc(p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)));
    return FJ_OK;
}

fj_status ensure_fwd(fj_mpnn *m, int64_t n)
{
    if (n <= m->cap) return FJ_OK;
    m->cap = 0;  // stays 0 if an allocation fails, so the next call grows again
    FJ_CHECK(grow(&m->x, 4 * n));
    FJ_CHECK(grow(&m->g0, 4 * n));
    for (auto &p : m->h) FJ_CHECK(grow(&p, kHid * n));
    for (auto &p : m->g) FJ_CHECK(grow(&p, kHid * n));
    FJ_CHECK(grow(&m->z0, n));
    FJ_CHECK(grow(&m->mv, n));
    FJ_CHECK(grow(&m->base, n));
    m->cap = n;
    return FJ_OK;
}

fj_status ensure_bwd(fj_mpnn *m, int64_t n)
{
    if (n <= m->cap_bwd) return FJ_OK;
    m->cap_bwd = 0;
    FJ_CHECK(grow(&m->dh, kHid * n));
    FJ_CHECK(grow(&m->dg, kHid * n));
    m->cap_bwd = n;
    return FJ_OK;
}

fj_status stage(fj_mpnn *m, int64_t n, const double *src, double **dst_slot, const double **out, int mem,
                cudaStream_t st)
{
    if (mem == FJ_MEM_DEVICE || src == nullptr) {
        *out = src;
        return FJ_OK;
    }
    if (n > m->cap_stage) {
        m->cap_stage = 0;
        FJ_CHECK(grow(&m->sin, n));
        FJ_CHECK(grow(&m->zin, n));
        FJ_CHECK(grow(&m->zout, n));
        m->cap_stage = n;
    }
    FJ_CUDA(cudaMemcpyAsync(*dst_slot, src, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    *out = *dst_slot;
    return FJ_OK;
}

// Forward pass (every activation stays for the backward pass).
fj_status forward(fj_mpnn *m, fj_graph *g, const double *sd, cudaStream_t st)
{
    const DevCSR &c = g->csr;
    const int64_t n = c.n;
    FJ_CHECK(ensure_fwd(m, n));
    const ItemPlan *ip = nullptr;
    FJ_CHECK(plain_items(g, st, &ip));
    if (ip->nparts * 64 > m->cap_part) {
        m->cap_part = 0;
        FJ_CHECK(grow(&m->part, ip->nparts * 64));
        m->cap_part = ip->nparts * 64;
    }
    const unsigned agrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ip->nitems, 8), 152 * 8));
    k_agg_s<<<agrid, 256, 0, st>>>(ip->items, ip->nitems, c.row_ptr, c.col, c.w, c.deg64, sd, m->mv, ip->part,
                                   ip->cnt, ip->slot_first, ip->slot_nchunk, n, m->err);
    k_features<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, c.deg64, c.indeg, sd, m->mv, m->x, m->base);
    k_agg4<<<agrid, 256, 0, st>>>(ip->items, ip->nitems, c.row_ptr, c.col, c.w, c.deg64, m->x, m->g0, m->part,
                                  ip->cnt, ip->slot_first, ip->slot_nchunk, n, m->err);
    const unsigned tiles = (unsigned)std::max<int64_t>(1, (n + kTile - 1) / kTile);
    const float *th = m->theta;
    const int ho = head_off();
    k_layer_fwd<kFin0, false><<<tiles, 128, kSmemFwd4, st>>>(n, m->x, m->g0, m->img_fwd[0], th + layer_off(0).b,
                                                             th + ho, m->base, m->h[0], m->z0, m->err);
    for (int l = 1; l < 3; ++l) {
        k_agg64<<<agrid, 256, 0, st>>>(ip->items, ip->nitems, c.row_ptr, c.col, c.w, c.deg64, m->h[l - 1],
                                       m->g[l - 1], m->part, ip->cnt, ip->slot_first, ip->slot_nchunk, n, m->err);
        if (l == 1)
            k_layer_fwd<kHid, false><<<tiles, 128, kSmemFwd64, st>>>(n, m->h[0], m->g[0], m->img_fwd[1],
                                                                    th + layer_off(1).b, th + ho, m->base, m->h[1],
                                                                    m->z0, m->err);
        else
            k_layer_fwd<kHid, true><<<tiles, 128, kSmemFwd64, st>>>(n, m->h[1], m->g[1], m->img_fwd[2],
                                                                   th + layer_off(2).b, th + ho, m->base, m->h[2],
                                                                   m->z0, m->err);
    }
    FJ_CUDA(cudaGetLastError());
    return FJ_OK;
}

bool g_attrs_set[64] = {};

fj_status set_attrs(int dev)
{
    if (dev >= 0 && dev < 64 && g_attrs_set[dev]) return FJ_OK;
    FJ_CUDA(cudaFuncSetAttribute(k_layer_fwd<kFin0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd4));
    FJ_CUDA(cudaFuncSetAttribute(k_layer_fwd<kHid, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd64));
    FJ_CUDA(cudaFuncSetAttribute(k_layer_fwd<kHid, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd64));
    FJ_CUDA(cudaFuncSetAttribute(k_layer_dx, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDx));
    FJ_CUDA(cudaFuncSetAttribute(k_layer_dw<kFin0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDw));
    FJ_CUDA(cudaFuncSetAttribute(k_layer_dw<kHid>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDw));
    if (dev >= 0 && dev < 64) g_attrs_set[dev] = true;
    return FJ_OK;
}

}  // namespace

extern "C" {

int64_t fj_mpnn_param_count(void) { return param_count(); }

fj_status fj_mpnn_create(const float *params, fj_mpnn **out)
{
    FJ_ARG(params != nullptr && out != nullptr, "NULL pointer");
    *out = nullptr;
    fj_mpnn *m = new fj_mpnn();
    const int np = param_count();
    auto fail = [&](fj_status s) {
        fj_mpnn_destroy(m);
        return s;
    };
    if (cudaGetDevice(&m->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "device", __FILE__, __LINE__));
    fj_status s = set_attrs(m->device);
    if (s != FJ_OK) return fail(s);
    float **fb[] = {&m->theta, &m->m, &m->v, &m->grad};
    for (float **p : fb)
        if ((s = grow(p, np)) != FJ_OK) return fail(s);
    for (int l = 0; l < 3; ++l) {
        const LayerOff o = layer_off(l);
        const int kp = o.fin == kFin0 ? 16 : 2 * o.fin;
        if ((s = grow(&m->img_fwd[l], kHid * kp)) != FJ_OK) return fail(s);
        if ((s = grow(&m->img_bwd[l], 2 * o.fin * kHid)) != FJ_OK) return fail(s);
    }
    if ((s = grow(&m->loss, 1)) != FJ_OK) return fail(s);
    if ((s = grow(&m->mm, 2)) != FJ_OK) return fail(s);
    if ((s = grow(&m->err, 1)) != FJ_OK) return fail(s);
    if (cudaMemcpy(m->theta, params, sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m, 0, sizeof(float) * np) != cudaSuccess || cudaMemset(m->v, 0, sizeof(float) * np) != cudaSuccess ||
        cudaMemset(m->grad, 0, sizeof(float) * np) != cudaSuccess || cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "network init", __FILE__, __LINE__));
    if ((s = pack_all(m, nullptr)) != FJ_OK) return fail(s);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "network init", __FILE__, __LINE__));
    *out = m;
    return FJ_OK;
}

void fj_mpnn_destroy(fj_mpnn *m)
{
    if (!m) return;
    dev_free(m->theta); dev_free(m->m); dev_free(m->v); dev_free(m->grad);
    for (auto p : m->img_fwd) dev_free(p);
    for (auto p : m->img_bwd) dev_free(p);
    dev_free(m->x); dev_free(m->g0); dev_free(m->z0);
    for (auto p : m->h) dev_free(p);
    for (auto p : m->g) dev_free(p);
    dev_free(m->dh); dev_free(m->dg); dev_free(m->mv); dev_free(m->part); dev_free(m->base);
    dev_free(m->sin); dev_free(m->zin); dev_free(m->zout);
    dev_free(m->loss); dev_free(m->mm); dev_free(m->err);
    delete m;
}

fj_status fj_mpnn_get_params(const fj_mpnn *m, float *params)
{
    FJ_ARG(m && params, "NULL pointer");
    FJ_CUDA(cudaMemcpy(params, m->theta, sizeof(float) * param_count(), cudaMemcpyDeviceToHost));
    return FJ_OK;
}

fj_status fj_mpnn_set_params(fj_mpnn *m, const float *params)
{
    FJ_ARG(m && params, "NULL pointer");
    FJ_CUDA(cudaMemcpy(m->theta, params, sizeof(float) * param_count(), cudaMemcpyHostToDevice));
    FJ_CHECK(pack_all(m, nullptr));
    FJ_CUDA(cudaDeviceSynchronize());
    return FJ_OK;
}

fj_status fj_mpnn_predict(fj_mpnn *m, fj_graph *g, const double *s, double *z0, int mem, void *stream)
{
    FJ_ARG(m && g && s && z0, "NULL pointer");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g->csr.n;
    const double *sd = nullptr;
    FJ_CHECK(stage(m, n, s, &m->sin, &sd, mem, st));
    FJ_CHECK(forward(m, g, sd, st));
    const unsigned long long init[2] = {~0ULL, 0ULL};
    FJ_CUDA(cudaMemcpyAsync(m->mm, init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_range<<<grid_for(n, 256, 152 * 4), 256, 0, st>>>(n, sd, m->mm);
    double *dst = mem == FJ_MEM_DEVICE ? z0 : nullptr;
    if (!dst) {
        if (n > m->cap_stage) {
            m->cap_stage = 0;
            FJ_CHECK(grow(&m->sin, n));
            FJ_CHECK(grow(&m->zin, n));
            FJ_CHECK(grow(&m->zout, n));
            m->cap_stage = n;
        }
        dst = m->zout;
    }
    k_clamp_out<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, m->z0, m->mm, g->csr.deg64, sd, dst);
    FJ_CUDA(cudaGetLastError());
    if (mem == FJ_MEM_HOST) FJ_CUDA(cudaMemcpyAsync(z0, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    return mpnn_check(m, st);
}

fj_status fj_mpnn_grad(fj_mpnn *m, fj_graph *g, const double *s, const double *z, double *loss, float *grad,
                       int mem, void *stream)
{
    FJ_ARG(m && g && s && z, "NULL pointer");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    cudaStream_t st = (cudaStream_t)stream;
    const DevCSR &c = g->csr;
    const int64_t n = c.n;
    FJ_ARG(n > 0, "empty graph");
    const double *sd = nullptr, *zd = nullptr;
    FJ_CHECK(stage(m, n, s, &m->sin, &sd, mem, st));
    FJ_CHECK(stage(m, n, z, &m->zin, &zd, mem, st));
    FJ_CHECK(ensure_bwd(m, n));
    FJ_CHECK(forward(m, g, sd, st));
    const int np = param_count();
    FJ_CUDA(cudaMemsetAsync(m->grad, 0, sizeof(float) * np, st));
    FJ_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), st));
    const int ho = head_off();
    k_loss_head<<<grid_for(n * 32, 256, 152 * 8), 256, 0, st>>>(n, m->z0, zd, m->h[2], m->theta + ho, m->dh,
                                                                m->grad + ho, m->loss);
    const ItemPlan *ip = nullptr;
    FJ_CHECK(plain_items(g, st, &ip));
    const unsigned agrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ip->nitems, 8), 152 * 8));
    const unsigned tiles = (unsigned)std::max<int64_t>(1, (n + kTile - 1) / kTile);
    const unsigned dwgrid = (unsigned)std::min<int64_t>(tiles, 152 * 3);
    for (int l = 2; l >= 0; --l) {
        const LayerOff o = layer_off(l);
        const __nv_bfloat16 *hin = l == 0 ? m->x : m->h[l - 1];
        const __nv_bfloat16 *gin = l == 0 ? m->g0 : m->g[l - 1];
        if (l == 0)
            k_layer_dw<kFin0><<<dwgrid, 128, kSmemDw, st>>>(n, hin, gin, m->dh, m->h[l], m->grad + o.ws,
                                                              m->grad + o.b, m->err);
        else
            k_layer_dw<kHid><<<dwgrid, 128, kSmemDw, st>>>(n, hin, gin, m->dh, m->h[l], m->grad + o.ws,
                                                             m->grad + o.b, m->err);
        if (l > 0) {
            // dh <- gradient through h_{l-1} itself, then + the adjoint of the aggregation
            k_layer_dx<<<tiles, 128, kSmemDx, st>>>(n, m->dh, m->h[l], m->img_bwd[l], m->dg, m->err);
            k_scatter64<<<agrid, 256, 0, st>>>(ip->items, ip->nitems, c.row_ptr, c.col, c.w, c.deg64, m->dg, m->dh,
                                               n, m->err);
        }
        FJ_CUDA(cudaGetLastError());
    }
    double hl = 0.0;
    FJ_CUDA(cudaMemcpyAsync(&hl, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad) FJ_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * np, cudaMemcpyDeviceToHost, st));
    FJ_CHECK(mpnn_check(m, st));
    if (loss) *loss = hl;
    m->have_grad = true;
    return FJ_OK;
}

fj_status fj_mpnn_adam_step(fj_mpnn *m, double lr, void *stream)
{
    FJ_ARG(m != nullptr, "NULL pointer");
    FJ_ARG(m->have_grad, "no gradient: call fj_mpnn_grad first");
    FJ_ARG(lr > 0.0 && lr < 1.0, "lr must be in (0, 1)");
    cudaStream_t st = (cudaStream_t)stream;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(0.9, (double)m->step), c2 = 1.f - (float)std::pow(0.999, (double)m->step);
    const int np = param_count();
    k_adam<<<grid_for(np, 256), 256, 0, st>>>(np, m->theta, m->m, m->v, m->grad, (float)lr, b1, b2, 1e-8f, c1, c2);
    FJ_CUDA(cudaGetLastError());
    FJ_CHECK(pack_all(m, st));
    m->have_grad = false;
    return FJ_OK;
}

}  // extern "C"
