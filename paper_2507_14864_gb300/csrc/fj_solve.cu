// The FJ push solver on the GPU: ImprovedBLISOR (Alg. 2 + Alg. 3) with the
// pushes of a sweep applied class by class (Gauss-Seidel order, Theorem 2) or
// as synchronous rounds, an FP64 certificate (Lemmas 3-5) and FP64 restarts.
//
// State per node u (shifted system s' = s + c_eff, Alg. 2):
//   r_u     residual of s' - (I + L) zhat'          (T = float or double)
//   h_u     threshold eps' s'_u                      (T; FP32 rounded down)
//   delta_u last push increment of u, kept in two buffers (this sweep's and
//           the previous one's) until every in-neighbour has pulled it
//   zhat_u  estimate of z'_u                         (FP64)
// With d_u the weighted out-degree, a push of u (Eqs. sor1-sor3) is
// delta = omega r_u / (1 + d_u), zhat_u += delta, r_u <- (1 - omega) r_u, and
// r_x += a_xu delta for every x with a_xu > 0.  The kernels apply the last
// step in pull form: when row x is visited it adds sum_j a_xj delta_j over
// its row.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fj_tc.cuh"
#include "fj_internal.cuh"

namespace fj {

// ============================================================== small kernels

__device__ __forceinline__ unsigned long long order_key(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

__host__ __device__ inline double order_key_inv(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

// gstat layout per graph (8 words): 0 min-s order key, 1 c_eff, 2 resid_inf,
// 3 resid_rel, 4 z_inf, 5 violators, 6 non-finite count, 7 spare.
constexpr int kGs = 8;

__global__ void k_gstat_reset(int ng, unsigned long long *gs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng * kGs; i += gridDim.x * blockDim.x)
        gs[i] = (i % kGs == 0) ? ~0ULL : 0ULL;
}

// Per-graph minimum of s (original order; graphs are contiguous id ranges)
// and a finiteness check.  Each thread scans a contiguous chunk and flushes
// one atomic per graph it meets.
__global__ void k_min_s(int64_t n, const double *__restrict__ s, const int32_t *__restrict__ graph_of,
                        unsigned long long *gs, int *err)
{
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t chunk = ceil_div(n, nt);
    int64_t a = t * chunk, b = min(n, a + chunk);
    if (a >= b) return;
    int gcur = graph_of ? graph_of[a] : 0;
    unsigned long long best = ~0ULL;
    for (int64_t v = a; v < b; ++v) {
        double x = s[v];
        if (!isfinite(x)) dev_error(err, DEV_BAD_OPINION);
        int gv = graph_of ? graph_of[v] : 0;
        if (gv != gcur) {
            atomicMin(&gs[(int64_t)gcur * kGs], best);
            best = ~0ULL;
            gcur = gv;
        }
        unsigned long long k = order_key(x);
        best = k < best ? k : best;
    }
    atomicMin(&gs[(int64_t)gcur * kGs], best);
}

// c_eff = c + max(0, -min s) per graph (Alg. 2 shift, extended to signed s).
__global__ void k_shift(int ng, unsigned long long *gs, double c)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    double mn = order_key_inv(gs[(int64_t)i * kGs]);
    double ce = c - (mn < 0.0 ? mn : 0.0);
    reinterpret_cast<double *>(gs)[(int64_t)i * kGs + 1] = ce;
}

template <typename T>
__device__ __forceinline__ T threshold_of(double x);
template <>
__device__ __forceinline__ float threshold_of<float>(double x) { return __double2float_rd(x); }
template <>
__device__ __forceinline__ double threshold_of<double>(double x) { return x; }

// Residual stored in the push precision with its magnitude rounded up, so a
// stored |r| below its threshold proves the FP64 residual is below it too.
template <typename T>
__device__ __forceinline__ T resid_store(double x);
template <>
__device__ __forceinline__ float resid_store<float>(double x)
{
    return x >= 0.0 ? __double2float_ru(x) : __double2float_rd(x);
}
template <>
__device__ __forceinline__ double resid_store<double>(double x) { return x; }

// Initial state over new ids i (o = perm[i] the caller's id): s', zhat, r, h,
// and the relaxation factor of node i: omega, lowered for a node with weight
// din_i to neighbours of its own colour class so that
// (2 / omega_i - 1)(1 + d_i) >= din_i / 0.98.
template <typename T>
__global__ void k_init(int64_t n, const double *__restrict__ s, const double *__restrict__ z0,
                       const int32_t *__restrict__ perm, const int32_t *__restrict__ graph_of,
                       const unsigned long long *__restrict__ gs, double epsp, double omega,
                       const double *__restrict__ deg, const double *__restrict__ din, double *__restrict__ sp,
                       double *__restrict__ zhat, T *__restrict__ r, T *__restrict__ h, T *__restrict__ da,
                       T *__restrict__ db, T *__restrict__ om)
{
    const double *gsd = reinterpret_cast<const double *>(gs);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = perm ? perm[i] : i;
        int gph = graph_of ? graph_of[i] : 0;
        double ce = gsd[(int64_t)gph * kGs + 1];
        double spv = s[o] + ce;
        sp[i] = spv;
        zhat[i] = z0 ? z0[o] + ce : 0.0;
        r[i] = (T)spv;
        h[i] = threshold_of<T>(epsp * spv);
        da[i] = T(0);
        db[i] = T(0);
        double oi = omega;
        if (din && din[i] > 0.0) {
            double bound = 0.98 * 2.0 * (1.0 + deg[i]) / (1.0 + deg[i] + din[i]);
            oi = fmin(omega, bound);
        }
        om[i] = (T)oi;
    }
}

// z_out[o] = zhat[i] - c_eff (Alg. 2's unshift), scattered back to caller ids.
__global__ void k_unshift(int64_t n, const double *__restrict__ zhat, const int32_t *__restrict__ perm,
                          const int32_t *__restrict__ graph_of, const unsigned long long *__restrict__ gs,
                          double *__restrict__ z)
{
    const double *gsd = reinterpret_cast<const double *>(gs);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = perm ? perm[i] : i;
        int gph = graph_of ? graph_of[i] : 0;
        z[o] = zhat[i] - gsd[(int64_t)gph * kGs + 1];
    }
}

__global__ void k_pass_reset(Counters *c, long long max_sweeps)
{
    c->done = 0;
    c->pass_sweeps = 0;
    c->sweep_pushes = 0;
    c->max_sweeps = max_sweeps;
    c->ticket = 0;
}

// End of a sweep (or round): stop when nothing was pushed, at the cap, or on
// a non-finite residual.
__global__ void k_end_sweep(Counters *c)
{
    c->ticket = 0;
    if (c->done) return;
    c->sweeps += 1;
    c->pass_sweeps += 1;
    if (c->nonfinite != 0.0) c->done = 3;
    else if (c->sweep_pushes == 0) c->done = 1;
    else if (c->pass_sweeps >= c->max_sweeps) c->done = 2;
    c->sweep_pushes = 0;
    c->ticket = 0;
}

// ============================================================== helpers

template <typename T, bool W>
__device__ __forceinline__ T arc_w(const float *__restrict__ w, int64_t k)
{
    if constexpr (W) return (T)__ldg(w + k);
    else return T(1);
}

// ============================================================== push round

// Bounds-checked indexing: the sweep and certificate kernels verify every
// row, block and column index against its array before using it.  The first
// index out of range is stored here as (site, block, index, limit), the access
// is skipped, and the host turns the record into an error.  The checks cost one
// compare per nonzero in kernels that are bound by memory traffic.
__device__ long long g_fj_dbg[4];
#define FJ_IDX_OK(site, idx, lim) FJ_IDX_OK_REC(g_fj_dbg, site, idx, lim)
}  // namespace fj
#include "fj_tile.cuh"
namespace fj {

// ============================================================== sweep: gather and apply

// One colour class of a sweep (Theorem 2's Gauss-Seidel order realised by
// colour classes taken in turn; the whole graph as one class is a synchronous
// round): for every row x of the class,
//   r_x += sum_j a_xj delta_j, then if |r_x| > h_x push x (Eqs. sor1-sor3):
//   delta = omega_x r_x / (1 + d_x), zhat_x += delta, r_x <- (1 - omega_x) r_x.
// delta_j is node j's latest increment in the sweep order: for j in an
// earlier class (those classes ran in earlier launches of this sweep) the
// one made in this sweep, in dcur; for j in this or a later class the one
// made in the previous sweep, in dprev.  Every row writes its own increment
// (0 when it does not push) into dcur.
//
// Two kernels per class.  k_sweep_gather streams the class's nonzeros in
// 32-element chunks, lane l of a warp taking element 32 C + l of chunk C with
// several chunks' gathers in flight per thread, and sums every row's products
// inside each chunk by a segmented inclusive scan across the warp (segments
// start where the chunk plan's start bits say a row begins).  A segment that
// ends its row is written to the row sums at the row's rank (its slot among
// the non-empty rows); the segment of a row that goes on into the next chunk
// is the chunk's carry.  k_sweep_apply then gives every row of the class its
// sum, the carries of the chunks it crosses in chunk order and then its last
// segment (a fixed order: deterministic), and applies the push.  Rows over
// kLongChunks chunks are combined by a warp each.
//
// Hot table: node ids below nhot (the hub prefix of the colour order: the
// nodes of largest in-degree, ordered by class) have their increments staged
// in shared memory when a gather block starts, from this sweep's buffer for
// ids below hlo (hubs of earlier classes) and the previous sweep's otherwise,
// so that the gathers most rows make (a few percent of the nodes draw a third
// of the gathers on an R-MAT graph) are shared-memory loads.
// Launch shape of the gather kernel and size of its hot table (tuning knobs;
// the defaults give one block per SM holding every hub's FP32 increment).
#ifndef FJ_GATHER_THREADS
#define FJ_GATHER_THREADS 1024
#endif
#ifndef FJ_HOT_KB
#define FJ_HOT_KB 192
#endif
constexpr int kGatherThreads = FJ_GATHER_THREADS;
constexpr int64_t kFp32PassSweeps = 48;  // sweeps of an FP32 pass before a restart from the FP64 residual
constexpr int kHotBytes = FJ_HOT_KB * 1024;
static_assert(kHotBytes <= kHubMax * 4 + 1024, "the hot table holds at most the hub prefix");

__device__ __forceinline__ int32_t ld_stream_i32(const int32_t *p)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream_f32(const float *p)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// L2 policy for the increments: kept in L2 ahead of the streams around them
// (columns, weights and row state are read with evict-first loads).
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float ld_keep(const float *ptr, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *ptr, uint64_t pol)
{
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}

template <typename T, bool W>
__global__ void __launch_bounds__(kGatherThreads, kHotBytes > 110 * 1024 ? 1 : 2048 / kGatherThreads)
k_sweep_gather(int64_t ka0, int64_t ka1, int64_t kb0, int64_t kb1, const int32_t *__restrict__ col,
               const float *__restrict__ w, const uint32_t *__restrict__ starts, const int32_t *__restrict__ endbase,
               int lo, int nhot, int nhub, int hlo, const T *__restrict__ dcur, const T *__restrict__ dprev,
               T *__restrict__ rsum, T *__restrict__ carry, const Counters *ctr, int64_t n_rows, int64_t n_ranks)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char gather_dyn[];
    T *hot = reinterpret_cast<T *>(gather_dyn);
    if (*reinterpret_cast<const volatile int *>(&ctr->done)) return;
    // stage the hot table, eight independent loads in flight per thread
    for (int i0 = threadIdx.x; i0 < nhot; i0 += 8 * blockDim.x) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            v[u] = i < nhot ? (i < hlo ? dcur[i] : dprev[i]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            if (i < nhot) hot[i] = v[u];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // chunks of the two ranges, numbered 0 .. na + nb - 1
    const int64_t ca0 = ka0 / kChunkE, cb0 = kb0 / kChunkE;
    const int64_t na = ka1 > ka0 ? (ka1 - 1) / kChunkE - ca0 + 1 : 0;
    const int64_t nb = kb1 > kb0 ? (kb1 - 1) / kChunkE - cb0 + 1 : 0;
    const int64_t total = na + nb;
    // consecutive chunks go to consecutive blocks (a short class spreads over the SMs)
    const int64_t warp = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t keep = l2_keep_policy();
    auto delta = [&](int32_t j) -> T {
        if ((unsigned)j < (unsigned)nhot) return hot[j];
        if (!FJ_IDX_OK(15, j, n_rows)) return T(0);
        const bool earlier = j < nhub ? j < hlo : j < lo;
        return ld_keep((earlier ? dcur : dprev) + j, keep);
    };
    // one chunk per warp iteration; the next chunk's columns and plan words
    // load while this chunk's gathers are in flight (the weights, needed only
    // after the gathers, load beside them)
    struct ChunkRegs {
        int64_t C, e0;
        unsigned inm;
        int4 c0, c1;
        uint32_t word, word_next;
        int32_t ebase;
    };
    auto load_chunk = [&](int64_t t, ChunkRegs &q) {
        const bool first = t < na;
        q.C = first ? ca0 + t : cb0 + (t - na);
        q.e0 = q.C * kChunkE + lane * 8;  // this lane's eight nonzeros
        // which of them lie in the range (the range is whole rows)
        const int64_t lo_off = (first ? ka0 : kb0) - q.e0, hi_off = (first ? ka1 : kb1) - q.e0;
        unsigned inm = 0xFFu;
        if (lo_off > 0) inm = lo_off >= 8 ? 0u : (inm << lo_off) & 0xFFu;
        if (hi_off < 8) inm &= hi_off <= 0 ? 0u : (0xFFu >> (8 - hi_off));
        q.inm = inm;
        q.c0 = __ldcs(reinterpret_cast<const int4 *>(col + q.e0));
        q.c1 = __ldcs(reinterpret_cast<const int4 *>(col + q.e0 + 4));
        q.word = __ldg(starts + q.C * 8 + (lane >> 2));
        // the last lane of each word also needs the next word's first bit
        q.word_next = (lane & 3) == 3 ? __ldg(starts + q.C * 8 + (lane >> 2) + 1) : 0u;
        q.ebase = __ldg(endbase + q.C);
    };
    ChunkRegs nxt;
    if (warp < total) load_chunk(warp, nxt);
    for (int64_t t = warp; t < total; t += nwarps) {
        const ChunkRegs q = nxt;
        if (t + nwarps < total) load_chunk(t + nwarps, nxt);
        const int64_t C = q.C;
        const unsigned inm = q.inm;
        T v[8];
        {
            const int32_t jj[8] = {q.c0.x, q.c0.y, q.c0.z, q.c0.w, q.c1.x, q.c1.y, q.c1.z, q.c1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = ((inm >> i) & 1u) ? delta(jj[i]) : T(0);
            if constexpr (W) {
                const float4 w0 = __ldcs(reinterpret_cast<const float4 *>(w + q.e0));
                const float4 w1 = __ldcs(reinterpret_cast<const float4 *>(w + q.e0 + 4));
                v[0] *= (T)w0.x; v[1] *= (T)w0.y; v[2] *= (T)w0.z; v[3] *= (T)w0.w;
                v[4] *= (T)w1.x; v[5] *= (T)w1.y; v[6] *= (T)w1.z; v[7] *= (T)w1.w;
            }
        }
        // start bits of the lane's elements (sb) and end bits (eb: element i ends its row)
        const unsigned sb = (q.word >> ((lane & 3) * 8)) & 0xFFu;
        const unsigned nx = (lane & 3) == 3 ? (q.word_next & 1u) : ((q.word >> ((lane & 3) * 8 + 8)) & 1u);
        const unsigned eb = (sb >> 1) | (nx << 7);
        // ranks: row ends before this lane in the chunk, one ballot per element slot
        const unsigned lt = lanemask_lt();
        int ebefore = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) ebefore += __popc(__ballot_sync(FULL, (eb >> i) & 1u) & lt);
        const int64_t rbase = (int64_t)q.ebase + ebefore;
        // the lane's own pass: segments that start and end in the lane are
        // written now; the one open at its start (started in an earlier lane)
        // waits for the carry-in
        T run = T(0), open_part = T(0);
        bool seen = false;
        int ei = 0, open_i = -1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if ((sb >> i) & 1u) {
                seen = true;
                run = T(0);
            }
            run += v[i];
            if ((eb >> i) & 1u) {
                if (seen) {
                    if (((inm >> i) & 1u) && FJ_IDX_OK(19, rbase + ei, n_ranks)) rsum[rbase + ei] = run;
                } else {
                    open_i = i;
                    open_part = run;
                }
                ++ei;
            }
        }
        // carry across lanes: a lane's outgoing value is its open tail, or (no
        // start and no end in it) the incoming value plus all eight elements
        const bool closed = (eb >> 7) & 1u;
        T x = closed ? T(0) : run;
        // segmented inclusive scan: a lane with a start or a closed end heads a
        // segment (its value does not depend on earlier lanes)
        const unsigned heads = __ballot_sync(FULL, seen || closed) & (lt | (1u << lane));
        const int hs = heads ? 31 - __clz(heads) : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T y = __shfl_up_sync(FULL, x, d);
            if (lane - d >= hs) x += y;
        }
        T in = __shfl_up_sync(FULL, x, 1);
        if (lane == 0) in = T(0);  // the chunk's first segment: earlier chunks reach it through their carries
        if (open_i >= 0) {
            const int64_t rk = rbase;  // the open segment's end is the lane's first end
            if (((inm >> open_i) & 1u) && FJ_IDX_OK(19, rk, n_ranks)) rsum[rk] = in + open_part;
        }
        if (lane == 31 && !closed && ((inm >> 7) & 1u)) carry[C] = x;
    }
}

// Combines and applies the sums of the class's rows: rows [xa0, xa1) and
// [xb0, xb1) one thread each (a row over kLongChunks chunks is left to the
// warps below), then the class's long rows one warp each, in blocks from
// first_long_block on.
template <typename T>
__global__ void __launch_bounds__(256)
k_sweep_apply(int64_t xa0, int64_t xa1, int64_t xb0, int64_t xb1, const int32_t *__restrict__ long_rows,
              int64_t nlong, unsigned first_long_block, const int64_t *__restrict__ rp,
              const int32_t *__restrict__ rank, const T *__restrict__ rsum, const T *__restrict__ carry, T *dcur,
              T *__restrict__ r, const T *__restrict__ h, const T *__restrict__ inv, double *__restrict__ zhat,
              const int32_t *__restrict__ indeg, const T *__restrict__ om, Counters *ctr, int64_t n_rows)
{
    __shared__ unsigned long long red[2][8];
    __shared__ int sbad;
    if (*reinterpret_cast<volatile int *>(&ctr->done)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    unsigned long long my_push = 0, my_edges = 0;
    bool bad = false;
    // row state streams through L2 with evict-first loads and stores, so that
    // the increments the gathers read stay resident
    auto apply = [&](int64_t x, T acc) {
        T rx = __ldcs(r + x) + acc;
        T dx = T(0);
        if (abs_t(rx) > __ldcs(h + x)) {
            const T ox = __ldcs(om + x);
            dx = ox * rx * __ldcs(inv + x);
            __stcs(zhat + x, __ldcs(zhat + x) + (double)dx);
            rx = (T(1) - ox) * rx;
            my_push += 1;
            my_edges += (unsigned long long)__ldcs(indeg + x);
        }
        if (!isfinite(rx)) bad = true;
        __stcs(r + x, rx);
        dcur[x] = dx;
    };
    if (blockIdx.x < first_long_block) {
        const int64_t na = xa1 - xa0, total = na + (xb1 - xb0);
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
             t += (int64_t)first_long_block * blockDim.x) {
            const int64_t x = t < na ? xa0 + t : xb0 + (t - na);
            if (!FJ_IDX_OK(11, x, n_rows)) continue;
            const int64_t a = __ldcs(rp + x), b = __ldcs(rp + x + 1);
            T acc = T(0);
            if (b > a) {
                const int64_t cs = a / kChunkE, ce = (b - 1) / kChunkE;
                if (ce - cs > kLongChunks) continue;  // a warp combines it
                for (int64_t c = cs; c < ce; ++c) acc += __ldcs(carry + c);
                acc += __ldcs(rsum + __ldcs(rank + x));
            }
            apply(x, acc);
        }
    } else {
        const int64_t warp = ((int64_t)(blockIdx.x - first_long_block) * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)(gridDim.x - first_long_block) * blockDim.x) >> 5;
        for (int64_t i = warp; i < nlong; i += nwarps) {
            const int64_t x = long_rows[i];
            if (!FJ_IDX_OK(12, x, n_rows)) continue;
            const int64_t cs = rp[x] / kChunkE, ce = (rp[x + 1] - 1) / kChunkE;
            T acc = T(0);
            for (int64_t c = cs + lane; c < ce; c += 32) acc += carry[c];
            acc = warp_sum(acc);
            if (lane == 0) apply(x, acc + rsum[rank[x]]);
        }
    }
    my_push = warp_sum(my_push);
    my_edges = warp_sum(my_edges);
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (lane == 0) {
        red[0][wl] = my_push;
        red[1][wl] = my_edges;
        if (anybad) sbad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long pp = 0, ee = 0;
        for (int i = 0; i < 8; ++i) {
            pp += red[0][i];
            ee += red[1][i];
        }
        if (sbad) ctr->nonfinite = 1.0;
        if (pp) {
            atomicAdd(&ctr->pushes, pp);
            atomicAdd(&ctr->sweep_pushes, pp);
            atomicAdd(&ctr->edges, ee);
        }
    }
}

// ---- chunk plan construction

__global__ void k_start_bits(int64_t n, int64_t nnz, const int64_t *__restrict__ rp, uint32_t *__restrict__ starts,
                             int32_t *__restrict__ nonempty)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += (int64_t)gridDim.x * blockDim.x) {
        if (x == n) {
            atomicOr(&starts[nnz >> 5], 1u << (nnz & 31));  // closes the last row
            continue;
        }
        const int64_t a = rp[x];
        const bool ne = rp[x + 1] > a;
        nonempty[x] = ne ? 1 : 0;
        if (ne) atomicOr(&starts[a >> 5], 1u << (a & 31));
    }
}

// rows that end in chunk C: its end bits are the start bits one position on
struct EndCount {
    const uint32_t *starts;
    __device__ long long operator()(int64_t c) const
    {
        long long k = 0;
        for (int64_t i = 8 * c; i < 8 * c + 8; ++i) k += __popc((starts[i] >> 1) | (starts[i + 1] << 31));
        return k;
    }
};

__global__ void k_narrow_i32(int64_t n, const long long *__restrict__ in, int32_t *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

// ============================================================== FP64 certificate

// r64_x = s'_x - (1 + d_x) zhat_x + sum_j a_xj zhat_j  (= s' - (I + L) zhat').
// The off-diagonal sum runs in FP32 pair arithmetic: zhat_j is read as a pair
// of floats hi + lo (k_split_absmax; |zhat - hi - lo| <= 2^-47 |zhat|), every
// product a hi is split exactly into p + pe (fma), and the running sum is
// carried as an unevaluated pair S + C with Knuth's error-free addition (the
// Sum2/Dot2 scheme of Ogita, Rump and Oishi, in single precision).  S + C
// then meets the a-priori bound of pair_bound below, about n^2 2^-46 d_x
// max|zhat| for n terms per lane, without one FP64 operation per nonzero (the
// FP64 pipe of this part is narrow).  The diagonal part and the pair are
// combined in FP64.  The decision |r64| > max(eps' s', resid_floor) is taken
// in FP32 only when |r64| is farther from the threshold than the bound plus
// the FP32 rounding of both sides; otherwise the row is summed again exactly
// in FP64 double-double (Dot2 over zhat), so the decision is always the exact
// one.  Per graph: max |r64|, max |r64| / s', max |zhat - c_eff|, the number
// above threshold.  Stores r64 into the push residual (magnitude rounded up
// for FP32) and the FP64 residual, and clears both increment buffers: the push
// restarts from this residual (a refinement pass).
//
// One warp per warp tile (grid-strided): a row of at most kShortRow nonzeros
// is summed by one lane, a longer row by the whole warp; a chunk of a long row
// is summed by the warp and the last chunk to finish completes the row.
constexpr int kShortRow = 8;

// An unevaluated FP32 sum s + c.
struct FF {
    float s, c;
};

// acc += a * (z.x + z.y): the product a z.x exactly as p + pe, a z.y rounded
// (it is 2^-24 below a z.x), p added to s error-free, every error term into c.
// The _rn intrinsics keep the compiler from contracting these steps.
template <bool W>
__device__ __forceinline__ void ff_fma(FF &acc, float a, float2 z)
{
    float p, pe, q;
    if constexpr (W) {
        p = __fmul_rn(a, z.x);
        pe = __fmaf_rn(a, z.x, -p);
        q = __fmul_rn(a, z.y);
    } else {
        p = z.x;
        pe = 0.f;
        q = z.y;
    }
    const float s = __fadd_rn(acc.s, p);
    const float bp = __fsub_rn(s, acc.s);
    const float e = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    acc.s = s;
    acc.c = __fadd_rn(acc.c, __fadd_rn(e, __fadd_rn(pe, q)));
}

// Butterfly sum of the lanes' pairs; every lane ends with the same pair
// (error-free addition gives the same error term in either operand order).
__device__ __forceinline__ FF warp_ff_sum(FF a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bs = __shfl_xor_sync(0xffffffffu, a.s, o), bc = __shfl_xor_sync(0xffffffffu, a.c, o);
        const float s = __fadd_rn(a.s, bs);
        const float bp = __fsub_rn(s, a.s);
        const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(bs, bp));
        a.s = s;
        a.c = __fadd_rn(__fadd_rn(a.c, bc), e);
    }
    return a;
}

// Upper bound on |r64 - r_exact| for a row whose off-diagonal sum took at most
// n terms per lane in pair arithmetic (a warp reduction counts as at most 8
// more) and whose pair values were then combined with m64 FP64 roundings.
// The pair sum errs by at most (2 n (n + 2) + 2) u^2 sum|a zhat| with
// u = 2^-24, the hi + lo split by 2^-47 sum|a zhat|; 3 (n + 8)^2 + 8 covers
// both with the tree levels.  The FP64 steps add gamma_{m64} (2^-53) times the
// magnitudes involved; sum|a zhat| <= d_x max|zhat|, and 2^-100 (1 + d_x)
// covers subnormal halves.  Evaluated in FP32 and inflated by 1 %.
__device__ __forceinline__ float pair_bound(int n, int64_t m64, float deg, float zmax, float dpl_zx, float spx)
{
    const float nn = (float)(n + 8);
    const float kpair = (3.f * nn * nn + 8.f) * 0x1p-48f;
    const float mm = (float)(m64 + 4);
    const float g64 = mm * 0x1p-53f / (1.f - mm * 0x1p-53f);
    const float dz = deg * zmax;
    return 1.01f * (kpair * dz + g64 * (dz + fabsf(dpl_zx) + fabsf(spx)) + 0x1p-100f * (1.f + deg));
}

// gamma_m of the standard bound on an m-term FP64 sum (u = 2^-53), times an
// upper bound of the sum of |terms|: d_x max|zhat| for the row's products plus
// the two diagonal terms (the batch certificate's plain FP64 sums).  Evaluated
// in FP32 and inflated to stay an upper bound.
__device__ __forceinline__ double plain_bound(int64_t m, double deg, double zmax, double dpl_zx, double spx)
{
    const float mm = (float)(m + 4);
    const float gam = mm * 0x1p-53f / (1.f - mm * 0x1p-53f);
    const float mag = (float)deg * (float)zmax + fabsf((float)dpl_zx) + fabsf((float)spx);
    return (double)(gam * mag * 1.001f);
}

// FP32 batch path: the increments a check interval accumulated in FP32 per
// entry are added to the FP64 estimate and cleared (the batch sweep then does
// an FP32 instead of an FP64 read-modify-write per push; measured: fewer
// bytes win for 64 vectors, while for one vector the few extra sweeps that
// the coarser accumulation costs do not pay).
__global__ void k_fold(int64_t n, float *__restrict__ z32, double *__restrict__ zhat)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = z32[i];
        if (d != 0.f) {
            zhat[i] += (double)d;
            z32[i] = 0.f;
        }
    }
}

// max |zhat| over n entries into *out (ordered bits of a non-negative double).
__global__ void k_absmax(int64_t n, const double *__restrict__ z, unsigned long long *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(z[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(reinterpret_cast<double *>(out), m);
}

// k_absmax, and zhat split into float pairs: hi = fl32(zhat), lo =
// fl32(zhat - hi) (zhat - hi is exact in FP64), so zhat - hi - lo is the
// rounding error of lo, at most 2^-24 |lo| <= 2^-48 |zhat| for normal floats.
__global__ void k_split_absmax(int64_t n, const double *__restrict__ z, float2 *__restrict__ zs,
                               unsigned long long *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = z[i];
        const float hi = __double2float_rn(v);
        zs[i] = make_float2(hi, __double2float_rn(v - (double)hi));
        m = fmax(m, fabs(v));
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(reinterpret_cast<double *>(out), m);
}

// Fixed-point sums of the long-row certificate.  With |a zhat| < 2^E for
// every product a zhat of the graph, a finite value t is taken as the integer
// trunc(t 2^(94-E)) (below 2^94 in magnitude; the dropped part is under one
// unit 2^(E-94)), and a row's integers are added exactly in 128 bits, within a
// chunk and across its chunks (a row of up to 2^32 terms stays below 2^126).
// The off-diagonal sum thus errs by under one unit per term, taken into the
// decision as a bound, and no nonzero costs an FP64 operation beyond the
// product of a weighted graph.  (GB300's FP64 rate is a small fraction of its
// integer rate.)
typedef unsigned __int128 u128;
constexpr int kFixBits = 94;

__device__ __forceinline__ void fix_add(u128 &acc, double t, int E, bool &bad)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    const int e = (int)((b >> 52) & 0x7ffu);
    const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    const int sh = (e ? e : 1) - (1075 - kFixBits) - E;  // at most kFixBits - 53 when |t| < 2^E
    bad |= (e == 0x7ff) | (sh > kFixBits - 52);
    u128 q;
    if (sh >= 0)
        q = (u128)m << min(sh, kFixBits - 52);
    else
        q = sh > -64 ? (u128)(m >> -sh) : (u128)0;
    acc = (long long)b < 0 ? acc - q : acc + q;
}

__device__ __forceinline__ u128 warp_u128_sum(u128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
        v += ((u128)hi << 64) | (u128)lo;
    }
    return v;
}

// The exponent E of the fixed-point scale: max|zhat| < 2^Ez, max|a| < 2^Ew,
// one bit more for the product's rounding; kept where the unit 2^(E-94) is a
// normal double and a sum (below 2^(E+32)) is finite.  Out of range (a
// non-finite or huge max): *bad.
__device__ __forceinline__ int fix_exponent(double zmax, int ew, bool &bad)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(zmax);
    const int e = (int)((b >> 52) & 0x7ffu);
    int E = (e ? e : 1) - 1022 + ew + 1;
    bad |= e == 0x7ff;
    E = max(E, -900);
    if (E > 950) {  // sums up to 2^(E+32) stay finite
        bad = true;
        E = 950;
    }
    return E;
}

// The signed 128-bit sum v (units 2^(E-94)) as a double-double: four 32-bit
// limbs, each exact in FP64, joined largest first.
__device__ __forceinline__ DD fix_value(u128 v, int E)
{
    const bool neg = (long long)(unsigned long long)(v >> 64) < 0;
    const u128 a = neg ? (u128)0 - v : v;
    const double unit = __longlong_as_double((long long)(E - kFixBits + 1023) << 52);
    DD acc{(double)(unsigned)(a >> 96) * 0x1p96, 0.0};
    dd_add(acc, (double)(unsigned)(a >> 64) * 0x1p64);
    dd_add(acc, (double)(unsigned)(a >> 32) * 0x1p32);
    dd_add(acc, (double)(unsigned)a);
    const double sg = neg ? -unit : unit;
    return DD{acc.hi * sg, acc.lo * sg};
}

template <typename T, bool W>
__global__ void __launch_bounds__(256)
k_certify(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
          const int32_t *__restrict__ col, const float *__restrict__ w, const double *__restrict__ zhat,
          const float2 *__restrict__ zs, const double *__restrict__ sp, const double *__restrict__ deg,
          const int32_t *__restrict__ graph_of, double epsp, T *__restrict__ r, T *__restrict__ da,
          T *__restrict__ db, unsigned long long *gs, const int32_t *__restrict__ slot_first,
          const int32_t *__restrict__ slot_nchunk, double *part, int32_t *cnt, double *__restrict__ r64,
          const unsigned long long *__restrict__ zmaxp, int wexp, int64_t n_rows)
{
    constexpr unsigned FULL = 0xffffffffu;
    const double zmaxd = __longlong_as_double((long long)*zmaxp);
    const float zmaxf = (float)zmaxd;
    bool fix_bad = false;
    const int fixE = fix_exponent(zmaxd, W ? wexp : 0, fix_bad);
    const float epsf = (float)epsp;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double *gsd = reinterpret_cast<const double *>(gs);
    int cur_g = -1;
    float cef = 0.f, m_rel = 0.f, m_z = 0.f;
    double m_abs = 0.0, viol = 0.0;

    auto flush = [&]() {  // warp-uniform
        const double a = warp_max(m_abs), v = warp_sum(viol);
        const double rl = warp_max((double)m_rel), zz = warp_max((double)m_z);
        if (lane == 0 && cur_g >= 0) {
            unsigned long long *g = gs + (int64_t)cur_g * kGs;
            atomic_max_nonneg(reinterpret_cast<double *>(g + 2), a);
            atomic_max_nonneg(reinterpret_cast<double *>(g + 3), rl);
            atomic_max_nonneg(reinterpret_cast<double *>(g + 4), zz);
            if (v > 0) atomicAdd(reinterpret_cast<double *>(g + 5), v);
        }
        m_abs = viol = 0.0;
        m_rel = m_z = 0.f;
    };
    // pair-arithmetic pass over [a, e) by one thread
    auto pair_terms = [&](int64_t a, int64_t e, int64_t step, FF &acc) {
        for (int64_t k = a; k < e; k += step) {
            const int32_t cj = __ldg(col + k);
            if (!FJ_IDX_OK(4, cj, n_rows)) continue;
            ff_fma<W>(acc, W ? __ldg(w + k) : 1.f, __ldg(zs + cj));
        }
    };
    auto exact_terms = [&](int64_t a, int64_t e, int64_t step, DD &acc) {
        for (int64_t k = a; k < e; k += step) {
            const int32_t cj = __ldg(col + k);
            if (FJ_IDX_OK(4, cj, n_rows)) dd_fma(acc, arc_w<double, W>(w, k), zhat[cj]);
        }
    };
    // The residual from the pair sum (given as an FP64 value `off` after
    // m64 FP64 roundings) and, when it is decidable in FP32, the decision:
    // dec = 1 above threshold, 0 not, -1 undecided (needs the exact sum).
    auto pair_residual = [&](int64_t x, int n, int64_t m64, double off, int &dec) -> double {
        const double zx = zhat[x], spx = sp[x], dx = deg[x];
        const double dpl = 1.0 + dx;
        const double rx = fma(-dpl, zx, spx) + off;
        const float degf = (float)dx, spf = (float)spx, zxf = zs[x].x;
        const float bnd = pair_bound(n, m64, degf, zmaxf, (1.f + degf) * zxf, spf);
        const float arf = fabsf((float)rx);
        const float thrf = fmaxf(epsf * spf, 0x1p-51f * (1.f + degf) * fabsf(zxf));
        const float slack = bnd + 0x1p-20f * (arf + thrf);
        const float gap = arf - thrf;
        dec = gap > slack ? 1 : (-gap > slack ? 0 : -1);  // NaN or inf: undecided
        return rx;
    };
    auto fix_terms = [&](int64_t a, int64_t e, int64_t step, u128 &acc, bool &bad) {
        for (int64_t k = a; k < e; k += step) {
            const int32_t cj = __ldg(col + k);
            if (!FJ_IDX_OK(4, cj, n_rows)) continue;
            const double z = zhat[cj];
            if (W) {
                const double av = (double)__ldg(w + k);
                const double pr = __dmul_rn(av, z);
                fix_add(acc, pr, fixE, bad);
                fix_add(acc, fma(av, z, -pr), fixE, bad);  // the product's rounding error, exactly
            } else {
                fix_add(acc, z, fixE, bad);
            }
        }
    };
    auto exact_residual = [&](int64_t x, DD acc, int &dec) -> double {
        dd_add(acc, sp[x]);
        dd_fma(acc, -(1.0 + deg[x]), zhat[x]);
        const double rx = dd_value(acc);
        dec = fabs(rx) > fmax(epsp * sp[x], resid_floor(deg[x], zhat[x])) ? 1 : 0;
        return rx;
    };
    auto finish = [&](int64_t x, double rx, int dec) {
        double ax = fabs(rx);
        if (!(ax <= 1e300)) {
            ax = INFINITY;
            dec = 1;
        }
        const float af = (float)ax;
        m_abs = fmax(m_abs, ax);
        m_rel = fmaxf(m_rel, af / (float)sp[x]);  // reported, FP32 is enough
        m_z = fmaxf(m_z, fabsf(zs[x].x - cef));   // reported, FP32 is enough
        if (dec) viol += 1.0;
        r[x] = resid_store<T>(rx);
        r64[x] = rx;
        da[x] = T(0);
        db[x] = T(0);
    };

    for (int64_t ii = warp; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (!FJ_IDX_OK(1, r0, n_rows) || !FJ_IDX_OK(2, r1, n_rows + 1) ||
            (it.slot < 0 && !FJ_IDX_OK(3, r1 - r0, kWarpRows + 1)))
            continue;
        const int gph = graph_of ? graph_of[r0] : 0;
        if (!FJ_IDX_OK(6, gph, 1 << 20)) continue;
        if (gph != cur_g) {
            flush();
            cur_g = gph;
            cef = (float)gsd[(int64_t)gph * kGs + 1];
        }
        if (it.slot < 0) {
            // off-diagonal pair sums of the tile's rows: a short row by its own
            // lane, a longer one by the warp with the sum handed to the row's
            // lane; then every lane takes its rows' FP64 steps in parallel
            int64_t ra[2], re[2];
            bool mine[2], shrt[2];
            FF acc[2];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int64_t x = r0 + lane + 32 * half;
                mine[half] = x < r1;
                ra[half] = re[half] = 0;
                if (mine[half]) {
                    ra[half] = rp[x];
                    re[half] = rp[x + 1];
                }
                shrt[half] = re[half] - ra[half] <= kShortRow;
                acc[half] = FF{0.f, 0.f};
                if (mine[half] && shrt[half]) pair_terms(ra[half], re[half], 1, acc[half]);
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                unsigned longs = __ballot_sync(FULL, mine[half] && !shrt[half]);
                while (longs) {
                    const int src = __ffs(longs) - 1;
                    longs &= longs - 1;
                    const int64_t al = __shfl_sync(FULL, ra[half], src), el = __shfl_sync(FULL, re[half], src);
                    FF t{0.f, 0.f};
                    pair_terms(al + lane, el, 32, t);
                    t = warp_ff_sum(t);
                    if (lane == src) acc[half] = t;
                }
            }
            double rx[2];
            int dec[2];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                rx[half] = 0.0;
                dec[half] = 0;
                if (mine[half]) {
                    const int64_t len = re[half] - ra[half];
                    const int nl = shrt[half] ? (int)len : (int)((len + 31) / 32);
                    rx[half] = pair_residual(r0 + lane + 32 * half, nl, 1, (double)acc[half].s + (double)acc[half].c,
                                             dec[half]);
                }
            }
            // rows the FP32 decision left open: exact sums
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int64_t x = r0 + lane + 32 * half;
                if (mine[half] && shrt[half] && dec[half] < 0) {
                    DD d{0.0, 0.0};
                    exact_terms(ra[half], re[half], 1, d);
                    rx[half] = exact_residual(x, d, dec[half]);
                }
                unsigned open = __ballot_sync(FULL, mine[half] && !shrt[half] && dec[half] < 0);
                while (open) {
                    const int src = __ffs(open) - 1;
                    open &= open - 1;
                    const int64_t al = __shfl_sync(FULL, ra[half], src), el = __shfl_sync(FULL, re[half], src);
                    DD d{0.0, 0.0};
                    exact_terms(al + lane, el, 32, d);
                    d = warp_dd_sum(d);
                    if (lane == src) rx[half] = exact_residual(x, d, dec[half]);
                }
                if (mine[half]) finish(x, rx[half], dec[half]);
            }
        } else {
            // a chunk of a long row: its compensated (Dot2) partial; the last
            // chunk to finish joins the chunks' partials and decides exactly.
            // (A long row's pair-arithmetic bound grows with its length, so the
            // FP32 decision would leave it open near convergence, and one warp
            // re-summing a hub row of 10^5-10^6 nonzeros would serialise the
            // certificate; the chunks share that work instead.)
            u128 acc = 0;
            bool bad = fix_bad;
            fix_terms(it.k0 + lane, it.k1, 32, acc, bad);
            acc = warp_u128_sum(acc);
            bad = __any_sync(FULL, bad);
            const int slot = it.slot;
            const int first = slot_first[slot], nch = slot_nchunk[slot];
            const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
            unsigned long long *pw = reinterpret_cast<unsigned long long *>(part);
            int last = 0;
            if (lane == 0) {
                // a chunk's sum is below 2^104, so a top word of INT64_MIN marks a bad chunk
                pw[2 * (first + ci)] = bad ? 0ull : (unsigned long long)acc;
                pw[2 * (first + ci) + 1] = bad ? 0x8000000000000000ull : (unsigned long long)(acc >> 64);
                __threadfence();
                last = atomicAdd(&cnt[slot], 1) == nch - 1;
            }
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
                u128 d = 0;
                bool dbad = false;
                for (int c = lane; c < nch; c += 32) {
                    const unsigned long long lo = __ldcg(pw + 2 * (first + c)), hi = __ldcg(pw + 2 * (first + c) + 1);
                    dbad |= hi == 0x8000000000000000ull;
                    d += ((u128)hi << 64) | (u128)lo;
                }
                d = warp_u128_sum(d);
                dbad = __any_sync(FULL, dbad);
                const int64_t len = rp[r0 + 1] - rp[r0];
                const DD off = fix_value(d, fixE);
                int dec;
                double rx = exact_residual(r0, off, dec);
                // under one unit per term (two for a weighted product), and
                // the double-double steps' rounding, on the safe side
                const double unit = __longlong_as_double((long long)(fixE - kFixBits + 1023) << 52);
                const double slack = (double)((W ? 2 : 1) * len + 4) * unit +
                                     0x1p-100 * (fabs(off.hi) + (1.0 + deg[r0]) * fabs(zhat[r0]) + fabs(sp[r0]));
                if (dbad) rx = __longlong_as_double(0x7ff8000000000000ll);  // non-finite input: NaN
                else if (!dec && fabs(rx) + slack > fmax(epsp * sp[r0], resid_floor(deg[r0], zhat[r0])))
                    dec = 1;
                if (lane == 0) {
                    cnt[slot] = 0;
                    finish(r0, rx, dec);
                }
            }
        }
    }
    flush();
}

// Clears the per-graph certificate slots (2..6) before a certify pass.
__global__ void k_cert_reset(int ng, unsigned long long *gs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x)
        for (int j = 2; j < kGs; ++j) gs[(int64_t)i * kGs + j] = 0ULL;
}

// ============================================================== FP64 frontier push

// Entries e = v k + j (node v, vector j; k = 1 for one vector) whose FP64
// residual, as left by the certificate and the frontier pushes since, is
// above the certificate's threshold.
struct CleanPred {
    const double *r64, *sp, *zhat, *deg;
    double epsp;
    int k;
    __device__ bool operator()(int64_t e) const
    {
        // the FP64 resolution term is read only for an entry above eps' s'
        // (a NaN residual fails both tests)
        const double a = fabs(r64[e]), t = epsp * sp[e];
        if (!(a > t)) return false;
        const int64_t v = k == 1 ? e : e / k;
        return a > fmax(t, resid_floor(deg[v], zhat[e]));
    }
};

// One round of the scatter-form push (Alg. 1, omega = 1) over the frontier
// list, one warp per entry: zhat_e moves by r_e / (1 + d_v), and the change
// zhat actually took (exact, a difference of neighbouring doubles) is taken out
// of r_e and added, times a_uv, to r_u j for every in-neighbour u of v.
// Pushes of one round run concurrently, so every residual update is an
// atomic addition; an entry's own residual is read once and what was read is
// what is moved (asynchronous relaxation of the diagonally dominant I + L).
// An entry whose in-neighbour list is longer than long_min leaves its
// scatter to k_frontier_push_long (a block per such entry), so a hub does not
// serialise a round on one warp: the entry and its step are appended to
// (lng_e, lng_dz), counted by *lng_n, which is zero when the kernel starts.

template <bool W>
__global__ void __launch_bounds__(256)
k_frontier_push(const int32_t *__restrict__ list, const long long *__restrict__ count, int k,
                const int64_t *__restrict__ tp, const int32_t *__restrict__ tc, const float *__restrict__ tw,
                const double *__restrict__ deg, double *r64, double *__restrict__ zhat, Counters *ctr,
                int64_t n_rows, int64_t long_min, unsigned long long *lng_n, int64_t *__restrict__ lng_e,
                double *__restrict__ lng_dz)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const long long cnt = *count;
    const int64_t n_ent = n_rows * k;
    unsigned long long my_edges = 0;
    for (int64_t i = warp; i < cnt; i += nwarps) {
        const int64_t e = list[i];
        if (!FJ_IDX_OK(20, e, n_ent)) continue;
        const int64_t v = e / k;
        const int j = (int)(e - v * k);
        double dz = 0.0;
        if (lane == 0) {
            const double rv = __ldcg(r64 + e);
            const double dpl = 1.0 + deg[v];
            const double z0 = zhat[e];
            const double z1 = __dadd_rn(z0, rv / dpl);
            zhat[e] = z1;
            dz = __dsub_rn(z1, z0);
            atomicAdd(r64 + e, -__dmul_rn(dpl, dz));
        }
        dz = __shfl_sync(0xffffffffu, dz, 0);
        const int64_t a0 = tp[v], a1 = tp[v + 1];
        if (a1 - a0 > long_min) {
            if (lane == 0) {
                const unsigned long long slot = atomicAdd(lng_n, 1ull);
                lng_e[slot] = e;  // slot < cnt: one slot per list entry at most
                lng_dz[slot] = dz;
            }
            continue;
        }
        for (int64_t kk = a0 + lane; kk < a1; kk += 32) {
            const int32_t u = tc[kk];
            if (!FJ_IDX_OK(21, u, n_rows)) continue;
            const double a = W ? (double)tw[kk] : 1.0;
            atomicAdd(r64 + (int64_t)u * k + j, __dmul_rn(a, dz));
        }
        if (lane == 0) my_edges += (unsigned long long)(a1 - a0);
    }
    my_edges = warp_sum(my_edges);
    if (lane == 0 && my_edges) atomicAdd(&ctr->fedges, my_edges);
}

// The scatter of the long entries of a frontier round: persistent blocks take
// the entries k_frontier_push set aside in turn and a block spreads an entry's
// in-neighbours over its threads (the step dz was computed and applied to the
// entry itself by k_frontier_push).
template <bool W>
__global__ void __launch_bounds__(1024)
k_frontier_push_long(const unsigned long long *__restrict__ lng_n, const int64_t *__restrict__ lng_e,
                     const double *__restrict__ lng_dz, const long long *__restrict__ count, int k,
                     const int64_t *__restrict__ tp, const int32_t *__restrict__ tc, const float *__restrict__ tw,
                     double *r64, Counters *ctr, int64_t n_rows)
{
    const long long nl = (long long)*lng_n;
    const long long cnt = *count;
    const int64_t n_ent = n_rows * k;
    unsigned long long my_edges = 0;
    for (int64_t i = blockIdx.x; i < nl && i < cnt; i += gridDim.x) {
        const int64_t e = lng_e[i];
        if (!FJ_IDX_OK(22, e, n_ent)) continue;
        const int64_t v = e / k;
        const int j = (int)(e - v * k);
        const int64_t a0 = tp[v], a1 = tp[v + 1];
        const double dz = lng_dz[i];
        for (int64_t kk = a0 + threadIdx.x; kk < a1; kk += blockDim.x) {
            const int32_t u = tc[kk];
            if (!FJ_IDX_OK(23, u, n_rows)) continue;
            const double a = W ? (double)tw[kk] : 1.0;
            atomicAdd(r64 + (int64_t)u * k + j, __dmul_rn(a, dz));
        }
        if (threadIdx.x == 0) my_edges += (unsigned long long)(a1 - a0);
    }
    if (threadIdx.x == 0 && my_edges) atomicAdd(&ctr->fedges, my_edges);
}

// ============================================================== frontier

template <typename T>
struct FrontierPred {
    const T *r, *h;
    __device__ bool operator()(int64_t v) const { return abs_t(r[v]) > h[v]; }
};

// ============================================================== residual API

__global__ void k_residual(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const float *__restrict__ w, const double *__restrict__ s, const double *__restrict__ z,
                           double ce, double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp0; x < n; x += nwarps) {
        double zx = z[x] + ce;
        double acc = 0.0;
        for (int64_t k = rp[x] + lane; k < rp[x + 1]; k += 32)
            acc += (w ? (double)w[k] : 1.0) * ((z[col[k]] + ce) - zx);
        acc = warp_sum(acc);
        if (lane == 0) out[x] = (s[x] + ce) - zx + acc;
    }
}

// ============================================================== warm-start judge

// The zero start is the judge of a warm start (its fallback).  The push's
// work is driven down by the residual sum (the running-time argument of
// Section 5.1.2, Theorem 1), so a start z0 is kept only when its exact
// residual sum, sum_v |r_v| of r = s' - (I + L)(z0 + c_eff), is below the
// zero start's, sum_v s'_v.  Per right-hand side j (node-major [n][k]),
// block b writes its two sums to part[(j * gridDim.x + b) * 2 + {0, 1}], each
// in a fixed order; the host adds the blocks in order (deterministic).
constexpr int kJudgeBlocks = 256;

__global__ void __launch_bounds__(256)
k_warm_judge(int64_t n, int k, const double *__restrict__ r64, const double *__restrict__ sp, double *__restrict__ part)
{
    __shared__ double sa[8], sb[8];
    const int j = blockIdx.y;
    double a = 0.0, b = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        a += fabs(r64[v * k + j]);
        b += sp[v * k + j];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < 8; ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        part[((int64_t)j * gridDim.x + blockIdx.x) * 2] = ta;
        part[((int64_t)j * gridDim.x + blockIdx.x) * 2 + 1] = tb;
    }
}

// Right-hand sides whose start lost to the zero start restart from zero: the
// state a zero start's initialisation gives (zhat' = 0, r = s').
template <typename T>
__global__ void k_zero_start_cols(int64_t n, int k, const int *__restrict__ cold, const double *__restrict__ sp,
                                  double *__restrict__ zhat, T *__restrict__ r, double *__restrict__ r64,
                                  T *__restrict__ da, T *__restrict__ db)
{
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * k;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx % k);
        if (!cold[j]) continue;
        zhat[idx] = 0.0;
        r[idx] = (T)sp[idx];
        r64[idx] = sp[idx];
        da[idx] = T(0);
        db[idx] = T(0);
    }
}

// keep[j] = 1 when start j beats the zero start (see k_warm_judge).
static fj_status warm_judge(fj_graph *g, int64_t n, int k, const double *r64, const double *sp, cudaStream_t st,
                            std::vector<int> &keep)
{
    Workspace &ws = g->ws;
    const int64_t need = (int64_t)kJudgeBlocks * k * 2;
    if (need + 64 > ws.cap_judge) {  // the sums, then room for 64 restart flags
        dev_free(ws.judge);
        ws.judge = nullptr;
        ws.cap_judge = 0;  // stays 0 if the allocation fails
        FJ_CUDA(dev_malloc(&ws.judge, sizeof(double) * (size_t)(need + 64)));
        ws.cap_judge = need + 64;
    }
    k_warm_judge<<<dim3(kJudgeBlocks, k), 256, 0, st>>>(n, k, r64, sp, ws.judge);
    FJ_CUDA(cudaGetLastError());
    std::vector<double> h((size_t)need);
    FJ_CUDA(cudaMemcpyAsync(h.data(), ws.judge, sizeof(double) * (size_t)need, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    keep.assign((size_t)k, 0);
    for (int j = 0; j < k; ++j) {
        double a = 0.0, b = 0.0;
        for (int bl = 0; bl < kJudgeBlocks; ++bl) {
            a += h[((size_t)j * kJudgeBlocks + bl) * 2];
            b += h[((size_t)j * kJudgeBlocks + bl) * 2 + 1];
        }
        keep[(size_t)j] = (std::isfinite(a) && a < b) ? 1 : 0;
    }
    return FJ_OK;
}

// ============================================================== host driver

template <typename T>
static fj_status ws_grow(fj_graph *g, int64_t entries, int ngraphs)
{
    Workspace &ws = g->ws;
    if (entries > ws.cap_n) {
        ws.cap_n = 0;  // stays 0 if an allocation fails, so the next call grows again
        void **bufs[] = {&ws.r, &ws.h, &ws.da, &ws.db, &ws.om, &ws.rsum};
        for (void **p : bufs) {
            dev_free(*p);
            *p = nullptr;
            FJ_CUDA(dev_malloc(p, sizeof(double) * (size_t)entries));
        }
        double **dbufs[] = {&ws.zhat, &ws.sp, &ws.sin, &ws.zout, &ws.r64};
        for (double **p : dbufs) {
            dev_free(*p);
            *p = nullptr;
            FJ_CUDA(dev_malloc(p, sizeof(double) * (size_t)entries));
        }
        dev_free(ws.list);
        ws.list = nullptr;
        FJ_CUDA(dev_malloc(&ws.list, sizeof(int32_t) * (size_t)entries));
        dev_free(ws.zs);
        ws.zs = nullptr;
        FJ_CUDA(dev_malloc(&ws.zs, sizeof(float2) * (size_t)entries));
        ws.cap_n = entries;
        ws.gen++;
    }
    if (ngraphs > ws.cap_graphs) {
        ws.cap_graphs = 0;
        dev_free(ws.gstat);
        ws.gstat = nullptr;
        if (ws.gstat_host) cudaFreeHost(ws.gstat_host);
        ws.gstat_host = nullptr;
        FJ_CUDA(dev_malloc(&ws.gstat, sizeof(double) * kGs * ngraphs));
        FJ_CUDA(cudaMallocHost(&ws.gstat_host, sizeof(double) * kGs * ngraphs));
        ws.cap_graphs = ngraphs;
    }
    if (!ws.ctr) {
        FJ_CUDA(dev_malloc(&ws.ctr, sizeof(Counters)));
        FJ_CUDA(cudaMallocHost(&ws.ctr_host, sizeof(Counters)));
    }
    if (!ws.zmax) FJ_CUDA(dev_malloc(&ws.zmax, sizeof(unsigned long long)));
    return FJ_OK;
}

struct Plan {
    const DevCSR *c = nullptr;  // CSR the push runs on
    const int32_t *perm = nullptr;
    const ItemPlan *wip = nullptr;  // warp-tile items (certificate, batch sweep)
    const ChunkPlan *cp = nullptr;  // chunk plan (single-vector sweep)
    bool mc = false;
};

// Launch bookkeeping of one solve: every kernel launched, and with profiling
// a CUDA-event pair around every sweep-kernel launch on the solve's stream.
struct Run {
    int64_t launches = 0;
    int64_t push_launches = 0;
    bool profile = false;
    std::vector<cudaEvent_t> ev;  // pairs
    size_t used = 0;
    double push_ms = 0.0;

    fj_status before(cudaStream_t st)
    {
        if (!profile) return FJ_OK;
        if (used + 2 > ev.size()) {
            cudaEvent_t a, b;
            FJ_CUDA(cudaEventCreate(&a));
            FJ_CUDA(cudaEventCreate(&b));
            ev.push_back(a);
            ev.push_back(b);
        }
        FJ_CUDA(cudaEventRecord(ev[used], st));
        return FJ_OK;
    }
    fj_status after(cudaStream_t st)
    {
        ++launches;
        ++push_launches;
        if (!profile) return FJ_OK;
        FJ_CUDA(cudaEventRecord(ev[used + 1], st));
        used += 2;
        return FJ_OK;
    }
    // after a stream synchronisation: fold the recorded pairs into push_ms
    fj_status harvest()
    {
        for (size_t i = 0; i < used; i += 2) {
            float ms = 0.f;
            FJ_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            push_ms += ms;
        }
        used = 0;
        return FJ_OK;
    }
    ~Run()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

static fj_status check_opts(const fj_solve_opts *o)
{
    FJ_ARG(o != nullptr, "opts is NULL");
    FJ_ARG(o->eps > 0.0 && o->eps < 1.0, "eps must be in (0, 1)");
    FJ_ARG(o->omega > 0.0 && o->omega < 2.0, "omega must be in (0, 2)");
    FJ_ARG(o->c > 0.0 && std::isfinite(o->c), "c must be positive");
    FJ_ARG(o->sigma > 0.0 && std::isfinite(o->sigma), "sigma must be positive");
    FJ_ARG(o->precision == FJ_PREC_FP64 || o->precision == FJ_PREC_FP32, "unknown precision");
    FJ_ARG(o->schedule >= FJ_SCHED_AUTO && o->schedule <= FJ_SCHED_MULTICOLOUR, "unknown schedule");
    FJ_ARG(!(o->schedule == FJ_SCHED_JACOBI && o->omega > 1.0), "JACOBI rounds need omega <= 1");
    FJ_ARG(o->max_sweeps >= 1, "max_sweeps must be >= 1");
    FJ_ARG(o->max_refine >= 0, "max_refine must be >= 0");
    FJ_ARG(o->palette >= 0 && o->palette <= 32, "palette must be 0 (unbounded) or 1..32");
    return FJ_OK;
}

__global__ void k_gather_rp(int64_t nb, const int32_t *__restrict__ blk_row, const int64_t *__restrict__ rp,
                            long long *__restrict__ out)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += (int64_t)gridDim.x * blockDim.x)
        out[b] = rp[blk_row[b]];
}

// Work items of a CSR: every row block, with rows longer than two tiles cut
// into chunks, grouped by colour class (items of class c are
// [class_item[c], class_item[c+1]), in row order inside the class: first the
// class's hub rows, then its other rows).  With a colouring (multicolour)
// each item carries the first row of its class, the first hub row of its
// class and the hub count; without one every item is in the one class 0.
static fj_status build_items(fj_graph *g, const DevCSR &c, const Colouring *cl, ItemPlan &ip, cudaStream_t st,
                             TileKind kind)
{
    const bool warp_tiles = kind == kTileWarp;
    const int64_t nb = warp_tiles ? c.nwblocks : c.nblocks;
    const int32_t *blk_row = warp_tiles ? c.wblk_row : c.blk_row;
    const int64_t long_row = warp_tiles ? 2 * kWarpNnz : 2 * kBlockNnz;
    const int64_t chunk = warp_tiles ? kWarpChunk : kChunkNnz;
    std::vector<int32_t> br((size_t)nb + 1);
    std::vector<long long> bk((size_t)nb + 1);
    long long *bk_d = nullptr;
    FJ_CUDA(dev_malloc(&bk_d, sizeof(long long) * (nb + 1)));
    k_gather_rp<<<grid_for(nb + 1, 256), 256, 0, st>>>(nb, blk_row, c.row_ptr, bk_d);
    FJ_CUDA(cudaGetLastError());
    FJ_CUDA(cudaMemcpyAsync(br.data(), blk_row, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(bk.data(), bk_d, sizeof(long long) * (nb + 1), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    dev_free(bk_d);
    std::vector<Item> items;
    std::vector<int32_t> icls;  // class of every item
    std::vector<int32_t> sfirst, snch;
    items.reserve((size_t)nb + 16);
    int64_t nparts = 0;
    const int ncls = cl ? cl->ncolours : 1;
    auto class_of = [&](int64_t x) -> int {
        if (!cl) return 0;
        const std::vector<int64_t> &bnd = x < cl->nhub ? cl->hub_row : cl->class_row;
        return (int)(std::upper_bound(bnd.begin(), bnd.end(), x) - bnd.begin()) - 1;
    };
    for (int64_t b = 0; b < nb; ++b) {
        Item it;
        it.r0 = br[(size_t)b];
        it.r1 = br[(size_t)b + 1];
        it.lo = 0;
        it.hlo = 0;
        it.nhub = 0;
        const int cls = std::min(std::max(class_of(it.r0), 0), ncls - 1);
        if (cl) {
            it.lo = (int32_t)cl->class_row[(size_t)cls];
            it.nhub = (int32_t)cl->nhub;
            it.hlo = cl->nhub > 0 ? (int32_t)cl->hub_row[(size_t)cls] : 0;
        }
        const int64_t k0 = bk[(size_t)b], k1 = bk[(size_t)b + 1];
        if (k1 - k0 > long_row) {
            const int64_t nch = ceil_div(k1 - k0, chunk);
            it.slot = (int32_t)sfirst.size();
            sfirst.push_back((int32_t)nparts);
            snch.push_back((int32_t)nch);
            nparts += nch;
            for (int64_t ch = 0; ch < nch; ++ch) {
                it.k0 = k0 + ch * chunk;
                it.k1 = std::min(k1, it.k0 + chunk);
                items.push_back(it);
                icls.push_back(cls);
            }
        } else {
            it.slot = -1;
            it.k0 = k0;
            it.k1 = k1;
            items.push_back(it);
            icls.push_back(cls);
        }
    }
    ip.nitems = (int64_t)items.size();
    ip.nslots = (int64_t)sfirst.size();
    // group by class, stable (a class's hub items come before its other items)
    ip.class_item.assign((size_t)ncls + 1, 0);
    for (int32_t k : icls) ++ip.class_item[(size_t)k + 1];
    for (int k = 0; k < ncls; ++k) ip.class_item[(size_t)k + 1] += ip.class_item[(size_t)k];
    {
        std::vector<int64_t> at(ip.class_item.begin(), ip.class_item.end() - 1);
        std::vector<Item> grouped(items.size());
        for (size_t i = 0; i < items.size(); ++i) grouped[(size_t)at[(size_t)icls[i]]++] = items[i];
        items.swap(grouped);
    }
    ip.nparts = nparts;
    FJ_CUDA(dev_malloc(&ip.items, sizeof(Item) * std::max<size_t>(items.size(), 1)));
    FJ_CUDA(dev_malloc(&ip.slot_first, sizeof(int32_t) * std::max<size_t>(sfirst.size(), 1)));
    FJ_CUDA(dev_malloc(&ip.slot_nchunk, sizeof(int32_t) * std::max<size_t>(snch.size(), 1)));
    FJ_CUDA(dev_malloc(&ip.cnt, sizeof(int32_t) * std::max<size_t>(sfirst.size(), 1)));
    FJ_CUDA(dev_malloc(&ip.part, 2 * sizeof(double) * std::max<int64_t>(nparts, 1)));
    FJ_CUDA(cudaMemcpyAsync(ip.items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, st));
    if (!sfirst.empty()) {
        FJ_CUDA(cudaMemcpyAsync(ip.slot_first, sfirst.data(), sizeof(int32_t) * sfirst.size(), cudaMemcpyHostToDevice,
                                st));
        FJ_CUDA(cudaMemcpyAsync(ip.slot_nchunk, snch.data(), sizeof(int32_t) * snch.size(), cudaMemcpyHostToDevice,
                                st));
    }
    FJ_CUDA(cudaMemsetAsync(ip.cnt, 0, sizeof(int32_t) * std::max<size_t>(sfirst.size(), 1), st));
    FJ_CUDA(cudaStreamSynchronize(st));
    ip.built = true;
    return FJ_OK;
}

static fj_status make_plan(fj_graph *g, const fj_solve_opts *o, cudaStream_t st, Plan &p)
{
    p.mc = o->schedule != FJ_SCHED_JACOBI;
    if (!p.mc) {
        p.c = &g->csr;
        if (!g->wplan_csr.built) FJ_CHECK(build_items(g, g->csr, nullptr, g->wplan_csr, st, kTileWarp));
        p.wip = &g->wplan_csr;
        return FJ_OK;
    }
    FJ_CHECK(ensure_colouring(g, o->palette, st));
    p.c = &g->colr.pcsr;
    p.perm = g->colr.perm;
    if (!g->wplan_pcsr.built) FJ_CHECK(build_items(g, g->colr.pcsr, &g->colr, g->wplan_pcsr, st, kTileWarp));
    p.wip = &g->wplan_pcsr;
    return FJ_OK;
}

// Warp-tile items of the caller-order CSR (built on first use): the balanced
// work list other passes over the graph (the network's aggregations) share.
fj_status plain_items(fj_graph *g, cudaStream_t st, const ItemPlan **out)
{
    if (!g->wplan_csr.built) FJ_CHECK(build_items(g, g->csr, nullptr, g->wplan_csr, st, kTileWarp));
    *out = &g->wplan_csr;
    return FJ_OK;
}


struct FlagLoad {
    const int32_t *a;
    __device__ long long operator()(int64_t i) const { return (long long)a[i]; }
};

struct LongRowPred {
    const int64_t *rp;
    __device__ bool operator()(int64_t x) const
    {
        const int64_t a = rp[x], b = rp[x + 1];
        return b > a && (b - 1) / kChunkE - a / kChunkE > kLongChunks;
    }
};

// Chunk plan of CSR c: start bits, ranks, per-class row and nonzero ranges
// (cl = nullptr: the whole graph as one class), long rows grouped by class.
static fj_status build_chunk_plan(fj_graph *g, const DevCSR &c, const Colouring *cl, ChunkPlan &cp, cudaStream_t st)
{
    const int64_t n = c.n, nnz = c.nnz;
    cp.nch = std::max<int64_t>(1, ceil_div(nnz, kChunkE));
    const int64_t nwords = 8 * (cp.nch + 1);
    FJ_CUDA(dev_malloc(&cp.starts, sizeof(uint32_t) * (size_t)nwords));
    FJ_CUDA(dev_malloc(&cp.endbase, sizeof(int32_t) * (size_t)cp.nch));
    FJ_CUDA(dev_malloc(&cp.rank, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
    int32_t *nonempty = nullptr;
    long long *excl = nullptr;
    FJ_CUDA(dev_malloc(&nonempty, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
    FJ_CUDA(dev_malloc(&excl, sizeof(long long) * (size_t)(std::max(n, cp.nch) + 1)));
    FJ_CUDA(cudaMemsetAsync(cp.starts, 0, sizeof(uint32_t) * (size_t)nwords, st));
    k_start_bits<<<grid_for(n + 1, 256), 256, 0, st>>>(n, nnz, c.row_ptr, cp.starts, nonempty);
    FJ_CUDA(cudaGetLastError());
    Workspace &ws = g->ws;
    FJ_CHECK(ws_status(ws, scan_tiles(std::max(n, cp.nch), 256 * 8)));
    if (n > 0) {
        FJ_CUDA(scan<256, 8>(n, FlagLoad{nonempty}, excl, ws.count, ws.status, ws.tile_ctr, g->err, st));
        k_narrow_i32<<<grid_for(n, 256), 256, 0, st>>>(n, excl, cp.rank);
    }
    FJ_CUDA(scan<256, 8>(cp.nch, EndCount{cp.starts}, excl, ws.count, ws.status, ws.tile_ctr, g->err, st));
    k_narrow_i32<<<grid_for(cp.nch, 256), 256, 0, st>>>(cp.nch, excl, cp.endbase);
    FJ_CUDA(cudaGetLastError());
    // class ranges
    const int ncls = cl ? cl->ncolours : 1;
    cp.row0.clear();
    cp.row1.clear();
    for (int k = 0; k < ncls; ++k) {
        if (cl) {
            const bool hubs = cl->nhub > 0;
            cp.row0.push_back(hubs ? cl->hub_row[(size_t)k] : 0);
            cp.row1.push_back(hubs ? cl->hub_row[(size_t)k + 1] : 0);
            cp.row0.push_back(cl->class_row[(size_t)k]);
            cp.row1.push_back(cl->class_row[(size_t)k + 1]);
        } else {
            cp.row0.push_back(0);
            cp.row1.push_back(0);
            cp.row0.push_back(0);
            cp.row1.push_back(n);
        }
    }
    std::vector<int64_t> hrp((size_t)n + 1);
    FJ_CUDA(cudaMemcpyAsync(hrp.data(), c.row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToHost, st));
    // long rows, in row order
    int32_t *lr = nonempty;  // reused: the flags are no longer needed
    FJ_CUDA(compact<256, 8>(n, LongRowPred{c.row_ptr}, lr, ws.count, ws.status, ws.tile_ctr, g->err, st));
    long long nl = 0;
    FJ_CUDA(cudaMemcpyAsync(&nl, ws.count, sizeof(long long), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> hl((size_t)nl);
    if (nl > 0) FJ_CUDA(cudaMemcpy(hl.data(), lr, sizeof(int32_t) * (size_t)nl, cudaMemcpyDeviceToHost));
    cp.k0.assign(cp.row0.size(), 0);
    cp.k1.assign(cp.row0.size(), 0);
    for (size_t i = 0; i < cp.row0.size(); ++i) {
        cp.k0[i] = hrp[(size_t)cp.row0[i]];
        cp.k1[i] = hrp[(size_t)cp.row1[i]];
    }
    // group the long rows by class (each class's two ranges)
    std::vector<int32_t> grouped;
    grouped.reserve(hl.size());
    cp.long_off.assign((size_t)ncls + 1, 0);
    for (int k = 0; k < ncls; ++k) {
        for (int part = 0; part < 2; ++part) {
            const int64_t a = cp.row0[(size_t)(2 * k + part)], b = cp.row1[(size_t)(2 * k + part)];
            auto lo_it = std::lower_bound(hl.begin(), hl.end(), (int32_t)a);
            for (auto it = lo_it; it != hl.end() && *it < b; ++it) grouped.push_back(*it);
        }
        cp.long_off[(size_t)k + 1] = (int64_t)grouped.size();
    }
    FJ_CUDA(dev_malloc(&cp.long_rows, sizeof(int32_t) * std::max<size_t>(grouped.size(), 1)));
    if (!grouped.empty())
        FJ_CUDA(cudaMemcpy(cp.long_rows, grouped.data(), sizeof(int32_t) * grouped.size(), cudaMemcpyHostToDevice));
    dev_free(nonempty);
    dev_free(excl);
    cp.built = true;
    return read_dev_error(g, st);
}

// Resident gather blocks per device for dyn bytes of hot table (persistent grid).
template <typename T, bool W>
static int64_t gather_blocks(int dyn)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sweep_gather<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHotBytes);
        attr = true;
    }
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_gather<T, W>, kGatherThreads, dyn);
    return std::max(1, sms * std::max(1, per));
}

static int device_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            sms = 152;
    }
    return sms;
}

template <typename T, bool W>
static fj_status launch_classes(fj_graph *g, const Plan &p, cudaStream_t st, Run &run, T *dcur, const T *dprev)
{
    Workspace &ws = g->ws;
    const DevCSR &c = *p.c;
    const ChunkPlan &cp = *p.cp;
    T *r = reinterpret_cast<T *>(ws.r);
    const T *h = reinterpret_cast<const T *>(ws.h);
    const T *inv;
    if constexpr (sizeof(T) == 4) inv = reinterpret_cast<const T *>(c.inv32);
    else inv = reinterpret_cast<const T *>(c.inv64);
    const T *om = reinterpret_cast<const T *>(ws.om);
    T *rsum = reinterpret_cast<T *>(ws.rsum), *carry = reinterpret_cast<T *>(ws.carry);
    // hub prefix of the colour order (multicolour only): its first nhot ids go to the hot table
    const int nhub = p.mc ? (int)g->colr.nhub : 0;
    const int hot_cap = std::max(0, std::min<int>(nhub, kHotBytes / (int)sizeof(T)));
    const int64_t nres = gather_blocks<T, W>(hot_cap * (int)sizeof(T));
    const int sms = device_sms();
    const int ncls = (int)cp.long_off.size() - 1;
    for (int cl = 0; cl < ncls; ++cl) {
        const int64_t ka0 = cp.k0[(size_t)2 * cl], ka1 = cp.k1[(size_t)2 * cl];
        const int64_t kb0 = cp.k0[(size_t)2 * cl + 1], kb1 = cp.k1[(size_t)2 * cl + 1];
        const int64_t xa0 = cp.row0[(size_t)2 * cl], xa1 = cp.row1[(size_t)2 * cl];
        const int64_t xb0 = cp.row0[(size_t)2 * cl + 1], xb1 = cp.row1[(size_t)2 * cl + 1];
        const int64_t rows = (xa1 - xa0) + (xb1 - xb0);
        if (rows <= 0) continue;
        const int64_t chunks = (ka1 > ka0 ? ceil_div(ka1 - ka0, kChunkE) + 1 : 0) +
                               (kb1 > kb0 ? ceil_div(kb1 - kb0, kChunkE) + 1 : 0);
        // the class's first row (first hub row): every column below it belongs to an earlier class
        const int lo = p.mc ? (int)g->colr.class_row[(size_t)cl] : 0;
        const int hlo = nhub > 0 ? (int)g->colr.hub_row[(size_t)cl] : 0;
        FJ_CHECK(run.before(st));
        if (chunks > 0) {
            unsigned grid =
                (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(chunks, kGatherThreads / 32), nres));
            // a block stages the table only when its share of the class's
            // gathers is large beside it (a small graph's increments stay in
            // L2 anyway, and the copy would dominate its short launches);
            // without it, a short class takes one chunk per SM at a time
            const int64_t per_block = ((ka1 - ka0) + (kb1 - kb0)) / (int64_t)grid;
            const int nhot = per_block >= 2 * (int64_t)hot_cap ? hot_cap : 0;
            if (nhot == 0) grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, nres));
            const int dyn = nhot * (int)sizeof(T);
            k_sweep_gather<T, W><<<grid, kGatherThreads, dyn, st>>>(ka0, ka1, kb0, kb1, c.col, c.w, cp.starts,
                                                                     cp.endbase, lo, nhot, nhub, hlo, dcur, dprev,
                                                                     rsum, carry, ws.ctr, c.n, c.n);
            FJ_CUDA(cudaGetLastError());
        }
        const int64_t nlong = cp.long_off[(size_t)cl + 1] - cp.long_off[(size_t)cl];
        const unsigned rgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, 256), (int64_t)sms * 8));
        const unsigned lgrid = nlong > 0 ? (unsigned)std::min<int64_t>(ceil_div(nlong, 8), (int64_t)sms * 4) : 0;
        k_sweep_apply<T><<<rgrid + lgrid, 256, 0, st>>>(xa0, xa1, xb0, xb1, cp.long_rows + cp.long_off[(size_t)cl],
                                                        nlong, rgrid, c.row_ptr, cp.rank, rsum, carry, dcur, r, h,
                                                        inv, ws.zhat, c.indeg, om, ws.ctr, c.n);
        FJ_CUDA(cudaGetLastError());
        FJ_CHECK(run.after(st));
        ++run.launches;  // the gather launch
    }
    return FJ_OK;
}

// One sweep (multicolour: two launches per colour class, in order) or round
// (Jacobi: the whole graph as one class), then the stop test.  The two
// increment buffers swap roles every sweep.
template <typename T>
static fj_status launch_sweep(fj_graph *g, const Plan &p, cudaStream_t st, Run &run, int64_t sweep)
{
    Workspace &ws = g->ws;
    T *bufs[2] = {reinterpret_cast<T *>(ws.da), reinterpret_cast<T *>(ws.db)};
    T *dcur = bufs[sweep & 1];
    const T *dprev = bufs[(sweep - 1) & 1];
    if (p.c->w) FJ_CHECK((launch_classes<T, true>(g, p, st, run, dcur, dprev)));
    else FJ_CHECK((launch_classes<T, false>(g, p, st, run, dcur, dprev)));
    k_end_sweep<<<1, 1, 0, st>>>(ws.ctr);
    FJ_CUDA(cudaGetLastError());
    ++run.launches;
    return FJ_OK;
}

// A batch of `nsweeps` (even) sweeps captured once into a CUDA graph and
// replayed; the buffer parity repeats every two sweeps, and a pass always
// starts from cleared increment buffers, so every replay is exact.
template <typename T>
static fj_status sweep_graph(fj_graph *g, const Plan &p, int nsweeps, cudaGraphExec_t *out, int *launches)
{
    Workspace &ws = g->ws;
    const int a = sizeof(T) == 8 ? 1 : 0, b = p.mc ? 1 : 0;
    if (ws.gexec[a][b] && ws.gkey[a][b] == ws.gen && ws.gsweeps[a][b] == nsweeps) {
        *out = ws.gexec[a][b];
        *launches = ws.glaunch[a][b];
        return FJ_OK;
    }
    if (ws.gexec[a][b]) cudaGraphExecDestroy(ws.gexec[a][b]);
    ws.gexec[a][b] = nullptr;
    if (!ws.cap_stream) FJ_CUDA(cudaStreamCreateWithFlags(&ws.cap_stream, cudaStreamNonBlocking));
    Run dummy;
    FJ_CUDA(cudaStreamBeginCapture(ws.cap_stream, cudaStreamCaptureModeThreadLocal));
    fj_status s = FJ_OK;
    for (int j = 0; j < nsweeps && s == FJ_OK; ++j) s = launch_sweep<T>(g, p, ws.cap_stream, dummy, j);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ws.cap_stream, &graph);
    if (s != FJ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    FJ_CUDA(e);
    e = cudaGraphInstantiate(&ws.gexec[a][b], graph, 0);
    cudaGraphDestroy(graph);
    FJ_CUDA(e);
    ws.gkey[a][b] = ws.gen;
    ws.gsweeps[a][b] = nsweeps;
    ws.glaunch[a][b] = (int)dummy.launches;
    *out = ws.gexec[a][b];
    *launches = (int)dummy.launches;
    return FJ_OK;
}

// max |w| over the nonzeros into *out (ordered bits of a non-negative double).
__global__ void k_absmax_w(int64_t nnz, const float *__restrict__ w, unsigned long long *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, (double)fabsf(w[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(reinterpret_cast<double *>(out), m);
}

// Ew with max|w| < 2^Ew for the certificate's fixed-point scale; computed on
// the first certificate of a weighted CSR and kept (the weights are fixed).
static fj_status weight_exponent(const DevCSR &c, Workspace &ws, cudaStream_t st, int *ew)
{
    if (c.wexp == INT32_MIN) {
        FJ_CUDA(cudaMemsetAsync(ws.zmax, 0, sizeof(unsigned long long), st));
        k_absmax_w<<<grid_for(c.nnz, 256, 152 * 8), 256, 0, st>>>(c.nnz, c.w, ws.zmax);
        FJ_CUDA(cudaGetLastError());
        unsigned long long bits = 0;
        FJ_CUDA(cudaMemcpyAsync(&bits, ws.zmax, sizeof(bits), cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
        double wm = 0.0;
        std::memcpy(&wm, &bits, sizeof(wm));
        if (!std::isfinite(wm)) return FJ_ERR_INVALID_ARG;
        int e = 0;
        std::frexp(wm, &e);  // wm < 2^e
        c.wexp = wm > 0.0 ? e : -126;
    }
    *ew = c.wexp;
    return FJ_OK;
}

template <typename T>
static fj_status launch_certify(fj_graph *g, const Plan &p, double epsp, cudaStream_t st, Run &run)
{
    run.launches += 2;
    Workspace &ws = g->ws;
    const DevCSR &c = *p.c;
    const ItemPlan &ip = *p.wip;
    k_cert_reset<<<grid_for(g->ngraphs, 256), 256, 0, st>>>(g->ngraphs, reinterpret_cast<unsigned long long *>(ws.gstat));
    T *r = reinterpret_cast<T *>(ws.r), *da = reinterpret_cast<T *>(ws.da), *db = reinterpret_cast<T *>(ws.db);
    unsigned long long *gs = reinterpret_cast<unsigned long long *>(ws.gstat);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ip.nitems, 8), 152 * 8));
    int wexp = 0;
    if (c.w) FJ_CHECK(weight_exponent(c, ws, st, &wexp));
    FJ_CUDA(cudaMemsetAsync(ws.zmax, 0, sizeof(unsigned long long), st));
    k_split_absmax<<<grid_for(c.n, 256, 152 * 8), 256, 0, st>>>(c.n, ws.zhat, ws.zs, ws.zmax);
    run.launches += 1;
    if (c.w)
        k_certify<T, true><<<grid, 256, 0, st>>>(ip.items, ip.nitems, c.row_ptr, c.col, c.w, ws.zhat, ws.zs, ws.sp,
                                                 c.deg64, c.graph_of, epsp, r, da, db, gs, ip.slot_first,
                                                 ip.slot_nchunk, ip.part, ip.cnt, ws.r64, ws.zmax, wexp, c.n);
    else
        k_certify<T, false><<<grid, 256, 0, st>>>(ip.items, ip.nitems, c.row_ptr, c.col, c.w, ws.zhat, ws.zs, ws.sp,
                                                  c.deg64, c.graph_of, epsp, r, da, db, gs, ip.slot_first,
                                                  ip.slot_nchunk, ip.part, ip.cnt, ws.r64, ws.zmax, 0, c.n);
    FJ_CUDA(cudaGetLastError());
    return FJ_OK;
}

static fj_status check_index_record()
{
    long long dbg[4] = {0, 0, 0, 0};
    FJ_CUDA(cudaMemcpyFromSymbol(dbg, g_fj_dbg, sizeof(dbg)));
    if (dbg[0]) {
        set_error("index check failed: site %lld block %lld index %lld limit %lld", dbg[0], dbg[1], dbg[2], dbg[3]);
        return FJ_ERR_INVALID_ARG;
    }
    return FJ_OK;
}

// In-neighbour lists of the solve's row order: the CSR itself for an
// undirected graph (symmetric), the transposed CSR for a directed one
// (renumbered into the colour order for the multicolour schedule).
struct InLists {
    const int64_t *tp = nullptr;
    const int32_t *tc = nullptr;
    const float *tw = nullptr;
};

static fj_status in_lists(fj_graph *g, const Plan &p, cudaStream_t st, InLists &out)
{
    if (!g->directed) {
        out.tp = p.c->row_ptr;
        out.tc = p.c->col;
        out.tw = p.c->w;
    } else if (p.mc) {
        FJ_CHECK(ensure_ptranspose(g, st));
        out.tp = g->colr.tptr;
        out.tc = g->colr.tcol;
        out.tw = g->colr.tw;
    } else {
        out.tp = g->tptr;
        out.tc = g->tcol;
        out.tw = g->tw;
    }
    return FJ_OK;
}

// In-neighbour lists longer than this are scattered by a block each
// (k_frontier_push_long); FJ_FRONTIER_LONG overrides it (0: every entry).
static int64_t frontier_long_min()
{
    const char *e = std::getenv("FJ_FRONTIER_LONG");
    if (e && *e) {
        char *end = nullptr;
        const long long v = std::strtoll(e, &end, 10);
        if (end && *end == 0 && v >= 0) return (int64_t)v;
    }
    return 4096;
}

// Largest frontier the FP64 push takes on (entries); beyond it another pass
// of sweeps is cheaper.
static int64_t frontier_limit(int64_t entries) { return std::max<int64_t>(1024, entries / 64); }
constexpr int kMaxCleanups = 4;     // frontier-push episodes per solve
constexpr int kCleanupRounds = 64;  // rounds per episode

// FP64 frontier push rounds on the entries above threshold, until the
// frontier is empty (*cleared), grows past frontier_limit, or max_rounds.
static fj_status frontier_cleanup(fj_graph *g, const Plan &p, int k, double *r64, double *zhat, const double *sp,
                                  double epsp, int32_t *list, int max_rounds, cudaStream_t st, Run &run,
                                  int64_t *rounds, int64_t *pushes, bool *cleared)
{
    Workspace &ws = g->ws;
    const DevCSR &c = *p.c;
    const int64_t ne = c.n * k;
    const int64_t limit = frontier_limit(ne);
    InLists L;
    FJ_CHECK(in_lists(g, p, st, L));
    FJ_CHECK(ws_status(ws, scan_tiles(ne, 256 * 8)));
    if (limit > ws.cap_fdz) {  // [count, pad][entries: limit x int64][steps: limit x double]
        dev_free(ws.fdz);
        ws.fdz = nullptr;
        ws.cap_fdz = 0;
        FJ_CUDA(dev_malloc(&ws.fdz, 16 + 16 * (size_t)limit));
        ws.cap_fdz = limit;
    }
    unsigned long long *lng_n = reinterpret_cast<unsigned long long *>(ws.fdz);
    int64_t *lng_e = reinterpret_cast<int64_t *>(ws.fdz + 16);
    double *lng_dz = reinterpret_cast<double *>(ws.fdz + 16 + 8 * (size_t)limit);
    const int64_t long_min = frontier_long_min();
    *cleared = false;
    for (int it = 0; it < max_rounds; ++it) {
        FJ_CUDA(compact<256, 8>(ne, CleanPred{r64, sp, zhat, c.deg64, epsp, k}, list, ws.count, ws.status,
                                ws.tile_ctr, g->err, st));
        long long cnt = 0;
        FJ_CUDA(cudaMemcpyAsync(&cnt, ws.count, sizeof(long long), cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
        ++run.launches;
        if (cnt == 0) {
            *cleared = true;
            break;
        }
        if (cnt > limit) break;
        const unsigned grid = grid_for(cnt * 32, 256, 152 * 16);
        const unsigned lgrid = (unsigned)std::max<long long>(1, std::min<long long>(cnt, 152 * 2));
        FJ_CUDA(cudaMemsetAsync(lng_n, 0, sizeof(unsigned long long), st));
        if (L.tw) {
            k_frontier_push<true><<<grid, 256, 0, st>>>(list, ws.count, k, L.tp, L.tc, L.tw, c.deg64, r64, zhat,
                                                        ws.ctr, c.n, long_min, lng_n, lng_e, lng_dz);
            k_frontier_push_long<true><<<lgrid, 1024, 0, st>>>(lng_n, lng_e, lng_dz, ws.count, k, L.tp, L.tc, L.tw,
                                                               r64, ws.ctr, c.n);
        } else {
            k_frontier_push<false><<<grid, 256, 0, st>>>(list, ws.count, k, L.tp, L.tc, L.tw, c.deg64, r64, zhat,
                                                         ws.ctr, c.n, long_min, lng_n, lng_e, lng_dz);
            k_frontier_push_long<false><<<lgrid, 1024, 0, st>>>(lng_n, lng_e, lng_dz, ws.count, k, L.tp, L.tc,
                                                                L.tw, r64, ws.ctr, c.n);
        }
        FJ_CUDA(cudaGetLastError());
        run.launches += 2;
        ++*rounds;
        *pushes += cnt;
    }
    FJ_CHECK(check_index_record());
    return read_dev_error(g, st);
}

// Convergence trace of a solve (fj_solve_trace): rows of
// [ms since the first sweep, sweeps so far, max_v |r_v| / s'_v, kind].
struct Trace {
    double *rows = nullptr;
    int cap = 0;
    int count = 0;
};

// max_v |r_v| / s'_v of the residual r = s' - (I + L) zhat of the current
// estimate, in FP64, one warp per row, into *out (ordered bits of a
// non-negative double).  The push's own residual array lags: in the pull form
// a row's stored residual leaves out the increments its neighbours made after
// it in the sweep, so the trace evaluates the residual afresh.
__global__ void k_trace_resid(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const float *__restrict__ w, const double *__restrict__ deg,
                              const double *__restrict__ sp, const double *__restrict__ zhat, unsigned long long *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double m = 0.0;
    for (int64_t x = warp0; x < n; x += nwarps) {
        double acc = 0.0;
        for (int64_t k = rp[x] + lane; k < rp[x + 1]; k += 32) {
            const int32_t c = col[k];
            if (c >= 0 && c < n) acc = fma(w ? (double)w[k] : 1.0, zhat[c], acc);
        }
        acc = warp_sum(acc);
        const double r = fma(-(1.0 + deg[x]), zhat[x], sp[x]) + acc;
        const double rel = fabs(r) / sp[x];
        m = rel > m ? rel : m;  // a NaN never wins
    }
    if (lane == 0) atomic_max_nonneg(reinterpret_cast<double *>(out), m);
}

template <typename T>
static fj_status solve_t(fj_graph *g, const double *s, const double *z0, const fj_solve_opts *o, double *z_out,
                         fj_solve_info *info, int mem, Trace *tr = nullptr)
{
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)o->stream;
    const int64_t n = g->csr.n;
    const int ng = g->ngraphs;
    FJ_CHECK(ws_grow<T>(g, n, ng));
    Workspace &ws = g->ws;
    Plan p;
    FJ_CHECK(make_plan(g, o, st, p));
    {
        ChunkPlan &cpl = p.mc ? g->cplan_pcsr : g->cplan_csr;
        if (!cpl.built) FJ_CHECK(build_chunk_plan(g, *p.c, p.mc ? &g->colr : nullptr, cpl, st));
        p.cp = &cpl;
        if (cpl.nch > ws.cap_carry) {
            dev_free(ws.carry);
            ws.carry = nullptr;
            ws.cap_carry = 0;
            FJ_CUDA(dev_malloc(&ws.carry, sizeof(double) * (size_t)cpl.nch));
            ws.cap_carry = cpl.nch;
            ws.gen++;
        }
    }
    const DevCSR &c = *p.c;
    const double epsp = o->sigma * o->eps / (o->c + o->sigma);

    // stage s (and z0) on the device
    const double *sd = s, *z0d = z0;
    if (mem == FJ_MEM_HOST) {
        FJ_CUDA(cudaMemcpyAsync(ws.sin, s, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        sd = ws.sin;
        if (z0) {
            FJ_CUDA(cudaMemcpyAsync(ws.zout, z0, sizeof(double) * n, cudaMemcpyHostToDevice, st));
            z0d = ws.zout;
        }
    }
    unsigned long long *gs = reinterpret_cast<unsigned long long *>(ws.gstat);
    k_gstat_reset<<<1, 256, 0, st>>>(ng, gs);
    k_min_s<<<grid_for(n, 256, 152 * 4), 256, 0, st>>>(n, sd, g->csr.graph_of, gs, g->err);
    k_shift<<<grid_for(ng, 256), 256, 0, st>>>(ng, gs, o->c);
    T *r = reinterpret_cast<T *>(ws.r), *h = reinterpret_cast<T *>(ws.h);
    T *da = reinterpret_cast<T *>(ws.da), *db = reinterpret_cast<T *>(ws.db);
    const double *din = p.mc ? g->colr.din_p : nullptr;
    k_init<T><<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, sd, z0d, p.perm, c.graph_of, gs, epsp, o->omega, c.deg64,
                                                         din, ws.sp, ws.zhat, r, h, da, db,
                                                         reinterpret_cast<T *>(ws.om));
    FJ_CUDA(cudaGetLastError());
    FJ_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(Counters), st));
    FJ_CHECK(read_dev_error(g, st));
    Run run;
    run.profile = o->profile != 0;
    run.launches += 4;  // gstat reset, min s, shift, init
    int warm = z0 ? 1 : -1;
    if (z0) {
        // warm start: exact FP64 residual of z0, judged against the zero start
        FJ_CHECK(launch_certify<T>(g, p, epsp, st, run));
        std::vector<int> keep;
        FJ_CHECK(warm_judge(g, n, 1, ws.r64, ws.sp, st, keep));
        run.launches += 1;
        if (!keep[0]) {
            warm = 0;
            k_init<T><<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, sd, nullptr, p.perm, c.graph_of, gs, epsp,
                                                                 o->omega, c.deg64, din, ws.sp, ws.zhat, r, h, da,
                                                                 db, reinterpret_cast<T *>(ws.om));
            FJ_CUDA(cudaGetLastError());
            run.launches += 1;
        }
    }

    // profiling times every sweep launch, so no sweep may run past the stop flag;
    // otherwise sweeps run in captured batches of an even count
    int check = run.profile ? 1 : (o->check_every > 0 ? o->check_every : 8);
    if (!run.profile) check += check & 1;
    cudaGraphExec_t batch = nullptr;
    int batch_launches = 0;
    if (!run.profile) FJ_CHECK(sweep_graph<T>(g, p, check, &batch, &batch_launches));
    int refine = 0, cleanups = 0;
    int64_t f_rounds = 0, f_pushes = 0;
    fj_status result = FJ_OK;
    cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};
    float excluded_ms = 0.f;  // time the trace's own evaluations took, left out of the rows' times
    if (tr) {
        tr->count = 0;
        for (cudaEvent_t &e : tev) FJ_CUDA(cudaEventCreate(&e));
        FJ_CUDA(cudaEventRecord(tev[0], st));
    }
    // one trace row at this point of the stream (the stream is idle: every
    // caller has just synchronised); rel < 0 asks for the push residual
    auto trace_row = [&](double rel, double kind) -> fj_status {
        if (!tr || tr->count >= tr->cap) return FJ_OK;
        if (rel < 0.0) {
            FJ_CUDA(cudaEventRecord(tev[1], st));  // the sweeps end here; the evaluation is not timed
            FJ_CUDA(cudaMemsetAsync(ws.zmax, 0, sizeof(unsigned long long), st));
            k_trace_resid<<<152 * 16, 256, 0, st>>>(n, c.row_ptr, c.col, c.w, c.deg64, ws.sp, ws.zhat, ws.zmax);
            FJ_CUDA(cudaGetLastError());
            unsigned long long bits = 0;
            FJ_CUDA(cudaMemcpyAsync(&bits, ws.zmax, sizeof(bits), cudaMemcpyDeviceToHost, st));
            FJ_CUDA(cudaEventRecord(tev[2], st));
            FJ_CUDA(cudaStreamSynchronize(st));
            double d;
            std::memcpy(&d, &bits, sizeof(d));
            rel = d;
        } else {
            FJ_CUDA(cudaEventRecord(tev[1], st));
            FJ_CUDA(cudaEventRecord(tev[2], st));
            FJ_CUDA(cudaStreamSynchronize(st));
        }
        float ms = 0.f, ev_ms = 0.f;
        FJ_CUDA(cudaEventElapsedTime(&ms, tev[0], tev[1]));
        FJ_CUDA(cudaEventElapsedTime(&ev_ms, tev[1], tev[2]));
        ms -= excluded_ms;
        excluded_ms += ev_ms;
        double *row = tr->rows + 4 * (int64_t)tr->count++;
        row[0] = ms;
        row[1] = (double)ws.ctr_host->sweeps;
        row[2] = rel;
        row[3] = kind;
        return FJ_OK;
    };
    struct EvFree {
        cudaEvent_t *e;
        ~EvFree()
        {
            for (int i = 0; i < 3; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } ev_free{tev};
    // FP32 passes are restarted from the exact FP64 residual every
    // kFp32PassSweeps sweeps (iterative refinement): past that the FP32
    // residual drifts from the true one and further sweeps stall (a capped
    // pass on undirected R-MAT s24 cut the sweeps to certify from 163 to 96)
    const int64_t pass_cap = sizeof(T) == 4 ? std::min<int64_t>(o->max_sweeps, kFp32PassSweeps) : o->max_sweeps;
    double prev_rel = INFINITY, last_rel = INFINITY;
    int strikes = 0;  // restarts that did not halve the relative residual (bounded by max_refine)
    for (;;) {
        k_pass_reset<<<1, 1, 0, st>>>(ws.ctr, pass_cap);
        FJ_CUDA(cudaGetLastError());
        ++run.launches;
        for (;;) {
            if (batch) {
                FJ_CUDA(cudaGraphLaunch(batch, st));
                run.launches += batch_launches;
                run.push_launches += batch_launches - check;
            } else {
                for (int j = 0; j < check; ++j) FJ_CHECK(launch_sweep<T>(g, p, st, run, ++ws.sweep_parity));
            }
            FJ_CUDA(cudaMemcpyAsync(ws.ctr_host, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
            FJ_CUDA(cudaStreamSynchronize(st));
            FJ_CHECK(run.harvest());
            FJ_CHECK(check_index_record());
            FJ_CHECK(trace_row(-1.0, 0.0));
            if (ws.ctr_host->done) break;
        }
        const int done = ws.ctr_host->done;
        if (done == 3) {
            result = FJ_ERR_DIVERGED;
            set_error("residual became non-finite (omega %.3f)", o->omega);
            break;
        }
        auto certify_count = [&](double &viol) -> fj_status {
            FJ_CHECK(launch_certify<T>(g, p, epsp, st, run));
            FJ_CUDA(cudaMemcpyAsync(ws.gstat_host, ws.gstat, sizeof(double) * kGs * ng, cudaMemcpyDeviceToHost, st));
            FJ_CUDA(cudaStreamSynchronize(st));
            FJ_CHECK(check_index_record());
            viol = 0.0;
            double rel = 0.0;
            for (int i = 0; i < ng; ++i) {
                viol += ws.gstat_host[i * kGs + 5];
                rel = std::max(rel, ws.gstat_host[i * kGs + 3]);
            }
            last_rel = rel;
            return trace_row(rel, 1.0);
        };
        double viol = 0.0;
        FJ_CHECK(certify_count(viol));
        // few nodes left above threshold: FP64 frontier pushes on them, then
        // the exact certificate again (it also re-syncs the push residual)
        while (viol > 0.0 && viol <= (double)frontier_limit(n) && cleanups < kMaxCleanups) {
            bool cleared = false;
            ++cleanups;
            FJ_CHECK(frontier_cleanup(g, p, 1, ws.r64, ws.zhat, ws.sp, epsp, ws.list, kCleanupRounds, st, run,
                                      &f_rounds, &f_pushes, &cleared));
            FJ_CHECK(certify_count(viol));
            if (!cleared) break;
        }
        if (viol == 0.0) break;
        // a pass that reached its sweep cap is restarted from the FP64
        // residual like one that stopped pushing (a refinement pass); an FP32
        // pass stopped by its own length that at least halved the certified
        // relative residual does not count against max_refine
        const bool progress = done == 2 && pass_cap < o->max_sweeps && last_rel < 0.5 * prev_rel;
        // over-relaxation that made the certified residual grow from one pass
        // to the next is divergence (before the residual overflows)
        if (o->omega > 1.0 && done == 2 && last_rel > 2.0 * prev_rel) {
            result = FJ_ERR_DIVERGED;
            set_error("residual grew from pass to pass (omega %.3f)", o->omega);
            break;
        }
        prev_rel = last_rel;
        if (!progress) {
            if (strikes >= o->max_refine) {
                result = FJ_ERR_NOT_CONVERGED;
                set_error("refinement cap %d reached with %.0f nodes above threshold", o->max_refine, viol);
                break;
            }
            ++strikes;
        }
        ++refine;
    }
    // unshift into caller order
    double *zdst = mem == FJ_MEM_DEVICE ? z_out : ws.zout;
    k_unshift<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, ws.zhat, p.perm, c.graph_of, gs, zdst);
    FJ_CUDA(cudaGetLastError());
    ++run.launches;
    if (mem == FJ_MEM_HOST)
        FJ_CUDA(cudaMemcpyAsync(z_out, ws.zout, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(ws.gstat_host, ws.gstat, sizeof(double) * kGs * ng, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(ws.ctr_host, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    FJ_CHECK(read_dev_error(g, st));
    if (info) {
        for (int i = 0; i < ng; ++i) {
            const double *q = ws.gstat_host + (size_t)i * kGs;
            fj_solve_info &f = info[i];
            std::memset(&f, 0, sizeof(f));
            f.sweeps = ws.ctr_host->sweeps;
            f.pushes = (int64_t)ws.ctr_host->pushes;
            f.edges = (int64_t)(ws.ctr_host->edges + ws.ctr_host->fedges);
            f.frontier_edges = (int64_t)ws.ctr_host->fedges;
            f.refine_passes = refine;
            f.c_eff = q[1];
            f.eps_prime = epsp;
            f.resid_inf = q[2];
            f.resid_rel_max = q[3];
            f.z_inf = q[4];
            f.err_bound = q[2];
            f.cert_rel_err = q[4] > q[2] ? q[2] / (q[4] - q[2]) : INFINITY;
            f.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            f.converged = (q[5] == 0.0 && result == FJ_OK) ? 1 : 0;
            f.launches = run.launches;
            f.push_launches = run.push_launches;
            f.push_ms = run.push_ms;
            // every effective sweep reads each row and nonzero once; pushes add their own traffic
            const double tb = (double)sizeof(T);
            const double per_sweep = (double)c.nnz * (4.0 + (c.w ? 4.0 : 0.0) + tb) + (double)c.n * (8.0 + 5.0 * tb);
            f.push_bytes = (double)ws.ctr_host->sweeps * per_sweep + (double)ws.ctr_host->pushes * 20.0;
            f.method_bytes = (double)ws.ctr_host->edges * (4.0 + (c.w ? 4.0 : 0.0) + tb) +
                             (double)ws.ctr_host->pushes * 32.0;
            f.frontier_rounds = f_rounds;
            f.frontier_pushes = f_pushes;
            f.omega_used = o->omega;
            f.warm_start = warm;
        }
    }
    return result;
}

}  // namespace fj

using namespace fj;

// FJ_SCHED_AUTO: a solve whose residual becomes non-finite at omega > 1 (SOR
// over colour classes is proven for symmetric systems only, Section 5.2) is
// restarted from its start with omega = 1, where the sweep is Gauss-Seidel on
// the diagonally dominant M-matrix I + L and converges.
template <typename F>
static fj_status with_omega_fallback(const fj_solve_opts *opts, F run)
{
    const fj_status st = run(opts);
    if (st != FJ_ERR_DIVERGED || opts->schedule != FJ_SCHED_AUTO || !(opts->omega > 1.0)) return st;
    fj_solve_opts o = *opts;
    o.omega = 1.0;
    return run(&o);
}

extern "C" {

fj_status fj_solve(fj_graph *g, const double *s, const fj_solve_opts *opts, double *z_out, fj_solve_info *info,
                   int mem)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s != nullptr && z_out != nullptr, "s or z_out is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(check_opts(opts));
    return with_omega_fallback(opts, [&](const fj_solve_opts *o) {
        if (o->precision == FJ_PREC_FP32) return solve_t<float>(g, s, nullptr, o, z_out, info, mem);
        return solve_t<double>(g, s, nullptr, o, z_out, info, mem);
    });
}

fj_status fj_solve_trace(fj_graph *g, const double *s, const fj_solve_opts *opts, double *z_out, fj_solve_info *info,
                         int mem, double *trace, int cap, int *count)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s != nullptr && z_out != nullptr, "s or z_out is NULL");
    FJ_ARG(trace != nullptr && count != nullptr && cap >= 1, "trace, count or cap");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(check_opts(opts));
    Trace tr;
    tr.rows = trace;
    tr.cap = cap;
    const fj_status st = with_omega_fallback(opts, [&](const fj_solve_opts *o) {
        if (o->precision == FJ_PREC_FP32) return solve_t<float>(g, s, nullptr, o, z_out, info, mem, &tr);
        return solve_t<double>(g, s, nullptr, o, z_out, info, mem, &tr);
    });
    *count = tr.count;
    return st;
}

fj_status fj_solve_warm(fj_graph *g, const double *s, const double *z0, const fj_solve_opts *opts, double *z_out,
                        fj_solve_info *info, int mem)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s != nullptr && z0 != nullptr && z_out != nullptr, "s, z0 or z_out is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(check_opts(opts));
    return with_omega_fallback(opts, [&](const fj_solve_opts *o) {
        if (o->precision == FJ_PREC_FP32) return solve_t<float>(g, s, z0, o, z_out, info, mem);
        return solve_t<double>(g, s, z0, o, z_out, info, mem);
    });
}

fj_status fj_frontier(int64_t n, const void *r, const void *h, int precision, int32_t *list, int64_t *count,
                      void *stream)
{
    FJ_ARG(n >= 0 && n < (int64_t(1) << 31), "n must be in [0, 2^31)");
    FJ_ARG(r && h && list && count, "NULL pointer");
    FJ_ARG(precision == FJ_PREC_FP64 || precision == FJ_PREC_FP32, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t tiles = scan_tiles(n, 256 * 8);
    unsigned long long *status = nullptr;
    unsigned int *tctr = nullptr;
    int *err = nullptr;
    FJ_CUDA(cudaMallocAsync(&status, sizeof(unsigned long long) * tiles, st));
    FJ_CUDA(cudaMallocAsync(&tctr, sizeof(unsigned int), st));
    FJ_CUDA(cudaMallocAsync(&err, sizeof(int), st));
    FJ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    cudaError_t e;
    if (n == 0) {
        e = cudaMemsetAsync(count, 0, sizeof(int64_t), st);
    } else if (precision == FJ_PREC_FP32) {
        e = compact<256, 8>(n, FrontierPred<float>{(const float *)r, (const float *)h}, list, (long long *)count,
                            status, tctr, err, st);
    } else {
        e = compact<256, 8>(n, FrontierPred<double>{(const double *)r, (const double *)h}, list,
                            (long long *)count, status, tctr, err, st);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(status, st);
    cudaFreeAsync(tctr, st);
    cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "frontier", __FILE__, __LINE__);
    if (herr) {
        set_error("frontier look-back timed out");
        return FJ_ERR_TIMEOUT;
    }
    return FJ_OK;
}

fj_status fj_residual(fj_graph *g, const double *s, const double *z, double c_eff, double *r, int mem, void *stream)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s && z && r, "NULL pointer");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g->csr.n;
    const double *sd = s, *zd = z;
    double *rd = r;
    double *tmp = nullptr;
    if (mem == FJ_MEM_HOST) {
        FJ_CUDA(cudaMallocAsync(&tmp, sizeof(double) * 3 * n, st));
        FJ_CUDA(cudaMemcpyAsync(tmp, s, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        FJ_CUDA(cudaMemcpyAsync(tmp + n, z, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        sd = tmp;
        zd = tmp + n;
        rd = tmp + 2 * n;
    }
    const DevCSR &c = g->csr;
    k_residual<<<grid_for(n * 32, 256), 256, 0, st>>>(n, c.row_ptr, c.col, c.w, sd, zd, c_eff, rd);
    FJ_CUDA(cudaGetLastError());
    if (mem == FJ_MEM_HOST) {
        FJ_CUDA(cudaMemcpyAsync(r, rd, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaFreeAsync(tmp, st));
    }
    FJ_CUDA(cudaStreamSynchronize(st));
    return FJ_OK;
}

}  // extern "C"

// ============================================================== multi-RHS batch

namespace fj {

// Per right-hand side: minimum of s (column j of the node-major [n][k] S).
__global__ void k_min_s_batch(int64_t n, int k, const double *__restrict__ S, unsigned long long *gs, int *err)
{
    __shared__ unsigned long long sm[8];
    const int j = blockIdx.y;
    unsigned long long best = ~0ULL;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double x = S[v * k + j];
        if (!isfinite(x)) dev_error(err, DEV_BAD_OPINION);
        const unsigned long long key = order_key(x);
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, best, o);
        best = u < best ? u : best;
    }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < 8; ++i) best = sm[i] < best ? sm[i] : best;
        atomicMin(&gs[(int64_t)j * kGs], best);
    }
}

// Node-major initial state: s', zhat, r, h per (node, right-hand side); omega per node.
template <typename T>
__global__ void k_init_batch(int64_t n, int k, const double *__restrict__ S, const double *__restrict__ Z0,
                             const int32_t *__restrict__ perm, const unsigned long long *__restrict__ gs,
                             double epsp, double omega, const double *__restrict__ deg,
                             const double *__restrict__ din, double *__restrict__ sp, double *__restrict__ zhat,
                             T *__restrict__ r, T *__restrict__ h, T *__restrict__ da, T *__restrict__ db,
                             T *__restrict__ om)
{
    const double *gsd = reinterpret_cast<const double *>(gs);
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx - i * k);
        const int64_t o = perm ? perm[i] : i;
        const double ce = gsd[(int64_t)j * kGs + 1];
        const double spv = S[o * k + j] + ce;
        sp[idx] = spv;
        zhat[idx] = Z0 ? Z0[o * k + j] + ce : 0.0;
        r[idx] = (T)spv;
        h[idx] = threshold_of<T>(epsp * spv);
        da[idx] = T(0);
        db[idx] = T(0);
        if (j == 0) {
            double oi = omega;
            if (din && din[i] > 0.0) oi = fmin(omega, 0.98 * 2.0 * (1.0 + deg[i]) / (1.0 + deg[i] + din[i]));
            om[i] = (T)oi;
        }
    }
}

template <typename T>
__global__ void k_unshift_batch(int64_t n, int k, const double *__restrict__ zhat, const int32_t *__restrict__ perm,
                                const unsigned long long *__restrict__ gs, double *__restrict__ Z)
{
    const double *gsd = reinterpret_cast<const double *>(gs);
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx - i * k);
        const int64_t o = perm ? perm[i] : i;
        Z[o * k + j] = zhat[idx] - gsd[(int64_t)j * kGs + 1];
    }
}

// One colour class of a multi-RHS sweep: the update of k_sweep applied to k
// opinion vectors at once, one warp per warp tile.  A long row's chunks keep
// k partial sums each and the last chunk to finish applies the update.
template <typename T, bool W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_sweep_batch(const Item *__restrict__ items, int64_t item0, int64_t nitems, const int64_t *__restrict__ rp,
              const int32_t *__restrict__ col, const float *__restrict__ w, int k, T *dcur,
              const T *__restrict__ dprev, T *__restrict__ r, const T *__restrict__ h, const T *__restrict__ inv,
              T *__restrict__ zacc, const T *__restrict__ om, const int32_t *__restrict__ indeg,
              const int32_t *__restrict__ slot_first, const int32_t *__restrict__ slot_nchunk, double *partk,
              int32_t *cnt, Counters *ctr, unsigned int *tick, int64_t n_rows)
{
    __shared__ unsigned long long red[2][8];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (*reinterpret_cast<volatile int *>(&ctr->done)) return;
    const bool has1 = lane < k, has2 = lane + 32 < k;
    unsigned long long my_push = 0, my_edges = 0;
    bool bad = false;

    // row state loaded when the row becomes current, used when it completes
    T pr[2] = {T(0), T(0)}, ph[2] = {T(0), T(0)}, pom = T(0), pinv = T(0);
    int32_t pdeg = 0;
    auto begin = [&](int64_t x) {
        const int64_t q = x * k + lane;
        if (has1) {
            pr[0] = r[q];
            ph[0] = h[q];
        }
        if (has2) {
            pr[1] = r[q + 32];
            ph[1] = h[q + 32];
        }
        pom = om[x];
        pinv = inv[x];
        pdeg = indeg[x];
    };
    auto upd = [&](int64_t x, int hh, T acc) {
        const int64_t q = x * k + lane + 32 * hh;
        T rx = pr[hh] + acc;
        T dx = T(0);
        if (abs_t(rx) > ph[hh]) {
            dx = pom * rx * pinv;
            zacc[q] += dx;
            rx = (T(1) - pom) * rx;
            my_push += 1;
            my_edges += (unsigned long long)pdeg;
        }
        if (!isfinite(rx)) bad = true;
        r[q] = rx;
        dcur[q] = dx;
    };
    auto apply_row = [&](int64_t x, T s1, T s2) {
        if (has1) upd(x, 0, s1);
        if (has2) upd(x, 1, s2);
    };
    auto no_begin = [](int64_t) {};

    // tiles are drawn from tick[0] one at a time (dynamic balance across warps);
    // the last warp to retire resets tick[0..1] for the next launch
    for (;;) {
        unsigned int got = 0;
        if (lane == 0) got = atomicAdd(&tick[0], 1u);
        got = __shfl_sync(0xffffffffu, got, 0);
        if ((int64_t)got >= nitems) break;
        const Item it = items[item0 + got];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (!FJ_IDX_OK(11, r0, n_rows) || !FJ_IDX_OK(12, r1, n_rows + 1) ||
            (it.slot < 0 && !FJ_IDX_OK(13, r1 - r0, kWarpRows + 1)))
            continue;
        const int32_t lo = it.lo, hlo = it.hlo, nhub = it.nhub;
        auto src = [&](int32_t c) -> const T * {
            const bool earlier = c < nhub ? c < hlo : c < lo;
            return (earlier ? (const T *)dcur : dprev) + (int64_t)c * k;
        };
        auto add = [](T &acc, float a, T v) { acc += (T)a * v; };
        if (it.slot < 0) {
            warp_tile_k<T, T, W, D>(r0, r1, it.k0, it.k1, false, rp, col, w, begin, src, add, apply_row, lane,
                                    has1, has2, n_rows);
        } else {
            const int slot = it.slot;
            const int first = slot_first[slot], nch = slot_nchunk[slot];
            const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
            auto store_part = [&](int64_t, T s1, T s2) {
                if (has1) partk[(int64_t)(first + ci) * k + lane] = (double)s1;
                if (has2) partk[(int64_t)(first + ci) * k + lane + 32] = (double)s2;
            };
            warp_tile_k<T, T, W, D>(r0, r1, it.k0, it.k1, true, rp, col, w, no_begin, src, add, store_part, lane,
                                    has1, has2, n_rows);
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&cnt[slot], 1) == nch - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                double a1 = 0.0, a2 = 0.0;
                for (int c = 0; c < nch; ++c) {
                    if (has1) a1 += __ldcg(partk + (int64_t)(first + c) * k + lane);
                    if (has2) a2 += __ldcg(partk + (int64_t)(first + c) * k + lane + 32);
                }
                if (lane == 0) cnt[slot] = 0;
                begin(r0);
                apply_row(r0, (T)a1, (T)a2);
            }
        }
    }
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&tick[1], 1u) == gridDim.x * 8u - 1u) {
            tick[0] = 0u;
            tick[1] = 0u;
        }
    }
    my_push = warp_sum(my_push);
    my_edges = warp_sum(my_edges);
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[0][wl] = my_push;
        red[1][wl] = my_edges;
        if (anybad) ctr->nonfinite = 1.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long pp = 0, ee = 0;
        for (int i = 0; i < 8; ++i) {
            pp += red[0][i];
            ee += red[1][i];
        }
        if (pp) {
            atomicAdd(&ctr->pushes, pp);
            atomicAdd(&ctr->sweep_pushes, pp);
            atomicAdd(&ctr->edges, ee);
        }
    }
}

// FP64 certificate of every (node, right-hand side), as k_certify: a plain
// FP64 sum per (row, vector) with an FP32 magnitude sum beside it, and the
// compensated (Dot2) re-evaluation of the few entries whose residual lies
// within the plain sum's error bound of the threshold; long rows' chunks sum
// in 128-bit fixed point (fix_add) from the start.  Per-vector statistics
// are reduced per block in shared memory (maxima of non-negative doubles
// compare as integers) and added with one atomic per vector and field.
struct PlainAcc {
    double s;
};
struct FixAcc {
    u128 v;
    bool bad;
};

template <typename T, bool W>
__global__ void __launch_bounds__(256)
k_certify_batch(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
                const int32_t *__restrict__ col, const float *__restrict__ w, int k, const double *__restrict__ zhat,
                const double *__restrict__ sp, const double *__restrict__ deg, double epsp, T *__restrict__ r,
                T *__restrict__ da, T *__restrict__ db, unsigned long long *gs, const int32_t *__restrict__ slot_first,
                const int32_t *__restrict__ slot_nchunk, double *partk, int32_t *cnt, double *__restrict__ r64,
                const unsigned long long *__restrict__ zmaxp, int wexp, int64_t n_rows)
{
    __shared__ unsigned long long sred[4][64];
    const double zmax = __longlong_as_double((long long)*zmaxp);
    bool fix_bad = false;
    const int fixE = fix_exponent(zmax, W ? wexp : 0, fix_bad);
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 4 * 64; i += 256) (&sred[0][0])[i] = 0ULL;
    __syncthreads();
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    const bool has1 = lane < k, has2 = lane + 32 < k;
    double m_abs[2] = {0, 0}, m_rel[2] = {0, 0}, m_z[2] = {0, 0}, viol[2] = {0, 0};
    const double *gsd = reinterpret_cast<const double *>(gs);

    // row x, vector j = lane + 32 hh, from the plain sums over `len` terms
    auto finish = [&](int64_t x, int hh, PlainAcc acc, int64_t len) {
        const int j = lane + 32 * hh;
        const int64_t q = x * k + j;
        const double zx = zhat[q], spx = sp[q], dpl = 1.0 + deg[x];
        double rx = fma(-dpl, zx, spx) + acc.s;
        const double thr = fmax(epsp * spx, resid_floor(deg[x], zx));
        const double bnd = plain_bound(len, deg[x], zmax, dpl * zx, spx);
        if (fabs(fabs(rx) - thr) <= bnd || !(fabs(rx) <= 1e300)) {
            DD d{0.0, 0.0};  // exact re-evaluation of this entry, by this lane
            for (int64_t kk = rp[x]; kk < rp[x + 1]; ++kk) {
                const int32_t c = __ldg(col + kk);
                if (FJ_IDX_OK(4, c, n_rows)) dd_fma(d, W ? (double)__ldg(w + kk) : 1.0, zhat[(int64_t)c * k + j]);
            }
            dd_add(d, spx);
            dd_fma(d, -dpl, zx);
            rx = dd_value(d);
        }
        const double ce = gsd[(int64_t)j * kGs + 1];
        const double ax = fabs(rx) <= 1e300 ? fabs(rx) : INFINITY;
        m_abs[hh] = fmax(m_abs[hh], ax);
        m_rel[hh] = fmax(m_rel[hh], (double)((float)ax / (float)spx));
        m_z[hh] = fmax(m_z[hh], fabs(zx - ce));
        if (ax > thr) viol[hh] += 1.0;
        r[q] = resid_store<T>(rx);
        r64[q] = rx;
        da[q] = T(0);
        db[q] = T(0);
    };
    // row x, vector lane + 32 hh, from the fixed-point sum of a_xc zhat_c
    // over the row's len nonzeros; the sum's error bound counts against the
    // row (a row within it of the threshold is not certified)
    auto finish_fix = [&](int64_t x, int hh, u128 sum, bool bad, int64_t len) {
        const int j = lane + 32 * hh;
        const int64_t q = x * k + j;
        const double zx = zhat[q], spx = sp[q], dpl = 1.0 + deg[x];
        const DD off = fix_value(sum, fixE);
        DD acc = off;
        dd_add(acc, spx);
        dd_fma(acc, -dpl, zx);
        double rx = dd_value(acc);
        if (bad) rx = __longlong_as_double(0x7ff8000000000000ll);  // non-finite input: NaN
        const double unit = __longlong_as_double((long long)(fixE - kFixBits + 1023) << 52);
        const double slack =
            (double)((W ? 2 : 1) * len + 4) * unit + 0x1p-100 * (fabs(off.hi) + dpl * fabs(zx) + fabs(spx));
        const double thr = fmax(epsp * spx, resid_floor(deg[x], zx));
        const double ce = gsd[(int64_t)j * kGs + 1];
        const double ax = fabs(rx) <= 1e300 ? fabs(rx) : INFINITY;
        m_abs[hh] = fmax(m_abs[hh], ax);
        m_rel[hh] = fmax(m_rel[hh], ax / spx);
        m_z[hh] = fmax(m_z[hh], fabs(zx - ce));
        if (ax + slack > thr) viol[hh] += 1.0;
        r[q] = resid_store<T>(rx);
        r64[q] = rx;
        da[q] = T(0);
        db[q] = T(0);
    };
    auto src = [&](int32_t c) -> const double * { return zhat + (int64_t)c * k; };
    auto add = [](PlainAcc &acc, float a, double v) { acc.s = W ? fma((double)a, v, acc.s) : acc.s + v; };
    auto no_begin = [](int64_t) {};
    for (int64_t ii = (int64_t)blockIdx.x * 8 + wl; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (!FJ_IDX_OK(1, r0, n_rows) || !FJ_IDX_OK(2, r1, n_rows + 1) ||
            (it.slot < 0 && !FJ_IDX_OK(13, r1 - r0, kWarpRows + 1)))
            continue;
        auto add_fix = [&](FixAcc &acc, float a, double v) {
            if (W) {
                const double av = (double)a, pr = __dmul_rn(av, v);
                fix_add(acc.v, pr, fixE, acc.bad);
                fix_add(acc.v, fma(av, v, -pr), fixE, acc.bad);  // the product's rounding error
            } else {
                fix_add(acc.v, v, fixE, acc.bad);
            }
        };
        if (it.slot < 0) {
            auto short_row = [&](int64_t x, PlainAcc s1, PlainAcc s2) {
                const int64_t len = rp[x + 1] - rp[x];
                if (has1) finish(x, 0, s1, len);
                if (has2) finish(x, 1, s2, len);
            };
            warp_tile_k<PlainAcc, double, W, 8>(r0, r1, it.k0, it.k1, false, rp, col, w, no_begin, src, add,
                                                short_row, lane, has1, has2, n_rows);
        } else {
            // chunks of long rows: fixed-point sums from the start (a hub's
            // plain-sum bound always straddles its threshold); a chunk's sum
            // is below 2^104, so a top word of INT64_MIN marks a bad chunk
            const int slot = it.slot;
            const int first = slot_first[slot], nch = slot_nchunk[slot];
            const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
            unsigned long long *pc =
                reinterpret_cast<unsigned long long *>(partk) + 2 * ((int64_t)(first + ci) * k + lane);
            auto put = [&](unsigned long long *q, const FixAcc &a) {
                const bool b = a.bad || fix_bad;
                q[0] = b ? 0ull : (unsigned long long)a.v;
                q[1] = b ? 0x8000000000000000ull : (unsigned long long)(a.v >> 64);
            };
            auto store_part = [&](int64_t, FixAcc s1, FixAcc s2) {
                if (has1) put(pc, s1);
                if (has2) put(pc + 64, s2);
            };
            warp_tile_k<FixAcc, double, W, 8>(r0, r1, it.k0, it.k1, true, rp, col, w, no_begin, src, add_fix,
                                              store_part, lane, has1, has2, n_rows);
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&cnt[slot], 1) == nch - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                u128 a1 = 0, a2 = 0;
                bool b1 = false, b2 = false;
                const unsigned long long *pw = reinterpret_cast<const unsigned long long *>(partk);
                for (int c = 0; c < nch; ++c) {
                    const unsigned long long *q = pw + 2 * ((int64_t)(first + c) * k + lane);
                    if (has1) {
                        const unsigned long long lo = __ldcg(q), hi = __ldcg(q + 1);
                        b1 |= hi == 0x8000000000000000ull;
                        a1 += ((u128)hi << 64) | (u128)lo;
                    }
                    if (has2) {
                        const unsigned long long lo = __ldcg(q + 64), hi = __ldcg(q + 65);
                        b2 |= hi == 0x8000000000000000ull;
                        a2 += ((u128)hi << 64) | (u128)lo;
                    }
                }
                if (lane == 0) cnt[slot] = 0;
                const int64_t len = rp[r0 + 1] - rp[r0];
                if (has1) finish_fix(r0, 0, a1, b1, len);
                if (has2) finish_fix(r0, 1, a2, b2, len);
            }
        }
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        if (!(hh == 0 ? has1 : has2)) continue;
        const int j = lane + 32 * hh;
        atomicMax(&sred[0][j], (unsigned long long)__double_as_longlong(m_abs[hh]));
        atomicMax(&sred[1][j], (unsigned long long)__double_as_longlong(m_rel[hh]));
        atomicMax(&sred[2][j], (unsigned long long)__double_as_longlong(m_z[hh]));
        atomicAdd(&sred[3][j], (unsigned long long)viol[hh]);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += 256) {
        unsigned long long *gj = gs + (int64_t)j * kGs;
        atomic_max_nonneg(reinterpret_cast<double *>(gj + 2), __longlong_as_double((long long)sred[0][j]));
        atomic_max_nonneg(reinterpret_cast<double *>(gj + 3), __longlong_as_double((long long)sred[1][j]));
        atomic_max_nonneg(reinterpret_cast<double *>(gj + 4), __longlong_as_double((long long)sred[2][j]));
        if (sred[3][j]) atomicAdd(reinterpret_cast<double *>(gj + 5), (double)sred[3][j]);
    }
}

// ---------------------------------------------------------------- bulk-copy batch sweep
//
// The batch sweep with the neighbours' k-vectors gathered by the copy engine:
// for each batch of kBulkRows nonzeros of a tile, lane l issues one bulk
// asynchronous copy (cp.async.bulk, completion counted in bytes on an
// mbarrier) of row col[l] of the increment buffer (k FP32 values, 16-byte
// aligned because k is a multiple of 4) into a per-warp shared-memory ring of
// two stages, then the warp consumes the previous batch from shared memory
// while this one is in flight.  Each warp keeps up to 2 kBulkRows rows in flight with
// no registers held for them, which the per-lane loads of k_sweep_batch
// cannot.  Otherwise the update is k_sweep_batch's.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
constexpr uint32_t kBulkWaitLimit = 1u << 22;  // polls of an mbarrier before the kernel reports a timeout
constexpr int kBulkRows = 16;                  // nonzeros (gathered rows) per stage

template <bool W>
__global__ void __launch_bounds__(256, 3)
k_sweep_batch_bulk(const Item *__restrict__ items, int64_t item0, int64_t nitems, const int64_t *__restrict__ rp,
                   const int32_t *__restrict__ col, const float *__restrict__ w, int k, float *dcur,
                   const float *__restrict__ dprev, float *__restrict__ r, const float *__restrict__ h,
                   const float *__restrict__ inv, float *__restrict__ zacc, const float *__restrict__ om,
                   const int32_t *__restrict__ indeg, const int32_t *__restrict__ slot_first,
                   const int32_t *__restrict__ slot_nchunk, double *partk, int32_t *cnt, Counters *ctr,
                   unsigned int *tick, int *err, int64_t n_rows)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) float ring_all[];  // [8 warps][2 stages][kBulkRows rows][k]
    __shared__ uint64_t bars[8][2];
    __shared__ unsigned long long red[2][8];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (*reinterpret_cast<volatile int *>(&ctr->done)) return;
    float *ring = ring_all + (size_t)wl * 2 * kBulkRows * k;
    if (lane == 0) {
        tc::mbar_init(&bars[wl][0], 1);
        tc::mbar_init(&bars[wl][1], 1);
    }
    __syncwarp();
    uint32_t phase = 0;  // bit s: parity of the next completion of stage s
    bool timed_out = false;
    const bool has1 = lane < k, has2 = lane + 32 < k;
    const uint32_t row_bytes = (uint32_t)k * 4u;
    unsigned long long my_push = 0, my_edges = 0;
    bool bad = false;

    float pr[2] = {0.f, 0.f}, ph[2] = {0.f, 0.f}, pom = 0.f, pinv = 0.f;
    int32_t pdeg = 0;
    auto begin = [&](int64_t x) {
        const int64_t q = x * k + lane;
        if (has1) {
            pr[0] = r[q];
            ph[0] = h[q];
        }
        if (has2) {
            pr[1] = r[q + 32];
            ph[1] = h[q + 32];
        }
        pom = om[x];
        pinv = inv[x];
        pdeg = indeg[x];
    };
    auto upd = [&](int64_t x, int hh, float acc) {
        const int64_t q = x * k + lane + 32 * hh;
        float rx = pr[hh] + acc;
        float dx = 0.f;
        if (fabsf(rx) > ph[hh]) {
            dx = pom * rx * pinv;
            zacc[q] += dx;
            rx = (1.f - pom) * rx;
            my_push += 1;
            my_edges += (unsigned long long)pdeg;
        }
        if (!isfinite(rx)) bad = true;
        r[q] = rx;
        dcur[q] = dx;
    };
    auto apply_row = [&](int64_t x, float s1, float s2) {
        if (has1) upd(x, 0, s1);
        if (has2) upd(x, 1, s2);
    };

    // Walk of [k0, k1): rows r0.. (a tile) or one chunk of row r0.  Returns
    // false after a wait that timed out (the warp then stops).
    auto walk = [&](int64_t r0, int64_t r1, int64_t k0, int64_t k1, bool chunk, int32_t lo, int32_t hlo,
                    int32_t nhub, float &o1, float &o2) -> bool {
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
        if (!chunk && x < r1) begin(x);
        float a1 = 0.f, a2 = 0.f;
        auto flush_until = [&](int64_t pos) {
            while (x < r1 && xe <= pos) {
                if (!chunk) apply_row(x, a1, a2);
                else {
                    o1 = a1;
                    o2 = a2;
                }
                a1 = a2 = 0.f;
                ++x;
                if (x < r1) {
                    xe = row_end(x);
                    if (!chunk) begin(x);
                }
            }
        };
        // issue the copies of the batch at `base` into stage s; returns the lane's weight
        auto issue = [&](int64_t base, int s) -> float {
            const int64_t kk = base + lane;
            int32_t cl = 0;
            float al = 0.f;
            const bool in = lane < kBulkRows && kk < k1;
            if (in) {
                cl = __ldg(col + kk);
                al = W ? __ldg(w + kk) : 1.f;
                if (!FJ_IDX_OK(15, cl, n_rows)) {
                    cl = 0;
                    al = 0.f;
                }
            }
            const int64_t left = k1 - base;
            const uint32_t m = (uint32_t)(left < kBulkRows ? left : kBulkRows);
            if (lane == 0) mbar_expect_tx(&bars[wl][s], m * row_bytes);
            __syncwarp();
            if (in) {
                const bool earlier = cl < nhub ? cl < hlo : cl < lo;
                const float *srcp = (earlier ? (const float *)dcur : dprev) + (int64_t)cl * k;
                bulk_g2s(ring + ((size_t)s * kBulkRows + lane) * k, srcp, row_bytes, &bars[wl][s]);
            }
            return al;
        };
        int s = 0;
        float al_cur = 0.f;
        if (k0 < k1) al_cur = issue(k0, 0);
        for (int64_t base = k0; base < k1; base += kBulkRows) {
            float al_nxt = 0.f;
            if (base + kBulkRows < k1) al_nxt = issue(base + kBulkRows, s ^ 1);
            if (!tc::mbar_wait_bounded(&bars[wl][s], (phase >> s) & 1u, kBulkWaitLimit)) return false;
            phase ^= 1u << s;
            const int64_t left = k1 - base;
            const int m = (int)(left < kBulkRows ? left : kBulkRows);
            const float *st = ring + (size_t)s * kBulkRows * k;
            for (int t = 0; t < m; ++t) {
                flush_until(base + t);
                const float a = __shfl_sync(FULL, al_cur, t);
                if (has1) a1 += a * st[t * k + lane];
                if (has2) a2 += a * st[t * k + lane + 32];
            }
            __syncwarp();
            tc::fence_async_smem();  // these reads come before the next copies into stage s
            al_cur = al_nxt;
            s ^= 1;
        }
        flush_until(k1);
        return true;
    };

    for (;;) {
        unsigned int got = 0;
        if (lane == 0) got = atomicAdd(&tick[0], 1u);
        got = __shfl_sync(FULL, got, 0);
        if ((int64_t)got >= nitems) break;
        const Item it = items[item0 + got];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (!FJ_IDX_OK(11, r0, n_rows) || !FJ_IDX_OK(12, r1, n_rows + 1) ||
            (it.slot < 0 && !FJ_IDX_OK(13, r1 - r0, kWarpRows + 1)))
            continue;
        float o1 = 0.f, o2 = 0.f;
        if (!walk(r0, r1, it.k0, it.k1, it.slot >= 0, it.lo, it.hlo, it.nhub, o1, o2)) {
            timed_out = true;
            break;
        }
        if (it.slot >= 0) {
            const int slot = it.slot;
            const int first = slot_first[slot], nch = slot_nchunk[slot];
            const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
            if (has1) partk[(int64_t)(first + ci) * k + lane] = (double)o1;
            if (has2) partk[(int64_t)(first + ci) * k + lane + 32] = (double)o2;
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&cnt[slot], 1) == nch - 1;
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
                double a1 = 0.0, a2 = 0.0;
                for (int c = 0; c < nch; ++c) {
                    if (has1) a1 += __ldcg(partk + (int64_t)(first + c) * k + lane);
                    if (has2) a2 += __ldcg(partk + (int64_t)(first + c) * k + lane + 32);
                }
                if (lane == 0) cnt[slot] = 0;
                begin(r0);
                apply_row(r0, (float)a1, (float)a2);
            }
        }
    }
    if (timed_out) {
        // report, then let every copy this warp issued land before the block
        // leaves (both stages' outstanding phases, each wait bounded)
        if (lane == 0) dev_error(err, DEV_SPIN_TIMEOUT);
        for (int s = 0; s < 2; ++s) tc::mbar_wait_bounded(&bars[wl][s], (phase >> s) & 1u, kBulkWaitLimit);
    }
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&tick[1], 1u) == gridDim.x * 8u - 1u) {
            tick[0] = 0u;
            tick[1] = 0u;
        }
    }
    my_push = warp_sum(my_push);
    my_edges = warp_sum(my_edges);
    const unsigned anybad = __ballot_sync(FULL, bad);
    if (lane == 0) {
        red[0][wl] = my_push;
        red[1][wl] = my_edges;
        if (anybad) ctr->nonfinite = 1.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long pp = 0, ee = 0;
        for (int i = 0; i < 8; ++i) {
            pp += red[0][i];
            ee += red[1][i];
        }
        if (pp) {
            atomicAdd(&ctr->pushes, pp);
            atomicAdd(&ctr->sweep_pushes, pp);
            atomicAdd(&ctr->edges, ee);
        }
    }
}

// Resident blocks of the batch sweep kernel (its persistent grid).
template <typename T>
static int64_t batch_sweep_blocks(bool weighted)
{
    static int cached[2] = {0, 0};
    int &nres = cached[weighted ? 1 : 0];
    if (nres == 0) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_batch<T, true, 8>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_batch<T, false, 8>, 256, 0);
        nres = std::max(1, sms * std::max(1, per));
    }
    return nres;
}

static fj_status bws_grow(fj_graph *g, int k, int64_t nparts, int64_t nclasses)
{
    BatchWorkspace &b = g->bws;
    if (nclasses > b.cap_tick) {
        b.cap_tick = 0;  // stays 0 if an allocation fails, so the next call grows again
        dev_free(b.tick);
        b.tick = nullptr;
        FJ_CUDA(dev_malloc(&b.tick, sizeof(unsigned int) * 2 * (size_t)nclasses));
        FJ_CUDA(cudaMemset(b.tick, 0, sizeof(unsigned int) * 2 * (size_t)nclasses));
        b.cap_tick = nclasses;
    }
    const int64_t need = g->csr.n * k;
    if (need > b.cap) {
        b.cap = 0;
        void **vb[] = {&b.r, &b.h, &b.da, &b.db, &b.z32};
        for (void **p : vb) {
            dev_free(*p);
            *p = nullptr;
            FJ_CUDA(dev_malloc(p, sizeof(double) * (size_t)need));
        }
        double **db_[] = {&b.zhat, &b.sp, &b.sin, &b.zout, &b.r64};
        for (double **p : db_) {
            dev_free(*p);
            *p = nullptr;
            FJ_CUDA(dev_malloc(p, sizeof(double) * (size_t)need));
        }
        dev_free(b.list);
        b.list = nullptr;
        FJ_CUDA(dev_malloc(&b.list, sizeof(int32_t) * (size_t)need));
        b.cap = need;
    }
    if (!b.om) FJ_CUDA(dev_malloc(&b.om, sizeof(double) * (size_t)g->csr.n));
    if (k > b.cap_k) {
        b.cap_k = 0;
        dev_free(b.gstat);
        b.gstat = nullptr;
        if (b.gstat_host) cudaFreeHost(b.gstat_host);
        b.gstat_host = nullptr;
        FJ_CUDA(dev_malloc(&b.gstat, sizeof(double) * kGs * k));
        FJ_CUDA(cudaMallocHost(&b.gstat_host, sizeof(double) * kGs * k));
        b.cap_k = k;
    }
    const int64_t np = 2 * std::max<int64_t>(nparts, 1) * k;
    if (np > b.cap_partk) {
        b.cap_partk = 0;
        dev_free(b.partk);
        b.partk = nullptr;
        FJ_CUDA(dev_malloc(&b.partk, sizeof(double) * (size_t)np));
        b.cap_partk = np;
    }
    return FJ_OK;
}

template <typename T>
static fj_status solve_batch_t(fj_graph *g, const double *S, const double *Z0, int k, const fj_solve_opts *o,
                               double *Z, fj_solve_info *info, int mem)
{
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)o->stream;
    const int64_t n = g->csr.n;
    Workspace &ws = g->ws;
    if (!ws.ctr) {
        FJ_CUDA(dev_malloc(&ws.ctr, sizeof(Counters)));
        FJ_CUDA(cudaMallocHost(&ws.ctr_host, sizeof(Counters)));
    }
    if (!ws.zmax) FJ_CUDA(dev_malloc(&ws.zmax, sizeof(unsigned long long)));
    Plan p;
    FJ_CHECK(make_plan(g, o, st, p));
    const DevCSR &c = *p.c;
    const ItemPlan &wp = *p.wip;
    FJ_CHECK(bws_grow(g, k, wp.nparts, (int64_t)wp.class_item.size()));
    BatchWorkspace &b = g->bws;
    const double epsp = o->sigma * o->eps / (o->c + o->sigma);
    const double *Sd = S, *Z0d = Z0;
    if (mem == FJ_MEM_HOST) {
        FJ_CUDA(cudaMemcpyAsync(b.sin, S, sizeof(double) * n * k, cudaMemcpyHostToDevice, st));
        Sd = b.sin;
        if (Z0) {
            FJ_CUDA(cudaMemcpyAsync(b.zout, Z0, sizeof(double) * n * k, cudaMemcpyHostToDevice, st));
            Z0d = b.zout;
        }
    }
    unsigned long long *gs = reinterpret_cast<unsigned long long *>(b.gstat);
    k_gstat_reset<<<1, 256, 0, st>>>(k, gs);
    k_min_s_batch<<<dim3(grid_for(n, 256, 64), k), 256, 0, st>>>(n, k, Sd, gs, g->err);
    k_shift<<<1, 64, 0, st>>>(k, gs, o->c);
    T *r = reinterpret_cast<T *>(b.r), *h = reinterpret_cast<T *>(b.h);
    T *da = reinterpret_cast<T *>(b.da), *db = reinterpret_cast<T *>(b.db);
    T *om = reinterpret_cast<T *>(b.om);
    T *zacc = sizeof(T) == 4 ? reinterpret_cast<T *>(b.z32) : reinterpret_cast<T *>(b.zhat);
    if (sizeof(T) == 4) FJ_CUDA(cudaMemsetAsync(b.z32, 0, sizeof(float) * n * k, st));
    const double *din = p.mc ? g->colr.din_p : nullptr;
    k_init_batch<T><<<grid_for(n * k, 256, 152 * 16), 256, 0, st>>>(n, k, Sd, Z0d, p.perm, gs, epsp, o->omega,
                                                                    c.deg64, din, b.sp, b.zhat, r, h, da, db, om);
    FJ_CUDA(cudaGetLastError());
    FJ_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(Counters), st));
    FJ_CHECK(read_dev_error(g, st));
    const T *inv;
    if constexpr (sizeof(T) == 4) inv = reinterpret_cast<const T *>(c.inv32);
    else inv = reinterpret_cast<const T *>(c.inv64);
    const unsigned cgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(wp.nitems, 8), 152 * 8));
    int wexp = 0;
    if (c.w) FJ_CHECK(weight_exponent(c, ws, st, &wexp));
    auto certify = [&]() -> fj_status {
        k_cert_reset<<<1, 64, 0, st>>>(k, gs);
        if (sizeof(T) == 4)
            k_fold<<<grid_for(n * k, 256, 152 * 8), 256, 0, st>>>(n * k, reinterpret_cast<float *>(b.z32), b.zhat);
        FJ_CUDA(cudaMemsetAsync(ws.zmax, 0, sizeof(unsigned long long), st));
        k_absmax<<<grid_for(n * k, 256, 152 * 8), 256, 0, st>>>(n * k, b.zhat, ws.zmax);
        if (c.w)
            k_certify_batch<T, true><<<cgrid, 256, 0, st>>>(wp.items, wp.nitems, c.row_ptr, c.col, c.w, k, b.zhat,
                                                            b.sp, c.deg64, epsp, r, da, db, gs, wp.slot_first,
                                                            wp.slot_nchunk, b.partk, wp.cnt, b.r64, ws.zmax, wexp, c.n);
        else
            k_certify_batch<T, false><<<cgrid, 256, 0, st>>>(wp.items, wp.nitems, c.row_ptr, c.col, c.w, k, b.zhat,
                                                             b.sp, c.deg64, epsp, r, da, db, gs, wp.slot_first,
                                                             wp.slot_nchunk, b.partk, wp.cnt, b.r64, ws.zmax, wexp, c.n);
        FJ_CUDA(cudaGetLastError());
        return FJ_OK;
    };
    std::vector<int> warm((size_t)k, Z0 ? 1 : -1);
    if (Z0) {
        // every vector's start is judged against its zero start; the losers restart from zero
        FJ_CHECK(certify());
        std::vector<int> keep;
        FJ_CHECK(warm_judge(g, n, k, b.r64, b.sp, st, keep));
        bool any = false;
        for (int j = 0; j < k; ++j) {
            warm[(size_t)j] = keep[(size_t)j];
            any = any || !keep[(size_t)j];
        }
        if (any) {
            std::vector<int> cold((size_t)k);
            for (int j = 0; j < k; ++j) cold[(size_t)j] = keep[(size_t)j] ? 0 : 1;
            // the flags go after the judge's sums (the buffer holds room for 64)
            int *cold_d = reinterpret_cast<int *>(g->ws.judge + (size_t)kJudgeBlocks * k * 2);
            FJ_CUDA(cudaMemcpyAsync(cold_d, cold.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
            k_zero_start_cols<T><<<grid_for(n * k, 256, 152 * 16), 256, 0, st>>>(n, k, cold_d, b.sp, b.zhat, r,
                                                                                  b.r64, da, db);
            FJ_CUDA(cudaGetLastError());
            FJ_CUDA(cudaStreamSynchronize(st));
        }
    }
    Run run;
    run.profile = o->profile != 0;
    run.launches = 6;
    // bulk-copy gathers (depth 0): FP32 rows of k values, a multiple of 16 bytes
    const bool bulk = sizeof(T) == 4 && b.depth == 0 && k % 4 == 0 && k >= 4 && k <= 64;
    const size_t bulk_smem = (size_t)8 * 2 * kBulkRows * (size_t)k * sizeof(float);
    int64_t sms = 152;
    if (bulk) {
        int dev = 0, nsm = 0;
        FJ_CUDA(cudaGetDevice(&dev));
        FJ_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        sms = std::max(1, nsm);
        FJ_CUDA(cudaFuncSetAttribute(k_sweep_batch_bulk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bulk_smem));
        FJ_CUDA(cudaFuncSetAttribute(k_sweep_batch_bulk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bulk_smem));
    }
    int64_t sweep = 0;
    const int check = o->check_every > 0 ? o->check_every : 8;
    const int64_t pass_cap = sizeof(T) == 4 ? std::min<int64_t>(o->max_sweeps, kFp32PassSweeps) : o->max_sweeps;
    double prev_rel = INFINITY, last_rel = INFINITY;
    int strikes = 0;
    int refine = 0, cleanups = 0;
    int64_t f_rounds = 0, f_pushes = 0;
    fj_status result = FJ_OK;
    for (;;) {
        k_pass_reset<<<1, 1, 0, st>>>(ws.ctr, pass_cap);
        for (;;) {
            for (int jj = 0; jj < check; ++jj) {
                ++sweep;
                T *dcur = (sweep & 1) ? db : da;
                const T *dprev = (sweep & 1) ? da : db;
                for (size_t cl = 0; cl + 1 < wp.class_item.size(); ++cl) {
                    const int64_t i0 = wp.class_item[cl], ni = wp.class_item[cl + 1] - i0;
                    if (ni <= 0) continue;
                    const unsigned grid =
                        (unsigned)std::min<int64_t>(ceil_div(ni, 8), batch_sweep_blocks<T>(c.w != nullptr));
                    unsigned int *tk = b.tick + 2 * cl;
                    FJ_CHECK(run.before(st));
#define FJ_SWEEP_BATCH(WW, DD)                                                                                \
    k_sweep_batch<T, WW, DD><<<grid, 256, 0, st>>>(wp.items, i0, ni, c.row_ptr, c.col, c.w, k, dcur, dprev, r, h, \
                                                   inv, zacc, om, c.indeg, wp.slot_first, wp.slot_nchunk, b.partk, \
                                                   wp.cnt, ws.ctr, tk, c.n)
                    if constexpr (sizeof(T) == 4) {
                        if (bulk) {
                            const unsigned bgrid = (unsigned)std::min<int64_t>(ceil_div(ni, 8), 3 * sms);
                            if (c.w)
                                k_sweep_batch_bulk<true><<<bgrid, 256, bulk_smem, st>>>(
                                    wp.items, i0, ni, c.row_ptr, c.col, c.w, k, dcur, dprev, r, h, inv, zacc, om,
                                    c.indeg, wp.slot_first, wp.slot_nchunk, b.partk, wp.cnt, ws.ctr, tk, g->err, c.n);
                            else
                                k_sweep_batch_bulk<false><<<bgrid, 256, bulk_smem, st>>>(
                                    wp.items, i0, ni, c.row_ptr, c.col, c.w, k, dcur, dprev, r, h, inv, zacc, om,
                                    c.indeg, wp.slot_first, wp.slot_nchunk, b.partk, wp.cnt, ws.ctr, tk, g->err, c.n);
                            FJ_CUDA(cudaGetLastError());
                            FJ_CHECK(run.after(st));
                            continue;
                        }
                    }
                    if (c.w) {
                        if (b.depth == 4) FJ_SWEEP_BATCH(true, 4);
                        else FJ_SWEEP_BATCH(true, 8);
                    } else {
                        if (b.depth == 4) FJ_SWEEP_BATCH(false, 4);
                        else FJ_SWEEP_BATCH(false, 8);
                    }
#undef FJ_SWEEP_BATCH
                    FJ_CUDA(cudaGetLastError());
                    FJ_CHECK(run.after(st));
                }
                k_end_sweep<<<1, 1, 0, st>>>(ws.ctr);
                ++run.launches;
            }
            if (sizeof(T) == 4) {
                k_fold<<<grid_for(n * k, 256, 152 * 8), 256, 0, st>>>(n * k, reinterpret_cast<float *>(b.z32), b.zhat);
                ++run.launches;
            }
            FJ_CUDA(cudaMemcpyAsync(ws.ctr_host, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
            FJ_CUDA(cudaStreamSynchronize(st));
            FJ_CHECK(run.harvest());
            FJ_CHECK(check_index_record());
            if (bulk) FJ_CHECK(read_dev_error(g, st));
            if (ws.ctr_host->done) break;
        }
        const int done = ws.ctr_host->done;
        if (done == 3) {
            result = FJ_ERR_DIVERGED;
            set_error("residual became non-finite (omega %.3f)", o->omega);
            break;
        }
        auto certify_count = [&](double &viol) -> fj_status {
            FJ_CHECK(certify());
            run.launches += 2;
            FJ_CUDA(cudaMemcpyAsync(b.gstat_host, b.gstat, sizeof(double) * kGs * k, cudaMemcpyDeviceToHost, st));
            FJ_CUDA(cudaStreamSynchronize(st));
            FJ_CHECK(check_index_record());
            viol = 0.0;
            last_rel = 0.0;
            for (int j = 0; j < k; ++j) {
                viol += b.gstat_host[j * kGs + 5];
                last_rel = std::max(last_rel, b.gstat_host[j * kGs + 3]);
            }
            return FJ_OK;
        };
        double viol = 0.0;
        FJ_CHECK(certify_count(viol));
        while (viol > 0.0 && viol <= (double)frontier_limit(n * k) && cleanups < kMaxCleanups) {
            bool cleared = false;
            ++cleanups;
            FJ_CHECK(frontier_cleanup(g, p, k, b.r64, b.zhat, b.sp, epsp, b.list, kCleanupRounds, st, run, &f_rounds,
                                      &f_pushes, &cleared));
            FJ_CHECK(certify_count(viol));
            if (!cleared) break;
        }
        if (viol == 0.0) break;
        // as fj_solve: FP32 passes of kFp32PassSweeps, free restarts while the
        // certified relative residual (largest over the vectors) halves
        const bool progress = done == 2 && pass_cap < o->max_sweeps && last_rel < 0.5 * prev_rel;
        if (o->omega > 1.0 && done == 2 && last_rel > 2.0 * prev_rel) {
            result = FJ_ERR_DIVERGED;
            set_error("residual grew from pass to pass (omega %.3f)", o->omega);
            break;
        }
        prev_rel = last_rel;
        if (!progress) {
            if (strikes >= o->max_refine) {
                result = FJ_ERR_NOT_CONVERGED;
                set_error("batch did not certify (%.0f entries above threshold)", viol);
                break;
            }
            ++strikes;
        }
        ++refine;
        sweep = 0;
    }
    double *Zd = mem == FJ_MEM_DEVICE ? Z : b.zout;
    k_unshift_batch<T><<<grid_for(n * k, 256, 152 * 16), 256, 0, st>>>(n, k, b.zhat, p.perm, gs, Zd);
    FJ_CUDA(cudaGetLastError());
    if (mem == FJ_MEM_HOST) FJ_CUDA(cudaMemcpyAsync(Z, b.zout, sizeof(double) * n * k, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(b.gstat_host, b.gstat, sizeof(double) * kGs * k, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(ws.ctr_host, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    FJ_CHECK(read_dev_error(g, st));
    if (info) {
        for (int j = 0; j < k; ++j) {
            const double *q = b.gstat_host + (size_t)j * kGs;
            fj_solve_info &f = info[j];
            std::memset(&f, 0, sizeof(f));
            f.sweeps = ws.ctr_host->sweeps;
            f.pushes = (int64_t)ws.ctr_host->pushes;
            f.edges = (int64_t)(ws.ctr_host->edges + ws.ctr_host->fedges);
            f.frontier_edges = (int64_t)ws.ctr_host->fedges;
            f.refine_passes = refine;
            f.c_eff = q[1];
            f.eps_prime = epsp;
            f.resid_inf = q[2];
            f.resid_rel_max = q[3];
            f.z_inf = q[4];
            f.err_bound = q[2];
            f.cert_rel_err = q[4] > q[2] ? q[2] / (q[4] - q[2]) : INFINITY;
            f.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            f.converged = (q[5] == 0.0 && result == FJ_OK) ? 1 : 0;
            f.launches = run.launches + 1;
            f.push_launches = run.push_launches;
            f.push_ms = run.push_ms;
            f.frontier_rounds = f_rounds;
            f.frontier_pushes = f_pushes;
            f.warm_start = warm[(size_t)j];
            const double tb = (double)sizeof(T);
            // per sweep: columns and weights once, k increments per nonzero, k row records per row
            f.push_bytes = (double)ws.ctr_host->sweeps *
                           ((double)c.nnz * (4.0 + (c.w ? 4.0 : 0.0) + tb * k) + (double)c.n * (8.0 + 5.0 * tb * k));
            f.method_bytes = (double)ws.ctr_host->sweeps * (double)c.nnz * (4.0 + (c.w ? 4.0 : 0.0)) +
                             (double)ws.ctr_host->edges * tb + (double)ws.ctr_host->pushes * 32.0;
        }
    }
    return result;
}

}  // namespace fj

extern "C" fj_status fj_solve_batch(fj_graph *g, const double *S, int k, const fj_solve_opts *opts, double *Z_out,
                                    fj_solve_info *info, int mem)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(S != nullptr && Z_out != nullptr, "S or Z_out is NULL");
    FJ_ARG(k >= 1 && k <= 64, "k must be in 1..64");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_ARG(g->ngraphs == 1, "a ragged handle takes one opinion vector per graph (use fj_solve)");
    FJ_CHECK(fj::check_opts(opts));
    return with_omega_fallback(opts, [&](const fj_solve_opts *o) {
        if (o->precision == FJ_PREC_FP32) return fj::solve_batch_t<float>(g, S, nullptr, k, o, Z_out, info, mem);
        return fj::solve_batch_t<double>(g, S, nullptr, k, o, Z_out, info, mem);
    });
}

extern "C" fj_status fj_solve_batch_warm(fj_graph *g, const double *S, const double *Z0, int k,
                                         const fj_solve_opts *opts, double *Z_out, fj_solve_info *info, int mem)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(S != nullptr && Z0 != nullptr && Z_out != nullptr, "S, Z0 or Z_out is NULL");
    FJ_ARG(k >= 1 && k <= 64, "k must be in 1..64");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_ARG(g->ngraphs == 1, "a ragged handle takes one opinion vector per graph (use fj_solve_warm)");
    FJ_CHECK(fj::check_opts(opts));
    return with_omega_fallback(opts, [&](const fj_solve_opts *o) {
        if (o->precision == FJ_PREC_FP32) return fj::solve_batch_t<float>(g, S, Z0, k, o, Z_out, info, mem);
        return fj::solve_batch_t<double>(g, S, Z0, k, o, Z_out, info, mem);
    });
}

// ============================================================== autotuner

// ============================================================== optimal omega (Eq. 17)

// y = (x + (I + D)^{-1} A x) / 2 over the warp-tile items of the caller-order
// CSR: a row of at most 32 nonzeros is summed by one lane, a longer row of a
// tile by the whole warp, a chunk of a long row by the warp with the chunks'
// sums added in chunk order by the last one to finish.  FP64, fixed order.
template <bool W>
__global__ void __launch_bounds__(256)
k_jacobi_half(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ rp,
              const int32_t *__restrict__ col, const float *__restrict__ w, const double *__restrict__ inv64,
              const double *__restrict__ x, double *__restrict__ y, const int32_t *__restrict__ slot_first,
              const int32_t *__restrict__ slot_nchunk, double *part, int32_t *cnt, int64_t n_rows)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto terms = [&](int64_t a, int64_t e, int64_t step) -> double {
        double acc = 0.0;
        for (int64_t k = a; k < e; k += step) {
            const int32_t c = __ldg(col + k);
            if (!FJ_IDX_OK(4, c, n_rows)) continue;
            acc = fma(W ? (double)__ldg(w + k) : 1.0, x[c], acc);
        }
        return acc;
    };
    auto finish = [&](int64_t v, double ax) { y[v] = 0.5 * (x[v] + inv64[v] * ax); };
    for (int64_t ii = warp; ii < nitems; ii += nwarps) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (!FJ_IDX_OK(1, r0, n_rows) || !FJ_IDX_OK(2, r1, n_rows + 1) ||
            (it.slot < 0 && !FJ_IDX_OK(3, r1 - r0, kWarpRows + 1)))
            continue;
        if (it.slot < 0) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int64_t v = r0 + lane + 32 * half;
                const bool mine = v < r1;
                int64_t a = 0, e = 0;
                if (mine) {
                    a = rp[v];
                    e = rp[v + 1];
                }
                const bool shrt = e - a <= 32;
                if (mine && shrt) finish(v, terms(a, e, 1));
                unsigned longs = __ballot_sync(FULL, mine && !shrt);
                while (longs) {
                    const int src = __ffs(longs) - 1;
                    longs &= longs - 1;
                    const int64_t al = __shfl_sync(FULL, a, src), el = __shfl_sync(FULL, e, src);
                    const double s = warp_sum(terms(al + lane, el, 32));
                    if (lane == src) finish(v, s);
                }
            }
        } else {
            const double s = warp_sum(terms(it.k0 + lane, it.k1, 32));
            const int slot = it.slot;
            const int first = slot_first[slot], nch = slot_nchunk[slot];
            int last = 0;
            if (lane == 0) {
                const int ci = (int)((it.k0 - rp[r0]) / kWarpChunk);
                part[2 * (first + ci)] = s;
                __threadfence();
                last = atomicAdd(&cnt[slot], 1) == nch - 1;
            }
            last = __shfl_sync(FULL, last, 0);
            if (last && lane == 0) {
                __threadfence();
                double t = 0.0;
                for (int c = 0; c < nch; ++c) t += __ldcg(part + 2 * (first + c));
                cnt[slot] = 0;
                finish(r0, t);
            }
        }
    }
}

// Per-block sums of y (fixed tree), then one block adds them in block order.
__global__ void __launch_bounds__(256) k_block_sum(int64_t n, const double *__restrict__ y, double *__restrict__ part)
{
    __shared__ double sm[8];
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += y[i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sm[i];
        part[blockIdx.x] = t;
    }
}

// sums[it] = sum of y; x = y * n / sum (x keeps the sum n)
__global__ void __launch_bounds__(256)
k_rescale(int64_t n, int nb, const double *__restrict__ part, const double *__restrict__ y, double *__restrict__ x,
          double *__restrict__ sums, int it)
{
    __shared__ double tot;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        tot = t;
        if (blockIdx.x == 0) sums[it] = t;
    }
    __syncthreads();
    const double f = tot > 0.0 ? (double)n / tot : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = y[i] * f;
}

__global__ void k_fill(int64_t n, double *__restrict__ x, double v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

namespace fj {
// mu = rho((I + D)^{-1} A) by power iteration on (I + M) / 2 (see the header).
fj_status jacobi_radius(fj_graph *g, int iters, cudaStream_t st, double *mu)
{
    const ItemPlan *ip = nullptr;
    FJ_CHECK(plain_items(g, st, &ip));
    const DevCSR &c = g->csr;
    const int64_t n = c.n;
    constexpr int kNb = 152 * 4;
    double *x = nullptr, *y = nullptr, *part = nullptr, *sums = nullptr;
    fj_status s = FJ_OK;
    cudaError_t e = dev_malloc(&x, sizeof(double) * n);
    if (e == cudaSuccess) e = dev_malloc(&y, sizeof(double) * n);
    if (e == cudaSuccess) e = dev_malloc(&part, sizeof(double) * kNb);
    if (e == cudaSuccess) e = dev_malloc(&sums, sizeof(double) * iters);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ip->nitems, 8), 152 * 8));
        k_fill<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, x, 1.0);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) {
            if (c.w)
                k_jacobi_half<true><<<grid, 256, 0, st>>>(ip->items, ip->nitems, c.row_ptr, c.col, c.w, c.inv64, x,
                                                          y, ip->slot_first, ip->slot_nchunk, ip->part, ip->cnt, n);
            else
                k_jacobi_half<false><<<grid, 256, 0, st>>>(ip->items, ip->nitems, c.row_ptr, c.col, c.w, c.inv64, x,
                                                           y, ip->slot_first, ip->slot_nchunk, ip->part, ip->cnt, n);
            k_block_sum<<<kNb, 256, 0, st>>>(n, y, part);
            k_rescale<<<kNb, 256, 0, st>>>(n, kNb, part, y, x, sums, it);
            e = cudaGetLastError();
        }
    }
    double last = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last, sums + (iters - 1), sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "omega_opt", __FILE__, __LINE__);
    dev_free(x);
    dev_free(y);
    dev_free(part);
    dev_free(sums);
    FJ_CHECK(s);
    FJ_CHECK(check_index_record());
    // the iterate entering the last step had sum n, so nu = sum(y) / n
    *mu = 2.0 * last / (double)n - 1.0;
    return FJ_OK;
}
}  // namespace fj

extern "C" fj_status fj_graph_omega_opt(fj_graph *g, int iters, double *mu_out, double *omega_out, void *stream)
{
    FJ_ARG(g, "NULL graph");
    FJ_ARG(iters >= 1 && iters <= 100000, "iters must be in 1..100000");
    FJ_ARG(g->csr.n > 0, "empty graph");
    double mu = 0.0;
    FJ_CHECK(fj::jacobi_radius(g, iters, (cudaStream_t)stream, &mu));
    mu = std::min(std::max(mu, 0.0), 1.0);
    const double r = mu / (1.0 + std::sqrt(1.0 - mu * mu));
    if (mu_out) *mu_out = mu;
    if (omega_out) *omega_out = 1.0 + r * r;
    return FJ_OK;
}

namespace {

constexpr int kTuneOmegaIters = 200;  // power-iteration steps behind the tuner's Eq. 17 candidate

struct TuneCand {
    int schedule, palette, depth;
    double omega;
};

// Candidates in palette order, so each colouring is built once.  wopt > 0
// adds the omega of Eq. 17 (fj_graph_omega_opt) to the fixed grid.
std::vector<TuneCand> tune_candidates(bool batch, double wopt)
{
    std::vector<TuneCand> c;
    c.push_back({FJ_SCHED_JACOBI, 0, 4, 1.0});
    std::vector<double> ws = {1.2, 1.5, 1.6, 1.7, 1.8};
    if (wopt > 1.0 && wopt < 2.0) ws.push_back(wopt);
    for (int K : {4, 8, 16, 32})
        for (double w : ws)
            for (int d : {0, 4, 8}) {
                if (!batch && d != 4) continue;
                c.push_back({FJ_SCHED_MULTICOLOUR, K, d, w});
            }
    if (batch) c.push_back({FJ_SCHED_JACOBI, 0, 8, 1.0});
    return c;
}

// Times `reps` calls of run() after one untimed call; returns the mean ms, or
// a negative value when the untimed call did not certify.
template <typename F>
fj_status time_candidate(cudaStream_t st, int reps, F run, double *ms)
{
    *ms = -1.0;
    fj_status s0 = run();
    if (s0 == FJ_ERR_NOT_CONVERGED || s0 == FJ_ERR_DIVERGED) return FJ_OK;
    FJ_CHECK(s0);
    cudaEvent_t e0, e1;
    FJ_CUDA(cudaEventCreate(&e0));
    FJ_CUDA(cudaEventCreate(&e1));
    FJ_CUDA(cudaEventRecord(e0, st));
    fj_status s = FJ_OK;
    for (int i = 0; i < reps && s == FJ_OK; ++i) s = run();
    FJ_CUDA(cudaEventRecord(e1, st));
    FJ_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    FJ_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == FJ_OK) *ms = (double)t / reps;
    else if (s != FJ_ERR_NOT_CONVERGED && s != FJ_ERR_DIVERGED) return s;
    return FJ_OK;
}

}  // namespace

extern "C" fj_status fj_graph_tune(fj_graph *g, const double *s, const fj_solve_opts *base, int reps,
                                   fj_solve_opts *best, double *best_ms, int mem)
{
    FJ_ARG(g && s && base && best, "NULL pointer");
    FJ_ARG(reps >= 1 && reps <= 100, "reps must be in 1..100");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(fj::check_opts(base));
    cudaStream_t st = (cudaStream_t)base->stream;
    const int64_t n = g->csr.n;
    std::vector<double> zh;
    double *zd = nullptr;
    if (mem == FJ_MEM_DEVICE) FJ_CUDA(dev_malloc(&zd, sizeof(double) * std::max<int64_t>(n, 1)));
    else zh.resize((size_t)std::max<int64_t>(n, 1));
    double *z = mem == FJ_MEM_DEVICE ? zd : zh.data();
    double best_t = -1.0;
    fj_solve_opts bo = *base;
    fj_status result = FJ_OK;
    double wopt = 0.0;
    FJ_CHECK(fj_graph_omega_opt(g, kTuneOmegaIters, nullptr, &wopt, base->stream));
    for (const TuneCand &cd : tune_candidates(false, wopt)) {
        fj_solve_opts o = *base;
        o.schedule = cd.schedule;
        o.palette = cd.schedule == FJ_SCHED_JACOBI ? base->palette : cd.palette;
        o.omega = cd.omega;
        o.profile = 0;
        double ms = -1.0;
        result = time_candidate(st, reps, [&]() { return fj_solve(g, s, &o, z, nullptr, mem); }, &ms);
        if (result != FJ_OK) break;
        if (ms >= 0.0 && (best_t < 0.0 || ms < best_t)) {
            best_t = ms;
            bo = o;
        }
    }
    if (zd) cudaFree(zd);
    FJ_CHECK(result);
    if (best_t < 0.0) {
        set_error("no candidate certified");
        return FJ_ERR_NOT_CONVERGED;
    }
    if (bo.schedule == FJ_SCHED_MULTICOLOUR) FJ_CHECK(fj::ensure_colouring(g, bo.palette, st));
    *best = bo;
    if (best_ms) *best_ms = best_t;
    return FJ_OK;
}

extern "C" fj_status fj_graph_tune_batch(fj_graph *g, const double *S, int k, const fj_solve_opts *base, int reps,
                                         fj_solve_opts *best, double *best_ms, int mem)
{
    FJ_ARG(g && S && base && best, "NULL pointer");
    FJ_ARG(k >= 1 && k <= 64, "k must be in 1..64");
    FJ_ARG(reps >= 1 && reps <= 100, "reps must be in 1..100");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(fj::check_opts(base));
    cudaStream_t st = (cudaStream_t)base->stream;
    const int64_t n = g->csr.n;
    std::vector<double> zh;
    double *zd = nullptr;
    if (mem == FJ_MEM_DEVICE) FJ_CUDA(dev_malloc(&zd, sizeof(double) * std::max<int64_t>(n * k, 1)));
    else zh.resize((size_t)std::max<int64_t>(n * k, 1));
    double *z = mem == FJ_MEM_DEVICE ? zd : zh.data();
    double best_t = -1.0;
    fj_solve_opts bo = *base;
    int best_depth = g->bws.depth;
    fj_status result = FJ_OK;
    double wopt = 0.0;
    FJ_CHECK(fj_graph_omega_opt(g, kTuneOmegaIters, nullptr, &wopt, base->stream));
    for (const TuneCand &cd : tune_candidates(true, wopt)) {
        fj_solve_opts o = *base;
        o.schedule = cd.schedule;
        o.palette = cd.schedule == FJ_SCHED_JACOBI ? base->palette : cd.palette;
        o.omega = cd.omega;
        o.profile = 0;
        g->bws.depth = cd.depth;
        double ms = -1.0;
        result = time_candidate(st, reps, [&]() { return fj_solve_batch(g, S, k, &o, z, nullptr, mem); }, &ms);
        if (result != FJ_OK) break;
        if (ms >= 0.0 && (best_t < 0.0 || ms < best_t)) {
            best_t = ms;
            bo = o;
            best_depth = cd.depth;
        }
    }
    g->bws.depth = best_depth;
    if (zd) cudaFree(zd);
    FJ_CHECK(result);
    if (best_t < 0.0) {
        set_error("no candidate certified");
        return FJ_ERR_NOT_CONVERGED;
    }
    if (bo.schedule == FJ_SCHED_MULTICOLOUR) FJ_CHECK(fj::ensure_colouring(g, bo.palette, st));
    *best = bo;
    if (best_ms) *best_ms = best_t;
    return FJ_OK;
}

// ============================================================== failure-path self-test

namespace fj {

// The library's two kinds of bounded device wait, each on something that
// nothing completes: the look-back's wait on a tile status word (zero: never
// published) and the bulk-copy ring's wait on an mbarrier (no arrival).
// Each must give up after `limit` polls and say so.
__global__ void k_wait_selftest(const unsigned long long *word, long long limit, int *gave_up)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    unsigned long long w;
    if (!wait_published(word, limit, w)) gave_up[0] = 1;
    tc::mbar_init(&bar, 1);
    if (!tc::mbar_wait_bounded(&bar, 0, (uint32_t)limit)) gave_up[1] = 1;
}

}  // namespace fj

extern "C" fj_status fj_wait_selftest(int64_t polls, void *stream)
{
    FJ_ARG(polls >= 1 && polls <= fj::kSpinLimit, "polls must be in 1..2^24");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *word = nullptr;
    FJ_CUDA(fj::dev_malloc(&word, sizeof(unsigned long long) + 2 * sizeof(int)));
    int *flags = reinterpret_cast<int *>(word + 1);
    cudaError_t e = cudaMemsetAsync(word, 0, sizeof(unsigned long long) + 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        fj::k_wait_selftest<<<1, 32, 0, st>>>(word, (long long)polls, flags);
        e = cudaGetLastError();
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    fj::dev_free(word);
    if (e != cudaSuccess) return fj::cuda_fail(e, "wait self-test", __FILE__, __LINE__);
    if (h[0] && h[1]) {
        fj::set_error("both bounded waits gave up after %lld polls", (long long)polls);
        return FJ_ERR_TIMEOUT;
    }
    fj::set_error("a bounded wait returned although nothing completed it (status word %d, mbarrier %d)", h[0], h[1]);
    return FJ_OK;
}

