// Shared internals of the FJ CUDA library: error plumbing, device helpers and
// the per-solve device counters.  Target: sm_103a (GB300), one GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "fj.h"

namespace fj {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
fj_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

// Every device allocation of the library goes through dev_malloc, so that a
// test can make one fail on the host (fj_debug_fail_allocation) as a full
// device would, without touching the GPU.
cudaError_t dev_malloc_raw(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

#define FJ_CUDA(...)                                                                       \
    do {                                                                                   \
        cudaError_t fj_e_ = (__VA_ARGS__);                                                 \
        if (fj_e_ != cudaSuccess) return ::fj::cuda_fail(fj_e_, #__VA_ARGS__, __FILE__, __LINE__); \
    } while (0)

#define FJ_CHECK(...)                                \
    do {                                             \
        fj_status fj_s_ = (__VA_ARGS__);             \
        if (fj_s_ != FJ_OK) return fj_s_;            \
    } while (0)

// Bounds-checked index for a kernel: true when 0 <= idx < lim; otherwise
// the first failure is stored in rec[4] (a __device__ long long array of the
// translation unit) as (site, block, index, limit) and the caller skips the
// access; the host turns the record into an error.
#define FJ_IDX_OK_REC(rec, site, idx, lim)                                                            \
    ((idx) >= 0 && (idx) < (lim)                                                                      \
         ? true                                                                                       \
         : (atomicCAS((unsigned long long *)&(rec)[0], 0ULL, (unsigned long long)(site)) == 0ULL     \
                ? ((rec)[1] = blockIdx.x, (rec)[2] = (long long)(idx), (rec)[3] = (long long)(lim), false) \
                : false))

#define FJ_ARG(cond, msg)                                                 \
    do {                                                                  \
        if (!(cond)) {                                                    \
            ::fj::set_error("invalid argument: %s", msg);                 \
            return FJ_ERR_INVALID_ARG;                                    \
        }                                                                 \
    } while (0)

// Device-side error codes written (first writer wins) into a device int.
enum DevErr : int {
    DEV_OK = 0,
    DEV_BAD_ROW_PTR = 1,
    DEV_BAD_COL = 2,
    DEV_SELF_LOOP = 3,
    DEV_UNSORTED_ROW = 4,
    DEV_BAD_WEIGHT = 5,
    DEV_CROSS_GRAPH = 6,
    DEV_SPIN_TIMEOUT = 7,
    DEV_NONFINITE = 8,
    DEV_BAD_OPINION = 9
};

// Bounded spin: every device wait gives up after this many polls and records
// DEV_SPIN_TIMEOUT instead of hanging the GPU.
constexpr long long kSpinLimit = 1LL << 24;

__device__ __forceinline__ void dev_error(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------------ warp helpers

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Block-wide sum for blockDim.x <= 1024, result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *smem /* >= 32 */)
{
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[wid] = v;
    __syncthreads();
    T r = 0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? smem[lane] : T(0);
        r = warp_sum(r);
    }
    return r;
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T *smem)
{
    v = warp_max(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[wid] = v;
    __syncthreads();
    T r = 0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? smem[lane] : T(0);
        r = warp_max(r);
    }
    return r;
}

// Max of non-negative doubles: their IEEE bit patterns order like unsigned ints.
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}

// ------------------------------------------------------------------ compensated FP64

// A sum carried as an unevaluated pair hi + lo.  two_sum is Knuth's
// error-free addition (s + e = a + b exactly); a product's rounding error is
// fma(a, b, -p).  Accumulating a dot product this way is Ogita, Rump and
// Oishi's Dot2 (SIAM J. Sci. Comput. 26, 2005): the result is as accurate as
// if computed in twice the working precision, then rounded.  The _rn
// intrinsics keep the compiler from contracting these steps into FMAs.
struct DD {
    double hi, lo;
};

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    const double bp = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bp)), __dsub_rn(b, bp));
}

__device__ __forceinline__ void dd_add(DD &acc, double x)
{
    double s, e;
    two_sum(acc.hi, x, s, e);
    acc.hi = s;
    acc.lo = __dadd_rn(acc.lo, e);
}

// acc += a * b
__device__ __forceinline__ void dd_fma(DD &acc, double a, double b)
{
    const double p = __dmul_rn(a, b);
    const double pe = fma(a, b, -p);
    dd_add(acc, p);
    acc.lo = __dadd_rn(acc.lo, pe);
}

__device__ __forceinline__ DD dd_merge(DD a, DD b)
{
    double s, e;
    two_sum(a.hi, b.hi, s, e);
    return DD{s, __dadd_rn(__dadd_rn(a.lo, b.lo), e)};
}

__device__ __forceinline__ DD warp_dd_sum(DD v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DD u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = dd_merge(v, u);
    }
    return v;
}

__device__ __forceinline__ double dd_value(DD v) { return __dadd_rn(v.hi, v.lo); }

// FP64 resolution of row x's residual: moving zhat'_x by one ulp moves r_x by
// (1 + d_x) ulp(zhat'_x) <= 2^-52 (1 + d_x) |zhat'_x|, so a threshold below
// this may be unreachable.  The certificate test takes the larger of the two.
__device__ __forceinline__ double resid_floor(double deg, double zp)
{
    return 0x1p-51 * (1.0 + deg) * fabs(zp);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T abs_t(T x) { return x < T(0) ? -x : x; }

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ counters

// Device-resident solve state read by the host between batches of sweeps.
struct Counters {
    unsigned long long pushes;        // node pushes, whole solve
    unsigned long long edges;         // residual updates (sum of in-degrees of pushed nodes)
    unsigned long long sweep_pushes;  // pushes in the current sweep / round
    long long sweeps;                 // completed sweeps / rounds, whole solve
    long long pass_sweeps;            // completed sweeps in the current refinement pass
    long long max_sweeps;             // cap per pass
    int done;                         // 0 running, 1 converged, 2 sweep cap, 3 diverged
    int err;                          // DevErr
    double nonfinite;                 // set when a residual became NaN/Inf
    unsigned int ticket;              // next work item of the running sweep
    unsigned int pad;
    unsigned long long fedges;        // residual updates of the FP64 frontier push rounds
};

// Launch helper: grid size for a grid-stride loop over `work` items.
inline unsigned grid_for(int64_t work, int threads, int max_blocks = 152 * 16)
{
    int64_t b = ceil_div(work, threads);
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

}  // namespace fj
