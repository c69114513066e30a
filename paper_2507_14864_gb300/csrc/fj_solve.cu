// The FJ push solver on the GPU: ImprovedBLISOR (Alg. 2 + Alg. 3) with the
// pushes of a sweep applied class by class (Gauss-Seidel order, Theorem 2) or
// as synchronous rounds, an FP64 certificate (Lemmas 3-5) and FP64 restarts.
//
// State per node u (shifted system s' = s + c_eff, Alg. 2):
//   r_u    residual of s' - (I + L) zhat'          (T = float or double)
//   h_u    threshold eps' s'_u                      (T; FP32 rounded down)
//   d_u    last push increment of u not yet pulled by every in-neighbour
//   zhat_u estimate of z'_u                         (FP64)
// A push of u (Eqs. sor1-sor3) is delta = omega r_u / (1 + d_u),
// zhat_u += delta, r_u <- (1 - omega) r_u, and r_x += a_xu delta for every x
// with a_xu > 0.  The kernels apply the last step in pull form: when row x is
// visited it adds sum_j a_xj delta_j over its row.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

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

// Initial state over new ids i (o = perm[i] the caller's id): s', zhat, r, h.
template <typename T>
__global__ void k_init(int64_t n, const double *__restrict__ s, const double *__restrict__ z0,
                       const int32_t *__restrict__ perm, const int32_t *__restrict__ graph_of,
                       const unsigned long long *__restrict__ gs, double epsp, double *__restrict__ sp,
                       double *__restrict__ zhat, T *__restrict__ r, T *__restrict__ h, T *__restrict__ da,
                       T *__restrict__ db)
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
}

// End of a sweep (or round): stop when nothing was pushed, at the cap, or on
// a non-finite residual.
__global__ void k_end_sweep(Counters *c)
{
    if (c->done) return;
    c->sweeps += 1;
    c->pass_sweeps += 1;
    if (c->nonfinite != 0.0) c->done = 3;
    else if (c->sweep_pushes == 0) c->done = 1;
    else if (c->pass_sweeps >= c->max_sweeps) c->done = 2;
    c->sweep_pushes = 0;
}

// ============================================================== row-block machinery

// Segmented inclusive scan of prod[0, nz) in place (segments start where
// head[i] != 0), by 8 warps over contiguous chunks.  Afterwards the last
// element of every row holds that row's sum.
template <typename T>
__device__ __forceinline__ void block_segscan(T *prod, const unsigned char *head, int nz, T *wcarry, int *whas)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int C = (((nz + 7) >> 3) + 31) & ~31;
    const int beg = wid * C;
    const int end = min(beg + C, nz);
    T carry = T(0);
    int seen = 0;
    int first_head = end;
    for (int base = beg; base < end; base += 32) {
        int i = base + lane;
        bool valid = i < end;
        T v = valid ? prod[i] : T(0);
        int f = valid ? (int)head[i] : 0;
        unsigned hb = __ballot_sync(0xffffffffu, f != 0);
        if (hb && !seen) first_head = base + __ffs(hb) - 1;
        seen |= (hb != 0u);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T vu = __shfl_up_sync(0xffffffffu, v, o);
            int fu = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) {
                if (!f) v += vu;
                f |= fu;
            }
        }
        if (!f) v += carry;
        if (valid) prod[i] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) {
        wcarry[wid] = carry;
        whas[wid] = seen;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T cin = T(0);
        for (int w = 0; w < 8; ++w) {
            T out = whas[w] ? wcarry[w] : cin + wcarry[w];
            wcarry[w] = cin;  // becomes the carry-in of warp w
            cin = out;
        }
    }
    __syncthreads();
    const T cin = wcarry[wid];
    for (int i = beg + lane; i < first_head; i += 32) prod[i] += cin;
}

template <typename T, bool W>
__device__ __forceinline__ T arc_w(const float *__restrict__ w, int64_t k)
{
    if constexpr (W) return (T)__ldg(w + k);
    else return T(1);
}

// ============================================================== push round

// Bounds-checked indexing: the push and certificate kernels verify every
// row, block and column index against its array before using it.  The first
// index out of range is stored here as (site, block, index, limit), the access
// is skipped, and the host turns the record into an error.  The checks cost one
// compare per nonzero in kernels that are bound by memory traffic.
__device__ long long g_fj_dbg[4];
#define FJ_IDX_OK(site, idx, lim)                                                     \
    ((idx) >= 0 && (idx) < (lim)                                                      \
         ? true                                                                       \
         : (atomicCAS((unsigned long long *)&g_fj_dbg[0], 0ULL, (unsigned long long)(site)) == 0ULL \
                ? (g_fj_dbg[1] = blockIdx.x, g_fj_dbg[2] = (long long)(idx), g_fj_dbg[3] = (long long)(lim), false) \
                : false))

// One pull pass over row blocks [blk0, blk0 + gridDim.x): for every row x,
//   r_x += sum_j a_xj din_j;  if |r_x| > h_x push x:
//   delta = omega r_x / (1 + d_x), zhat_x += delta, r_x <- (1 - omega) r_x;
//   dout_x = delta (0 when x did not push).
// Jacobi rounds pass din != dout (double buffer).  A colour class passes
// din == dout: no row of an independent set reads a value another row of the
// same launch writes.
template <typename T, bool W>
__global__ void __launch_bounds__(256)
k_pull(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ w,
       const int32_t *__restrict__ blk_row, int64_t blk0, const T *din, T *dout, T *__restrict__ r,
       const T *__restrict__ h, const T *__restrict__ inv, double *__restrict__ zhat,
       const int32_t *__restrict__ indeg, T omega, Counters *ctr, int64_t n_rows)
{
    __shared__ T prod[2 * kBlockNnz];
    __shared__ unsigned char head[2 * kBlockNnz];
    __shared__ T wcarry[8];
    __shared__ int whas[8];
    __shared__ unsigned long long red[2][8];
    if (*reinterpret_cast<volatile int *>(&ctr->done)) return;
    const int64_t b = blk0 + blockIdx.x;
    const int64_t r0 = blk_row[b], r1 = blk_row[b + 1];
    if (!FJ_IDX_OK(11, r0, n_rows) || !FJ_IDX_OK(12, r1, n_rows + 1) || !FJ_IDX_OK(13, r1 - r0, kBlockRows + 1))
        return;
    const int64_t k0 = rp[r0], k1 = rp[r1];
    const int64_t nz = k1 - k0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long my_push = 0, my_edges = 0;
    bool bad = false;

    auto epilogue = [&](int64_t x, T acc) {
        T rx = r[x] + acc;
        T dx = T(0);
        if (abs_t(rx) > h[x]) {
            dx = omega * rx * inv[x];
            zhat[x] += (double)dx;
            rx = (T(1) - omega) * rx;
            my_push += 1;
            my_edges += (unsigned long long)indeg[x];
        }
        if (!isfinite(rx)) bad = true;
        r[x] = rx;
        dout[x] = dx;
    };

    if (nz > 2 * kBlockNnz) {
        // one long row
        T acc = T(0);
        for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
            int32_t cj = __ldg(col + k);
            if (FJ_IDX_OK(14, cj, n_rows)) acc += arc_w<T, W>(w, k) * __ldg(din + cj);
        }
        acc = warp_sum(acc);
        if (lane == 0) wcarry[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            T t = T(0);
            for (int i = 0; i < 8; ++i) t += wcarry[i];
            epilogue(r0, t);
        }
    } else {
        const int nzi = (int)nz;
        for (int i = threadIdx.x; i < nzi; i += 256) {
            int64_t k = k0 + i;
            int32_t cj = __ldg(col + k);
            prod[i] = FJ_IDX_OK(15, cj, n_rows) ? arc_w<T, W>(w, k) * __ldg(din + cj) : T(0);
            head[i] = 0;
        }
        __syncthreads();
        for (int64_t x = r0 + threadIdx.x; x < r1; x += 256) {
            int64_t a = rp[x];
            if (rp[x + 1] > a && FJ_IDX_OK(16, a - k0, nz)) head[a - k0] = 1;
        }
        __syncthreads();
        block_segscan<T>(prod, head, nzi, wcarry, whas);
        __syncthreads();
        for (int64_t x = r0 + threadIdx.x; x < r1; x += 256) {
            int64_t a = rp[x], e = rp[x + 1];
            epilogue(x, e > a ? prod[e - 1 - k0] : T(0));
        }
    }
    // block totals -> three atomics
    my_push = warp_sum(my_push);
    my_edges = warp_sum(my_edges);
    unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[0][wid] = my_push;
        red[1][wid] = my_edges;
        if (anybad) ctr->nonfinite = 1.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long p = 0, e = 0;
        for (int i = 0; i < 8; ++i) {
            p += red[0][i];
            e += red[1][i];
        }
        if (p) {
            atomicAdd(&ctr->pushes, p);
            atomicAdd(&ctr->sweep_pushes, p);
            atomicAdd(&ctr->edges, e);
        }
    }
}

// ============================================================== FP64 certificate


// r64_x = s'_x - (1 + d_x) zhat_x + sum_j a_xj zhat_j  (= s' - (I + L) zhat'; a long
// row sums a_xj (zhat_j - zhat_x) instead, which cancels less),
// per graph: max |r64|, max |r64| / s', max |zhat - c_eff|, number of nodes
// with |r64| > eps' s'.  Stores r64 into the push residual (magnitude rounded
// up for FP32) and clears both increment buffers: the push restarts from an
// exact residual (a refinement pass).
template <typename T, bool W>
__global__ void __launch_bounds__(256)
k_certify(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ w,
          const int32_t *__restrict__ blk_row, const double *__restrict__ zhat, const double *__restrict__ sp,
          const double *__restrict__ deg, const int32_t *__restrict__ graph_of, double epsp, T *__restrict__ r, T *__restrict__ da,
          T *__restrict__ db, unsigned long long *gs, int64_t n_rows)
{
    __shared__ double prod[2 * kBlockNnz];
    __shared__ unsigned char head[2 * kBlockNnz];
    __shared__ double wcarry[8];
    __shared__ int whas[8];
    __shared__ double red[4][8];
    const int64_t b = blockIdx.x;
    const int64_t r0 = blk_row[b], r1 = blk_row[b + 1];
    if (!FJ_IDX_OK(1, r0, n_rows) || !FJ_IDX_OK(2, r1, n_rows + 1) || !FJ_IDX_OK(3, r1 - r0, kBlockRows + 1)) return;
    const int64_t k0 = rp[r0], k1 = rp[r1];
    const int64_t nz = k1 - k0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gph = graph_of ? graph_of[r0] : 0;
    if (!FJ_IDX_OK(6, gph, 1 << 20)) return;
    const double ce = reinterpret_cast<const double *>(gs)[(int64_t)gph * kGs + 1];
    double m_abs = 0.0, m_rel = 0.0, m_z = 0.0, viol = 0.0;

    auto epilogue = [&](int64_t x, double acc) {
        double zx = zhat[x];
        double rx = sp[x] - zx + acc;
        double ax = fabs(rx);
        if (!(ax <= 1e300)) ax = INFINITY;
        m_abs = fmax(m_abs, ax);
        m_rel = fmax(m_rel, ax / sp[x]);
        m_z = fmax(m_z, fabs(zx - ce));
        if (ax > epsp * sp[x]) viol += 1.0;
        r[x] = resid_store<T>(rx);
        da[x] = T(0);
        db[x] = T(0);
    };

    if (nz > 2 * kBlockNnz) {
        const double zx = zhat[r0];
        double acc = 0.0;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
            int32_t cj = __ldg(col + k);
            if (FJ_IDX_OK(7, cj, n_rows)) acc += arc_w<double, W>(w, k) * (zhat[cj] - zx);
        }
        acc = warp_sum(acc);
        if (lane == 0) wcarry[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < 8; ++i) t += wcarry[i];
            epilogue(r0, t);
        }
    } else {
        const int nzi = (int)nz;
        for (int i = threadIdx.x; i < nzi; i += 256) head[i] = 0;
        __syncthreads();
        for (int64_t x = r0 + threadIdx.x; x < r1; x += 256) {
            int64_t a = rp[x];
            if (rp[x + 1] > a && FJ_IDX_OK(5, a - k0, nz)) head[a - k0] = 1;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nzi; i += 256) {
            int64_t k = k0 + i;
            int32_t cj = __ldg(col + k);
            prod[i] = FJ_IDX_OK(4, cj, n_rows) ? arc_w<double, W>(w, k) * zhat[cj] : 0.0;
        }
        __syncthreads();
        block_segscan<double>(prod, head, nzi, wcarry, whas);
        __syncthreads();
        for (int64_t x = r0 + threadIdx.x; x < r1; x += 256) {
            int64_t a = rp[x], e = rp[x + 1];
            // sum_j a_xj zhat_j - d_x zhat_x
            epilogue(x, (e > a ? prod[e - 1 - k0] : 0.0) - deg[x] * zhat[x]);
        }
    }
    m_abs = warp_max(m_abs);
    m_rel = warp_max(m_rel);
    m_z = warp_max(m_z);
    viol = warp_sum(viol);
    if (lane == 0) {
        red[0][wid] = m_abs;
        red[1][wid] = m_rel;
        red[2][wid] = m_z;
        red[3][wid] = viol;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, rl = 0, zz = 0, v = 0;
        for (int i = 0; i < 8; ++i) {
            a = fmax(a, red[0][i]);
            rl = fmax(rl, red[1][i]);
            zz = fmax(zz, red[2][i]);
            v += red[3][i];
        }
        unsigned long long *g = gs + (int64_t)gph * kGs;
        atomic_max_nonneg(reinterpret_cast<double *>(g + 2), a);
        atomic_max_nonneg(reinterpret_cast<double *>(g + 3), rl);
        atomic_max_nonneg(reinterpret_cast<double *>(g + 4), zz);
        if (v > 0) atomicAdd(reinterpret_cast<double *>(g + 5), v);
    }
}

// Clears the per-graph certificate slots (2..6) before a certify pass.
__global__ void k_cert_reset(int ng, unsigned long long *gs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x)
        for (int j = 2; j < kGs; ++j) gs[(int64_t)i * kGs + j] = 0ULL;
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

// ============================================================== host driver

template <typename T>
static fj_status ws_grow(fj_graph *g, int64_t entries, int ngraphs)
{
    Workspace &ws = g->ws;
    if (entries > ws.cap_n) {
        void **bufs[] = {&ws.r, &ws.h, &ws.da, &ws.db};
        for (void **p : bufs) {
            dev_free(*p);
            *p = nullptr;
            FJ_CUDA(cudaMalloc(p, sizeof(double) * (size_t)entries));
        }
        double **dbufs[] = {&ws.zhat, &ws.sp, &ws.sin, &ws.zout};
        for (double **p : dbufs) {
            dev_free(*p);
            *p = nullptr;
            FJ_CUDA(cudaMalloc(p, sizeof(double) * (size_t)entries));
        }
        dev_free(ws.list);
        ws.list = nullptr;
        FJ_CUDA(cudaMalloc(&ws.list, sizeof(int32_t) * (size_t)entries));
        ws.cap_n = entries;
    }
    if (ngraphs > ws.cap_graphs) {
        dev_free(ws.gstat);
        ws.gstat = nullptr;
        if (ws.gstat_host) cudaFreeHost(ws.gstat_host);
        ws.gstat_host = nullptr;
        FJ_CUDA(cudaMalloc(&ws.gstat, sizeof(double) * kGs * ngraphs));
        FJ_CUDA(cudaMallocHost(&ws.gstat_host, sizeof(double) * kGs * ngraphs));
        ws.cap_graphs = ngraphs;
    }
    if (!ws.ctr) {
        FJ_CUDA(cudaMalloc(&ws.ctr, sizeof(Counters)));
        FJ_CUDA(cudaMallocHost(&ws.ctr_host, sizeof(Counters)));
    }
    return FJ_OK;
}

struct Plan {
    const DevCSR *c = nullptr;  // CSR the push runs on
    const int32_t *perm = nullptr;
    bool mc = false;
    int head_classes = 0;       // classes launched one by one
    int64_t tail_row = 0;       // first row of the merged tail block (== n when none)
    int64_t tail_blk0 = 0, tail_blk1 = 0;
};

// Launch bookkeeping of one solve: every kernel launched, and with profiling
// a CUDA-event pair around every push launch on the solve's stream.
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
    return FJ_OK;
}

static fj_status make_plan(fj_graph *g, const fj_solve_opts *o, cudaStream_t st, Plan &p)
{
    p.mc = o->schedule != FJ_SCHED_JACOBI;
    if (!p.mc) {
        p.c = &g->csr;
        p.tail_row = g->csr.n;
        return FJ_OK;
    }
    FJ_CHECK(ensure_colouring(g, st));
    const Colouring &cl = g->colr;
    p.c = &cl.pcsr;
    p.perm = cl.perm;
    // the tail: the longest run of final classes that are each smaller than tail_rows
    int64_t tail_rows = o->tail_rows > 0 ? o->tail_rows : 4096;
    int k = cl.ncolours;
    while (k > 1 && cl.class_row[k] - cl.class_row[k - 1] < tail_rows) --k;
    if (k == cl.ncolours - 1) k = cl.ncolours;  // a single small last class is launched on its own
    p.head_classes = k;
    p.tail_row = cl.class_row[k];
    p.tail_blk0 = cl.class_blk[k];
    p.tail_blk1 = cl.pcsr.nblocks;
    return FJ_OK;
}

template <typename T>
static fj_status launch_pull(const DevCSR &c, int64_t blk0, int64_t blk1, const T *din, T *dout, Workspace &ws,
                             double omega, cudaStream_t st, Run &run)
{
    if (blk1 <= blk0) return FJ_OK;
    FJ_CHECK(run.before(st));
    const unsigned nb = (unsigned)(blk1 - blk0);
    T *r = reinterpret_cast<T *>(ws.r);
    const T *h = reinterpret_cast<const T *>(ws.h);
    const T *inv;
    if constexpr (sizeof(T) == 4) inv = reinterpret_cast<const T *>(c.inv32);
    else inv = reinterpret_cast<const T *>(c.inv64);
    if (c.w)
        k_pull<T, true><<<nb, 256, 0, st>>>(c.row_ptr, c.col, c.w, c.blk_row, blk0, din, dout, r, h, inv, ws.zhat,
                                            c.indeg, (T)omega, ws.ctr, c.n);
    else
        k_pull<T, false><<<nb, 256, 0, st>>>(c.row_ptr, c.col, c.w, c.blk_row, blk0, din, dout, r, h, inv, ws.zhat,
                                             c.indeg, (T)omega, ws.ctr, c.n);
    FJ_CUDA(cudaGetLastError());
    return run.after(st);
}

// One sweep (multicolour) or round (Jacobi).  Jacobi alternates the two
// increment buffers, so `parity` selects the direction.
template <typename T>
static fj_status launch_sweep(fj_graph *g, const Plan &p, double omega, int parity, cudaStream_t st, Run &run)
{
    Workspace &ws = g->ws;
    const DevCSR &c = *p.c;
    T *da = reinterpret_cast<T *>(ws.da), *db = reinterpret_cast<T *>(ws.db);
    if (!p.mc) {
        const T *din = parity ? db : da;
        T *dout = parity ? da : db;
        FJ_CHECK(launch_pull<T>(c, 0, c.nblocks, din, dout, ws, omega, st, run));
    } else {
        const Colouring &cl = g->colr;
        for (int k = 0; k < p.head_classes; ++k)
            FJ_CHECK(launch_pull<T>(c, cl.class_blk[k], cl.class_blk[k + 1], da, da, ws, omega, st, run));
        if (p.tail_blk1 > p.tail_blk0) {
            // unrelaxed Jacobi step over the merged small classes, then commit its increments
            FJ_CHECK(launch_pull<T>(c, p.tail_blk0, p.tail_blk1, da, db, ws, std::min(omega, 1.0), st, run));
            FJ_CUDA(cudaMemcpyAsync(da + p.tail_row, db + p.tail_row, sizeof(T) * (c.n - p.tail_row),
                                    cudaMemcpyDeviceToDevice, st));
        }
    }
    k_end_sweep<<<1, 1, 0, st>>>(ws.ctr);
    FJ_CUDA(cudaGetLastError());
    ++run.launches;
    return FJ_OK;
}

template <typename T>
static fj_status launch_certify(fj_graph *g, const Plan &p, double epsp, cudaStream_t st, Run &run)
{
    run.launches += 2;
    Workspace &ws = g->ws;
    const DevCSR &c = *p.c;
    k_cert_reset<<<grid_for(g->ngraphs, 256), 256, 0, st>>>(g->ngraphs, reinterpret_cast<unsigned long long *>(ws.gstat));
    T *r = reinterpret_cast<T *>(ws.r), *da = reinterpret_cast<T *>(ws.da), *db = reinterpret_cast<T *>(ws.db);
    unsigned long long *gs = reinterpret_cast<unsigned long long *>(ws.gstat);
    if (c.w)
        k_certify<T, true><<<(unsigned)c.nblocks, 256, 0, st>>>(c.row_ptr, c.col, c.w, c.blk_row, ws.zhat, ws.sp,
                                                                c.deg64, c.graph_of, epsp, r, da, db, gs, c.n);
    else
        k_certify<T, false><<<(unsigned)c.nblocks, 256, 0, st>>>(c.row_ptr, c.col, c.w, c.blk_row, ws.zhat, ws.sp,
                                                                 c.deg64, c.graph_of, epsp, r, da, db, gs, c.n);
    FJ_CUDA(cudaGetLastError());
    return FJ_OK;
}

template <typename T>
static fj_status solve_t(fj_graph *g, const double *s, const double *z0, const fj_solve_opts *o, double *z_out,
                         fj_solve_info *info, int mem)
{
    cudaStream_t st = (cudaStream_t)o->stream;
    const int64_t n = g->csr.n;
    const int ng = g->ngraphs;
    FJ_CHECK(ws_grow<T>(g, n, ng));
    Workspace &ws = g->ws;
    Plan p;
    FJ_CHECK(make_plan(g, o, st, p));
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
    k_init<T><<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, sd, z0d, p.perm, c.graph_of, gs, epsp, ws.sp, ws.zhat, r,
                                                         h, da, db);
    FJ_CUDA(cudaGetLastError());
    FJ_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(Counters), st));
    FJ_CHECK(read_dev_error(g, st));
    Run run;
    run.profile = o->profile != 0;
    run.launches += 5;  // gstat reset, min s, shift, init, (memset)
    if (z0) FJ_CHECK(launch_certify<T>(g, p, epsp, st, run));  // warm start: exact FP64 residual of z0

    // profiling times every push launch, so no sweep may run past the stop flag
    const int check = run.profile ? 1 : (o->check_every > 0 ? o->check_every : 8);
    int refine = 0;
    fj_status result = FJ_OK;
    int parity = 0;
    for (;;) {
        k_pass_reset<<<1, 1, 0, st>>>(ws.ctr, o->max_sweeps);
        FJ_CUDA(cudaGetLastError());
        ++run.launches;
        for (;;) {
            for (int j = 0; j < check; ++j) {
                FJ_CHECK(launch_sweep<T>(g, p, o->omega, parity, st, run));
                parity ^= 1;
            }
            FJ_CUDA(cudaMemcpyAsync(ws.ctr_host, ws.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
            FJ_CUDA(cudaStreamSynchronize(st));
            FJ_CHECK(run.harvest());
            {
                long long dbg[4] = {0, 0, 0, 0};
                FJ_CUDA(cudaMemcpyFromSymbol(dbg, g_fj_dbg, sizeof(dbg)));
                if (dbg[0]) {
                    set_error("index check failed: site %lld block %lld index %lld limit %lld", dbg[0], dbg[1], dbg[2],
                              dbg[3]);
                    return FJ_ERR_INVALID_ARG;
                }
            }
            if (ws.ctr_host->done) break;
        }
        // Jacobi rounds that ran after the stop flag were no-ops; re-align parity
        const int done = ws.ctr_host->done;
        if (done == 3) {
            result = FJ_ERR_DIVERGED;
            set_error("residual became non-finite (omega %.3f)", o->omega);
            break;
        }
        FJ_CHECK(launch_certify<T>(g, p, epsp, st, run));
        FJ_CUDA(cudaMemcpyAsync(ws.gstat_host, ws.gstat, sizeof(double) * kGs * ng, cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
        {
            long long dbg[4] = {0, 0, 0, 0};
            FJ_CUDA(cudaMemcpyFromSymbol(dbg, g_fj_dbg, sizeof(dbg)));
            if (dbg[0]) {
                set_error("index check failed: site %lld block %lld index %lld limit %lld", dbg[0], dbg[1], dbg[2], dbg[3]);
                return FJ_ERR_INVALID_ARG;
            }
        }
        double viol = 0.0;
        for (int i = 0; i < ng; ++i) viol += ws.gstat_host[i * kGs + 5];
        if (viol == 0.0) break;
        if (done == 2) {
            result = FJ_ERR_NOT_CONVERGED;
            set_error("sweep cap %lld reached", (long long)o->max_sweeps);
            break;
        }
        if (refine >= o->max_refine) {
            result = FJ_ERR_NOT_CONVERGED;
            set_error("refinement cap %d reached with %.0f nodes above threshold", o->max_refine, viol);
            break;
        }
        ++refine;
        parity = 0;  // certify cleared both increment buffers
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
            f.edges = (int64_t)ws.ctr_host->edges;
            f.refine_passes = refine;
            f.c_eff = q[1];
            f.eps_prime = epsp;
            f.resid_inf = q[2];
            f.resid_rel_max = q[3];
            f.z_inf = q[4];
            f.err_bound = q[2];
            f.converged = (q[5] == 0.0 && result == FJ_OK) ? 1 : 0;
            f.launches = run.launches;
            f.push_launches = run.push_launches;
            f.push_ms = run.push_ms;
            // every effective sweep reads each row and nonzero once; pushes add their own traffic
            const double tb = (double)sizeof(T);
            const double per_sweep = (double)c.nnz * (4.0 + (c.w ? 4.0 : 0.0) + tb) + (double)c.n * (8.0 + 5.0 * tb);
            f.push_bytes = (double)ws.ctr_host->sweeps * per_sweep + (double)ws.ctr_host->pushes * 20.0;
        }
    }
    return result;
}

}  // namespace fj

using namespace fj;

extern "C" {

fj_status fj_solve(fj_graph *g, const double *s, const fj_solve_opts *opts, double *z_out, fj_solve_info *info,
                   int mem)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s != nullptr && z_out != nullptr, "s or z_out is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(check_opts(opts));
    if (opts->precision == FJ_PREC_FP32) return solve_t<float>(g, s, nullptr, opts, z_out, info, mem);
    return solve_t<double>(g, s, nullptr, opts, z_out, info, mem);
}

fj_status fj_solve_warm(fj_graph *g, const double *s, const double *z0, const fj_solve_opts *opts, double *z_out,
                        fj_solve_info *info, int mem)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s != nullptr && z0 != nullptr && z_out != nullptr, "s, z0 or z_out is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_CHECK(check_opts(opts));
    if (opts->precision == FJ_PREC_FP32) return solve_t<float>(g, s, z0, opts, z_out, info, mem);
    return solve_t<double>(g, s, z0, opts, z_out, info, mem);
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
