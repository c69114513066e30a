// The measures of Table 1 (Section 3.4) for opinions s and equilibrium z:
//   C = sum z_i^2, P = sum (z_i - mean z)^2, I = sum (z_i - s_i)^2,
//   D = sum over edges a_ij (z_i - z_j)^2 (an undirected edge once).
// Two passes over the row blocks of the caller-order CSR: the mean first,
// then C, P, I and the disagreement gathered over the nonzeros.  All sums are
// FP64 in a fixed order (per-thread strided partials, shuffle trees, warps in
// order, blocks in order per graph), so the result is bit-reproducible.
#include <vector>

#include "fj_internal.cuh"

namespace fj {
// first out-of-range index of the batch measures (see FJ_IDX_OK_REC)
__device__ long long g_fj_metric_dbg[4];
}  // namespace fj
#define FJ_IDX_OK(site, idx, lim) FJ_IDX_OK_REC(fj::g_fj_metric_dbg, site, idx, lim)
#include "fj_tile.cuh"

namespace fj {

// Deterministic block sum of NV values (thread 0 ends with the totals).
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double (*smem)[8])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) smem[j][wid] = v[j];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += smem[j][w];
            v[j] = t;
        }
}

__global__ void __launch_bounds__(256)
k_metric_mean(const int32_t *__restrict__ blk_row, const double *__restrict__ z, double *__restrict__ part)
{
    __shared__ double sm[1][8];
    const int64_t r0 = blk_row[blockIdx.x], r1 = blk_row[blockIdx.x + 1];
    double v[1] = {0.0};
    for (int64_t x = r0 + threadIdx.x; x < r1; x += 256) v[0] += z[x];
    block_sums<1>(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

template <bool W>
__global__ void __launch_bounds__(256)
k_metric_main(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ w,
              const int32_t *__restrict__ blk_row, const double *__restrict__ s, const double *__restrict__ z,
              const int32_t *__restrict__ graph_of, const double *__restrict__ mean, double *__restrict__ part)
{
    __shared__ double sm[4][8];
    __shared__ int64_t srp[kBlockRows + 1];
    const int64_t r0 = blk_row[blockIdx.x], r1 = blk_row[blockIdx.x + 1];
    const int64_t k0 = rp[r0], k1 = rp[r1];
    const int nrows = (int)(r1 - r0);
    const double mu = mean[graph_of ? graph_of[r0] : 0];
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // C, P, I, D
    for (int64_t x = r0 + threadIdx.x; x < r1; x += 256) {
        double zx = z[x], dz = zx - mu, di = zx - s[x];
        v[0] += zx * zx;
        v[1] += dz * dz;
        v[2] += di * di;
    }
    if (nrows == 1) {
        const double zx = z[r0];
        for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
            double d = zx - z[col[k]];
            v[3] += (W ? (double)w[k] : 1.0) * d * d;
        }
    } else {
        for (int i = threadIdx.x; i <= nrows; i += 256) srp[i] = rp[r0 + i];
        __syncthreads();
        for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
            int lo = 0, hi = nrows;  // last row with srp[row] <= k
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (srp[mid] <= k) lo = mid; else hi = mid;
            }
            double d = z[r0 + lo] - z[col[k]];
            v[3] += (W ? (double)w[k] : 1.0) * d * d;
        }
    }
    block_sums<4>(v, sm);
    if (threadIdx.x == 0)
        for (int j = 0; j < 4; ++j) part[(int64_t)blockIdx.x * 4 + j] = v[j];
}

// One block per graph sums its blocks' partials (nf fields each): thread t
// adds partials t, t + 256, ... in order, then a fixed tree over the threads.
__global__ void __launch_bounds__(256)
k_metric_reduce(int ng, const int64_t *__restrict__ gblk, const double *__restrict__ part, int nf,
                double *__restrict__ out)
{
    __shared__ double sm[4][8];
    const int gi = blockIdx.x;
    if (gi >= ng) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t b = gblk[gi] + threadIdx.x; b < gblk[gi + 1]; b += 256)
        for (int f = 0; f < nf; ++f) v[f] += part[b * nf + f];
    block_sums<4>(v, sm);
    if (threadIdx.x == 0)
        for (int f = 0; f < nf; ++f) out[(int64_t)gi * nf + f] = v[f];
}

__global__ void k_metric_mean_div(int ng, const int64_t *__restrict__ node_off, double *__restrict__ mean)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi < ng) mean[gi] /= (double)(node_off[gi + 1] - node_off[gi]);
}

// Multi-vector measures: S and Z node-major [n][k], k <= 64, lanes owning
// vectors j = lane and lane + 32.  Pass 1 (k_metric_batch_sum): the sum of z
// per vector, warps taking rows with a fixed stride.  Pass 2
// (k_metric_batch_items): C, P, I and the arc sum of a (z_x - z_c)^2 over the
// warp-tile item plan, warps taking items with a fixed stride: a tile's rows
// are walked by warp_tile_k (D neighbour rows in flight for both halves), a
// long row's 512-nonzero chunks are items of their own spread over the warps
// (the arc sum is a plain sum over arcs, so a chunk's part joins the warp's
// running sum directly), and the row's own terms are taken with its first
// chunk.  Partials per block, reduced in block order by
// k_metric_batch_reduce: every sum has a fixed order.
constexpr int kMetricBatchBlocks = 152 * 4;

__global__ void __launch_bounds__(256)
k_metric_batch_sum(int64_t n, int k, const double *__restrict__ Z, double *__restrict__ part)
{
    __shared__ double red[8][64];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp = (int64_t)blockIdx.x * 8 + wl, nwarps = (int64_t)gridDim.x * 8;
    const bool has[2] = {lane < k, lane + 32 < k};
    double acc[2] = {0.0, 0.0};
    for (int64_t x = warp; x < n; x += nwarps)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
            if (has[hh]) acc[hh] += Z[x * k + lane + 32 * hh];
    for (int hh = 0; hh < 2; ++hh) red[wl][lane + 32 * hh] = acc[hh];
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += 256) {
        double t = 0.0;
        for (int ww = 0; ww < 8; ++ww) t += red[ww][j];
        part[(int64_t)blockIdx.x * k + j] = t;
    }
}

template <bool W>
__global__ void __launch_bounds__(256)
k_metric_batch_items(const Item *__restrict__ items, int64_t nitems, int64_t n, int k,
                     const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ w,
                     const double *__restrict__ S, const double *__restrict__ Z, const double *__restrict__ mean,
                     double *__restrict__ part)
{
    __shared__ double red[8][4][64];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const bool has1 = lane < k, has2 = lane + 32 < k;
    const bool has[2] = {has1, has2};
    double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    const double mu[2] = {has1 ? mean[lane] : 0.0, has2 ? mean[lane + 32] : 0.0};
    double zx[2] = {0.0, 0.0};  // the current row's z, per half
    auto begin = [&](int64_t x) {
        zx[0] = has1 ? Z[x * k + lane] : 0.0;
        zx[1] = has2 ? Z[x * k + lane + 32] : 0.0;
    };
    auto src = [&](int32_t c) -> const double * { return Z + (int64_t)c * k; };
    auto add = [&](double &a, float wt, double v, int h) {
        const double d = zx[h] - v;
        a += (W ? (double)wt : 1.0) * d * d;
    };
    auto row_terms = [&](int64_t x) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            if (!has[hh]) continue;
            const double sx = S[x * k + lane + 32 * hh], z = zx[hh];
            acc[hh][0] += z * z;
            acc[hh][1] += (z - mu[hh]) * (z - mu[hh]);
            acc[hh][2] += (z - sx) * (z - sx);
        }
    };
    for (int64_t ii = (int64_t)blockIdx.x * 8 + wl; ii < nitems; ii += (int64_t)gridDim.x * 8) {
        const Item it = items[ii];
        const int64_t r0 = it.r0, r1 = it.r1;
        if (!FJ_IDX_OK(1, r0, n) || !FJ_IDX_OK(2, r1, n + 1) ||
            (it.slot < 0 && !FJ_IDX_OK(3, r1 - r0, kWarpRows + 1)))
            continue;
        if (it.slot < 0) {
            auto apply = [&](int64_t x, double s1, double s2) {
                row_terms(x);  // zx is row x's until the next row begins
                acc[0][3] += s1;
                acc[1][3] += s2;
            };
            warp_tile_k<double, double, W, 8>(r0, r1, it.k0, it.k1, false, rp, col, w, begin, src, add, apply, lane,
                                              has1, has2, n);
        } else {
            auto apply = [&](int64_t, double s1, double s2) {
                acc[0][3] += s1;
                acc[1][3] += s2;
            };
            warp_tile_k<double, double, W, 8>(r0, r0 + 1, it.k0, it.k1, true, rp, col, w, begin, src, add, apply,
                                              lane, has1, has2, n);
            if (it.k0 == rp[r0]) row_terms(r0);  // the row's own terms, once
        }
    }
    for (int hh = 0; hh < 2; ++hh)
        for (int f = 0; f < 4; ++f) red[wl][f][lane + 32 * hh] = acc[hh][f];
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 64; i += 256) {
        const int f = i / 64, j = i % 64;
        if (j >= k) continue;
        double t = 0.0;
        for (int ww = 0; ww < 8; ++ww) t += red[ww][f][j];
        part[((int64_t)blockIdx.x * 4 + f) * k + j] = t;
    }
}

// out[f * k + j] = sum over blocks (in order) of part[b][f][j].
__global__ void k_metric_batch_reduce(int nblocks, int nf, int k, const double *__restrict__ part,
                                      double *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf * k; i += gridDim.x * blockDim.x) {
        const int f = i / k, j = i % k;
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += part[((int64_t)b * nf + f) * k + j];
        out[i] = t;
    }
}

__global__ void k_metric_batch_mean(int k, int64_t n, double *__restrict__ m)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) m[j] /= (double)n;
}

}  // namespace fj

using namespace fj;

extern "C" fj_status fj_metrics(fj_graph *g, const double *s, const double *z, fj_metrics_out *out, int mem,
                                void *stream)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(s && z && out, "NULL pointer");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    cudaStream_t st = (cudaStream_t)stream;
    const DevCSR &c = g->csr;
    const int64_t n = c.n, nb = c.nblocks;
    const int ng = g->ngraphs;
    // scratch: staged s and z, per-block partials, per-graph results and block ranges
    size_t bytes = sizeof(double) * (size_t)(4 * nb + 8 * ng) + sizeof(int64_t) * (size_t)(2 * ng + 2);
    if (mem == FJ_MEM_HOST) bytes += sizeof(double) * 2 * (size_t)n;
    char *buf = nullptr;
    FJ_CUDA(cudaMallocAsync(&buf, bytes, st));
    double *part = reinterpret_cast<double *>(buf);
    double *mean = part + 4 * nb;
    double *res = mean + ng;
    int64_t *gblk = reinterpret_cast<int64_t *>(res + 4 * ng + 3 * ng);
    int64_t *noff = gblk + ng + 1;
    const double *sd = s, *zd = z;
    std::vector<int64_t> hg((size_t)ng + 1), hn((size_t)ng + 1);
    for (int i = 0; i < ng; ++i) {
        hg[(size_t)i] = ng > 1 ? c.seg_blk[(size_t)i] : 0;
        hn[(size_t)i] = g->node_off[(size_t)i];
    }
    hg[(size_t)ng] = nb;
    hn[(size_t)ng] = n;
    FJ_CUDA(cudaMemcpyAsync(gblk, hg.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, st));
    FJ_CUDA(cudaMemcpyAsync(noff, hn.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, st));
    if (mem == FJ_MEM_HOST) {
        double *stage = reinterpret_cast<double *>(noff + ng + 1);
        FJ_CUDA(cudaMemcpyAsync(stage, s, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        FJ_CUDA(cudaMemcpyAsync(stage + n, z, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        sd = stage;
        zd = stage + n;
    }
    k_metric_mean<<<(unsigned)nb, 256, 0, st>>>(c.blk_row, zd, part);
    k_metric_reduce<<<(unsigned)ng, 256, 0, st>>>(ng, gblk, part, 1, mean);
    k_metric_mean_div<<<(unsigned)ceil_div(ng, 256), 256, 0, st>>>(ng, noff, mean);
    if (c.w)
        k_metric_main<true><<<(unsigned)nb, 256, 0, st>>>(c.row_ptr, c.col, c.w, c.blk_row, sd, zd, c.graph_of, mean,
                                                          part);
    else
        k_metric_main<false><<<(unsigned)nb, 256, 0, st>>>(c.row_ptr, c.col, c.w, c.blk_row, sd, zd, c.graph_of, mean,
                                                           part);
    k_metric_reduce<<<(unsigned)ng, 256, 0, st>>>(ng, gblk, part, 4, res);
    FJ_CUDA(cudaGetLastError());
    std::vector<double> hres((size_t)4 * ng), hmean((size_t)ng);
    FJ_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * 4 * ng, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(hmean.data(), mean, sizeof(double) * ng, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaFreeAsync(buf, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < ng; ++i) {
        out[i].C = hres[(size_t)4 * i + 0];
        out[i].P = hres[(size_t)4 * i + 1];
        out[i].I = hres[(size_t)4 * i + 2];
        out[i].D = g->directed ? hres[(size_t)4 * i + 3] : 0.5 * hres[(size_t)4 * i + 3];
        out[i].mean_z = hmean[(size_t)i];
    }
    return FJ_OK;
}

extern "C" fj_status fj_metrics_batch(fj_graph *g, const double *S, const double *Z, int k, fj_metrics_out *out,
                                      int mem, void *stream)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(S && Z && out, "NULL pointer");
    FJ_ARG(k >= 1 && k <= 64, "k must be in 1..64");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_ARG(g->ngraphs == 1, "a ragged handle takes fj_metrics");
    cudaStream_t st = (cudaStream_t)stream;
    const DevCSR &c = g->csr;
    const int64_t n = c.n;
    const int nb = kMetricBatchBlocks;
    size_t bytes = sizeof(double) * ((size_t)nb * 4 * k + 5 * (size_t)k);
    if (mem == FJ_MEM_HOST) bytes += sizeof(double) * 2 * (size_t)n * k;
    char *buf = nullptr;
    FJ_CUDA(cudaMallocAsync(&buf, bytes, st));
    double *part = reinterpret_cast<double *>(buf);
    double *mean = part + (size_t)nb * 4 * k;
    double *res = mean + k;
    const double *Sd = S, *Zd = Z;
    if (mem == FJ_MEM_HOST) {
        double *stage = res + 4 * k;
        FJ_CUDA(cudaMemcpyAsync(stage, S, sizeof(double) * n * k, cudaMemcpyHostToDevice, st));
        FJ_CUDA(cudaMemcpyAsync(stage + n * k, Z, sizeof(double) * n * k, cudaMemcpyHostToDevice, st));
        Sd = stage;
        Zd = stage + n * k;
    }
    const ItemPlan *ip = nullptr;
    FJ_CHECK(plain_items(g, st, &ip));
    k_metric_batch_sum<<<nb, 256, 0, st>>>(n, k, Zd, part);
    k_metric_batch_reduce<<<1, 64, 0, st>>>(nb, 1, k, part, mean);
    k_metric_batch_mean<<<1, 64, 0, st>>>(k, n, mean);
    if (c.w)
        k_metric_batch_items<true><<<nb, 256, 0, st>>>(ip->items, ip->nitems, n, k, c.row_ptr, c.col, c.w, Sd, Zd,
                                                       mean, part);
    else
        k_metric_batch_items<false><<<nb, 256, 0, st>>>(ip->items, ip->nitems, n, k, c.row_ptr, c.col, c.w, Sd, Zd,
                                                        mean, part);
    k_metric_batch_reduce<<<1, 256, 0, st>>>(nb, 4, k, part, res);
    FJ_CUDA(cudaGetLastError());
    std::vector<double> hres((size_t)4 * k), hmean((size_t)k);
    FJ_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * 4 * k, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaMemcpyAsync(hmean.data(), mean, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaFreeAsync(buf, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    long long dbg[4] = {0, 0, 0, 0};
    FJ_CUDA(cudaMemcpyFromSymbol(dbg, g_fj_metric_dbg, sizeof(dbg)));
    if (dbg[0]) {
        const long long zero[4] = {0, 0, 0, 0};
        FJ_CUDA(cudaMemcpyToSymbol(g_fj_metric_dbg, zero, sizeof(zero)));
        set_error("index check failed in the batch measures: site %lld block %lld index %lld limit %lld", dbg[0],
                  dbg[1], dbg[2], dbg[3]);
        return FJ_ERR_INVALID_ARG;
    }
    for (int j = 0; j < k; ++j) {
        out[j].C = hres[(size_t)0 * k + j];
        out[j].P = hres[(size_t)1 * k + j];
        out[j].I = hres[(size_t)2 * k + j];
        out[j].D = g->directed ? hres[(size_t)3 * k + j] : 0.5 * hres[(size_t)3 * k + j];
        out[j].mean_z = hmean[(size_t)j];
    }
    return FJ_OK;
}
