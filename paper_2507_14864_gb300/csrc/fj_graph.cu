// Graph ingest on the GPU (Section 3.2 matrices): CSR validation, FP64
// out-degrees and 1/(1+d), in-degrees, the transposed CSR, row blocks for the
// push kernels, arc-list ingest (drop self-loops, keep the first of repeated
// arcs), ragged block-diagonal batches, and the Jones-Plassmann colouring that
// gives the Gauss-Seidel order of the multicolour schedule.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <functional>
#include <string>

#include "fj_internal.cuh"

// ============================================================== error plumbing

namespace fj {

static thread_local char g_last_error[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

fj_status cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? FJ_ERR_OOM : FJ_ERR_CUDA;
}

void dev_free(void *p)
{
    if (p) cudaFree(p);
}

// Allocation-failure injection: -1 disarmed, else the number of allocations
// that still succeed before one fails.
static std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t dev_malloc_raw(void **p, size_t bytes)
{
    long long left = g_fail_alloc_after.load();
    while (left >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
            if (left == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
static cudaError_t dalloc(T **p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    return dev_malloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)count);
}

fj_status ws_status(Workspace &ws, int64_t tiles)
{
    if (tiles <= ws.cap_status && ws.status) return FJ_OK;
    dev_free(ws.status);
    ws.status = nullptr;
    ws.cap_status = 0;
    int64_t cap = std::max<int64_t>(tiles, 1024);
    FJ_CUDA(dalloc(&ws.status, cap));
    ws.cap_status = cap;
    if (!ws.tile_ctr) FJ_CUDA(dalloc(&ws.tile_ctr, 1));
    if (!ws.count) FJ_CUDA(dalloc(&ws.count, 4));
    return FJ_OK;
}

static const char *dev_err_text(int code)
{
    switch (code) {
    case DEV_BAD_ROW_PTR: return "row_ptr is not a nondecreasing offset array from 0 to nnz";
    case DEV_BAD_COL: return "column index out of range";
    case DEV_SELF_LOOP: return "self-loop in the CSR";
    case DEV_UNSORTED_ROW: return "row not strictly increasing (unsorted or repeated column)";
    case DEV_BAD_WEIGHT: return "weight not positive and finite";
    case DEV_CROSS_GRAPH: return "arc leaves its graph in a ragged batch";
    case DEV_SPIN_TIMEOUT: return "bounded device wait timed out";
    case DEV_NONFINITE: return "residual became non-finite";
    case DEV_BAD_OPINION: return "opinion vector holds a non-finite value";
    default: return "unknown device error";
    }
}

fj_status read_dev_error(fj_graph *g, cudaStream_t st)
{
    FJ_CUDA(cudaMemcpyAsync(g->err_host, g->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    int code = *g->err_host;
    if (code == DEV_OK) return FJ_OK;
    FJ_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), st));
    set_error("%s", dev_err_text(code));
    if (code == DEV_SPIN_TIMEOUT) return FJ_ERR_TIMEOUT;
    if (code == DEV_NONFINITE) return FJ_ERR_DIVERGED;
    return FJ_ERR_INVALID_ARG;
}

// ============================================================== kernels

// Warp per row: offsets, column range, no self-loop, strictly increasing,
// weights positive and finite, arcs inside their graph (ragged).
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const float *__restrict__ w, const int64_t *__restrict__ node_off,
                           const int32_t *__restrict__ graph_of, int *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (warp0 == 0 && lane == 0 && (rp[0] != 0 || rp[n] != nnz)) dev_error(err, DEV_BAD_ROW_PTR);
    for (int64_t u = warp0; u < n; u += nwarps) {
        int64_t a = rp[u], b = rp[u + 1];
        if (a > b || a < 0 || b > nnz) {
            if (lane == 0) dev_error(err, DEV_BAD_ROW_PTR);
            continue;
        }
        int64_t lo = 0, hi = n;
        if (graph_of) {
            int gph = graph_of[u];
            lo = node_off[gph];
            hi = node_off[gph + 1];
        }
        for (int64_t k = a + lane; k < b; k += 32) {
            int32_t c = col[k];
            if (c < 0 || c >= n) {
                dev_error(err, DEV_BAD_COL);
                continue;
            }
            if (c == u) dev_error(err, DEV_SELF_LOOP);
            if (k > a && col[k - 1] >= c) dev_error(err, DEV_UNSORTED_ROW);
            if (c < lo || c >= hi) dev_error(err, DEV_CROSS_GRAPH);
            if (w) {
                float x = w[k];
                if (!(x > 0.0f) || !isfinite(x)) dev_error(err, DEV_BAD_WEIGHT);
            }
        }
    }
}

// Warp per row: d_u = sum of the row's weights in FP64, 1/(1+d_u) in FP64 and FP32.
__global__ void k_degrees(int64_t n, const int64_t *__restrict__ rp, const float *__restrict__ w,
                          double *__restrict__ deg, double *__restrict__ inv64, float *__restrict__ inv32)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp0; u < n; u += nwarps) {
        int64_t a = rp[u], b = rp[u + 1];
        double acc = 0.0;
        if (w) {
            for (int64_t k = a + lane; k < b; k += 32) acc += (double)w[k];
            acc = warp_sum(acc);
        } else {
            acc = (double)(b - a);
        }
        if (lane == 0) {
            double iv = 1.0 / (1.0 + acc);
            deg[u] = acc;
            inv64[u] = iv;
            inv32[u] = (float)iv;
        }
    }
}

__global__ void k_count_cols(int64_t nnz, const int32_t *__restrict__ col, int32_t *__restrict__ cnt)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[k]], 1);
}

__global__ void k_iota(int64_t n, uint32_t *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)i;
}

// Warp per row: write the row id into every slot of the row.
__global__ void k_row_of(int64_t n, const int64_t *__restrict__ rp, uint32_t *__restrict__ row_of)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp0; u < n; u += nwarps)
        for (int64_t k = rp[u] + lane; k < rp[u + 1]; k += 32) row_of[k] = (uint32_t)u;
}

// out_col[i] = row_of[perm[i]], out_w[i] = w[perm[i]].
__global__ void k_gather_transposed(int64_t nnz, const uint32_t *__restrict__ perm, const uint32_t *__restrict__ row_of,
                                    const float *__restrict__ w, int32_t *__restrict__ tcol, float *__restrict__ tw)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k = perm[i];
        tcol[i] = (int32_t)row_of[k];
        if (w) tw[i] = w[k];
    }
}

struct I32Load {
    const int32_t *a;
    __device__ long long operator()(int64_t i) const { return (long long)a[i]; }
};

__global__ void k_finish_ptr(int64_t n, const long long *__restrict__ excl, long long total, int64_t *__restrict__ ptr)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        ptr[i] = i < n ? (int64_t)excl[i] : (int64_t)total;
}

__global__ void k_finish_ptr_dev(int64_t n, const long long *__restrict__ excl, const long long *__restrict__ total,
                                 int64_t *__restrict__ ptr)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        ptr[i] = i < n ? (int64_t)excl[i] : (int64_t)*total;
}

// A block starts at row 0, at every forced segment start, every max_rows
// rows, at and after every row longer than `bucket` nonzeros, and where the
// row's first nonzero enters a new bucket-sized stretch of the nonzero range;
// so a block of several rows holds at most 2 * bucket nonzeros.
struct BlockStartPred {
    const int64_t *rp;
    const int64_t *seg;  // sorted forced starts
    int nseg;
    int64_t bucket;
    int64_t max_rows;
    __device__ bool operator()(int64_t u) const
    {
        if (u == 0 || (u % max_rows) == 0) return true;
        int64_t a = rp[u], la = rp[u + 1] - a, b = rp[u - 1], lb = a - b;
        if (la > bucket || lb > bucket) return true;
        if ((a / bucket) != (b / bucket)) return true;
        int lo = 0, hi = nseg;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (seg[mid] < u) lo = mid + 1; else hi = mid;
        }
        return lo < nseg && seg[lo] == u;
    }
};

// seg_blk[i] = index of the block that starts at row seg[i].
__global__ void k_seg_blocks(int nseg, const int64_t *__restrict__ seg, const int32_t *__restrict__ blk_row,
                             int64_t nblocks, long long *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    int64_t lo = 0, hi = nblocks;  // first block with blk_row >= seg[i]
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (blk_row[mid] < seg[i]) lo = mid + 1; else hi = mid;
    }
    out[i] = lo;
}

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }

// ============================================================== host pieces

fj_status build_blocks(DevCSR &c, const std::vector<int64_t> &seg_rows, Workspace &ws, int *err, cudaStream_t st,
                       TileKind kind)
{
    const int64_t n = c.n;
    const bool warp_tiles = kind != kTileBlock;
    int32_t *&blk = warp_tiles ? c.wblk_row : c.blk_row;
    dev_free(blk);
    blk = nullptr;
    FJ_CUDA(dalloc(&blk, n + 2));
    int64_t *seg_d = nullptr;
    std::vector<int64_t> seg = seg_rows;
    std::sort(seg.begin(), seg.end());
    FJ_CUDA(dalloc(&seg_d, (int64_t)seg.size() + 1));
    if (!seg.empty())
        FJ_CUDA(cudaMemcpyAsync(seg_d, seg.data(), sizeof(int64_t) * seg.size(), cudaMemcpyHostToDevice, st));
    FJ_CHECK(ws_status(ws, scan_tiles(n, 256 * 8)));
    const int64_t bucket = warp_tiles ? kWarpNnz : kBlockNnz;
    const int64_t max_rows = warp_tiles ? kWarpRows : kBlockRows;
    FJ_CUDA(compact<256, 8>(n, BlockStartPred{c.row_ptr, seg_d, (int)seg.size(), bucket, max_rows}, blk, ws.count,
                            ws.status, ws.tile_ctr, err, st));
    long long nb = 0;
    FJ_CUDA(cudaMemcpyAsync(&nb, ws.count, sizeof(long long), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    k_set_i32<<<1, 1, 0, st>>>(blk + nb, (int32_t)n);
    FJ_CUDA(cudaGetLastError());
    if (warp_tiles) {
        c.nwblocks = nb;
        dev_free(seg_d);
        return FJ_OK;
    }
    c.nblocks = nb;
    c.seg_blk.assign(seg.size() + 1, nb);
    if (!seg.empty()) {
        long long *sb = nullptr;
        FJ_CUDA(dalloc(&sb, (int64_t)seg.size()));
        k_seg_blocks<<<(unsigned)ceil_div((int64_t)seg.size(), 256), 256, 0, st>>>((int)seg.size(), seg_d, c.blk_row,
                                                                               nb, sb);
        FJ_CUDA(cudaGetLastError());
        std::vector<long long> h(seg.size());
        FJ_CUDA(cudaMemcpyAsync(h.data(), sb, sizeof(long long) * seg.size(), cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < seg.size(); ++i) c.seg_blk[i] = h[i];
        dev_free(sb);
    }
    dev_free(seg_d);
    return FJ_OK;
}

static void csr_free(DevCSR &c)
{
    dev_free(c.row_ptr);
    dev_free(c.col);
    dev_free(c.w);
    dev_free(c.deg64);
    dev_free(c.inv32);
    dev_free(c.inv64);
    dev_free(c.indeg);
    dev_free(c.graph_of);
    dev_free(c.blk_row);
    dev_free(c.wblk_row);
    c = DevCSR();
}

// Degrees, in-degrees, the transposed CSR (directed) and row blocks.
static fj_status derive_arrays(fj_graph *g, DevCSR &c, bool transpose, const std::vector<int64_t> &segs,
                               cudaStream_t st)
{
    const int64_t n = c.n, nnz = c.nnz;
    FJ_CUDA(dalloc(&c.deg64, n));
    FJ_CUDA(dalloc(&c.inv64, n));
    FJ_CUDA(dalloc(&c.inv32, n));
    FJ_CUDA(dalloc(&c.indeg, n));
    k_degrees<<<grid_for(n * 32, 256), 256, 0, st>>>(n, c.row_ptr, c.w, c.deg64, c.inv64, c.inv32);
    FJ_CUDA(cudaGetLastError());
    FJ_CUDA(cudaMemsetAsync(c.indeg, 0, sizeof(int32_t) * n, st));
    if (nnz > 0) {
        k_count_cols<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, c.col, c.indeg);
        FJ_CUDA(cudaGetLastError());
    }
    if (transpose) {
        FJ_CUDA(dalloc(&g->tptr, n + 1));
        FJ_CUDA(dalloc(&g->tcol, nnz));
        if (c.w) FJ_CUDA(dalloc(&g->tw, nnz));
        long long *excl = nullptr;
        FJ_CUDA(dalloc(&excl, n + 1));
        FJ_CHECK(ws_status(g->ws, scan_tiles(n, 256 * 8)));
        FJ_CUDA(scan<256, 8>(n, I32Load{c.indeg}, excl, g->ws.count, g->ws.status, g->ws.tile_ctr, g->err, st));
        k_finish_ptr_dev<<<grid_for(n + 1, 256), 256, 0, st>>>(n, excl, g->ws.count, g->tptr);
        FJ_CUDA(cudaGetLastError());
        dev_free(excl);
        if (nnz > 0) {
            uint32_t *k0, *v0, *k1, *v1, *row_of;
            FJ_CUDA(dalloc(&k0, nnz));
            FJ_CUDA(dalloc(&v0, nnz));
            FJ_CUDA(dalloc(&k1, nnz));
            FJ_CUDA(dalloc(&v1, nnz));
            FJ_CUDA(dalloc(&row_of, nnz));
            FJ_CUDA(cudaMemcpyAsync(k0, c.col, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToDevice, st));
            k_iota<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, v0);
            k_row_of<<<grid_for(n * 32, 256), 256, 0, st>>>(n, c.row_ptr, row_of);
            FJ_CUDA(cudaGetLastError());
            bool in1 = false;
            FJ_CUDA(sort_pairs(nnz, bits_for(n - 1), k0, v0, k1, v1, g->sort, g->err, st, &in1));
            k_gather_transposed<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, in1 ? v1 : v0, row_of, c.w, g->tcol, g->tw);
            FJ_CUDA(cudaGetLastError());
            FJ_CUDA(cudaStreamSynchronize(st));
            dev_free(k0); dev_free(v0); dev_free(k1); dev_free(v1); dev_free(row_of);
        }
    }
    FJ_CHECK(build_blocks(c, segs, g->ws, g->err, st, kTileBlock));
    FJ_CHECK(build_blocks(c, segs, g->ws, g->err, st, kTileWarp));
    return FJ_OK;
}

fj_status graph_finish(fj_graph *g, cudaStream_t st)
{
    std::vector<int64_t> segs;
    if (g->ngraphs > 1) segs.assign(g->node_off.begin(), g->node_off.end() - 1);
    FJ_CHECK(derive_arrays(g, g->csr, g->directed != 0, segs, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    return read_dev_error(g, st);
}

static fj_status graph_alloc_shell(int64_t n, int directed, fj_graph **out)
{
    fj_graph *g = new (std::nothrow) fj_graph();
    if (!g) {
        set_error("host allocation failed");
        return FJ_ERR_OOM;
    }
    cudaGetDevice(&g->device);
    g->directed = directed ? 1 : 0;
    g->csr.n = n;
    cudaError_t e = dev_malloc(&g->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&g->err_host, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        fj_graph_destroy(g);
        return cuda_fail(e, "graph shell", __FILE__, __LINE__);
    }
    *out = g;
    return FJ_OK;
}

static cudaMemcpyKind kind_in(int mem) { return mem == FJ_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
static cudaMemcpyKind kind_out(int mem) { return mem == FJ_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

static fj_status create_common(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w, int directed,
                               int mem, cudaStream_t st, int ngraphs, const int64_t *node_off_host, fj_graph **out)
{
    // nnz from the last offset (read once through the copy below)
    int64_t nnz = 0;
    if (mem == FJ_MEM_DEVICE) {
        FJ_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
    } else {
        nnz = row_ptr[n];
    }
    FJ_ARG(nnz >= 0 && nnz < (int64_t(1) << 31), "nnz must be in [0, 2^31)");
    FJ_ARG(nnz == 0 || col != nullptr, "col is NULL");
    fj_graph *g = nullptr;
    FJ_CHECK(graph_alloc_shell(n, directed, &g));
    fj_status s = FJ_OK;
    do {
        DevCSR &c = g->csr;
        c.nnz = nnz;
        cudaError_t e;
        if ((e = dalloc(&c.row_ptr, n + 1)) != cudaSuccess) { s = cuda_fail(e, "alloc", __FILE__, __LINE__); break; }
        if ((e = dalloc(&c.col, nnz + kNnzPad)) != cudaSuccess) { s = cuda_fail(e, "alloc", __FILE__, __LINE__); break; }
        if (w && (e = dalloc(&c.w, nnz + kNnzPad)) != cudaSuccess) { s = cuda_fail(e, "alloc", __FILE__, __LINE__); break; }
        e = cudaMemcpyAsync(c.row_ptr, row_ptr, sizeof(int64_t) * (n + 1), kind_in(mem), st);
        if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(c.col, col, sizeof(int32_t) * nnz, kind_in(mem), st);
        if (e == cudaSuccess && w && nnz) e = cudaMemcpyAsync(c.w, w, sizeof(float) * nnz, kind_in(mem), st);
        if (e != cudaSuccess) { s = cuda_fail(e, "copy CSR", __FILE__, __LINE__); break; }
        g->ngraphs = ngraphs;
        if (ngraphs > 1) {
            g->node_off.assign(node_off_host, node_off_host + ngraphs + 1);
            if ((e = dalloc(&g->node_off_d, ngraphs + 1)) != cudaSuccess) { s = cuda_fail(e, "alloc", __FILE__, __LINE__); break; }
            if ((e = dalloc(&c.graph_of, n)) != cudaSuccess) { s = cuda_fail(e, "alloc", __FILE__, __LINE__); break; }
            e = cudaMemcpyAsync(g->node_off_d, node_off_host, sizeof(int64_t) * (ngraphs + 1), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { s = cuda_fail(e, "copy offsets", __FILE__, __LINE__); break; }
            // graph id per row: expand offsets on the host once (n int32)
            std::vector<int32_t> gof((size_t)n);
            for (int gi = 0; gi < ngraphs; ++gi)
                for (int64_t v = node_off_host[gi]; v < node_off_host[gi + 1]; ++v) gof[(size_t)v] = gi;
            e = cudaMemcpyAsync(c.graph_of, gof.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { s = cuda_fail(e, "copy graph ids", __FILE__, __LINE__); break; }
        } else {
            g->node_off = {0, n};
        }
        k_validate<<<grid_for(n * 32, 256), 256, 0, st>>>(n, nnz, c.row_ptr, c.col, c.w, g->node_off_d, c.graph_of,
                                                           g->err);
        if ((e = cudaGetLastError()) != cudaSuccess) { s = cuda_fail(e, "validate", __FILE__, __LINE__); break; }
        s = read_dev_error(g, st);
        if (s != FJ_OK) break;
        s = graph_finish(g, st);
    } while (0);
    if (s != FJ_OK) {
        fj_graph_destroy(g);
        return s;
    }
    *out = g;
    return FJ_OK;
}

// ---------------------------------------------------------------- arc ingest

struct NotLoopPred {
    const int32_t *src, *dst;
    __device__ bool operator()(int64_t e) const { return src[e] != dst[e]; }
};

__global__ void k_arc_check(int64_t m, int64_t n, const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            const float *__restrict__ w, int *err)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) dev_error(err, DEV_BAD_COL);
        if (w && (!(w[e] > 0.0f) || !isfinite(w[e]))) dev_error(err, DEV_BAD_WEIGHT);
    }
}

// keys[i] = field[ids[i]]
__global__ void k_gather_key(int64_t m, const uint32_t *__restrict__ ids, const int32_t *__restrict__ field,
                             uint32_t *__restrict__ keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)field[ids[i]];
}

// Position i of the (src, dst)-sorted arc order is kept when it is the first of its (src, dst) run.
struct FirstOfRunPred {
    const uint32_t *ids;
    const int32_t *src, *dst;
    __device__ bool operator()(int64_t i) const
    {
        if (i == 0) return true;
        uint32_t a = ids[i], b = ids[i - 1];
        return src[a] != src[b] || dst[a] != dst[b];
    }
};

__global__ void k_emit_arcs(int64_t nk, const int32_t *__restrict__ pos, const uint32_t *__restrict__ ids,
                            const int32_t *__restrict__ src, const int32_t *__restrict__ dst, const float *__restrict__ w,
                            int32_t *__restrict__ col, float *__restrict__ wout, int32_t *__restrict__ rowcnt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = ids[pos[i]];
        col[i] = dst[e];
        if (w) wout[i] = w[e];
        atomicAdd(&rowcnt[src[e]], 1);
    }
}

}  // namespace fj

using namespace fj;

// ============================================================== C ABI

extern "C" {

void fj_solve_opts_default(fj_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps = 1e-6;
    o->omega = 1.0;
    o->c = 1e-5;
    o->sigma = 1e-5;
    o->precision = FJ_PREC_FP64;
    o->schedule = FJ_SCHED_AUTO;
    o->max_sweeps = 100000;
    o->max_refine = 8;
    o->palette = 16;
    o->check_every = 0;
    o->stream = nullptr;
}

const char *fj_status_string(fj_status s)
{
    switch (s) {
    case FJ_OK: return "ok";
    case FJ_ERR_INVALID_ARG: return "invalid argument";
    case FJ_ERR_CUDA: return "CUDA error";
    case FJ_ERR_OOM: return "out of device memory";
    case FJ_ERR_NOT_CONVERGED: return "not converged";
    case FJ_ERR_DIVERGED: return "diverged";
    case FJ_ERR_UNSUPPORTED: return "unsupported";
    case FJ_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *fj_last_error(void) { return g_last_error; }

fj_status fj_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w, int directed,
                          int mem, void *stream, fj_graph **out)
{
    FJ_ARG(out != nullptr, "out is NULL");
    FJ_ARG(n >= 1 && n < (int64_t(1) << 31), "n must be in [1, 2^31)");
    FJ_ARG(row_ptr != nullptr, "row_ptr is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    *out = nullptr;
    return create_common(n, row_ptr, col, w, directed, mem, (cudaStream_t)stream, 1, nullptr, out);
}

fj_status fj_graph_create_ragged(int ngraphs, const int64_t *node_offsets, const int64_t *row_ptr,
                                 const int32_t *col, const float *w, int directed, int mem, void *stream,
                                 fj_graph **out)
{
    FJ_ARG(out != nullptr, "out is NULL");
    FJ_ARG(ngraphs >= 1, "ngraphs must be >= 1");
    FJ_ARG(node_offsets != nullptr && row_ptr != nullptr, "NULL offsets");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    std::vector<int64_t> off((size_t)ngraphs + 1);
    if (mem == FJ_MEM_DEVICE) {
        FJ_CUDA(cudaMemcpy(off.data(), node_offsets, sizeof(int64_t) * (ngraphs + 1), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(off.data(), node_offsets, sizeof(int64_t) * (ngraphs + 1));
    }
    FJ_ARG(off[0] == 0, "node_offsets[0] must be 0");
    for (int i = 0; i < ngraphs; ++i) FJ_ARG(off[i + 1] > off[i], "node_offsets must be strictly increasing");
    int64_t n = off[ngraphs];
    FJ_ARG(n < (int64_t(1) << 31), "total nodes must be < 2^31");
    *out = nullptr;
    return create_common(n, row_ptr, col, w, directed, mem, (cudaStream_t)stream, ngraphs, off.data(), out);
}

fj_status fj_graph_create_from_arcs(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w,
                                    int directed, int mem, void *stream, fj_graph **out)
{
    FJ_ARG(out != nullptr, "out is NULL");
    FJ_ARG(n >= 1 && n < (int64_t(1) << 31), "n must be in [1, 2^31)");
    FJ_ARG(m >= 0 && m < (int64_t(1) << 31), "m must be in [0, 2^31)");
    FJ_ARG(m == 0 || (src && dst), "NULL arc arrays");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    fj_graph *g = nullptr;
    FJ_CHECK(graph_alloc_shell(n, directed, &g));
    fj_status s = FJ_OK;
    int32_t *ds = nullptr, *dd = nullptr, *pos = nullptr;
    float *dw = nullptr;
    uint32_t *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr;
    auto fail = [&](cudaError_t e, const char *what) { s = cuda_fail(e, what, __FILE__, __LINE__); };
    do {
        cudaError_t e;
        if ((e = dalloc(&ds, m)) || (e = dalloc(&dd, m)) || (w && (e = dalloc(&dw, m)))) { fail(e, "alloc arcs"); break; }
        if (m) {
            e = cudaMemcpyAsync(ds, src, sizeof(int32_t) * m, kind_in(mem), st);
            if (!e) e = cudaMemcpyAsync(dd, dst, sizeof(int32_t) * m, kind_in(mem), st);
            if (!e && w) e = cudaMemcpyAsync(dw, w, sizeof(float) * m, kind_in(mem), st);
            if (e) { fail(e, "copy arcs"); break; }
            k_arc_check<<<grid_for(m, 256), 256, 0, st>>>(m, n, ds, dd, dw, g->err);
            if ((e = cudaGetLastError())) { fail(e, "arc check"); break; }
        }
        s = read_dev_error(g, st);
        if (s != FJ_OK) break;
        if ((e = dalloc(&k0, m)) || (e = dalloc(&v0, m)) || (e = dalloc(&k1, m)) || (e = dalloc(&v1, m)) ||
            (e = dalloc(&pos, m))) { fail(e, "alloc sort"); break; }
        // arcs that are not self-loops, in array order
        s = ws_status(g->ws, scan_tiles(m, 256 * 8));
        if (s != FJ_OK) break;
        long long mk = 0;
        if (m) {
            if ((e = compact<256, 8>(m, NotLoopPred{ds, dd}, reinterpret_cast<int32_t *>(v0), g->ws.count,
                                     g->ws.status, g->ws.tile_ctr, g->err, st))) { fail(e, "drop loops"); break; }
            if ((e = cudaMemcpyAsync(&mk, g->ws.count, sizeof(long long), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st))) { fail(e, "count"); break; }
        }
        // stable sort by dst, then stable sort by src: (src, dst, array order)
        bool in1 = false;
        uint32_t *ids = v0;
        if (mk > 1) {
            k_gather_key<<<grid_for(mk, 256), 256, 0, st>>>(mk, v0, dd, k0);
            if ((e = sort_pairs(mk, bits_for(n - 1), k0, v0, k1, v1, g->sort, g->err, st, &in1))) { fail(e, "sort dst"); break; }
            uint32_t *kA = in1 ? k1 : k0, *vA = in1 ? v1 : v0;  // dst-sorted ids live in vA
            uint32_t *kB = in1 ? k0 : k1, *vB = in1 ? v0 : v1;  // free pair
            k_gather_key<<<grid_for(mk, 256), 256, 0, st>>>(mk, vA, ds, kA);
            bool in2 = false;
            if ((e = sort_pairs(mk, bits_for(n - 1), kA, vA, kB, vB, g->sort, g->err, st, &in2))) { fail(e, "sort src"); break; }
            ids = in2 ? vB : vA;
        }
        // first arc of every (src, dst) run
        long long nk = 0;
        if (mk) {
            if ((e = compact<256, 8>(mk, FirstOfRunPred{ids, ds, dd}, pos, g->ws.count, g->ws.status, g->ws.tile_ctr,
                                     g->err, st))) { fail(e, "dedup"); break; }
            if ((e = cudaMemcpyAsync(&nk, g->ws.count, sizeof(long long), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st))) { fail(e, "count"); break; }
        }
        DevCSR &c = g->csr;
        c.nnz = nk;
        int32_t *rowcnt = nullptr;
        long long *excl = nullptr;
        if ((e = dalloc(&c.row_ptr, n + 1)) || (e = dalloc(&c.col, nk + kNnzPad)) || (w && (e = dalloc(&c.w, nk + kNnzPad))) ||
            (e = dalloc(&rowcnt, n)) || (e = dalloc(&excl, n + 1))) { fail(e, "alloc CSR"); break; }
        cudaMemsetAsync(rowcnt, 0, sizeof(int32_t) * n, st);
        if (nk) k_emit_arcs<<<grid_for(nk, 256), 256, 0, st>>>(nk, pos, ids, ds, dd, dw, c.col, c.w, rowcnt);
        s = ws_status(g->ws, scan_tiles(n, 256 * 8));
        if (s != FJ_OK) break;
        if ((e = scan<256, 8>(n, I32Load{rowcnt}, excl, g->ws.count, g->ws.status, g->ws.tile_ctr, g->err, st))) {
            fail(e, "row scan");
            break;
        }
        k_finish_ptr<<<grid_for(n + 1, 256), 256, 0, st>>>(n, excl, nk, c.row_ptr);
        if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(st))) { fail(e, "row_ptr"); break; }
        dev_free(rowcnt);
        dev_free(excl);
        g->node_off = {0, n};
        s = graph_finish(g, st);
    } while (0);
    dev_free(ds); dev_free(dd); dev_free(dw); dev_free(pos);
    dev_free(k0); dev_free(v0); dev_free(k1); dev_free(v1);
    if (s != FJ_OK) {
        fj_graph_destroy(g);
        return s;
    }
    *out = g;
    return FJ_OK;
}

void fj_graph_destroy(fj_graph *g)
{
    if (!g) return;
    csr_free(g->csr);
    dev_free(g->tptr);
    dev_free(g->tcol);
    dev_free(g->tw);
    dev_free(g->node_off_d);
    dev_free(g->colr.colour);
    dev_free(g->colr.perm);
    dev_free(g->colr.iperm);
    dev_free(g->colr.din_p);
    dev_free(g->colr.tptr);
    dev_free(g->colr.tcol);
    dev_free(g->colr.tw);
    csr_free(g->colr.pcsr);
    for (ItemPlan *ip : {&g->wplan_csr, &g->wplan_pcsr}) {
        dev_free(ip->items);
        dev_free(ip->slot_first);
        dev_free(ip->slot_nchunk);
        dev_free(ip->part);
        dev_free(ip->cnt);
    }
    chunk_plan_free(g->cplan_csr);
    chunk_plan_free(g->cplan_pcsr);
    Workspace &ws = g->ws;
    dev_free(ws.r); dev_free(ws.h); dev_free(ws.da); dev_free(ws.db); dev_free(ws.om); dev_free(ws.judge);
    dev_free(ws.rsum); dev_free(ws.carry); dev_free(ws.fdz);
    dev_free(ws.zhat); dev_free(ws.sp); dev_free(ws.sin); dev_free(ws.zout); dev_free(ws.r64); dev_free(ws.zs);
    dev_free(ws.gstat); dev_free(ws.ctr); dev_free(ws.status); dev_free(ws.tile_ctr); dev_free(ws.zmax);
    dev_free(ws.list); dev_free(ws.count); dev_free(ws.partial);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (ws.gexec[a][b]) cudaGraphExecDestroy(ws.gexec[a][b]);
    if (ws.cap_stream) cudaStreamDestroy(ws.cap_stream);
    if (ws.ctr_host) cudaFreeHost(ws.ctr_host);
    BatchWorkspace &b = g->bws;
    dev_free(b.r); dev_free(b.h); dev_free(b.da); dev_free(b.db); dev_free(b.zhat); dev_free(b.sp);
    dev_free(b.z32);
    dev_free(b.sin); dev_free(b.zout); dev_free(b.om); dev_free(b.gstat); dev_free(b.partk);
    dev_free(b.r64); dev_free(b.list); dev_free(b.tick);
    if (b.gstat_host) cudaFreeHost(b.gstat_host);
    if (ws.gstat_host) cudaFreeHost(ws.gstat_host);
    sort_scratch_free(g->sort);
    dev_free(g->err);
    if (g->err_host) cudaFreeHost(g->err_host);
    delete g;
}

fj_status fj_graph_info(const fj_graph *g, int64_t *n, int64_t *nnz, int *ngraphs, int *ncolours)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    if (n) *n = g->csr.n;
    if (nnz) *nnz = g->csr.nnz;
    if (ngraphs) *ngraphs = g->ngraphs;
    if (ncolours) *ncolours = g->colr.built ? g->colr.ncolours : 0;
    return FJ_OK;
}

fj_status fj_graph_export(const fj_graph *g, int transposed, int64_t *row_ptr, int32_t *col, float *w, double *deg64,
                          int mem, void *stream)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    cudaStream_t st = (cudaStream_t)stream;
    const DevCSR &c = g->csr;
    const int64_t *rp = c.row_ptr;
    const int32_t *cc = c.col;
    const float *ww = c.w;
    if (transposed && g->directed) {
        rp = g->tptr;
        cc = g->tcol;
        ww = g->tw;
    }
    if (row_ptr) FJ_CUDA(cudaMemcpyAsync(row_ptr, rp, sizeof(int64_t) * (c.n + 1), kind_out(mem), st));
    if (col && c.nnz) FJ_CUDA(cudaMemcpyAsync(col, cc, sizeof(int32_t) * c.nnz, kind_out(mem), st));
    if (w && ww && c.nnz) FJ_CUDA(cudaMemcpyAsync(w, ww, sizeof(float) * c.nnz, kind_out(mem), st));
    if (deg64) FJ_CUDA(cudaMemcpyAsync(deg64, c.deg64, sizeof(double) * c.n, kind_out(mem), st));
    FJ_CUDA(cudaStreamSynchronize(st));
    return FJ_OK;
}

}  // extern "C"

// ============================================================== colouring

namespace fj {

__device__ __forceinline__ uint32_t prio_hash(uint32_t v)
{
    // SplitMix64 output for state v: mix(v + gamma), high 32 bits
    unsigned long long z = (unsigned long long)v + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (uint32_t)(z >> 32);
}

// Symmetric degree |out(v) U in(v)| and the priority key (degree << 32 | hash).
__global__ void k_sym_degree(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const int64_t *__restrict__ tp, const int32_t *__restrict__ tc,
                             unsigned long long *__restrict__ key)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp0; v < n; v += nwarps) {
        int64_t a = rp[v], b = rp[v + 1];
        long long deg = b - a;
        if (tp) {
            int64_t ta = tp[v], tb = tp[v + 1];
            // count in-neighbours not already among the out-neighbours (binary search in the sorted out-row)
            long long extra = 0;
            for (int64_t k = ta + lane; k < tb; k += 32) {
                int32_t u = tc[k];
                int64_t lo = a, hi = b;
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if (col[mid] < u) lo = mid + 1; else hi = mid;
                }
                extra += (lo < b && col[lo] == u) ? 0 : 1;
            }
            deg += warp_sum(extra);
        }
        if (lane == 0) key[v] = ((unsigned long long)deg << 32) | prio_hash((uint32_t)v);
    }
}

__device__ __forceinline__ bool higher(unsigned long long ku, int64_t u, unsigned long long kv, int64_t v)
{
    return ku > kv || (ku == kv && u < v);
}

// Arc weight in 32.32 fixed point: conflict sums are integers, so their value
// does not depend on the order of the additions.
__device__ __forceinline__ unsigned long long fixed_q(const float *w, int64_t k)
{
    return w ? (unsigned long long)llrint((double)w[k] * 4294967296.0) : (1ULL << 32);
}

// Warp per node: weight to neighbours of the same colour (out-arcs, plus
// in-arcs for a directed graph), FP64.
__global__ void k_class_weight(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                               const float *__restrict__ w, const int64_t *__restrict__ tp,
                               const int32_t *__restrict__ tc, const float *__restrict__ tw,
                               const int32_t *__restrict__ colour, double *__restrict__ din)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp0; v < n; v += nwarps) {
        const int cv = colour[v];
        double acc = 0.0;
        for (int64_t k = rp[v] + lane; k < rp[v + 1]; k += 32)
            if (colour[col[k]] == cv) acc += w ? (double)w[k] : 1.0;
        if (tp)
            for (int64_t k = tp[v] + lane; k < tp[v + 1]; k += 32)
                if (colour[tc[k]] == cv) acc += tw ? (double)tw[k] : 1.0;
        acc = warp_sum(acc);
        if (lane == 0) din[v] = acc;
    }
}

__global__ void k_gather_f64(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                             double *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

__global__ void k_fill_i32(int64_t n, int32_t *p, int32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_inverse_perm(int64_t n, const uint32_t *__restrict__ perm, int32_t *__restrict__ perm_out,
                               int32_t *__restrict__ iperm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t old = perm[i];
        perm_out[i] = (int32_t)old;
        iperm[old] = (int32_t)i;
    }
}

__global__ void k_perm_rowlen(int64_t n, const int32_t *__restrict__ perm, const int64_t *__restrict__ rp,
                              int32_t *__restrict__ len)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = perm[i];
        len[i] = (int32_t)(rp[o + 1] - rp[o]);
    }
}

// Warp per new row: copy the old row with its columns renamed by iperm.
__global__ void k_perm_rows(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ iperm,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ w,
                            const int64_t *__restrict__ prp, int32_t *__restrict__ pcol, float *__restrict__ pw)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nwarps) {
        int32_t o = perm[i];
        int64_t a = rp[o], len = rp[o + 1] - a, pa = prp[i];
        for (int64_t k = lane; k < len; k += 32) {
            pcol[pa + k] = iperm[col[a + k]];
            if (w) pw[pa + k] = w[a + k];
        }
    }
}

__global__ void k_perm_node_arrays(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ deg,
                                   const double *__restrict__ inv64, const float *__restrict__ inv32,
                                   const int32_t *__restrict__ indeg, const int32_t *__restrict__ graph_of,
                                   double *__restrict__ pdeg, double *__restrict__ pinv64, float *__restrict__ pinv32,
                                   int32_t *__restrict__ pindeg, int32_t *__restrict__ pgraph)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = perm[i];
        pdeg[i] = deg[o];
        pinv64[i] = inv64[o];
        pinv32[i] = inv32[o];
        pindeg[i] = indeg[o];
        if (graph_of) pgraph[i] = graph_of[o];
    }
}

// A forced block start wherever the range key (sorted key >> shift: the hub
// flag and the colour) or, in a ragged batch, the graph changes.
struct SegStartPred {
    const uint32_t *key_sorted;
    const int32_t *graph;
    int shift;
    __device__ bool operator()(int64_t i) const
    {
        return i == 0 || (key_sorted[i] >> shift) != (key_sorted[i - 1] >> shift) ||
               (graph && graph[i] != graph[i - 1]);
    }
};

// Sort key of the colour permutation: the colour, and when indeg is given,
// above it a flag that is 0 for hubs (in-degree >= hub_min) and below it the
// in-degree descending (22 bits, clamped).  So the hubs come first, ordered
// by class, then every class's other nodes; inside each range the nodes most
// rows gather from sit together (their increments share cache sectors, and
// the hubs' fit the sweep's shared-memory table).  Ties keep id order (the
// sort is stable).
constexpr int kDegKeyBits = 22;

__global__ void k_colour_keys(int64_t n, const int32_t *__restrict__ colour, const int32_t *__restrict__ indeg,
                              int32_t hub_min, uint32_t *__restrict__ key)
{
    constexpr uint32_t dmax = (1u << kDegKeyBits) - 1u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!indeg) {
            key[i] = (uint32_t)colour[i];
        } else {
            const uint32_t d = (uint32_t)min(max(indeg[i], 0), (int32_t)dmax);
            const uint32_t cold = indeg[i] >= hub_min ? 0u : 1u;
            key[i] = (cold << 31) | ((uint32_t)colour[i] << kDegKeyBits) | (dmax - d);
        }
    }
}

// Smallest in-degree threshold whose hub set {v : indeg_v >= t} holds at most
// kHubMax nodes (every node when n <= kHubMax).
static int32_t hub_threshold(const int32_t *indeg_host, int64_t n)
{
    if (n <= kHubMax) return INT32_MIN;
    std::vector<int32_t> d(indeg_host, indeg_host + n);
    std::nth_element(d.begin(), d.begin() + (kHubMax - 1), d.end(), std::greater<int32_t>());
    const int32_t v = d[(size_t)kHubMax - 1];
    int64_t ge = 0;
    for (int64_t i = 0; i < n; ++i) ge += indeg_host[i] >= v;
    return ge <= kHubMax ? v : v + 1;
}

// Data-driven greedy colouring (the same colours as the sequential greedy in
// priority order): dep[v] counts v's neighbours of higher priority that are
// not yet coloured; a node is ready when it reaches zero, takes its colour from
// its neighbours coloured so far (exactly its higher-priority ones: a
// lower-priority neighbour waits for it), then releases its lower-priority
// neighbours.  Each arc is visited a bounded number of times in total.
__device__ __forceinline__ void append_warp(bool keep, int32_t v, int32_t *out, long long *cnt)
{
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    long long at = 0;
    if ((threadIdx.x & 31) == 0 && m)
        at = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(cnt), (unsigned long long)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (keep) out[at + __popc(m & lanemask_lt())] = v;
}

__global__ void k_dep_count(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int64_t *__restrict__ tp, const int32_t *__restrict__ tc,
                            const unsigned long long *__restrict__ key, int32_t *__restrict__ dep,
                            int32_t *__restrict__ ready, long long *ready_cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // warps walk nodes in groups of 32 so that the ready append is warp-uniform
    for (int64_t g0 = warp0 * 32; g0 < n; g0 += nwarps * 32) {
        int my = 0;
        for (int q = 0; q < 32 && g0 + q < n; ++q) {
            const int64_t v = g0 + q;
            const unsigned long long kv = key[v];
            int c = 0;
            for (int64_t k = rp[v] + lane; k < rp[v + 1]; k += 32) c += higher(key[col[k]], col[k], kv, v);
            if (tp)
                for (int64_t k = tp[v] + lane; k < tp[v + 1]; k += 32) c += higher(key[tc[k]], tc[k], kv, v);
            c = (int)warp_sum((unsigned long long)c);
            if (lane == q) my = c;
        }
        const int64_t v = g0 + lane;
        if (v < n) dep[v] = my;
        append_warp(v < n && my == 0, (int32_t)v, ready, ready_cnt);
    }
}

template <bool PAL>
__global__ void __launch_bounds__(256)
k_jp_ready(const long long *__restrict__ cntp, const int32_t *__restrict__ list, const int64_t *__restrict__ rp,
           const int32_t *__restrict__ col, const float *__restrict__ w, const int64_t *__restrict__ tp,
           const int32_t *__restrict__ tc, const float *__restrict__ tw, const unsigned long long *__restrict__ key,
           int K, int32_t *colour, int32_t *dep, int32_t *__restrict__ next, long long *next_cnt)
{
    __shared__ unsigned long long conf[8][32];
    __shared__ unsigned bits[8][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    volatile int32_t *vc = colour;
    const int64_t cnt = *cntp;
    for (int64_t i = warp0; i < cnt; i += nwarps) {
        const int32_t v = list[i];
        const unsigned long long kv = key[v];
        const int64_t a = rp[v], b = rp[v + 1];
        const int64_t ta = tp ? tp[v] : 0, tb = tp ? tp[v + 1] : 0;
        int best = 0;
        if (PAL) {
            conf[wl][lane] = 0ULL;
            __syncwarp();
            for (int64_t k = a + lane; k < b; k += 32) {
                const int c = vc[col[k]];
                if (c >= 0 && c < 32) atomicAdd(&conf[wl][c], fixed_q(w, k));
            }
            for (int64_t k = ta + lane; k < tb; k += 32) {
                const int c = vc[tc[k]];
                if (c >= 0 && c < 32) atomicAdd(&conf[wl][c], fixed_q(tw, k));
            }
            __syncwarp();
            const unsigned long long mine = lane < K ? conf[wl][lane] : ~0ULL;
            const unsigned zero = __ballot_sync(0xffffffffu, lane < K && mine == 0ULL);
            if (zero) {
                best = __ffs(zero) - 1;
            } else {
                unsigned long long m = mine;
                int bl = lane;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, m, o);
                    const int b2 = __shfl_xor_sync(0xffffffffu, bl, o);
                    if (m2 < m || (m2 == m && b2 < bl)) {
                        m = m2;
                        bl = b2;
                    }
                }
                best = bl;
            }
        } else {
            int found = -1;
            for (int base = 0; found < 0; base += 1024) {
                bits[wl][lane] = 0u;
                __syncwarp();
                for (int64_t k = a + lane; k < b; k += 32) {
                    const int c = vc[col[k]] - base;
                    if (c >= 0 && c < 1024) atomicOr(&bits[wl][c >> 5], 1u << (c & 31));
                }
                for (int64_t k = ta + lane; k < tb; k += 32) {
                    const int c = vc[tc[k]] - base;
                    if (c >= 0 && c < 1024) atomicOr(&bits[wl][c >> 5], 1u << (c & 31));
                }
                __syncwarp();
                const unsigned freebits = ~bits[wl][lane];
                const unsigned has = __ballot_sync(0xffffffffu, freebits != 0u);
                if (has) {
                    const int l = __ffs(has) - 1;
                    const unsigned fb = __shfl_sync(0xffffffffu, freebits, l);
                    found = base + 32 * l + (__ffs(fb) - 1);
                }
                __syncwarp();
            }
            best = found;
        }
        if (lane == 0) colour[v] = best;
        __threadfence();
        __syncwarp();
        // release the lower-priority neighbours
        for (int64_t k0 = a; k0 < b; k0 += 32) {
            const int64_t k = k0 + lane;
            bool go = false;
            int32_t u = 0;
            if (k < b) {
                u = col[k];
                go = higher(kv, v, key[u], u) && atomicSub(&dep[u], 1) == 1;
            }
            append_warp(go, u, next, next_cnt);
        }
        for (int64_t k0 = ta; k0 < tb; k0 += 32) {
            const int64_t k = k0 + lane;
            bool go = false;
            int32_t u = 0;
            if (k < tb) {
                u = tc[k];
                go = higher(kv, v, key[u], u) && atomicSub(&dep[u], 1) == 1;
            }
            append_warp(go, u, next, next_cnt);
        }
    }
}

static fj_status colour_graph(fj_graph *g, int palette, cudaStream_t st)
{
    DevCSR &c = g->csr;
    const int64_t n = c.n;
    Colouring &cl = g->colr;
    unsigned long long *key = nullptr;
    int32_t *list = nullptr;
    FJ_CUDA(dalloc(&key, n));
    FJ_CUDA(dalloc(&list, n));
    if (!cl.colour) FJ_CUDA(dalloc(&cl.colour, n));
    const int64_t *tp = g->directed ? g->tptr : nullptr;
    const int32_t *tc = g->directed ? g->tcol : nullptr;
    k_sym_degree<<<grid_for(n * 32, 256), 256, 0, st>>>(n, c.row_ptr, c.col, tp, tc, key);
    k_fill_i32<<<grid_for(n, 256), 256, 0, st>>>(n, cl.colour, -1);
    FJ_CUDA(cudaGetLastError());
    // data-driven rounds over the ready nodes (ping-pong lists, count on the
    // device); the host reads the count every kBatch rounds
    constexpr int kBatch = 16;
    int32_t *lists[2] = {list, nullptr};
    long long *cnts = nullptr;
    int32_t *dep = nullptr;
    FJ_CUDA(dalloc(&lists[1], n));
    FJ_CUDA(dalloc(&cnts, 2));
    FJ_CUDA(dalloc(&dep, n));
    FJ_CUDA(cudaMemsetAsync(cnts, 0, 2 * sizeof(long long), st));
    k_dep_count<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(n, c.row_ptr, c.col, tp, tc, key, dep, lists[0], cnts);
    FJ_CUDA(cudaGetLastError());
    long long left = 1;
    int64_t rounds = 0;
    int cur = 0;
    fj_status result = FJ_OK;
    const unsigned grid = 152 * 8;
    while (left > 0) {
        for (int bt = 0; bt < kBatch; ++bt) {
            const long long *cin = cnts + cur;
            FJ_CUDA(cudaMemsetAsync(cnts + (cur ^ 1), 0, sizeof(long long), st));
            if (palette > 0)
                k_jp_ready<true><<<grid, 256, 0, st>>>(cin, lists[cur], c.row_ptr, c.col, c.w, tp, tc,
                                                       g->directed ? g->tw : nullptr, key, palette, cl.colour, dep,
                                                       lists[cur ^ 1], cnts + (cur ^ 1));
            else
                k_jp_ready<false><<<grid, 256, 0, st>>>(cin, lists[cur], c.row_ptr, c.col, c.w, tp, tc,
                                                        g->directed ? g->tw : nullptr, key, 0, cl.colour, dep,
                                                        lists[cur ^ 1], cnts + (cur ^ 1));
            FJ_CUDA(cudaGetLastError());
            cur ^= 1;
        }
        rounds += kBatch;
        FJ_CUDA(cudaMemcpyAsync(&left, cnts + cur, sizeof(long long), cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
        if (left > 0 && rounds > 4000000) {
            set_error("colouring did not finish");
            result = FJ_ERR_TIMEOUT;
            break;
        }
    }
    dev_free(dep);
    dev_free(lists[1]);
    dev_free(cnts);
    if (result != FJ_OK) {
        dev_free(key);
        dev_free(list);
        return result;
    }
    dev_free(key);
    dev_free(list);
    return read_dev_error(g, st);
}

static void item_plan_free(ItemPlan &ip)
{
    dev_free(ip.items);
    dev_free(ip.slot_first);
    dev_free(ip.slot_nchunk);
    dev_free(ip.part);
    dev_free(ip.cnt);
    ip = ItemPlan();
}

void chunk_plan_free(ChunkPlan &cp)
{
    dev_free(cp.starts);
    dev_free(cp.endbase);
    dev_free(cp.rank);
    dev_free(cp.long_rows);
    cp = ChunkPlan();
}

static void colouring_free(fj_graph *g)
{
    Colouring &cl = g->colr;
    dev_free(cl.colour);
    dev_free(cl.perm);
    dev_free(cl.iperm);
    dev_free(cl.din_p);
    dev_free(cl.tptr);
    dev_free(cl.tcol);
    dev_free(cl.tw);
    csr_free(cl.pcsr);
    cl = Colouring();
    item_plan_free(g->wplan_pcsr);
    chunk_plan_free(g->cplan_pcsr);
    g->ws.gen++;
}

// In-neighbour list lengths in the permuted order: row i of the permuted
// transpose is row perm[i] of the transpose.
struct PermRowLen {
    const int64_t *tptr;
    const int32_t *perm;
    __device__ long long operator()(int64_t i) const
    {
        const int64_t v = perm[i];
        return (long long)(tptr[v + 1] - tptr[v]);
    }
};

// One warp per new row i: copy transposed row perm[i] with its columns
// renumbered into the permuted order.
__global__ void k_permute_transpose(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ iperm,
                                    const int64_t *__restrict__ tptr, const int32_t *__restrict__ tcol,
                                    const float *__restrict__ tw, const int64_t *__restrict__ pptr,
                                    int32_t *__restrict__ pcol, float *__restrict__ pw)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int64_t v = perm[i];
        const int64_t a = tptr[v], len = tptr[v + 1] - a, d = pptr[i];
        for (int64_t t = lane; t < len; t += 32) {
            pcol[d + t] = iperm[tcol[a + t]];
            if (tw) pw[d + t] = tw[a + t];
        }
    }
}

fj_status ensure_ptranspose(fj_graph *g, cudaStream_t st)
{
    Colouring &cl = g->colr;
    if (cl.tptr) return FJ_OK;
    if (!cl.built || !g->directed || !g->tptr) {
        set_error("internal: permuted transpose needs a colouring of a directed graph");
        return FJ_ERR_INVALID_ARG;
    }
    const int64_t n = g->csr.n, nnz = g->csr.nnz;
    long long *excl = nullptr;
    FJ_CUDA(dalloc(&cl.tptr, n + 1));
    FJ_CUDA(dalloc(&cl.tcol, std::max<int64_t>(nnz, 1)));
    if (g->tw) FJ_CUDA(dalloc(&cl.tw, std::max<int64_t>(nnz, 1)));
    FJ_CUDA(dalloc(&excl, n + 1));
    FJ_CHECK(ws_status(g->ws, scan_tiles(n, 256 * 8)));
    FJ_CUDA(scan<256, 8>(n, PermRowLen{g->tptr, cl.perm}, excl, g->ws.count, g->ws.status, g->ws.tile_ctr, g->err,
                         st));
    k_finish_ptr_dev<<<grid_for(n + 1, 256), 256, 0, st>>>(n, excl, g->ws.count, cl.tptr);
    FJ_CUDA(cudaGetLastError());
    k_permute_transpose<<<grid_for(n * 32, 256), 256, 0, st>>>(n, cl.perm, cl.iperm, g->tptr, g->tcol, g->tw,
                                                               cl.tptr, cl.tcol, cl.tw);
    FJ_CUDA(cudaGetLastError());
    FJ_CUDA(cudaStreamSynchronize(st));
    dev_free(excl);
    return read_dev_error(g, st);
}

fj_status ensure_colouring(fj_graph *g, int palette, cudaStream_t st)
{
    if (palette < 0 || palette > 32) {
        set_error("invalid argument: palette must be 0 (unbounded) or 1..32");
        return FJ_ERR_INVALID_ARG;
    }
    Colouring &cl = g->colr;
    if (cl.built && cl.palette == palette) return FJ_OK;
    if (cl.built) colouring_free(g);
    cl.palette = palette;
    DevCSR &c = g->csr;
    const int64_t n = c.n, nnz = c.nnz;
    FJ_CHECK(colour_graph(g, palette, st));
    // permutation: stable sort of node ids by colour
    uint32_t *k0, *v0, *k1, *v1;
    FJ_CUDA(dalloc(&k0, n));
    FJ_CUDA(dalloc(&v0, n));
    FJ_CUDA(dalloc(&k1, n));
    FJ_CUDA(dalloc(&v1, n));
    // in-degree order inside classes: one graph and a bounded palette (colours
    // then fit the key's top 10 bits)
    const bool deg_key = g->ngraphs == 1 && palette > 0 && palette <= 32;
    int32_t hub_min = INT32_MAX;
    if (deg_key) {
        std::vector<int32_t> hd((size_t)n);
        FJ_CUDA(cudaMemcpyAsync(hd.data(), c.indeg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        FJ_CUDA(cudaStreamSynchronize(st));
        hub_min = hub_threshold(hd.data(), n);
    }
    k_colour_keys<<<grid_for(n, 256), 256, 0, st>>>(n, cl.colour, deg_key ? c.indeg : nullptr, hub_min, k0);
    k_iota<<<grid_for(n, 256), 256, 0, st>>>(n, v0);
    FJ_CUDA(cudaGetLastError());
    bool in1 = false;
    FJ_CUDA(sort_pairs(n, 32, k0, v0, k1, v1, g->sort, g->err, st, &in1));
    uint32_t *sk = in1 ? k1 : k0, *sv = in1 ? v1 : v0;
    // range boundaries from the sorted keys: hubs by colour, then the rest by colour
    const int kshift = deg_key ? kDegKeyBits : 0;
    std::vector<uint32_t> hk((size_t)n);
    FJ_CUDA(cudaMemcpyAsync(hk.data(), sk, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    for (auto &x : hk) x >>= kshift;
    constexpr uint32_t kColdBit = 1u << (31 - kDegKeyBits);
    auto colour_at = [&](int64_t i) -> uint32_t {
        return deg_key ? (hk[(size_t)i] & (kColdBit - 1u)) : hk[(size_t)i];
    };
    uint32_t maxc = 0;
    int64_t nhub = 0;
    for (int64_t i = 0; i < n; ++i) {
        maxc = std::max(maxc, colour_at(i));
        if (deg_key && !(hk[(size_t)i] & kColdBit)) ++nhub;
    }
    cl.ncolours = (int)maxc + 1;
    cl.nhub = nhub;
    // class c's hub rows start at the first hub of colour >= c, its other rows at
    // the first non-hub of colour >= c (the ranges of an absent colour are empty)
    cl.hub_row.assign((size_t)cl.ncolours + 1, nhub);
    cl.class_row.assign((size_t)cl.ncolours + 1, n);
    for (int64_t i = 0, cc = 0; cc < cl.ncolours; ++cc) {
        while (i < nhub && colour_at(i) < (uint32_t)cc) ++i;
        cl.hub_row[(size_t)cc] = i;
    }
    for (int64_t i = nhub, cc = 0; cc < cl.ncolours; ++cc) {
        while (i < n && colour_at(i) < (uint32_t)cc) ++i;
        cl.class_row[(size_t)cc] = i;
    }
    if (!cl.perm) FJ_CUDA(dalloc(&cl.perm, n));
    if (!cl.iperm) FJ_CUDA(dalloc(&cl.iperm, n));
    k_inverse_perm<<<grid_for(n, 256), 256, 0, st>>>(n, sv, cl.perm, cl.iperm);
    FJ_CUDA(cudaGetLastError());
    // permuted CSR
    DevCSR &p = cl.pcsr;
    p.n = n;
    p.nnz = nnz;
    int32_t *len = reinterpret_cast<int32_t *>(in1 ? k0 : k1);  // the free key buffer
    long long *excl = nullptr;
    FJ_CUDA(dalloc(&excl, n + 1));
    k_perm_rowlen<<<grid_for(n, 256), 256, 0, st>>>(n, cl.perm, c.row_ptr, len);
    FJ_CHECK(ws_status(g->ws, scan_tiles(n, 256 * 8)));
    FJ_CUDA(scan<256, 8>(n, I32Load{len}, excl, g->ws.count, g->ws.status, g->ws.tile_ctr, g->err, st));
    FJ_CUDA(dalloc(&p.row_ptr, n + 1));
    k_finish_ptr<<<grid_for(n + 1, 256), 256, 0, st>>>(n, excl, nnz, p.row_ptr);
    FJ_CUDA(dalloc(&p.col, nnz + kNnzPad));
    if (c.w) FJ_CUDA(dalloc(&p.w, nnz + kNnzPad));
    k_perm_rows<<<grid_for(n * 32, 256), 256, 0, st>>>(n, cl.perm, cl.iperm, c.row_ptr, c.col, c.w, p.row_ptr, p.col,
                                                       p.w);
    FJ_CUDA(dalloc(&p.deg64, n));
    FJ_CUDA(dalloc(&p.inv64, n));
    FJ_CUDA(dalloc(&p.inv32, n));
    FJ_CUDA(dalloc(&p.indeg, n));
    if (c.graph_of) FJ_CUDA(dalloc(&p.graph_of, n));
    k_perm_node_arrays<<<grid_for(n, 256), 256, 0, st>>>(n, cl.perm, c.deg64, c.inv64, c.inv32, c.indeg, c.graph_of,
                                                         p.deg64, p.inv64, p.inv32, p.indeg, p.graph_of);
    FJ_CUDA(cudaGetLastError());
    {
        // weight of each node to neighbours of its own colour (0 for a proper colouring)
        double *din = nullptr;
        FJ_CUDA(dalloc(&din, n));
        FJ_CUDA(dalloc(&cl.din_p, n));
        k_class_weight<<<grid_for(n * 32, 256), 256, 0, st>>>(n, c.row_ptr, c.col, c.w, g->directed ? g->tptr : nullptr,
                                                              g->directed ? g->tcol : nullptr,
                                                              g->directed ? g->tw : nullptr, cl.colour, din);
        k_gather_f64<<<grid_for(n, 256), 256, 0, st>>>(n, cl.perm, din, cl.din_p);
        FJ_CUDA(cudaGetLastError());
        FJ_CUDA(cudaStreamSynchronize(st));
        dev_free(din);
    }
    // forced block starts: every class start and, in a ragged batch, every
    // change of graph inside a class, so that each row block lies in one
    // class of one graph
    int32_t *starts = reinterpret_cast<int32_t *>(in1 ? v0 : v1);  // free value buffer
    FJ_CUDA(compact<256, 8>(n, SegStartPred{sk, p.graph_of, kshift}, starts, g->ws.count, g->ws.status, g->ws.tile_ctr,
                            g->err, st));
    long long nseg = 0;
    FJ_CUDA(cudaMemcpyAsync(&nseg, g->ws.count, sizeof(long long), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> hs((size_t)nseg);
    FJ_CUDA(cudaMemcpy(hs.data(), starts, sizeof(int32_t) * nseg, cudaMemcpyDeviceToHost));
    std::vector<int64_t> segs(hs.begin(), hs.end());
    dev_free(excl);
    dev_free(k0); dev_free(v0); dev_free(k1); dev_free(v1);
    FJ_CHECK(build_blocks(p, segs, g->ws, g->err, st, kTileBlock));
    FJ_CHECK(build_blocks(p, segs, g->ws, g->err, st, kTileWarp));
    cl.built = true;
    return read_dev_error(g, st);
}

}  // namespace fj

extern "C" fj_status fj_graph_colour(fj_graph *g, int palette, int32_t *colour, int *ncolours, int mem,
                                     void *stream)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_ARG(palette >= 0 && palette <= 32, "palette must be 0 (unbounded) or 1..32");
    cudaStream_t st = (cudaStream_t)stream;
    FJ_CHECK(fj::ensure_colouring(g, palette, st));
    if (colour)
        FJ_CUDA(cudaMemcpyAsync(colour, g->colr.colour, sizeof(int32_t) * g->csr.n,
                                mem == FJ_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    if (ncolours) *ncolours = g->colr.ncolours;
    return FJ_OK;
}

extern "C" fj_status fj_graph_order(fj_graph *g, int palette, int32_t *perm, int64_t *nhub, int64_t *hub_row,
                                    int64_t *class_row, int mem, void *stream)
{
    FJ_ARG(g != nullptr, "graph is NULL");
    FJ_ARG(mem == FJ_MEM_HOST || mem == FJ_MEM_DEVICE, "mem must be FJ_MEM_HOST or FJ_MEM_DEVICE");
    FJ_ARG(palette >= 0 && palette <= 32, "palette must be 0 (unbounded) or 1..32");
    cudaStream_t st = (cudaStream_t)stream;
    FJ_CHECK(fj::ensure_colouring(g, palette, st));
    const fj::Colouring &cl = g->colr;
    if (perm)
        FJ_CUDA(cudaMemcpyAsync(perm, cl.perm, sizeof(int32_t) * g->csr.n,
                                mem == FJ_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    if (nhub) *nhub = cl.nhub;
    for (int c = 0; c <= cl.ncolours; ++c) {
        if (hub_row) hub_row[c] = cl.hub_row[(size_t)c];
        if (class_row) class_row[c] = cl.class_row[(size_t)c];
    }
    return FJ_OK;
}

extern "C" void fj_debug_fail_allocation(int64_t after)
{
    fj::g_fail_alloc_after.store(after < 0 ? -1 : (long long)after);
}
