// Frontier compaction that allocates nothing: the look-back scratch lives in
// a file-scope device array sized for at most kStaticMaxNodes nodes.
#include <mutex>

#include "fj_internal.cuh"

namespace fj {

constexpr int64_t kStaticMaxNodes = int64_t(1) << 26;
constexpr int64_t kStaticTiles = kStaticMaxNodes / (256 * 8);

// tile status words, then the tile counter and the device error word
struct StaticScratch {
    unsigned long long status[kStaticTiles];
    unsigned int tile_ctr;
    int err;
};

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) StaticScratch g_static_scratch;

template <typename T>
struct StaticFrontierPred {
    const T *r, *h;
    __device__ bool operator()(int64_t v) const { return abs_t(r[v]) > h[v]; }
};

// Device address of the array, looked up once per device (host code cannot
// use the symbol itself: in host code it names a host-side stand-in).
static StaticScratch *static_scratch_ptr(fj_status *st)
{
    static std::mutex mu;
    static StaticScratch *ptrs[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
        return nullptr;
    }
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range for the static scratch table", dev);
        *st = FJ_ERR_UNSUPPORTED;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
            return nullptr;
        }
        ptrs[dev] = static_cast<StaticScratch *>(p);
    }
    *st = FJ_OK;
    return ptrs[dev];
}

}  // namespace fj

using namespace fj;

extern "C" fj_status fj_frontier_static(int64_t n, const void *r, const void *h, int precision, int32_t *list,
                                        int64_t *count, void *stream)
{
    FJ_ARG(n >= 0, "n must be >= 0");
    if (n > kStaticMaxNodes) {
        set_error("invalid argument: n = %lld exceeds the static scratch limit of %lld nodes", (long long)n,
                  (long long)kStaticMaxNodes);
        return FJ_ERR_INVALID_ARG;
    }
    FJ_ARG(r && h && list && count, "NULL pointer");
    FJ_ARG(precision == FJ_PREC_FP64 || precision == FJ_PREC_FP32, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    fj_status s = FJ_OK;
    StaticScratch *sc = static_scratch_ptr(&s);
    if (!sc) return s;
    FJ_CUDA(cudaMemsetAsync(&sc->err, 0, sizeof(int), st));
    cudaError_t e;
    if (n == 0) {
        e = cudaMemsetAsync(count, 0, sizeof(int64_t), st);
    } else if (precision == FJ_PREC_FP32) {
        e = compact<256, 8>(n, StaticFrontierPred<float>{(const float *)r, (const float *)h}, list,
                            (long long *)count, sc->status, &sc->tile_ctr, &sc->err, st);
    } else {
        e = compact<256, 8>(n, StaticFrontierPred<double>{(const double *)r, (const double *)h}, list,
                            (long long *)count, sc->status, &sc->tile_ctr, &sc->err, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "frontier (static scratch)", __FILE__, __LINE__);
    int herr = 0;
    FJ_CUDA(cudaMemcpyAsync(&herr, &sc->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FJ_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        set_error("frontier look-back timed out");
        return FJ_ERR_TIMEOUT;
    }
    return FJ_OK;
}
