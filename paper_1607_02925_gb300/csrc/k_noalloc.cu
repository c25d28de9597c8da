// lra_sampling_table_noalloc: the sampling-distribution builder of
// lra_sampling_table with its scratch memory in a fixed device array of this
// library instead of memory allocated per call.
//
// Who needs it: a caller that cannot call cudaMalloc/cudaFree at the point it
// builds the table, e.g. an application whose framework has reserved the GPU's
// memory for its own pool allocator, or one that must not take the device-wide
// synchronisation that cudaFree implies in the middle of its own stream work.
// The caller still provides the inputs and outputs.
//
// The scratch array lives for as long as the library is loaded, on every GPU
// that loads it.  All calls share it: two calls whose work overlaps on the GPU
// (different streams or threads) race on it and must be serialised by the
// caller.  The first call on a device (and the first after a device reset,
// which gives the device a new context) looks up the array's device address
// with that device current; make that first call before any stream capture.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>

#include "engine.h"

namespace lra {
namespace {

// Tile sums of the scan (ceil(n/1024) uint64) and per-block maxima of the
// c-vector kernel (ceil(n/256) doubles, reusing the same words), plus 4
// doubles for sum, max and kappa.
constexpr int64_t kScratchWords = LRA_NOALLOC_MAX_N / 256 + 64;
__device__ __align__(256) uint64_t g_table_scratch[kScratchWords];

std::mutex g_addr_mu;

// The address is cached per device together with the CUDA context it was
// looked up in: after a device reset the primary context, and with it the
// array's address, is new, so a changed context triggers a fresh lookup.
struct CachedAddr {
    CUcontext ctx = nullptr;
    void *ptr = nullptr;
};
CachedAddr g_addr[64];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

CUcontext current_context() {
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            cudaGetLastError();
            set_error("cuCtxGetCurrent not available");
            throw Error{LRA_ECUDA};
        }
        fn = reinterpret_cast<CtxGetCurrentFn>(f);
    }
    CUcontext c = nullptr;
    if (fn(&c) != CUDA_SUCCESS) {
        set_error("cuCtxGetCurrent failed");
        throw Error{LRA_ECUDA};
    }
    return c;
}

// Device address of g_table_scratch on the current device, looked up with
// cudaGetSymbolAddress on the first call in each CUDA context.
uint64_t *scratch_address(int device) {
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (device < 0 || device >= 64) {
        set_error("device index out of range for the fixed scratch table");
        throw Error{LRA_EUNSUPPORTED};
    }
    const CUcontext cur = current_context();
    CachedAddr &e = g_addr[device];
    if (!e.ptr || e.ctx != cur) {
        void *ptr = nullptr;
        const cudaError_t st = cudaGetSymbolAddress(&ptr, g_table_scratch);
        if (st != cudaSuccess || !ptr) {
            cudaGetLastError();
            set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(st));
            throw Error{LRA_ECUDA};
        }
        e.ptr = ptr;
        e.ctx = current_context();
    }
    return static_cast<uint64_t *>(e.ptr);
}

}  // namespace
}  // namespace lra

extern "C" lra_status lra_sampling_table_noalloc(lra_ctx *ctx, int64_t n, const double *norm2, int mode,
                                                 uint64_t *cum, float *c, uint64_t *total,
                                                 double *kappa) {
    using namespace lra;
    if (!ctx || !norm2 || !cum || !c || n < 1) {
        set_error("null argument or n < 1");
        return LRA_EINVAL;
    }
    if (n > LRA_NOALLOC_MAX_N) {
        set_error("n exceeds LRA_NOALLOC_MAX_N, the size of the fixed scratch array");
        return LRA_EINVAL;
    }
    if (mode != LRA_SAMPLE_IMPORTANCE && mode != LRA_SAMPLE_UNIFORM) {
        set_error("bad mode");
        return LRA_EINVAL;
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    try {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != ctx->device) LRA_CUDA(cudaSetDevice(ctx->device));
        struct Restore {
            int d;
            ~Restore() {
                if (d >= 0) cudaSetDevice(d);
            }
        } restore{prev != ctx->device ? prev : -1};
        uint64_t *scr = scratch_address(ctx->device);
        const cudaStream_t s = ctx->stream;
        const int64_t words = ceil_div(n, 256) + 16;
        double *sm = reinterpret_cast<double *>(scr + kScratchWords - 8);  // sum, max, kappa
        // The array keeps the previous call's contents.  Every word this call
        // reads is written first by this call (tile sums, block maxima, and the
        // sum, max and kappa slots), so nothing needs clearing.
        (void)words;
        sum_max(s, norm2, n, sm, nullptr);
        sampling_table(s, norm2, n, mode, sm + 1, cum, c, sm + 2, scr);
        uint64_t tot = 0;
        double kp = 0.0, sum = 0.0;
        LRA_CUDA(cudaMemcpyAsync(&tot, cum + n - 1, sizeof(tot), cudaMemcpyDeviceToHost, s));
        LRA_CUDA(cudaMemcpyAsync(&kp, sm + 2, sizeof(kp), cudaMemcpyDeviceToHost, s));
        LRA_CUDA(cudaMemcpyAsync(&sum, sm, sizeof(sum), cudaMemcpyDeviceToHost, s));
        LRA_CUDA(cudaStreamSynchronize(s));
        if (!std::isfinite(sum)) {
            set_error("a column norm is not finite");
            return LRA_EINVAL;
        }
        if (total) *total = tot;
        if (kappa) *kappa = kp;
        return LRA_OK;
    } catch (const Error &e) {
        return e.st;
    } catch (...) {
        set_error("unexpected exception");
        return LRA_ECUDA;
    }
}
