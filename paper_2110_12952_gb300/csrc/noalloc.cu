// noalloc.cu -- fractal_step_noalloc: the multi-generation compact step
// without any device allocation, for callers that cannot allocate device
// memory while they run: applications whose device memory is handed out up
// front by their own pool or by another framework that reserves it, and
// real-time loops in which cudaMalloc/cudaFree are not acceptable because
// they may synchronise the whole device.
//
// fractal_step needs a k^r-byte ping-pong buffer when steps > 1 and
// allocates it on first need.  Here that buffer is the file-scope device
// array below instead.  Its size is fixed (kNoAllocScratchBytes); every GPU
// that loads this library holds it until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "handle.h"

namespace fr {

// 32 MiB: a state of up to 33,554,432 cells (e.g. the triangle up to r = 15,
// the carpet up to r = 8).
constexpr int64_t kNoAllocScratchBytes = (int64_t)32 << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// The host-side name g_noalloc_scratch is only a stand-in and must never be
// passed to a kernel.  Its device address belongs to the CUDA context that
// loaded the module: it is looked up (with the device current) the first
// time a device is used and again whenever that device's current context is
// a different one (after cudaDeviceReset, for example, the runtime creates a
// new primary context and reloads the module, so an older address would
// dangle).
struct ScratchAddr {
    void *ctx = nullptr;
    uint8_t *ptr = nullptr;
};
static std::mutex g_noalloc_mu;
static ScratchAddr g_noalloc_addr[kMaxDevices];

// cuCtxGetCurrent from the driver, through the runtime's entry-point query
// (no link-time dependency on libcuda); null if unavailable, in which case
// the address is looked up on every call.
using CtxGetCurrent = int (*)(void **);
static CtxGetCurrent ctx_get_current()
{
    static CtxGetCurrent fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrent>(p);
    }();
    return fn;
}

static void *current_ctx()
{
    CtxGetCurrent fn = ctx_get_current();
    void *ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of the array in the current context of device `dev`.
static int noalloc_scratch(int dev, uint8_t **out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        set_error(FR_EINVAL, "fractal_step_noalloc: device index out of range");
        return FR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    ScratchAddr &c = g_noalloc_addr[dev];
    void *ctx = current_ctx();
    if (ctx && c.ctx == ctx && c.ptr) {
        *out = c.ptr;
        return FR_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "fractal_step_noalloc: cudaGetSymbolAddress");
    c.ptr = static_cast<uint8_t *>(p);
    c.ctx = current_ctx();   // the lookup has made the context current if it was not
    *out = c.ptr;
    return FR_OK;
}

}  // namespace fr

using namespace fr;

extern "C" int fractal_step_noalloc(fractal_t *f, const uint8_t *in, uint8_t *out, int64_t steps,
                                    uint32_t birth, uint32_t survive, void *stream)
{
    clear_error();
    if (!f || !in || !out) {
        set_error(FR_EINVAL, "fractal_step_noalloc: NULL argument");
        return FR_EINVAL;
    }
    if (steps < 0) {
        set_error(FR_EINVAL, "fractal_step_noalloc: steps < 0");
        return FR_EINVAL;
    }
    if (f->cells > kNoAllocScratchBytes) {
        set_error(FR_EINVAL, "fractal_step_noalloc: k^r = " + std::to_string(f->cells) +
                                 " cells exceeds the fixed scratch of " +
                                 std::to_string(kNoAllocScratchBytes) + " bytes; use fractal_step");
        return FR_EINVAL;
    }
    const uint8_t *a = in, *b = out;
    if (a < b + f->cells && b < a + f->cells) {
        set_error(FR_EINVAL, "fractal_step_noalloc: in and out overlap");
        return FR_EINVAL;
    }
    if (!f->plan.pos) {
        set_error(FR_EINVAL,
                  "fractal_step_noalloc: the handle's tables are not built yet (they are built, "
                  "with allocations, by fractal_step, fractal_autotune or fractal_get_tile_levels)");
        return FR_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (steps == 0) return launch_copy_normalise(in, out, f->cells, f->num_sms, st);
    int dev = 0;
    FR_CUDA(cudaGetDevice(&dev));
    if (dev != f->device) {
        set_error(FR_EINVAL, "fractal_step_noalloc: the current device is not the handle's device");
        return FR_EINVAL;
    }
    uint8_t *scratch = nullptr;
    int rc = noalloc_scratch(dev, &scratch);
    if (rc) return rc;
    // generation i (1-based) writes `out` when steps - i is even, the
    // scratch array otherwise, so the last one lands in `out`
    const uint8_t *src = in;
    for (int64_t i = 1; i <= steps; ++i) {
        uint8_t *dst = ((steps - i) % 2 == 0) ? out : scratch;
        rc = launch_step_once(f, src, dst, birth, survive, st);
        if (rc) return rc;
        src = dst;
    }
    return FR_OK;
}
