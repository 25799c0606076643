// gfe_mad_noalloc: the block multiply-add C := W + A B over GF(p) (the same
// computation as gfe_mad) for callers that cannot allocate device memory.
//
// Who needs it: code that runs where a device allocation is not allowed or
// not wanted -- a caller that owns a fixed device-memory budget and forbids
// libraries to grow it, or a caller on a latency-critical path, where
// cudaMalloc / cudaFree may block or implicitly synchronise the device.
// gfe_mad needs a caller-provided workspace; this entry point needs none: it
// uses a scratch array that lives in the library's own device image.
//
// The scratch is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES
// (32 MiB).  The CUDA runtime loads a module's device code lazily, so the
// array is created on a device by the first call there (the one that looks
// up its address), not when the library is loaded: that first call reserves
// the 32 MiB and may fail if the device is full, which is why callers should
// make it once as a warm-up.  From then on the device holds the array until
// the process exits.  Host code may not use the array's name as a device
// address (it is a host-side stand-in), so the first call on each device,
// with that device current, looks the address up with cudaGetSymbolAddress
// and keeps it; make that first call on a device before any stream capture.
//
// All calls on a device share the one array and it keeps the last call's
// contents.  The only element that must start at zero is the call's status
// word (the last 256 bytes of its scratch), which gfe_mad zeroes on the
// stream before the product; every other scratch element the multiply-add
// reads is written earlier in the same call.  Calls whose work overlaps on
// the GPU (for example issued on two streams without ordering) race on the
// array and give wrong results; order them.
#include "gfe.h"
#include "gfe_internal.h"

#include <mutex>

namespace gfe {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEV = 64;
std::mutex g_na_mu;
void *g_na_ptr[NA_MAX_DEV] = {};

// once per device, with that device current: the array's device address
gfe_status scratch_for_current_device(void **out) {
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return GFE_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEV) return (set_error("device ordinal out of range"), GFE_EINVAL);
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress")) return GFE_ECUDA;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return GFE_OK;
}

}  // namespace
}  // namespace gfe

using namespace gfe;

extern "C" size_t gfe_mad_noalloc_max_bytes(void) { return NOALLOC_SCRATCH_BYTES; }

extern "C" gfe_status gfe_mad_noalloc(int32_t p, int64_t m, int64_t n, int64_t k, const uint8_t *W, int64_t ldw,
                                      const uint8_t *A, int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C,
                                      int64_t ldc, uint32_t flags, void *stream) {
    if (!field_ok(p)) return (set_error("p must be a prime <= 251"), GFE_EINVAL);
    if (m < 0 || n < 0 || k < 0) return (set_error("negative size"), GFE_EINVAL);
    if (m == 0 || n == 0) return GFE_OK;
    const size_t need = gfe_mad_workspace(p, m, n, k);
    if (need > NOALLOC_SCRATCH_BYTES) {
        set_error("gfe_mad_noalloc: this product needs " + std::to_string(need) +
                  " bytes of scratch, more than the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                  " bytes it holds; use gfe_mad with a workspace");
        return GFE_EINVAL;
    }
    void *scratch = nullptr;
    gfe_status st = scratch_for_current_device(&scratch);
    if (st) return st;
    return gfe_mad(p, m, n, k, W, ldw, A, lda, B, ldb, C, ldc, flags, scratch, NOALLOC_SCRATCH_BYTES, stream);
}
