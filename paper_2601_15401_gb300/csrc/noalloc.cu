// Allocation-free variant of the multi-level rescale (ckks_rescale_multi).
//
// Some callers cannot allocate device memory at the point where they need a
// rescale: code running inside a region that must not call cudaMalloc or a
// caching allocator (a stream being captured into a CUDA graph by someone
// else, a real-time loop that forbids allocator locks, or a host process that
// only received device pointers from another component and has no allocator
// of its own). For them ckks_rescale_multi_noalloc runs the same Algorithm 1
// kernels as ckks_rescale_multi, but its scratch lives in a fixed device array
// of this library (kNoAllocScratchBytes, 32 MiB) instead of a caller-supplied
// workspace. The array exists once per device that loads the library and is
// held until the process exits.
#include <mutex>

#include "../../include/ckks_mulk.h"
#include "engine.h"
#include "internal.h"

using namespace ckks;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

// The scratch itself. In host code `g_noalloc_scratch` names a host-side
// stand-in, not device memory: its device address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_addr[64] = {nullptr};

// Device address of the scratch on `device` (the caller's current device is
// set to it first). Returns nullptr if the symbol cannot be resolved.
void *scratch_address(int device) {
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        if (cudaSetDevice(device) != cudaSuccess) return nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        g_addr[device] = p;
    }
    return g_addr[device];
}

}  // namespace

struct ckks_context {
    Context c;
};

extern "C" size_t ckks_rescale_noalloc_capacity(void) { return kNoAllocScratchBytes; }

extern "C" int ckks_rescale_multi_noalloc(ckks_context *ctx, const ckks_tuple *in, uint32_t mu, ckks_tuple *out,
                                          void *stream) {
    if (!ctx || !in || !out || !out->data) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!in->data || in->level < 1 || in->level > (uint32_t)C.L || in->poly_stride < in->level ||
        in->n_polys < 1 || in->n_polys > CKKS_MAX_TUPLE || !in->ntt_form)
        return CKKS_EINVAL;
    if (mu < 1 || mu >= in->level) return CKKS_ELEVEL;
    const uint32_t ol = in->level - mu;
    if (out->poly_stride == 0) out->poly_stride = out->data == in->data ? in->poly_stride : ol;
    if (out->poly_stride < ol) return CKKS_EINVAL;
    if (out->data == in->data && out->poly_stride != in->poly_stride) return CKKS_EINVAL;
    const size_t need = rescale_ws_bytes(C, (int)in->n_polys, (int)in->level, (int)mu, 1);
    if (need > kNoAllocScratchBytes) return CKKS_ENOMEM;
    void *scratch = scratch_address(C.device);
    if (!scratch) return CKKS_ECUDA;
    cudaSetDevice(C.device);
    double scale = in->scale;
    for (uint32_t j = 0; j < mu; ++j) scale /= (double)C.primes[in->level - 1 - j];
    LimbView vi{(u64 *)in->data, 0, (i64)in->poly_stride * C.N};
    LimbView vo{(u64 *)out->data, 0, (i64)out->poly_stride * C.N};
    // the timing hook would create CUDA events; keep it off for this call
    Profiler &prof = const_cast<Context &>(C).prof;
    const bool prof_on = prof.on;
    prof.on = false;
    cudaError_t err;
    int rc = run_rescale_ws(C, 1, (int)in->n_polys, (int)in->level, (int)mu, vi, vo, scratch, kNoAllocScratchBytes,
                            (cudaStream_t)stream, err);
    prof.on = prof_on;
    if (err != cudaSuccess || rc != 0) {
        const_cast<Context &>(C).sticky.store((int)(err == cudaSuccess ? cudaErrorUnknown : err));
        return CKKS_ECUDA;
    }
    out->n_polys = in->n_polys;
    out->level = ol;
    out->ntt_form = 1;
    out->scale = scale;
    return CKKS_OK;
}
