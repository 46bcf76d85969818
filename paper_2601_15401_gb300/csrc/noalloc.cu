// Allocation-free variant of the multi-level rescale (ckks_rescale_multi).
//
// Some callers cannot allocate device memory at the point where they need a
// rescale: a component that only receives device pointers from another one
// and has no allocator of its own, or a loop that must not call cudaMalloc
// (which can synchronise the device) or take a caching allocator's locks. For
// them ckks_rescale_multi_noalloc runs Algorithm 1 (always that form, whatever
// the context's "inner_rescale" setting) with its scratch in a fixed device
// array of this library (kNoAllocScratchBytes, 32 MiB) instead of a
// caller-supplied workspace. The array exists once per device that loads the
// library and is held until the process exits.
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

// Makes `device` current for the lifetime of the guard and puts the caller's
// current device back afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == device || cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Device address of the scratch on `device` (which the caller has made
// current). Returns nullptr if the symbol cannot be resolved.
void *scratch_address(int device) {
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        g_addr[device] = p;
    }
    return g_addr[device];
}

}  // namespace

extern "C" size_t ckks_rescale_noalloc_capacity(void) { return kNoAllocScratchBytes; }

extern "C" int ckks_rescale_multi_noalloc(ckks_context *ctx, const ckks_tuple *in, uint32_t mu, ckks_tuple *out,
                                          void *stream) {
    if (!ctx || !in || !out || !out->data) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!in->data || in->level < 1 || in->level > (uint32_t)C.L || in->poly_stride < in->level ||
        in->n_polys < 1 || in->n_polys > CKKS_MAX_TUPLE || !in->ntt_form)
        return CKKS_EINVAL;
    // the timing hook records CUDA events per launch; this call does not
    // take part in it (and does not switch it off for other callers)
    if (C.prof.on) return CKKS_EINVAL;
    if (mu < 1 || mu >= in->level) return CKKS_ELEVEL;
    const uint32_t ol = in->level - mu;
    if (out->poly_stride == 0) out->poly_stride = out->data == in->data ? in->poly_stride : ol;
    if (out->poly_stride < ol) return CKKS_EINVAL;
    if (out->data == in->data && out->poly_stride != in->poly_stride) return CKKS_EINVAL;
    const size_t need = rescale_alg1_ws_bytes(C, (int)in->n_polys, (int)in->level, (int)mu, 1);
    if (need > kNoAllocScratchBytes) return CKKS_ENOMEM;
    DeviceGuard guard(C.device);
    if (!guard.ok) return CKKS_ECUDA;
    void *scratch = scratch_address(C.device);
    if (!scratch) return CKKS_ECUDA;
    double scale = in->scale;
    for (uint32_t j = 0; j < mu; ++j) scale /= (double)C.primes[in->level - 1 - j];
    LimbView vi{(u64 *)in->data, 0, (i64)in->poly_stride * C.N};
    LimbView vo{(u64 *)out->data, 0, (i64)out->poly_stride * C.N};
    cudaError_t err;
    int rc = run_rescale_alg1_ws(C, 1, (int)in->n_polys, (int)in->level, (int)mu, vi, vo, scratch,
                                 kNoAllocScratchBytes, (cudaStream_t)stream, err);
    if (err != cudaSuccess || rc != 0) {
        ctx->c.sticky.store((int)(err == cudaSuccess ? cudaErrorUnknown : err));
        return CKKS_ECUDA;
    }
    out->n_polys = in->n_polys;
    out->level = ol;
    out->ntt_form = 1;
    out->scale = scale;
    return CKKS_OK;
}
