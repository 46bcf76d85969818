// Copies by the GPU's own loads and stores. On a Grace-Blackwell node the
// GPU reaches the host's memory over NVLink-C2C with ordinary loads, so a
// kernel can pull a step's inputs from pinned host memory (mapped into the
// device's address space) into HBM without a copy engine, or read them in
// place. ckks_pull is that copy: 16-byte loads and stores, a grid of small
// CTAs (64 threads, 32 registers each: 2048 registers, so one fits beside
// three 256-thread NTT CTAs of 80 registers on an SM) striding over the
// buffer.
#include "../../include/ckks_mulk.h"
#include "common.cuh"

namespace {

__global__ void __launch_bounds__(64) pull_kernel(ulonglong2 *dst, const ulonglong2 *src, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    // four independent 16-byte loads in flight per thread
    for (; i + 3 * stride < n; i += 4 * stride) {
        const ulonglong2 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

}  // namespace

extern "C" int ckks_pull(void *dst, const void *src, size_t bytes, int blocks, void *stream) {
    if (!dst || !src || bytes % 16 || (size_t)dst % 16 || (size_t)src % 16 || blocks < 1) return CKKS_EINVAL;
    if (bytes == 0) return CKKS_OK;
    pull_kernel<<<blocks, 64, 0, (cudaStream_t)stream>>>((ulonglong2 *)dst, (const ulonglong2 *)src, bytes / 16);
    return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_ECUDA;
}

extern "C" int ckks_host_device_pointer(void *host, void **dev) {
    if (!host || !dev) return CKKS_EINVAL;
    *dev = nullptr;
    if (cudaHostGetDevicePointer(dev, host, 0) == cudaSuccess) return CKKS_OK;
    cudaGetLastError();  // not pinned or not mapped: clear the (non-sticky) error
    return CKKS_EINVAL;
}
