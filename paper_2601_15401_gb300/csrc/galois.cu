// Galois automorphisms sigma_g: a(X) -> a(X^g), g odd (slot rotation and
// conjugation of Section II's encoding). In the NTT domain of this library
// (evaluation at psi^(2 brv(i) + 1)) sigma_g permutes every limb the same
// way, independently of the prime:
//   (sigma_g a)^[i] = a(psi^(g (2 brv(i) + 1))) = A[brv((g (2 brv(i) + 1) mod 2N - 1) / 2)]
#include "internal.h"
#include "rns.h"

namespace ckks {

namespace {

constexpr int kThr = 256;
constexpr int kLogChunk = 12;  // 4096 elements = 32 KiB of shared memory

__device__ __forceinline__ uint32_t brv(uint32_t x, int bits) { return bits ? __brev(x) >> (32 - bits) : 0u; }

// source index of output index i: brv((g (2 brv(i) + 1) mod 2N - 1) / 2)
__device__ __forceinline__ uint32_t perm(uint32_t i, uint32_t g, int log_n) {
    const uint32_t bi = brv(i, log_n);
    // g (2 bi + 1) mod 2N: 2N divides 2^32, so the wrap of the 32-bit
    // product leaves the low bits exact
    const uint32_t e = (g * (2u * bi + 1u)) & ((2u << log_n) - 1u);
    return brv((e - 1u) >> 1, log_n);
}

// With u = brv(i), the source is brv(v), v = g u + (g - 1) / 2 mod N: the
// low t bits of v depend only on the low t bits of u, i.e. the high t bits
// of the source index only on the high t bits of i. So every chunk of
// 2^(log_n - t) consecutive outputs reads exactly one chunk of the input:
// the CTA stages that chunk in shared memory with coalesced loads and
// writes its outputs coalesced.
// blockIdx.x = (output poly, limb, chunk), blockIdx.y = batch element.
__global__ void __launch_bounds__(kThr) automorphism_kernel(LimbView in, LimbView out, AutoMap map, int level,
                                                            int log_n, uint32_t g) {
    extern __shared__ u64 stage[];
    const int log_c = log_n < kLogChunk ? log_n : kLogChunk;
    const int chunk = 1 << log_c;
    const int n_chunks = 1 << (log_n - log_c);
    int bid = blockIdx.x;
    const int D = bid % n_chunks;
    bid /= n_chunks;
    const int x = bid % level;
    const int p = bid / level;
    const int b = blockIdx.y;
    const i64 limb = (i64)x << log_n;
    u64 *dst = out.ptr + (i64)b * out.bstride + (i64)p * out.pstride + limb + ((i64)D << log_c);
    const int sp = map.src[p];
    if (sp < 0) {
        for (int k = threadIdx.x; k < chunk; k += blockDim.x) dst[k] = 0;
        return;
    }
    const uint32_t i0 = (uint32_t)D << log_c;
    const uint32_t S = perm(i0, g, log_n) >> log_c;
    const u64 *src = in.ptr + (i64)b * in.bstride + (i64)sp * in.pstride + limb + ((i64)S << log_c);
    for (int k = threadIdx.x; k < chunk; k += blockDim.x) stage[k] = src[k];
    __syncthreads();
    const uint32_t s0 = S << log_c;
    for (int k = threadIdx.x; k < chunk; k += blockDim.x) dst[k] = stage[perm(i0 + k, g, log_n) - s0];
}

}  // namespace

cudaError_t launch_automorphism(const Context &C, LimbView in, LimbView out, const AutoMap &map, int batch,
                                int level, uint32_t g, cudaStream_t st) {
    const i64 total = (i64)map.n_out * level * C.N;
    if (total == 0 || batch == 0) return cudaSuccess;
    count_kernel(C);
    int reads = 0;
    for (int p = 0; p < map.n_out; ++p) reads += map.src[p] >= 0;
    ProfScope ps(C, KC_AUTOMORPHISM, (double)batch * (reads + map.n_out) * level * C.N * sizeof(u64), st);
    const int log_c = C.log_n < kLogChunk ? C.log_n : kLogChunk;
    dim3 grid((unsigned)((i64)map.n_out * level << (C.log_n - log_c)), (unsigned)batch);
    automorphism_kernel<<<grid, kThr, (size_t)sizeof(u64) << log_c, st>>>(in, out, map, level, C.log_n, g);
    return cudaGetLastError();
}

}  // namespace ckks
