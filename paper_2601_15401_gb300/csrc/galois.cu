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

// out poly p <- sigma_g(in poly src[p]), or zeros where src[p] < 0;
// blockIdx.y = batch element
__global__ void __launch_bounds__(kThr) automorphism_kernel(LimbView in, LimbView out, AutoMap map, int level,
                                                            int log_n, uint32_t g) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = 1 << log_n;
    const i64 per_poly = (i64)level * N;
    if (gid >= per_poly * map.n_out) return;
    const int b = blockIdx.y;
    const int p = (int)(gid / per_poly);
    const i64 r = gid % per_poly;
    const int i = (int)(r % N);
    u64 *d = out.ptr + (i64)b * out.bstride + (i64)p * out.pstride + r;
    const int sp = map.src[p];
    if (sp < 0) {
        *d = 0;
        return;
    }
    const uint32_t bi = __brev((uint32_t)i) >> (32 - log_n);
    // g (2 bi + 1) mod 2N: 2N divides 2^32, so the wrap of the 32-bit
    // product leaves the low bits exact
    const uint32_t e = (g * (2u * bi + 1u)) & (uint32_t)(2 * N - 1);
    const uint32_t src = __brev((e - 1u) >> 1) >> (32 - log_n);
    *d = in.ptr[(i64)b * in.bstride + (i64)sp * in.pstride + (r - i) + src];
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
    dim3 grid((unsigned)((total + kThr - 1) / kThr), (unsigned)batch);
    automorphism_kernel<<<grid, kThr, 0, st>>>(in, out, map, level, C.log_n, g);
    return cudaGetLastError();
}

}  // namespace ckks
