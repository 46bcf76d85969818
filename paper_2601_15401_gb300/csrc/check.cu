// Integrity checks for debugging and failure detection (no counterpart in
// the paper): counting residues outside [0, q) in a set of limbs, and a
// position-dependent checksum of a resident key buffer. Both only read.
#include "internal.h"
#include "rns.h"

namespace ckks {

namespace {

constexpr int kThr = 256;

// counter += number of residues >= q over [batch][polys][level][N]
// (blockIdx.y = batch element)
__global__ void __launch_bounds__(kThr) range_check_kernel(LimbView v, int polys, int level, int N,
                                                           const ModQ *mods, unsigned long long *counter) {
    const i64 per_poly = (i64)level * N;
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    if (gid < per_poly * polys) {
        const int p = (int)(gid / per_poly);
        const i64 r = gid % per_poly;
        const int x = (int)(r / N);
        bad = v.ptr[(i64)blockIdx.y * v.bstride + (i64)p * v.pstride + r] >= mods[x].q;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(counter, (unsigned long long)__popc(mask));
}

// sum over i of mix(w_i, i) mod 2^64, mix a 64-bit finaliser of the word
// and its position (so a changed, moved or swapped word changes the sum)
__device__ __forceinline__ u64 mix(u64 w, u64 i) {
    u64 z = w ^ (i * 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kThr) checksum_kernel(const u64 *w, i64 n, unsigned long long *out) {
    __shared__ u64 part[kThr / 32];
    u64 s = 0;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
        s += mix(w[i], (u64)i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0;
        for (int k = 0; k < kThr / 32; ++k) t += part[k];
        atomicAdd(out, (unsigned long long)t);
    }
}

}  // namespace

cudaError_t launch_range_check(const Context &C, LimbView v, int batch, int polys, int level, cudaStream_t st) {
    const i64 total = (i64)polys * level * C.N;
    if (total == 0 || batch == 0) return cudaSuccess;
    count_kernel(C);
    dim3 grid((unsigned)((total + kThr - 1) / kThr), (unsigned)batch);
    range_check_kernel<<<grid, kThr, 0, st>>>(v, polys, level, C.N, C.d_mods, C.d_check);
    return cudaGetLastError();
}

cudaError_t launch_checksum(const Context &C, const u64 *w, long long n, unsigned long long *out, cudaStream_t st) {
    count_kernel(C);
    checksum_kernel<<<4 * 152, kThr, 0, st>>>(w, (i64)n, out);
    return cudaGetLastError();
}

}  // namespace ckks
