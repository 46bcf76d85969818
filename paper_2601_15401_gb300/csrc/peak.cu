// Integer-arithmetic peaks of this GPU for the operations the hot path is
// built from, measured with register-only kernels (no memory traffic):
//   kind 0  lazy Shoup product  x w - floor(x w'/2^64) q      (NTT twiddles,
//           fused scalings)
//   kind 1  Harvey's lazy Cooley-Tukey butterfly (one Shoup product plus its
//           additions and correction; the forward NTT's unit of work)
//   kind 2  64 x 64 -> 128-bit multiply-accumulate (BConv, key MAC, tensor
//           product dot products)
//   kind 3  Montgomery product with R = 2^64 (tensor product, key preparation)
//   kind 4  the exchange between two radix-16 passes of a 256-point block
//           (each of 16 threads holds 16 values; afterwards thread i holds
//           value i of every thread: a 16 x 16 transpose) through warp
//           shuffles: four XOR stages of 8 swaps, no barrier
//   kind 5  the same exchange through shared memory (store, __syncwarp,
//           load), the way the NTT kernels pass data between passes
//   kind 6  kind 1 for a modulus q = 1 (mod 2^32) (shoup_lazy_q1)
//   kind 7  kind 0 for a modulus q = 1 (mod 2^32)
// Kinds 4 and 5 count one operation per value moved.
// Each thread runs kChains independent dependency chains so that issue, not
// latency, limits the rate. The caller times the launch (CUDA events) and
// divides blocks x threads x kChains x iters operations by the time.
#include "../../include/ckks_mulk.h"
#include "common.cuh"

namespace {

constexpr int kChains = 8;

struct PeakConsts {
    u64 q, qinv;
    u64 w[kChains], wp[kChains];
};

__device__ __forceinline__ void ct_bfly_peak(u64 &X, u64 &Y, u64 w, u64 wp, u64 q) {
    const u64 q2 = q << 1;
    const u64 x = X >= q2 ? X - q2 : X;
    const u64 t = shoup_lazy(Y, w, wp, q);
    X = x + t;
    Y = x - t + q2;
}

__device__ __forceinline__ void ct_bfly_peak_q1(u64 &X, u64 &Y, u64 w, u64 wp, u64 q) {
    const u64 q2 = q << 1;
    const u64 x = X >= q2 ? X - q2 : X;
    const u64 t = shoup_lazy_q1(Y, w, wp, (uint32_t)(q >> 32));
    X = x + t;
    Y = x - t + q2;
}

// 16 x 16 transpose within each half-warp: lane i holds row i in v[0..15];
// afterwards it holds column i. Stage s swaps the elements whose index bit
// s differs from the lane's bit s with the partner lane i ^ 2^s.
__device__ __forceinline__ void transpose16_shfl(u64 (&v)[16]) {
    const int lane = threadIdx.x & 15;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int m = 1 << s;
        const bool hi = lane & m;
#pragma unroll
        for (int k0 = 0; k0 < 16; ++k0) {
            if (k0 & m) continue;
            const int k1 = k0 | m;
            const u64 send = hi ? v[k0] : v[k1];
            const unsigned lo32 = __shfl_xor_sync(0xffffffffu, (unsigned)send, m);
            const unsigned hi32 = __shfl_xor_sync(0xffffffffu, (unsigned)(send >> 32), m);
            const u64 r = ((u64)hi32 << 32) | lo32;
            v[k0] = hi ? r : v[k0];
            v[k1] = hi ? v[k1] : r;
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) peak_kernel(PeakConsts P, int iters, u64 *out) {
    const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = P.q;
    u64 x[kChains], y[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        x[i] = (tid * 0x9E3779B97F4A7C15ull + (u64)i * 0x632BE59BD9B4E019ull) % q;
        y[i] = (tid * 0xD1B54A32D192ED03ull + (u64)i) % q;
    }
    Acc128Lazy acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i].zero();
    const ModQ m{q, P.qinv};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (KIND == 0) {
                x[i] = shoup_lazy(x[i], P.w[i], P.wp[i], q);
            } else if (KIND == 1) {
                ct_bfly_peak(x[i], y[i], P.w[i], P.wp[i], q);
            } else if (KIND == 6) {
                ct_bfly_peak_q1(x[i], y[i], P.w[i], P.wp[i], q);
            } else if (KIND == 7) {
                x[i] = shoup_lazy_q1(x[i], P.w[i], P.wp[i], (uint32_t)(q >> 32));
            } else if (KIND == 2) {
                acc[i].mac(x[i], P.w[i]);
                x[i] += y[i];
            } else {
                x[i] = mont_mul(x[i], P.w[i], m);
            }
        }
    }
    u64 r = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) r ^= x[i] ^ y[i] ^ acc[i].hi ^ acc[i].lo;
    out[tid] = r;
}

template <int KIND>
__global__ void __launch_bounds__(256) exchange_kernel(int iters, u64 *out) {
    __shared__ u64 sm[256 * 17];  // one padded 16 x 16 tile per half-warp (16 per CTA)
    const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = tid * 16 + k;
    u64 *tile = sm + (threadIdx.x >> 4) * (16 * 17);
    const int lane = threadIdx.x & 15;
    for (int it = 0; it < iters; ++it) {
        if (KIND == 4) {
            transpose16_shfl(v);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) tile[lane * 17 + k] = v[k];
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = tile[k * 17 + lane];
            __syncwarp();
        }
        v[0] += 1;  // a data dependence between rounds
    }
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) r ^= v[k];
    out[tid] = r;
}

}  // namespace

extern "C" int ckks_peak_chains(void) { return kChains; }

extern "C" int ckks_peak_int(int kind, uint64_t q, const uint64_t *w, const uint64_t *wp, int blocks, int threads,
                             int iters, uint64_t *out, void *stream) {
    if (kind < 0 || kind > 7 || !w || !wp || !out || blocks < 1 || threads < 32 || threads > 256 ||
        threads % 32 || iters < 1 || q < 3 || q >= (1ull << 62) || !(q & 1))
        return CKKS_EINVAL;
    if ((kind == 6 || kind == 7) && (q & 0xffffffffull) != 1) return CKKS_EINVAL;
    PeakConsts P;
    P.q = q;
    u64 inv = 1;  // q^-1 mod 2^64 by Newton's iteration (q odd)
    for (int i = 0; i < 6; ++i) inv *= 2 - q * inv;
    P.qinv = inv;
    for (int i = 0; i < kChains; ++i) {
        if (w[i] >= q) return CKKS_EINVAL;
        P.w[i] = w[i];
        P.wp[i] = wp[i];
    }
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
    case 0: peak_kernel<0><<<blocks, threads, 0, st>>>(P, iters, (u64 *)out); break;
    case 1: peak_kernel<1><<<blocks, threads, 0, st>>>(P, iters, (u64 *)out); break;
    case 2: peak_kernel<2><<<blocks, threads, 0, st>>>(P, iters, (u64 *)out); break;
    case 3: peak_kernel<3><<<blocks, threads, 0, st>>>(P, iters, (u64 *)out); break;
    case 6: peak_kernel<6><<<blocks, threads, 0, st>>>(P, iters, (u64 *)out); break;
    case 7: peak_kernel<7><<<blocks, threads, 0, st>>>(P, iters, (u64 *)out); break;
    case 4: exchange_kernel<4><<<blocks, threads, 0, st>>>(iters, (u64 *)out); break;
    default: exchange_kernel<5><<<blocks, threads, 0, st>>>(iters, (u64 *)out); break;
    }
    return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_ECUDA;
}
