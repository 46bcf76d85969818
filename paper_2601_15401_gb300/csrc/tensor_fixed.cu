// Tensor products (Eq. 1, 8, 13) of tree nodes in fixed shapes.
//
// The tensor kernels of rns.cu unroll their product loops to a tuple-size
// bound and predicate every product on the run-time tuple sizes: a node of
// two 7-term tuples issues the instructions of 91 products for its 49. The
// kernels here are compiled for one node shape each: children sorted by
// size, largest first (the product is commutative and every step returns
// canonical residues, so the order does not change the result), every load
// of the node issued before the first product, each output term stored as
// soon as it is reduced. Shapes (tensor_fixed_code): two children of 4..7
// terms, three of 4 or 5 terms — among them the roots and the larger inner
// nodes of the paper's partitions for k = 6..12 (Table II).
//
// Operands are reduced residues and no term sums more than 7 products, so
// the 128-bit sums need no per-term reduction: B q^2 < q 2^64 for B <= 8
// and q < 2^61 keeps the high word below q, as REDC requires.
#include <utility>

#include "common.cuh"
#include "internal.h"
#include "rns.h"

#ifndef CKKS_TENSOR_PRESCALE
#define CKKS_TENSOR_PRESCALE 1
#endif

namespace ckks {

namespace {

constexpr int kThreads = 256;

// z = x * y (polynomials in s of A and B terms), each term REDC-reduced
template <int A, int B, bool Q1>
__device__ __forceinline__ void conv_redc(const u64 (&x)[A], const u64 (&y)[B], u64 (&z)[A + B - 1], const ModQ m) {
    static_assert(A >= B && B <= 8, "at most 8 products per term");
#pragma unroll
    for (int t = 0; t < A + B - 1; ++t) {
        Acc128Lazy acc;
        acc.zero();
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (t - b >= 0 && t - b < A) acc.mac(x[t - b], y[b]);
        z[t] = redc_t<Q1>(acc.hi, acc.lo, m);
    }
}

// the same, each term stored at dst + t ds as soon as it is formed (with
// CKKS_TENSOR_PRESCALE = 0 multiplied by the Shoup constant fix first)
template <int A, int B, bool Q1>
__device__ __forceinline__ void conv_redc_store(const u64 (&x)[A], const u64 (&y)[B], const ModQ m, const Shoup fix,
                                                u64 *dst, i64 ds) {
    static_assert(A >= B && B <= 8, "at most 8 products per term");
#pragma unroll
    for (int t = 0; t < A + B - 1; ++t) {
        Acc128Lazy acc;
        acc.zero();
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (t - b >= 0 && t - b < A) acc.mac(x[t - b], y[b]);
        const u64 z = redc_t<Q1>(acc.hi, acc.lo, m);
        dst[(i64)t * ds] = CKKS_TENSOR_PRESCALE ? z : shoup_t<Q1>(z, fix.w, fix.wp, m.q);
    }
}

template <int T>
__device__ __forceinline__ void load_terms(const u64 *src, i64 ps, u64 (&o)[T]) {
#pragma unroll
    for (int a = 0; a < T; ++a) o[a] = src[(i64)a * ps];
}

// the terms of the last (smallest) child times R^(m-1)
template <int T, bool Q1>
__device__ __forceinline__ void prescale(u64 (&o)[T], const Shoup fix, u64 q) {
    if (CKKS_TENSOR_PRESCALE)
#pragma unroll
        for (int a = 0; a < T; ++a) o[a] = shoup_t<Q1>(o[a], fix.w, fix.wp, q);
}

// One coefficient r (= limb j * N + coefficient) of a node with children of
// A, B (and C; 0 for two children) terms: m - 1 Montgomery products, which
// leave R^-(m-1), and R^(m-1) as a Shoup product by the per-prime constant
// rfix[j][m] on the terms of the last child.
template <int A, int B, int C, bool Q1, class View>
__device__ __forceinline__ void tensor_fixed_coeff(const View &v, i64 r, int j, const ModQ m, const Shoup *rfix) {
    u64 x[A], y[B];
    load_terms<A>(v.src(0) + r, v.pstride(0), x);
    load_terms<B>(v.src(1) + r, v.pstride(1), y);
    u64 *dst = v.dst() + r;
    const i64 ds = v.dstride();
    if constexpr (C == 0) {
        const Shoup fix = rfix[(i64)j * 16 + 2];
        prescale<B, Q1>(y, fix, m.q);
        conv_redc_store<A, B, Q1>(x, y, m, fix, dst, ds);
    } else {
        const Shoup fix = rfix[(i64)j * 16 + 3];
        u64 w[C];
        load_terms<C>(v.src(2) + r, v.pstride(2), w);
        u64 z[A + B - 1];
        conv_redc<A, B, Q1>(x, y, z, m);
        prescale<C, Q1>(w, fix, m.q);
        conv_redc_store<A + B - 1, C, Q1>(z, w, m, fix, dst, ds);
    }
}

template <int A, int B, int C, bool Q1>
__global__ void __launch_bounds__(kThreads, 3) tensor_fixed_kernel(TensorArgs T) {
    const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;  // limb * N + coefficient
    if (r >= (i64)T.level * T.N) return;
    const int j = (int)(r >> T.log_n);
    tensor_fixed_coeff<A, B, C, Q1>(TensorUniformView{T, (int)blockIdx.y}, r, j, T.mods[j], T.rfix);
}

// blockIdx.y = table entry (every entry of the launch has this shape); the
// entry is staged in shared memory, one word per thread
template <int A, int B, int C, bool Q1>
__global__ void __launch_bounds__(kThreads, 3) tensor_fixed_table_kernel(const TensorJob *jobs, int N, int log_n,
                                                                        const ModQ *mods, const Shoup *rfix) {
    __shared__ TensorJob J;
    {
        static_assert(sizeof(TensorJob) % sizeof(u64) == 0, "TensorJob is a whole number of words");
        constexpr int W = sizeof(TensorJob) / sizeof(u64);
        const u64 *src = reinterpret_cast<const u64 *>(jobs + blockIdx.y);
        u64 *dst = reinterpret_cast<u64 *>(&J);
        for (int i = threadIdx.x; i < W; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (i64)J.level * N) return;
    const int j = (int)(r >> log_n);
    tensor_fixed_coeff<A, B, C, Q1>(TensorTableView{J}, r, j, mods[j], rfix);
}

// The shape of each code (tensor_fixed_code), as template arguments.
template <class F>
cudaError_t with_shape(int code, F &&f) {
    switch (code) {
    case 0: return f(std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{}, std::integral_constant<int, 0>{});
    case 1: return f(std::integral_constant<int, 5>{}, std::integral_constant<int, 4>{}, std::integral_constant<int, 0>{});
    case 2: return f(std::integral_constant<int, 5>{}, std::integral_constant<int, 5>{}, std::integral_constant<int, 0>{});
    case 4: return f(std::integral_constant<int, 6>{}, std::integral_constant<int, 5>{}, std::integral_constant<int, 0>{});
    case 5: return f(std::integral_constant<int, 6>{}, std::integral_constant<int, 6>{}, std::integral_constant<int, 0>{});
    case 6: return f(std::integral_constant<int, 7>{}, std::integral_constant<int, 4>{}, std::integral_constant<int, 0>{});
    case 7: return f(std::integral_constant<int, 7>{}, std::integral_constant<int, 5>{}, std::integral_constant<int, 0>{});
    case 8: return f(std::integral_constant<int, 7>{}, std::integral_constant<int, 6>{}, std::integral_constant<int, 0>{});
    case 9: return f(std::integral_constant<int, 7>{}, std::integral_constant<int, 7>{}, std::integral_constant<int, 0>{});
    case 10: return f(std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{});
    case 11: return f(std::integral_constant<int, 5>{}, std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{});
    case 12: return f(std::integral_constant<int, 5>{}, std::integral_constant<int, 5>{}, std::integral_constant<int, 4>{});
    case 13: return f(std::integral_constant<int, 5>{}, std::integral_constant<int, 5>{}, std::integral_constant<int, 5>{});
    default: return cudaErrorInvalidValue;
    }
}

template <bool Q1>
cudaError_t launch_uniform(const TensorArgs &T, int code, cudaStream_t st) {
    dim3 blocks((unsigned)(((i64)T.level * T.N + kThreads - 1) / kThreads), T.n_batch);
    return with_shape(code, [&](auto a, auto b, auto c) {
        tensor_fixed_kernel<decltype(a)::value, decltype(b)::value, decltype(c)::value, Q1>
            <<<blocks, kThreads, 0, st>>>(T);
        return cudaGetLastError();
    });
}

template <bool Q1>
cudaError_t launch_table(const Context &C, const TensorJob *jobs, int n_jobs, int code, int max_level,
                         cudaStream_t st) {
    dim3 blocks((unsigned)(((i64)max_level * C.N + kThreads - 1) / kThreads), (unsigned)n_jobs);
    return with_shape(code, [&](auto a, auto b, auto c) {
        tensor_fixed_table_kernel<decltype(a)::value, decltype(b)::value, decltype(c)::value, Q1>
            <<<blocks, kThreads, 0, st>>>(jobs, C.N, C.log_n, C.d_mods, C.d_rfix);
        return cudaGetLastError();
    });
}

}  // namespace

int tensor_sort_children(TensorJob &T) {
    for (int c = 1; c < T.m; ++c)
        for (int d = c; d > 0 && T.cpolys[d] > T.cpolys[d - 1]; --d) {
            std::swap(T.child[d], T.child[d - 1]);
            std::swap(T.cstride[d], T.cstride[d - 1]);
            std::swap(T.cpolys[d], T.cpolys[d - 1]);
        }
    if (T.m < 2 || T.m > 3) return -1;
    return tensor_fixed_code(T.m, T.cpolys[0], T.cpolys[1], T.m > 2 ? T.cpolys[2] : 0);
}

int tensor_sort_children(TensorArgs &A) {
    for (int c = 1; c < A.m; ++c)
        for (int d = c; d > 0 && A.child_polys[d] > A.child_polys[d - 1]; --d) {
            std::swap(A.child[d], A.child[d - 1]);
            std::swap(A.child_polys[d], A.child_polys[d - 1]);
        }
    if (A.m < 2 || A.m > 3) return -1;
    return tensor_fixed_code(A.m, A.child_polys[0], A.child_polys[1], A.m > 2 ? A.child_polys[2] : 0);
}

cudaError_t launch_tensor_fixed(const Context &C, const TensorArgs &A, int code, cudaStream_t st) {
    return C.q1() ? launch_uniform<true>(A, code, st) : launch_uniform<false>(A, code, st);
}

cudaError_t launch_tensor_fixed_table(const Context &C, const TensorJob *jobs, int n_jobs, int code, int max_level,
                                      double bytes, double ops, cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    if (n_jobs > 65535) return cudaErrorInvalidValue;
    count_kernel(C);
    ProfScope ps(C, KC_TENSOR, bytes, st, ops);
    return C.q1() ? launch_table<true>(C, jobs, n_jobs, code, max_level, st)
                  : launch_table<false>(C, jobs, n_jobs, code, max_level, st);
}

}  // namespace ckks
