// Coefficient-wise RNS kernels of the k-input multiplication:
//   tensor product of child tuples (Eq. 1, 8, 13), fast basis conversion for
//   ModUp (Eq. 4), the evaluation-key inner product summed over every key
//   and digit before one ModDown (Eq. 15 and the combined form of
//   Section III), the rescale chain among the top limbs (Eq. 6, Algorithm 1
//   step 2), key preparation (P^-1 folded into the Q limbs, Eq. 12) and key
//   generation (Eq. 2, 9, 14).
//
// All are memory-bound streams over [batch][poly][limb][N]; each thread owns
// one coefficient and loops over what the formula sums, keeping partial sums
// in 128-bit accumulators reduced once (Montgomery REDC).
#include "common.cuh"
#include "internal.h"
#include "rns.h"

#include <algorithm>
#include <type_traits>

namespace ckks {

static constexpr int kThreads = 256;

// 1: the tensor kernels for the largest tuples (three children at a k >= 9
// root) load the next child's terms while multiplying by the current one
#ifndef CKKS_TENSOR_PREFETCH
#define CKKS_TENSOR_PREFETCH 1
#endif

// 1: the R^(m-1) correction of a node's m - 1 Montgomery products is applied
// to the terms of its last child (the smallest: the host sorts children by
// size) before they are multiplied, instead of to every output term
#ifndef CKKS_TENSOR_PRESCALE
#define CKKS_TENSOR_PRESCALE 1
#endif

// 1: the bounded kernels' 128-bit sums reduce their high word once, at the
// REDC (the bounds are stated where the sums are formed); 0: after every term
#ifndef CKKS_TENSOR_LAZY
#define CKKS_TENSOR_LAZY 1
#endif
using TensorAcc = std::conditional<CKKS_TENSOR_LAZY != 0, Acc128Lazy, Acc128>::type;

// V adjacent words at p (16-byte loads / stores for even V; p 16-byte aligned)
template <int V>
__device__ __forceinline__ void load_span(const u64 *p, u64 (&o)[V]) {
    if constexpr (V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) o[i] = p[i];
    }
}

template <int V>
__device__ __forceinline__ void store_span(u64 *p, const u64 (&v)[V]) {
    if constexpr (V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 2) *reinterpret_cast<ulonglong2 *>(p + i) = make_ulonglong2(v[i], v[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) p[i] = v[i];
    }
}

// ---------------------------------------------------------------------------
// tensor product: out = prod over children of (sum_l c_l s^l), coefficient-
// wise in the NTT domain. Each child product is a Montgomery product, so the
// m - 1 products leave R^-(m-1); the smallest child's terms are multiplied
// by R^(m-1) before they enter (a Shoup product by a per-prime constant).
// ---------------------------------------------------------------------------
// MAXT bounds every tuple size involved (children and output), so the
// unrolled, predicated product loops stay short for small nodes.
// r = limb * N + coefficient (the first of V adjacent ones), j = the limb's
// prime.
template <int MAXT, bool Q1, int V, class View>
__device__ __forceinline__ void tensor_coeff(const View &v, i64 r, int j, const ModQ m, const Shoup *rfix) {
    const u64 q = m.q;
    u64 cur[MAXT][V];
    int ncur = v.polys(0);
    {
        const u64 *src = v.src(0) + r;
        const i64 ps = v.pstride(0);
#pragma unroll
        for (int a = 0; a < MAXT; ++a) {
            if (a < ncur) load_span<V>(src + (i64)a * ps, cur[a]);
            else
#pragma unroll
                for (int e = 0; e < V; ++e) cur[a][e] = 0ull;
        }
    }
    // the largest tuples (three children at a k >= 9 root) load the next
    // child while multiplying by this one
    constexpr bool PF = CKKS_TENSOR_PREFETCH && MAXT > 9;
    auto load_child = [&](int c, u64 (&y)[MAXT][V]) {
        const int ny = v.polys(c);
        const u64 *src = v.src(c) + r;
        const i64 ps = v.pstride(c);
#pragma unroll
        for (int a = 0; a < MAXT; ++a) {
            if (a < ny) load_span<V>(src + (i64)a * ps, y[a]);
            else
#pragma unroll
                for (int e = 0; e < V; ++e) y[a][e] = 0ull;
        }
    };
    // m children take m - 1 Montgomery products, which leave R^-(m-1): the
    // terms of the last child are multiplied by R^(m-1) first (a Shoup
    // product by a per-prime constant), or else every output term after
    const Shoup fix = rfix[(i64)j * 16 + v.m()];
    u64 y[MAXT][V];
    if (PF && v.m() > 1) load_child(1, y);
    for (int c = 1; c < v.m(); ++c) {
        const int ny = v.polys(c);
        u64 yn[PF ? MAXT : 1][V];
        if constexpr (PF) {
            if (c + 1 < v.m()) load_child(c + 1, yn);
        } else {
            load_child(c, y);
        }
        if (CKKS_TENSOR_PRESCALE && c == v.m() - 1) {
#pragma unroll
            for (int a = 0; a < MAXT; ++a)
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (a < ny) y[a][e] = shoup_t<Q1>(y[a][e], fix.w, fix.wp, q);
        }
        u64 nxt[MAXT][V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if (ny == 2) {
                // times a ciphertext (y0 + y1 s): Karatsuba on pairs of the running
                // tuple (Fig. 2(b)): for (c_a, c_{a+1}) the cross term
                // c_a y1 + c_{a+1} y0 = (c_a + c_{a+1})(y0 + y1) - c_a y0 - c_{a+1} y1,
                // an exact non-negative integer, so it stays in the 128-bit sums.
                // A sum takes p1 of its own pair, the cross term (< 2 q^2) of
                // the pair below and p2 of the pair below that, or the
                // unpaired products: below 4 q^2 < q 2^64 (q < 2^61), so its
                // high word stays below q without a reduction per term.
                TensorAcc acc[MAXT];
#pragma unroll
                for (int t = 0; t < MAXT; ++t) acc[t].zero();
                const u64 y0 = y[0][e], y1 = y[1][e];
                const u64 ys = y0 + y1;  // < 2q, not reduced
#pragma unroll
                for (int a = 0; a < MAXT; a += 2) {
                    if (a + 1 < ncur && a + 2 < MAXT) {
                        const u64 ca = cur[a][e], cb = cur[a + 1][e];
                        const u64 p1h = mulhi64(ca, y0), p1l = ca * y0;
                        const u64 p2h = mulhi64(cb, y1), p2l = cb * y1;
                        const u64 sab = ca + cb;
                        u64 p3l = sab * ys, p3h = mulhi64(sab, ys);
                        // p3 -= p1 + p2 (128-bit; the result is c_a y1 + c_{a+1} y0 >= 0)
                        u64 bl = p1l + p2l, bh = p1h + p2h + (bl < p1l ? 1ull : 0ull);
                        u64 rl = p3l - bl, rh = p3h - bh - (p3l < bl ? 1ull : 0ull);
                        acc[a].add(p1h, p1l, q);
                        acc[a + 1].add(rh, rl, q);
                        acc[a + 2].add(p2h, p2l, q);
                    } else if (a < ncur && a + 1 >= ncur) {
                        acc[a].mac(cur[a][e], y0, q);
                        if (a + 1 < MAXT) acc[a + 1].mac(cur[a][e], y1, q);
                    }
                }
#pragma unroll
                for (int t = 0; t < MAXT; ++t)
                    nxt[t][e] = t < ncur + 1 ? redc_t<Q1>(acc[t].hi, acc[t].lo, m) : 0ull;
            } else {
                // a term sums at most min(ncur, ny) <= 7 products (ncur + ny
                // - 1 <= 13) of reduced residues: below q 2^64, no reduction
                // per term
#pragma unroll
                for (int t = 0; t < MAXT; ++t) {
                    TensorAcc acc;
                    acc.zero();
#pragma unroll
                    for (int a = 0; a <= t; ++a) {
                        if (a < ncur && t - a < ny) acc.mac(cur[a][e], y[t - a][e], q);
                    }
                    nxt[t][e] = t < ncur + ny - 1 ? redc_t<Q1>(acc.hi, acc.lo, m) : 0ull;
                }
            }
        }
        ncur = ncur + ny - 1;
#pragma unroll
        for (int t = 0; t < MAXT; ++t)
#pragma unroll
            for (int e = 0; e < V; ++e) cur[t][e] = nxt[t][e];
        if constexpr (PF) {
#pragma unroll
            for (int a = 0; a < MAXT; ++a)
#pragma unroll
                for (int e = 0; e < V; ++e) y[a][e] = yn[a][e];
        }
    }
    u64 *dst = v.dst() + r;
    const i64 ds = v.dstride();
#pragma unroll
    for (int t = 0; t < MAXT; ++t)
        if (t < ncur) {
            u64 o[V];
#pragma unroll
            for (int e = 0; e < V; ++e)
                o[e] = CKKS_TENSOR_PRESCALE ? cur[t][e] : shoup_t<Q1>(cur[t][e], fix.w, fix.wp, m.q);
            store_span<V>(dst + (i64)t * ds, o);
        }
}

// CTAs of 256 threads per SM: four (at most 64 registers) up to 4-term
// tuples, whose launches are bound by HBM and need the loads of more
// threads in flight; three (at most 85) up to 9 terms; two for the largest.
#ifndef CKKS_TENSOR_SMALL_MINB
#define CKKS_TENSOR_SMALL_MINB 4
#endif
template <int MAXT>
struct TensorOcc {
    static constexpr int minb = MAXT <= 4 ? CKKS_TENSOR_SMALL_MINB : MAXT <= 9 ? 3 : 2;
};

template <int MAXT, bool Q1, int V>
__global__ void __launch_bounds__(kThreads, TensorOcc<MAXT>::minb) tensor_kernel(TensorArgs A) {
    const i64 r = ((i64)blockIdx.x * blockDim.x + threadIdx.x) * V;  // limb * N + coefficient
    if (r >= (i64)A.level * A.N) return;
    const int j = (int)(r >> A.log_n);
    tensor_coeff<MAXT, Q1, V>(TensorUniformView{A, (int)blockIdx.y}, r, j, A.mods[j], A.rfix);
}

// Table launch: blockIdx.y = tree node; the node's entry is staged in shared
// memory (it is indexed by child at run time).
template <int MAXT, bool Q1, int V>
__global__ void __launch_bounds__(kThreads, TensorOcc<MAXT>::minb) tensor_table_kernel(const TensorJob *jobs, int N, int log_n,
                                                                const ModQ *mods, const Shoup *rfix) {
    __shared__ TensorJob J;
    {
        // the entry is copied by many threads, one word each
        static_assert(sizeof(TensorJob) % sizeof(u64) == 0, "TensorJob is a whole number of words");
        constexpr int W = sizeof(TensorJob) / sizeof(u64);
        const u64 *src = reinterpret_cast<const u64 *>(jobs + blockIdx.y);
        u64 *dst = reinterpret_cast<u64 *>(&J);
        for (int i = threadIdx.x; i < W; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const i64 r = ((i64)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (r >= (i64)J.level * N) return;
    const int j = (int)(r >> log_n);
    tensor_coeff<MAXT, Q1, V>(TensorTableView{J}, r, j, mods[j], rfix);
}

// 64 x 64 -> 128-bit products per coefficient of a node's tensor product
// (Karatsuba pairs when a ciphertext multiplies the running tuple: 3 per
// pair, 2 for an unpaired term; schoolbook otherwise), plus one reduction
// per term of every intermediate and of the output (counted alike).
double tensor_products_per_coeff(const int *polys, int m) {
    double ops = 0;
    int ncur = polys[0];
    for (int c = 1; c < m; ++c) {
        const int ny = polys[c];
        ops += ny == 2 ? 3.0 * (ncur / 2) + 2.0 * (ncur % 2) : (double)ncur * ny;
        ncur += ny - 1;
        ops += ncur;  // REDC of every term
    }
    // the R^(m-1) correction (Shoup products): on the smallest child's terms
    // (children sorted by size, CKKS_TENSOR_PRESCALE) or on the output's
    int corr = ncur;
    if (CKKS_TENSOR_PRESCALE)
        for (int c = 0; c < m; ++c) corr = std::min(corr, polys[c]);
    return ops + corr;
}

// Tuples of up to 5 terms take two adjacent coefficients per thread
// (16-byte loads and stores) when every pointer is 16-byte aligned and every
// stride even; larger tuples (more live terms per coefficient) one.
#ifndef CKKS_TENSOR_VEC_MAXT
#define CKKS_TENSOR_VEC_MAXT 5
#endif
constexpr int kTensorVecMaxT = CKKS_TENSOR_VEC_MAXT;

template <bool Q1, int V>
static void launch_tensor_sized(int maxt, dim3 blocks, const TensorArgs &A, cudaStream_t st) {
    if (maxt <= 3) tensor_kernel<3, Q1, V><<<blocks, kThreads, 0, st>>>(A);
    else if (maxt <= 4) tensor_kernel<4, Q1, V><<<blocks, kThreads, 0, st>>>(A);
    else if (maxt <= 5 && (V == 1 || kTensorVecMaxT >= 5)) tensor_kernel<5, Q1, V><<<blocks, kThreads, 0, st>>>(A);
    else if constexpr (V == 1) {
        if (maxt <= 7) tensor_kernel<7, Q1, 1><<<blocks, kThreads, 0, st>>>(A);
        else if (maxt <= 9) tensor_kernel<9, Q1, 1><<<blocks, kThreads, 0, st>>>(A);
        else tensor_kernel<CKKS_MAX_TUPLE, Q1, 1><<<blocks, kThreads, 0, st>>>(A);
    }
}

template <bool Q1, int V>
static void launch_tensor_table_sized(const Context &C, int maxt, dim3 blocks, const TensorJob *jobs,
                                      cudaStream_t st) {
#define CKKS_TT(MT, VV) tensor_table_kernel<MT, Q1, VV><<<blocks, kThreads, 0, st>>>(jobs, C.N, C.log_n, C.d_mods, C.d_rfix)
    if (maxt <= 3) CKKS_TT(3, V);
    else if (maxt <= 4) CKKS_TT(4, V);
    else if (maxt <= 5 && (V == 1 || kTensorVecMaxT >= 5)) CKKS_TT(5, V);
    else if constexpr (V == 1) {
        if (maxt <= 7) CKKS_TT(7, 1);
        else if (maxt <= 9) CKKS_TT(9, 1);
        else CKKS_TT(CKKS_MAX_TUPLE, 1);
    }
#undef CKKS_TT
}

static bool view_vec2(const LimbView &v) {
    return ((uintptr_t)v.ptr % 16) == 0 && v.bstride % 2 == 0 && v.pstride % 2 == 0;
}

cudaError_t launch_tensor(const Context &C, const TensorArgs &Ain, cudaStream_t st) {
    TensorArgs A = Ain;
    A.log_n = C.log_n;
    count_kernel(C);
    // children sorted by size, largest first (the smallest, last, takes the
    // R^(m-1) correction); a node shape with a fixed kernel takes it
    int code = tensor_sort_children(A);
    if (!C.tune_tensor_fixed) code = -1;
    int in_polys = 0, maxt = 0;
    bool vec2 = view_vec2(A.out);
    for (int c = 0; c < A.m; ++c) {
        in_polys += A.child_polys[c];
        maxt = std::max(maxt, A.child_polys[c]);
        vec2 = vec2 && view_vec2(A.child[c]);
    }
    int out_polys = in_polys - A.m + 1;
    maxt = std::max(maxt, out_polys);
    vec2 = vec2 && maxt <= kTensorVecMaxT;
    const double coeffs = (double)A.n_batch * A.level * A.N;
    ProfScope ps(C, KC_TENSOR, (double)(in_polys + out_polys) * coeffs * sizeof(u64), st,
                 coeffs * tensor_products_per_coeff(A.child_polys, A.m));
    if (code >= 0) return launch_tensor_fixed(C, A, code, st);
    const i64 per = vec2 ? 2 * kThreads : kThreads;
    dim3 blocks((unsigned)(((i64)A.level * A.N + per - 1) / per), A.n_batch);
    if (vec2) {
        if (C.q1()) launch_tensor_sized<true, 2>(maxt, blocks, A, st);
        else launch_tensor_sized<false, 2>(maxt, blocks, A, st);
    } else {
        if (C.q1()) launch_tensor_sized<true, 1>(maxt, blocks, A, st);
        else launch_tensor_sized<false, 1>(maxt, blocks, A, st);
    }
    return cudaGetLastError();
}

bool tensor_job_vec2(const TensorJob &T) {
    bool ok = ((uintptr_t)T.out % 16) == 0 && T.ostride % 2 == 0;
    for (int c = 0; c < T.m; ++c) ok = ok && ((uintptr_t)T.child[c] % 16) == 0 && T.cstride[c] % 2 == 0;
    return ok;
}

cudaError_t launch_tensor_table(const Context &C, const TensorJob *jobs, int n_jobs, int maxt, int max_level,
                                bool vec2, double bytes, double ops, cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    if (n_jobs > 65535) return cudaErrorInvalidValue;
    vec2 = vec2 && maxt <= kTensorVecMaxT;
    const i64 per = vec2 ? 2 * kThreads : kThreads;
    dim3 blocks((unsigned)(((i64)max_level * C.N + per - 1) / per), (unsigned)n_jobs);
    count_kernel(C);
    ProfScope ps(C, KC_TENSOR, bytes, st, ops);
    if (vec2) {
        if (C.q1()) launch_tensor_table_sized<true, 2>(C, maxt, blocks, jobs, st);
        else launch_tensor_table_sized<false, 2>(C, maxt, blocks, jobs, st);
    } else {
        if (C.q1()) launch_tensor_table_sized<true, 1>(C, maxt, blocks, jobs, st);
        else launch_tensor_table_sized<false, 1>(C, maxt, blocks, jobs, st);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ModUp basis conversion (Eq. 4), coefficient domain:
//   ext[x] = sum_{j in digit} y'_j [(Q_beta / q_j) mod x]   (mod x)
// y'_j = [y_j (Q_beta/q_j)^-1]_{q_j} was produced by the INTT's epilogue.
// blockIdx.y = (t, beta) job, blockIdx.z = batch.
// ---------------------------------------------------------------------------
// Coefficients per thread of the key MAC: four adjacent coefficients read
// with two 16-byte loads per stream (more bytes in flight per thread; the
// kernel is bound by load latency, not by its multiplies). Measured on the
// bench step: 17.5 ms at four, 18.1 at two, 19.4 at one.
#ifndef CKKS_MAC_VEC
#define CKKS_MAC_VEC 4
#endif
// Two products of the same shape per thread share each term's key loads
// (CKKS_MAC_PAIR, rns.h), two coefficients each.
#ifndef CKKS_MAC_VEC_PAIR
#define CKKS_MAC_VEC_PAIR 2
#endif
// Largest key-MAC block (the "mac_threads" tunable's upper bound). At 1024
// the four-coefficient form gets 64 registers and spills 96-196 bytes a
// thread to L1; bounding the block at 512 removed the spills (106
// registers) but cut the resident warps, and the MAC took 20.3 instead of
// 17.5 ms per bench step.
#define CKKS_MAC_MAX_THREADS 1024

// Coefficients per thread of BConv (1: measured fastest; 2 was 3 % slower)
#ifndef CKKS_BCONV_VEC
#define CKKS_BCONV_VEC 1
#endif

// One CTA: the constants of (level, digit) staged in shared memory, then one
// coefficient per thread. y: limb 0 of the prescaled d_t; dst: slot 0 of the
// (t, digit) ModUp output.
template <int AMAX, bool Q1>
__device__ __forceinline__ void bconv_block(const u64 *ctab, const u64 *y0, u64 *dst0, int level, int beta,
                                            int alpha, int L, int K, int n_primes, int N, const ModQ *mods, u64 *cs) {
    const int d0 = beta * alpha;
    int d1 = d0 + alpha;
    if (d1 > level) d1 = level;
    const int na = d1 - d0;
    // targets: Q limbs outside the digit, then every P limb
    const int nq_t = level - na;
    const int n_t = nq_t + K;
    for (int i = threadIdx.x; i < na * n_t; i += blockDim.x) {
        int jj = i / n_t, ti = i % n_t;
        int x = ti < nq_t ? (ti < d0 ? ti : ti + na) : L + (ti - nq_t);
        cs[i] = ctab[(i64)jj * n_primes + x];
    }
    __syncthreads();
    // CKKS_BCONV_VEC adjacent coefficients per thread (16-byte loads and
    // stores for two)
    constexpr int V = CKKS_BCONV_VEC;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (e >= N) return;
    const u64 *ysrc = y0 + e;
    u64 y[AMAX][V];
#pragma unroll
    for (int jj = 0; jj < AMAX; ++jj) {
        if (jj < na) load_span<V>(ysrc + (i64)(d0 + jj) * N, y[jj]);
        else
#pragma unroll
            for (int v = 0; v < V; ++v) y[jj][v] = 0ull;
    }
    u64 *dst = dst0 + e;
    for (int ti = 0; ti < n_t; ++ti) {
        const int slot = ti < nq_t ? (ti < d0 ? ti : ti + na) : level + (ti - nq_t);
        const int x = ti < nq_t ? slot : L + (ti - nq_t);
        const ModQ m = mods[x];
        // sum over the digit: hi stays below q because the digit's primes sum to < 2^64
        Acc128Lazy acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v].zero();
#pragma unroll
        for (int jj = 0; jj < AMAX; ++jj)
            if (jj < na) {
                const u64 c = cs[jj * n_t + ti];
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].mac(y[jj][v], c);
            }
        u64 r[V];
#pragma unroll
        for (int v = 0; v < V; ++v) r[v] = redc_t<Q1>(acc[v].hi, acc[v].lo, m);
        store_span<V>(dst + (i64)slot * N, r);
    }
}

template <int AMAX, bool Q1>
__global__ void __launch_bounds__(1024) bconv_kernel(BconvArgs A) {
    extern __shared__ u64 cs[];  // [alpha][n_targets] Montgomery constants
    const int job = blockIdx.y;
    const int b = blockIdx.z;
    const int t = job / A.n_digits;
    const int beta = job % A.n_digits;
    bconv_block<AMAX, Q1>(A.consts + (i64)beta * A.alpha * A.n_primes,
                      A.y.ptr + (i64)b * A.y.bstride + (i64)t * A.y.pstride,
                      A.ext.ptr + (i64)b * A.ext.bstride + (i64)(t * A.n_digits + beta) * A.ext.pstride, A.level, beta,
                      A.alpha, A.L, A.K, A.n_primes, A.N, A.mods, cs);
}

// Table launch: blockIdx.y = (product, d_t, digit) entry.
template <int AMAX, bool Q1>
__global__ void __launch_bounds__(1024) bconv_table_kernel(const BconvJob *jobs, int alpha, int L, int K,
                                                           int n_primes, int N, const ModQ *mods) {
    extern __shared__ u64 cs[];
    const BconvJob J = jobs[blockIdx.y];
    bconv_block<AMAX, Q1>(J.consts, J.y, J.ext, J.level, J.beta, alpha, L, K, n_primes, N, mods, cs);
}

template <bool Q1>
static void launch_bconv_sized(int alpha, dim3 grid, int thr, size_t smem, const BconvArgs &A, cudaStream_t st) {
    if (alpha <= 4) bconv_kernel<4, Q1><<<grid, thr, smem, st>>>(A);
    else if (alpha <= 8) bconv_kernel<8, Q1><<<grid, thr, smem, st>>>(A);
    else if (alpha <= 12) bconv_kernel<12, Q1><<<grid, thr, smem, st>>>(A);
    else bconv_kernel<16, Q1><<<grid, thr, smem, st>>>(A);
}

template <bool Q1>
static void launch_bconv_table_sized(const Context &C, dim3 grid, int thr, size_t smem, const BconvJob *jobs,
                                     cudaStream_t st) {
    const int np = C.L + C.K;
    if (C.alpha <= 4) bconv_table_kernel<4, Q1><<<grid, thr, smem, st>>>(jobs, C.alpha, C.L, C.K, np, C.N, C.d_mods);
    else if (C.alpha <= 8) bconv_table_kernel<8, Q1><<<grid, thr, smem, st>>>(jobs, C.alpha, C.L, C.K, np, C.N, C.d_mods);
    else if (C.alpha <= 12)
        bconv_table_kernel<12, Q1><<<grid, thr, smem, st>>>(jobs, C.alpha, C.L, C.K, np, C.N, C.d_mods);
    else bconv_table_kernel<16, Q1><<<grid, thr, smem, st>>>(jobs, C.alpha, C.L, C.K, np, C.N, C.d_mods);
}

cudaError_t launch_bconv(const Context &C, const BconvArgs &A, cudaStream_t st) {
    const int thr = C.tune_bconv_threads;
    dim3 grid((A.N + thr * CKKS_BCONV_VEC - 1) / (thr * CKKS_BCONV_VEC), A.n_t * A.n_digits, A.n_batch);
    size_t smem = (size_t)A.alpha * (A.level + A.K) * sizeof(u64);
    count_kernel(C);
    count_op(C, OP_BCONV, (unsigned long long)A.n_t * A.n_digits * A.n_batch);
    // reads y' once, writes level + K - |digit| limbs per (t, digit)
    double limbs_out = (double)A.n_t * ((double)A.n_digits * (A.level + A.K) - A.level);
    // multiply-accumulates: per (t, digit) and coefficient, |digit| per target
    double macs = 0;
    for (int beta = 0; beta < A.n_digits; ++beta) {
        const int na = std::min(A.level, (beta + 1) * A.alpha) - beta * A.alpha;
        macs += (double)na * (A.level - na + A.K);
    }
    macs *= (double)A.n_t * A.n_batch * A.N;
    ProfScope ps(C, KC_BCONV, ((double)A.n_t * A.level + limbs_out) * A.n_batch * A.N * sizeof(u64), st, macs);
    if (C.q1()) launch_bconv_sized<true>(A.alpha, grid, thr, smem, A, st);
    else launch_bconv_sized<false>(A.alpha, grid, thr, smem, A, st);
    return cudaGetLastError();
}

cudaError_t launch_bconv_table(const Context &C, const BconvJob *jobs, int n_jobs, double bytes, double macs,
                               cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    if (n_jobs > 65535) return cudaErrorInvalidValue;
    const int thr = C.tune_bconv_threads;
    dim3 grid((C.N + thr * CKKS_BCONV_VEC - 1) / (thr * CKKS_BCONV_VEC), (unsigned)n_jobs);
    size_t smem = (size_t)C.alpha * (C.L + C.K) * sizeof(u64);
    count_kernel(C);
    count_op(C, OP_BCONV, (unsigned long long)n_jobs);
    ProfScope ps(C, KC_BCONV, bytes, st, macs);
    if (C.q1()) launch_bconv_table_sized<true>(C, grid, thr, smem, jobs, st);
    else launch_bconv_table_sized<false>(C, grid, thr, smem, jobs, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Key inner product summed over every extra key t = 2..n and digit beta
// (Eq. 15 combined before ModDown):
//   acc_l[x] = sum_t sum_beta term(t, beta, x) * ek'_{t,beta,l}[x]
// term = d_t[x] when x lies in digit beta (the digit's own limbs), else the
// ModUp output. Keys are in Montgomery form, so one REDC per output.
// Grid: x = coefficient chunk, y = target limb, z = batch (fastest-varying
// batch would reuse key tiles in L2; see launch order below).
// ---------------------------------------------------------------------------
// V coefficients of accumulator limb x of one product: dsrc / esrc point at
// limb x, coefficient e of the D tuple / the first ModUp output; krow at the
// prime's row, coefficient e, of the first key.
// V coefficients of accumulator limb x of P products of the same shape
// (level, n, digits) at once: the key words of each term are loaded once
// for all P. dsrc / esrc point at limb x, coefficient e of each product's D
// tuple / first ModUp output; krow at the prime's row, coefficient e, of the
// first key.
template <int V, int P, bool Q1>
__device__ __forceinline__ void mac_span(const u64 *const *dsrc, const i64 *dstride, const u64 *const *esrc,
                                         const i64 *estride, int n, int nd, int my_digit, const u64 *krow,
                                         i64 key_pstride, int key_digits, const ModQ m, u64 *const *dst,
                                         const i64 *astride) {
    const u64 q = m.q;
    Acc128 a0[P][V], a1[P][V];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            a0[p][v].zero();
            a1[p][v].zero();
        }
    for (int t = 2; t <= n; ++t) {
        for (int beta = 0; beta < nd; ++beta) {
            const u64 *key = krow + ((i64)((t - 2) * key_digits + beta) * 2) * key_pstride;
            u64 tv[P][V], k0[V], k1[V];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const u64 *src = beta == my_digit ? dsrc[p] + (i64)t * dstride[p]
                                                  : esrc[p] + (i64)((t - 2) * nd + beta) * estride[p];
                load_span<V>(src, tv[p]);
            }
            load_span<V>(key, k0);
            load_span<V>(key + key_pstride, k1);
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    a0[p][v].mac(tv[p][v], k0[v], q);
                    a1[p][v].mac(tv[p][v], k1[v], q);
                }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        u64 r0[V], r1[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            r0[v] = redc_t<Q1>(a0[p][v].hi, a0[p][v].lo, m);
            r1[v] = redc_t<Q1>(a1[p][v].hi, a1[p][v].lo, m);
        }
        store_span<V>(dst[p], r0);
        store_span<V>(dst[p] + astride[p], r1);
    }
}

// Batch elements b_first + g P + p (p < P) of group g; blockIdx.x runs over
// groups fastest, then coefficient chunks, then accumulator limbs, so that
// blocks that share key rows run next to each other.
template <bool Q1, int P, int V>
__global__ void __launch_bounds__(CKKS_MAC_MAX_THREADS) mac_kernel(MacArgs A, int b_first, int n_groups) {
    const int chunks = (A.N + blockDim.x * V - 1) / (blockDim.x * V);
    int bid = blockIdx.x;
    const int g = bid % n_groups;
    bid /= n_groups;
    const int chunk = bid % chunks;
    const int x = bid / chunks;  // acc slot: Q limbs 0..level-1 then P limbs
    const int e = (chunk * blockDim.x + threadIdx.x) * V;
    if (e >= A.N) return;
    const bool isq = x < A.level;
    const int prime = isq ? x : A.L + (x - A.level);
    const i64 off = (i64)x * A.N + e;
    const u64 *ds[P], *es[P];
    u64 *os[P];
    i64 dstr[P], estr[P], astr[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const i64 b = b_first + (i64)g * P + p;
        ds[p] = A.d.ptr + b * A.d.bstride + off;
        es[p] = A.ext.ptr + b * A.ext.bstride + off;
        os[p] = A.acc.ptr + b * A.acc.bstride + off;
        dstr[p] = A.d.pstride;
        estr[p] = A.ext.pstride;
        astr[p] = A.acc.pstride;
    }
    mac_span<V, P, Q1>(ds, dstr, es, estr, A.n, A.n_digits, isq ? x / A.alpha : -1, A.keys + (i64)prime * A.N + e,
                       A.key_pstride, A.key_digits, A.mods[prime], os, astr);
}

template <int P, int V>
static void launch_mac_part(const Context &C, const MacArgs &A, int b_first, int n_groups, cudaStream_t st) {
    const int thr = C.tune_mac_threads;
    const int chunks = (A.N + thr * V - 1) / (thr * V);
    const long long blocks = (long long)chunks * (A.level + A.K) * n_groups;
    count_kernel(C);
    if (C.q1()) mac_kernel<true, P, V><<<(unsigned)blocks, thr, 0, st>>>(A, b_first, n_groups);
    else mac_kernel<false, P, V><<<(unsigned)blocks, thr, 0, st>>>(A, b_first, n_groups);
}

cudaError_t launch_mac(const Context &C, const MacArgs &A, cudaStream_t st) {
    // per batch element: (n-1) * digits terms and 2 outputs per target limb;
    // key limbs counted once per launch
    const double terms = (double)(A.n - 1) * A.n_digits;
    const double limbs = (double)(A.level + A.K);
    double bytes = ((terms + 2.0) * A.n_batch + 2.0 * terms) * limbs * A.N * sizeof(u64);
    const double macs = 2.0 * terms * limbs * A.n_batch * A.N;
    ProfScope ps(C, KC_MAC, bytes, st, macs);
    // pairs of batch elements share the key loads; an odd last one alone
    const int pairs = CKKS_MAC_PAIR ? A.n_batch / 2 : 0;
    if (pairs > 0) launch_mac_part<2, CKKS_MAC_VEC_PAIR>(C, A, 0, pairs, st);
    if (A.n_batch - 2 * pairs > 0) launch_mac_part<1, CKKS_MAC_VEC>(C, A, 2 * pairs, A.n_batch - 2 * pairs, st);
    return cudaGetLastError();
}

// Table launch of the key MAC: blockIdx.x = accumulator limb (products
// job [, job2], x), ordered by prime so that neighbouring blocks read the
// same key rows; blockIdx.y = coefficient chunk. P = 2: the target pairs
// two products of the same shape (job2), which share the key loads.
template <bool Q1, int P, int V>
__global__ void __launch_bounds__(CKKS_MAC_MAX_THREADS) mac_table_kernel(const MacJob *jobs, const MacTarget *targets,
                                                                         const u64 *keys, i64 key_pstride,
                                                                         int key_digits, int alpha, int L, int N,
                                                                         const ModQ *mods) {
    const MacTarget T = targets[blockIdx.x];
    const int e = (blockIdx.y * blockDim.x + threadIdx.x) * V;
    if (e >= N) return;
    const int x = T.x;
    const MacJob J0 = jobs[T.job];
    const bool isq = x < J0.level;
    const int prime = isq ? x : L + (x - J0.level);
    const i64 off = (i64)x * N + e;
    const u64 *ds[P], *es[P];
    u64 *os[P];
    i64 dstr[P], estr[P], astr[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const MacJob J = p == 0 ? J0 : jobs[T.job2];
        ds[p] = J.d + off;
        es[p] = J.ext + off;
        os[p] = J.acc + off;
        dstr[p] = J.dstride;
        estr[p] = J.estride;
        astr[p] = J.astride;
    }
    mac_span<V, P, Q1>(ds, dstr, es, estr, J0.n, J0.nd, isq ? x / alpha : -1, keys + (i64)prime * N + e, key_pstride,
                       key_digits, mods[prime], os, astr);
}

template <int P, int V>
static cudaError_t launch_mac_table_part(const Context &C, const MacJob *jobs, const MacTarget *targets, int n,
                                         const u64 *keys, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int thr = C.tune_mac_threads;
    const int chunks = (C.N + thr * V - 1) / (thr * V);
    if (chunks > 65535) return cudaErrorInvalidValue;
    count_kernel(C);
    dim3 grid((unsigned)n, (unsigned)chunks);
    const i64 kps = (i64)(C.L + C.K) * C.N;
    if (C.q1())
        mac_table_kernel<true, P, V><<<grid, thr, 0, st>>>(jobs, targets, keys, kps, C.dnum, C.alpha, C.L, C.N,
                                                           C.d_mods);
    else
        mac_table_kernel<false, P, V><<<grid, thr, 0, st>>>(jobs, targets, keys, kps, C.dnum, C.alpha, C.L, C.N,
                                                            C.d_mods);
    return cudaGetLastError();
}

cudaError_t launch_mac_table(const Context &C, const MacJob *jobs, const MacTarget *targets, int n_pairs,
                             int n_targets, const u64 *keys, double bytes, double macs, cudaStream_t st) {
    if (n_targets <= 0) return cudaSuccess;
    ProfScope ps(C, KC_MAC, bytes, st, macs);
    cudaError_t e = launch_mac_table_part<2, CKKS_MAC_VEC_PAIR>(C, jobs, targets, n_pairs, keys, st);
    if (e != cudaSuccess) return e;
    return launch_mac_table_part<1, CKKS_MAC_VEC>(C, jobs, targets + n_pairs, n_targets - n_pairs, keys, st);
}

// ---------------------------------------------------------------------------
// Rescale chain among the mu top limbs (coefficient domain), in place:
// a^{(t),{u}} = q_{l-u}^-1 (a^{(t),{u-1}} - a^{(l-u),{u-1}}) mod q_t for
// u = 1..mu-1 and t < l-u (Eq. 6 applied inside Algorithm 1, step 2).
// After it, limb t holds a^{(t),{l-1-t}}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rschain_coeff(u64 *base, int N, int level, int mu, const ModQ *mods, const Shoup *one,
                                              const Shoup *invq) {
    const int l0 = level - mu;
    u64 a[CKKS_MAX_PRIMES];
    for (int t = 0; t < mu; ++t) a[t] = base[(i64)t * N];
    for (int u = 1; u < mu; ++u) {
        const int top = mu - u;  // index of limb level-u
        const int ptop = l0 + top;
        for (int t = 0; t < top; ++t) {
            const int pt = l0 + t;
            const u64 qt = mods[pt].q;
            const Shoup o = one[pt];
            const u64 tr = shoup(a[top], o.w, o.wp, qt);  // a[top] mod q_t
            const Shoup inv = invq[ptop * CKKS_MAX_PRIMES + pt];
            a[t] = shoup(sub_mod(a[t], tr, qt), inv.w, inv.wp, qt);
        }
    }
    for (int t = 0; t < mu - 1; ++t) base[(i64)t * N] = a[t];
}

__global__ void __launch_bounds__(kThreads) rschain_kernel(RsChainArgs A) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 per = (i64)A.n_polys * A.N;
    if (gid >= per * A.n_batch) return;
    const int b = (int)(gid / per);
    const int p = (int)((gid % per) / A.N);
    const int e = (int)(gid % A.N);
    u64 *base = A.v.ptr + (i64)b * A.v.bstride + (i64)p * A.v.pstride + e;  // slot 0 = limb level - mu
    rschain_coeff(base, A.N, A.level, A.mu, A.mods, A.one, A.invq);
}

// Table launch: blockIdx.y = tuple entry, x over its polynomials x coefficients.
__global__ void __launch_bounds__(kThreads) rschain_table_kernel(const RsJob *jobs, int N, const ModQ *mods,
                                                                 const Shoup *one, const Shoup *invq) {
    const RsJob J = jobs[blockIdx.y];
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)J.n_polys * N) return;
    const int p = (int)(gid / N);
    const int e = (int)(gid % N);
    rschain_coeff(J.v + (i64)p * J.pstride + e, N, J.level, J.mu, mods, one, invq);
}

cudaError_t launch_rschain(const Context &C, const RsChainArgs &A, cudaStream_t st) {
    if (A.mu < 2) return cudaSuccess;
    i64 total = (i64)A.n_batch * A.n_polys * A.N;
    count_kernel(C);
    ProfScope ps(C, KC_RSCHAIN, 2.0 * A.n_batch * A.n_polys * A.mu * A.N * sizeof(u64), st);
    rschain_kernel<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_rschain_table(const Context &C, const RsJob *jobs, int n_jobs, int max_polys, double bytes,
                                 cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    if (n_jobs > 65535) return cudaErrorInvalidValue;
    count_kernel(C);
    ProfScope ps(C, KC_RSCHAIN, bytes, st);
    dim3 grid((unsigned)(((i64)max_polys * C.N + kThreads - 1) / kThreads), (unsigned)n_jobs);
    rschain_table_kernel<<<grid, kThreads, 0, st>>>(jobs, C.N, C.d_mods, C.d_one, C.d_invq);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
// In place: v <- v * fold[x] R^-1, fold = P^-1 R^2 on Q limbs, R^2 on P
// limbs, giving the Montgomery form of P^-1 ek (Q limbs) or ek (P limbs).
__global__ void __launch_bounds__(kThreads) keyprep_kernel(u64 *keys, i64 n_rows, int n_primes, int N,
                                                           const ModQ *mods, const u64 *fold) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_rows * N) return;
    const int x = (int)((gid / N) % n_primes);
    keys[gid] = mont_mul(keys[gid], fold[x], mods[x]);
}

cudaError_t launch_keyprep(const Context &C, u64 *keys, long long n_rows, cudaStream_t st) {
    i64 total = n_rows * C.N;
    count_kernel(C);
    keyprep_kernel<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        keys, n_rows, C.L + C.K, C.N, C.d_mods, C.d_keyfold);
    return cudaGetLastError();
}

// Small signed coefficients -> residues for every prime: out[x][i] = v[i] mod prime_x.
__global__ void __launch_bounds__(kThreads) signed_to_res_kernel(const i64 *v, u64 *out, int n_primes, int N,
                                                                 const ModQ *mods) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)n_primes * N) return;
    const int x = (int)(gid / N);
    const int i = (int)(gid % N);
    const i64 s = v[i];
    const u64 q = mods[x].q;
    const u64 r = s >= 0 ? ((u64)s) % q : ((u64)(-s)) % q;
    out[gid] = (s >= 0 || r == 0) ? r : q - r;
}

cudaError_t launch_signed_to_res(const Context &C, const long long *v, u64 *out, cudaStream_t st) {
    i64 total = (i64)(C.L + C.K) * C.N;
    count_kernel(C);
    signed_to_res_kernel<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        (const i64 *)v, out, C.L + C.K, C.N, C.d_mods);
    return cudaGetLastError();
}

__device__ __forceinline__ u64 mulmod_full(u64 a, u64 b, ModQ m, u64 r2) {
    return mont_mul(mont_mul(a, b, m), r2, m);
}

// St <- St * S (pointwise, every prime)
__global__ void __launch_bounds__(kThreads) pointwise_mul_kernel(u64 *St, const u64 *S, int n_primes, int N,
                                                                 const ModQ *mods, const u64 *r2) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)n_primes * N) return;
    const int x = (int)(gid / N);
    St[gid] = mulmod_full(St[gid], S[gid], mods[x], r2[x]);
}

cudaError_t launch_pointwise_mul(const Context &C, u64 *St, const u64 *S, cudaStream_t st) {
    i64 total = (i64)(C.L + C.K) * C.N;
    count_kernel(C);
    pointwise_mul_kernel<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        St, S, C.L + C.K, C.N, C.d_mods, C.d_r2);
    return cudaGetLastError();
}

// dst <- dst + src over [batch][polys][level][N] limb views (limb x mod q_x)
__global__ void __launch_bounds__(kThreads) add_limbs_kernel(LimbView dst, LimbView src, int polys, int level, int N,
                                                             const ModQ *mods) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 per_poly = (i64)level * N;
    if (gid >= per_poly * polys) return;
    const int b = blockIdx.y;
    const int p = (int)(gid / per_poly);
    const i64 r = gid % per_poly;
    const int x = (int)(r / N);
    u64 *d = dst.ptr + (i64)b * dst.bstride + (i64)p * dst.pstride + r;
    const u64 v = src.ptr[(i64)b * src.bstride + (i64)p * src.pstride + r];
    *d = add_mod(*d, v, mods[x].q);
}

cudaError_t launch_add_limbs(const Context &C, LimbView dst, LimbView src, int batch, int polys, int level,
                             cudaStream_t st) {
    const i64 total = (i64)polys * level * C.N;
    if (total == 0 || batch == 0) return cudaSuccess;
    count_kernel(C);
    dim3 grid((unsigned)((total + kThreads - 1) / kThreads), (unsigned)batch);
    add_limbs_kernel<<<grid, kThreads, 0, st>>>(dst, src, polys, level, C.N, C.d_mods);
    return cudaGetLastError();
}

// ek0 = E - a S + [P G_beta]_x S^t,  ek1 = a   (all L + K limbs, NTT domain)
__global__ void __launch_bounds__(kThreads) keygen_kernel(const u64 *S, const u64 *St, const u64 *E, const u64 *a,
                                                          u64 *ek, int n_primes, int N, const ModQ *mods,
                                                          const u64 *r2, const Shoup *pg) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 plane = (i64)n_primes * N;
    if (gid >= plane) return;
    const int x = (int)(gid / N);
    const ModQ m = mods[x];
    const u64 q = m.q;
    u64 as = mulmod_full(a[gid], S[gid], m, r2[x]);
    u64 v = sub_mod(E[gid], as, q);
    const Shoup c = pg[x];
    v = add_mod(v, shoup(St[gid], c.w, c.wp, q), q);
    ek[gid] = v;
    ek[plane + gid] = a[gid];
}

cudaError_t launch_keygen(const Context &C, const u64 *S, const u64 *St, const u64 *E, const u64 *a, u64 *ek,
                          int beta, cudaStream_t st) {
    i64 total = (i64)(C.L + C.K) * C.N;
    count_kernel(C);
    keygen_kernel<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        S, St, E, a, ek, C.L + C.K, C.N, C.d_mods, C.d_r2, C.d_pgadget + (i64)beta * (C.L + C.K));
    return cudaGetLastError();
}

}  // namespace ckks
