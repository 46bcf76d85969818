// Argument blocks of the coefficient-wise RNS kernels (rns.cu).
#pragma once
#include "common.cuh"

namespace ckks {

struct Context;

#define CKKS_MAX_CHILDREN 12

struct TensorArgs {
    int n_batch, level, N, m, log_n;
    LimbView child[CKKS_MAX_CHILDREN];   // limb j of poly a: ptr + b bstride + a pstride + j N
    int child_polys[CKKS_MAX_CHILDREN];
    LimbView out;
    const ModQ *mods;
    const Shoup *rfix;                   // [prime][16] R^(e-1) mod prime (Shoup constants)
};

struct BconvArgs {
    int n_batch, N, level, L, K, alpha, n_digits, n_t, n_primes;
    LimbView y;      // [b][t][level][N] prescaled INTT outputs
    LimbView ext;    // [b][t * n_digits + beta][level + K][N]
    const u64 *consts;  // this level's [dnum][alpha][L+K] Montgomery constants
    const ModQ *mods;
};

struct MacArgs {
    int n_batch, N, level, L, K, alpha, n_digits, key_digits, n;
    LimbView d;      // D tuple [b][n+1][level][N] (NTT domain)
    LimbView ext;    // ModUp outputs
    LimbView acc;    // [b][2][level + K][N]
    const u64 *keys; // [t-2][dnum][2][L+K][N] prepared keys
    i64 key_pstride; // (L+K) N
    const ModQ *mods;
};

struct RsChainArgs {
    int n_batch, n_polys, N, level, mu;
    LimbView v;      // slot 0 = limb level-mu of each poly
    const ModQ *mods;
    const Shoup *one;
    const Shoup *invq;
};

// Output polynomial p of an automorphism launch is sigma_g of input
// polynomial src[p], or zero where src[p] < 0.
struct AutoMap {
    int n_out;
    int src[16];
};

// Cross-shape launches: entries of different products, levels and tree
// nodes of one context in one launch, read from device tables.
struct TensorJob {                       // one tree node of one product
    const u64 *child[CKKS_MAX_CHILDREN]; // limb 0 of polynomial 0 of each child
    i64 cstride[CKKS_MAX_CHILDREN];      // polynomial stride of each child (elements)
    int cpolys[CKKS_MAX_CHILDREN];
    u64 *out;                            // limb 0 of polynomial 0 of the product tuple
    i64 ostride;
    int m, level;
};

struct RsJob {                           // the mu top limbs of every polynomial of one tuple
    u64 *v;                              // limb level - mu of polynomial 0
    i64 pstride;
    int n_polys, level, mu, pad;
};

struct BconvJob {                        // one (d_t, digit) of one product
    const u64 *y;                        // prescaled INTT of d_t, limb 0
    u64 *ext;                            // ModUp output tuple of (t, digit), slot 0
    const u64 *consts;                   // [alpha][L+K] constants of (level, digit)
    int level, beta;
};

struct MacJob {                          // the key MAC of one product
    const u64 *d;                        // D tuple (NTT domain), polynomial t at d + t dstride
    i64 dstride;
    const u64 *ext;                      // ModUp output (t, digit) at ext + ((t-2) nd + digit) estride
    i64 estride;
    u64 *acc;                            // [2][level + K] accumulators, polynomial stride astride
    i64 astride;
    int level, n, nd, pad;
};

// 1: the key MAC takes two products of the same shape per thread, so that
// each key word is loaded once for both (the keys were otherwise re-read
// from L2 for every product: seven times the kernel's DRAM bytes went
// through L2); 0: one product per thread
#ifndef CKKS_MAC_PAIR
#define CKKS_MAC_PAIR 1
#endif

struct MacTarget {                       // accumulator limb x of product `job` (and of `job2`, of the same
    int job, x, job2, pad;               // shape, when the target pairs two products; else job2 = -1)
};

// Where a tensor-product CTA finds its children and output: the uniform
// batch of a launch (TensorArgs, batch element b) or one table entry.
struct TensorUniformView {
    const TensorArgs &A;
    int b;
    __device__ __forceinline__ int m() const { return A.m; }
    __device__ __forceinline__ int polys(int c) const { return A.child_polys[c]; }
    __device__ __forceinline__ const u64 *src(int c) const { return A.child[c].ptr + (i64)b * A.child[c].bstride; }
    __device__ __forceinline__ i64 pstride(int c) const { return A.child[c].pstride; }
    __device__ __forceinline__ u64 *dst() const { return A.out.ptr + (i64)b * A.out.bstride; }
    __device__ __forceinline__ i64 dstride() const { return A.out.pstride; }
};

struct TensorTableView {
    const TensorJob &J;
    __device__ __forceinline__ int m() const { return J.m; }
    __device__ __forceinline__ int polys(int c) const { return J.cpolys[c]; }
    __device__ __forceinline__ const u64 *src(int c) const { return J.child[c]; }
    __device__ __forceinline__ i64 pstride(int c) const { return J.cstride[c]; }
    __device__ __forceinline__ u64 *dst() const { return J.out; }
    __device__ __forceinline__ i64 dstride() const { return J.ostride; }
};

cudaError_t launch_tensor(const Context &C, const TensorArgs &A, cudaStream_t st);
// Node shapes with exactly unrolled tensor kernels (children sorted by
// tuple size, largest first; c = 0 for two children): two children of 4..7
// terms (codes 0..9) except 6 and 4 (children of 5 and 3 inputs: no tree
// within the depth rule has that node for k <= 16), three of 4 or 5 terms
// (codes 10..13); -1 otherwise.
__host__ __device__ inline int tensor_fixed_code(int m, int a, int b, int c) {
    if (m == 2 && b >= 4 && b <= a && a <= 7 && !(a == 6 && b == 4)) return (a - 4) * (a - 3) / 2 + (b - 4);
    if (m == 3 && c >= 4 && c <= b && b <= a && a <= 5) return 10 + (a - 4) + (b - 4) + (c - 4);
    return -1;
}
// The node's children sorted by tuple size, largest first (the product is
// commutative, so the order does not change the result); the shape code of
// the sorted node, -1 when no fixed kernel covers it.
int tensor_sort_children(TensorJob &T);
int tensor_sort_children(TensorArgs &A);
// Uniform launch of a node of shape `code` (children sorted); the caller
// counts and times it.
cudaError_t launch_tensor_fixed(const Context &C, const TensorArgs &A, int code, cudaStream_t st);
// vec2: every entry's pointers are 16-byte aligned and its strides even
// (tensor_job_vec2), so tuples of up to 5 terms may take two coefficients
// per thread
bool tensor_job_vec2(const TensorJob &T);
cudaError_t launch_tensor_table(const Context &C, const TensorJob *jobs, int n_jobs, int maxt, int max_level,
                                bool vec2, double bytes, double ops, cudaStream_t st);
// Table launch of nodes that all have the (sorted) shape `code`.
cudaError_t launch_tensor_fixed_table(const Context &C, const TensorJob *jobs, int n_jobs, int code, int max_level,
                                      double bytes, double ops, cudaStream_t st);
double tensor_products_per_coeff(const int *polys, int m);
cudaError_t launch_rschain_table(const Context &C, const RsJob *jobs, int n_jobs, int max_polys, double bytes,
                                 cudaStream_t st);
cudaError_t launch_bconv_table(const Context &C, const BconvJob *jobs, int n_jobs, double bytes, double macs,
                               cudaStream_t st);
// targets[0 .. n_pairs) pair two products (job2 >= 0), the rest are single
cudaError_t launch_mac_table(const Context &C, const MacJob *jobs, const MacTarget *targets, int n_pairs,
                             int n_targets, const u64 *keys, double bytes, double macs, cudaStream_t st);
cudaError_t launch_bconv(const Context &C, const BconvArgs &A, cudaStream_t st);
cudaError_t launch_mac(const Context &C, const MacArgs &A, cudaStream_t st);
cudaError_t launch_rschain(const Context &C, const RsChainArgs &A, cudaStream_t st);
cudaError_t launch_keyprep(const Context &C, u64 *keys, long long n_rows, cudaStream_t st);
cudaError_t launch_signed_to_res(const Context &C, const long long *v, u64 *out, cudaStream_t st);
cudaError_t launch_pointwise_mul(const Context &C, u64 *St, const u64 *S, cudaStream_t st);
cudaError_t launch_automorphism(const Context &C, LimbView in, LimbView out, const AutoMap &map, int batch,
                                int level, uint32_t g, cudaStream_t st);
// integrity checks (check.cu): residues >= q are counted into C.d_check[0];
// the checksum of n words is added to *out (device)
cudaError_t launch_range_check(const Context &C, LimbView v, int batch, int polys, int level, cudaStream_t st);
cudaError_t launch_checksum(const Context &C, const u64 *w, long long n, unsigned long long *out, cudaStream_t st);
cudaError_t launch_add_limbs(const Context &C, LimbView dst, LimbView src, int batch, int polys, int level,
                             cudaStream_t st);
cudaError_t launch_keygen(const Context &C, const u64 *S, const u64 *St, const u64 *E, const u64 *a, u64 *ek,
                          int beta, cudaStream_t st);

}  // namespace ckks
