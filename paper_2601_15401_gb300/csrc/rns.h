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
    const u64 *rpow;                     // [prime][16] R^e
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

cudaError_t launch_tensor(const Context &C, const TensorArgs &A, cudaStream_t st);
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
