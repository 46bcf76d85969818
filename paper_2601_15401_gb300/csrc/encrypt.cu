// Steps on either side of the multiplication (Section II): public key,
// encryption and decryption, on the device.
//
//   pk = (-a s + e, a)                        a uniform (NTT domain), s, e small
//   ct = (v pk_0 + e_0 + m, v pk_1 + e_1)     v, e_0, e_1 small, m the message
//   m' = c_0 + c_1 s                          over the two lowest limbs, lifted
//                                             by CRT (Garner, exact 128-bit) and
//                                             centred, as a double
// Everything is in the NTT domain except the small signed inputs, which are
// reduced into every limb and transformed by the library's NTT.
#include "../../include/ckks_mulk.h"
#include "engine.h"
#include "internal.h"
#include "rns.h"

using namespace ckks;

struct ckks_context {
    Context c;
};

namespace {

constexpr int kThr = 256;

__device__ __forceinline__ u64 mulmod_full(u64 a, u64 b, ModQ m, u64 r2) {
    return mont_mul(mont_mul(a, b, m), r2, m);
}

// pk0 = E - a S over `limbs` limbs (prime index = limb index)
__global__ void pk_kernel(const u64 *S, const u64 *E, const u64 *a, u64 *pk, int limbs, int N, const ModQ *mods,
                          const u64 *r2) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 plane = (i64)limbs * N;
    if (gid >= plane) return;
    const int x = (int)(gid / N);
    const ModQ m = mods[x];
    pk[gid] = sub_mod(E[gid], mulmod_full(a[gid], S[gid], m, r2[x]), m.q);
    pk[plane + gid] = a[gid];
}

// c0 = V pk0 + E0 + M, c1 = V pk1 + E1
__global__ void enc_kernel(const u64 *V, const u64 *E0, const u64 *E1, const u64 *M, const u64 *pk, i64 pk_pstride,
                           u64 *c0, u64 *c1, int limbs, int N, const ModQ *mods, const u64 *r2) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)limbs * N) return;
    const int x = (int)(gid / N);
    const ModQ m = mods[x];
    const u64 q = m.q;
    c0[gid] = add_mod(add_mod(mulmod_full(V[gid], pk[gid], m, r2[x]), E0[gid], q), M[gid], q);
    c1[gid] = add_mod(mulmod_full(V[gid], pk[pk_pstride + gid], m, r2[x]), E1[gid], q);
}

// P = C0 + C1 S over the lowest `limbs` limbs
__global__ void dec_kernel(const u64 *c0, const u64 *c1, const u64 *S, u64 *P, int limbs, int N, const ModQ *mods,
                           const u64 *r2) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)limbs * N) return;
    const int x = (int)(gid / N);
    const ModQ m = mods[x];
    P[gid] = add_mod(c0[gid], mulmod_full(c1[gid], S[gid], m, r2[x]), m.q);
}

// Garner lift of (x0 mod q0, x1 mod q1) to [0, q0 q1), centred, as double.
__global__ void crt2_kernel(const u64 *P, double *out, int limbs, int N, u64 q0, u64 q1, Shoup q0inv_mod_q1,
                            u64 one_q1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const u64 x0 = P[i];
    if (limbs == 1) {
        out[i] = x0 > q0 / 2 ? -(double)(q0 - x0) : (double)x0;
        return;
    }
    const u64 x1 = P[N + i];
    const u64 x0r = shoup(x0, 1, one_q1, q1);  // x0 mod q1
    const u64 t = shoup(sub_mod(x1, x0r, q1), q0inv_mod_q1.w, q0inv_mod_q1.wp, q1);
    // x = x0 + q0 t < q0 q1 < 2^122
    unsigned __int128 x = (unsigned __int128)q0 * t + x0;
    const unsigned __int128 Q = (unsigned __int128)q0 * q1;
    if (x > Q / 2) {
        const unsigned __int128 y = Q - x;
        out[i] = -((double)(u64)(y >> 64) * 18446744073709551616.0 + (double)(u64)y);
    } else {
        out[i] = (double)(u64)(x >> 64) * 18446744073709551616.0 + (double)(u64)x;
    }
}

unsigned blocks(i64 n) { return (unsigned)((n + kThr - 1) / kThr); }

// NTT of `limbs` limbs in place (prime index = limb index)
cudaError_t ntt_limbs(const Context &C, u64 *buf, int limbs, cudaStream_t st) {
    LimbView v{buf, 0, (i64)limbs * C.N};
    return transform_plain(C, true, 1, 1, limbs, v, v, st);
}

u64 host_inv(u64 a, u64 q) {
    unsigned __int128 r = 1, b = a % q;
    u64 e = q - 2;
    while (e) {
        if (e & 1) r = r * b % q;
        b = b * b % q;
        e >>= 1;
    }
    return (u64)r;
}

}  // namespace

extern "C" {

int ckks_encrypt_workspace_size(const ckks_context *ctx, size_t *bytes) {
    if (!ctx || !bytes) return CKKS_EINVAL;
    *bytes = (size_t)4 * (ctx->c.L + ctx->c.K) * ctx->c.N * sizeof(u64);
    return CKKS_OK;
}

int ckks_public_key(ckks_context *ctx, const int64_t *s, const uint64_t *a, const int64_t *e, uint64_t *pk,
                    void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !s || !a || !e || !pk || !workspace) return CKKS_EINVAL;
    const Context &C = ctx->c;
    size_t need;
    ckks_encrypt_workspace_size(ctx, &need);
    if (ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)(C.L + C.K) * C.N;
    u64 *S = (u64 *)workspace, *E = S + plane;
    cudaError_t err = launch_signed_to_res(C, (const long long *)s, S, st);
    if (err == cudaSuccess) err = launch_signed_to_res(C, (const long long *)e, E, st);
    if (err == cudaSuccess) err = ntt_limbs(C, S, C.L, st);
    if (err == cudaSuccess) err = ntt_limbs(C, E, C.L, st);
    if (err == cudaSuccess) {
        count_kernel(C);
        pk_kernel<<<blocks((i64)C.L * C.N), kThr, 0, st>>>(S, E, (const u64 *)a, (u64 *)pk, C.L, C.N, C.d_mods, C.d_r2);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

int ckks_encrypt(ckks_context *ctx, const int64_t *m, const int64_t *v, const int64_t *e0, const int64_t *e1,
                 const uint64_t *pk, uint32_t level, ckks_tuple *out, void *workspace, size_t ws_bytes,
                 void *stream) {
    if (!ctx || !m || !v || !e0 || !e1 || !pk || !out || !out->data || !workspace) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (level < 1 || level > (uint32_t)C.L) return CKKS_ELEVEL;
    if (out->poly_stride == 0) out->poly_stride = level;
    if (out->poly_stride < level) return CKKS_EINVAL;
    size_t need;
    ckks_encrypt_workspace_size(ctx, &need);
    if (ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)(C.L + C.K) * C.N;
    u64 *V = (u64 *)workspace, *E0 = V + plane, *E1 = E0 + plane, *M = E1 + plane;
    const int64_t *src[4] = {v, e0, e1, m};
    u64 *dst[4] = {V, E0, E1, M};
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < 4 && err == cudaSuccess; ++i) {
        err = launch_signed_to_res(C, (const long long *)src[i], dst[i], st);
        if (err == cudaSuccess) err = ntt_limbs(C, dst[i], (int)level, st);
    }
    if (err == cudaSuccess) {
        u64 *c0 = (u64 *)out->data, *c1 = c0 + (size_t)out->poly_stride * C.N;
        count_kernel(C);
        enc_kernel<<<blocks((i64)level * C.N), kThr, 0, st>>>(V, E0, E1, M, (const u64 *)pk, (i64)C.L * C.N, c0, c1,
                                                              (int)level, C.N, C.d_mods, C.d_r2);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    out->n_polys = 2;
    out->level = level;
    out->ntt_form = 1;
    return CKKS_OK;
}

int ckks_decrypt(ckks_context *ctx, const ckks_tuple *ct, const int64_t *s, double *out, void *workspace,
                 size_t ws_bytes, void *stream) {
    if (!ctx || !ct || !ct->data || !s || !out || !workspace) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (ct->n_polys != 2 || !ct->ntt_form || ct->level < 1 || ct->level > (uint32_t)C.L ||
        ct->poly_stride < ct->level)
        return CKKS_EINVAL;
    size_t need;
    ckks_encrypt_workspace_size(ctx, &need);
    if (ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    const int limbs = ct->level >= 2 ? 2 : 1;
    const size_t plane = (size_t)(C.L + C.K) * C.N;
    u64 *S = (u64 *)workspace, *P = S + plane;
    cudaError_t err = launch_signed_to_res(C, (const long long *)s, S, st);
    if (err == cudaSuccess) err = ntt_limbs(C, S, limbs, st);
    if (err == cudaSuccess) {
        const u64 *c0 = (const u64 *)ct->data, *c1 = c0 + (size_t)ct->poly_stride * C.N;
        count_kernel(C);
        dec_kernel<<<blocks((i64)limbs * C.N), kThr, 0, st>>>(c0, c1, S, P, limbs, C.N, C.d_mods, C.d_r2);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) {
        LimbView v{P, 0, (i64)limbs * C.N};
        err = transform_plain(C, false, 1, 1, limbs, v, v, st);
    }
    if (err == cudaSuccess) {
        const u64 q0 = C.primes[0], q1 = limbs > 1 ? C.primes[1] : 1;
        Shoup inv{0, 0};
        u64 one_q1 = 0;
        if (limbs > 1) {
            inv.w = host_inv(q0 % q1, q1);
            inv.wp = (u64)(((unsigned __int128)inv.w << 64) / q1);
            one_q1 = (u64)(((unsigned __int128)1 << 64) / q1);
        }
        count_kernel(C);
        crt2_kernel<<<blocks(C.N), kThr, 0, st>>>(P, out, limbs, C.N, q0, q1, inv, one_q1);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

}  // extern "C"
