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
#include <algorithm>

#include "../../include/ckks_mulk.h"
#include "engine.h"
#include "internal.h"
#include "rns.h"

using namespace ckks;


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

// Garner lift of (x0 mod q0, x1 mod q1) to [0, q0 q1), centred, as double.
__global__ void crt2_kernel(const u64 *P, double *out, int limbs, int N, u64 q0, u64 q1, Shoup q0inv_mod_q1,
                            u64 one_q1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    P += (i64)blockIdx.y * limbs * N;  // batch element
    out += (i64)blockIdx.y * N;
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

struct Src4 {
    const i64 *p[4];
};

// signed [4][batch][N] (v, e0, e1, m) -> W[b][p][x][N] residues, x < level;
// blockIdx.y = b * 4 + p
__global__ void signed4_kernel(Src4 src, u64 *W, int level, int N, const ModQ *mods) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)level * N) return;
    const int b = blockIdx.y / 4, p = blockIdx.y % 4;
    const int x = (int)(gid / N), i = (int)(gid % N);
    const i64 v = src.p[p][(i64)b * N + i];
    const u64 q = mods[x].q;
    const u64 r = v >= 0 ? ((u64)v) % q : ((u64)(-v)) % q;
    W[((i64)blockIdx.y * level) * N + gid] = (v >= 0 || r == 0) ? r : q - r;
}

// c0 = V pk0 + E0 + M, c1 = V pk1 + E1 for every batch element (blockIdx.y)
__global__ void enc_batch_kernel(const u64 *W, const u64 *pk, i64 pk_pstride, u64 *out, i64 out_bstride,
                                 i64 out_pstride, int level, int N, const ModQ *mods, const u64 *r2) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)level * N) return;
    const int b = blockIdx.y;
    const int x = (int)(gid / N);
    const ModQ m = mods[x];
    const u64 q = m.q;
    const i64 plane = (i64)level * N;
    const u64 *w = W + (i64)b * 4 * plane + gid;  // V, E0, E1, M
    u64 *c0 = out + (i64)b * out_bstride + gid, *c1 = c0 + out_pstride;
    *c0 = add_mod(add_mod(mulmod_full(w[0], pk[gid], m, r2[x]), w[plane], q), w[3 * plane], q);
    *c1 = add_mod(mulmod_full(w[0], pk[pk_pstride + gid], m, r2[x]), w[2 * plane], q);
}

// P[b][x] = C0 + C1 S over the lowest `limbs` limbs of every batch element
__global__ void dec_batch_kernel(const u64 *ct, i64 bstride, i64 pstride, const u64 *S, u64 *P, int limbs, int N,
                                 const ModQ *mods, const u64 *r2) {
    const i64 gid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (i64)limbs * N) return;
    const int b = blockIdx.y;
    const int x = (int)(gid / N);
    const ModQ m = mods[x];
    const u64 *c0 = ct + (i64)b * bstride + gid;
    P[(i64)b * limbs * N + gid] = add_mod(c0[0], mulmod_full(c0[pstride], S[gid], m, r2[x]), m.q);
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

size_t enc_batch_ws(const Context &C, uint32_t level, uint32_t batch) {
    const uint32_t chunk = std::min<uint32_t>(16383u, 65535u / (4u * level));
    return (size_t)std::min(batch, chunk) * 4 * level * C.N * sizeof(u64);
}

size_t dec_batch_ws(const Context &C, uint32_t batch) {
    return ((size_t)(C.L + C.K) * C.N + (size_t)batch * 2 * C.N) * sizeof(u64);
}

// evenly spaced tuple array: batch stride in elements, -1 if not
i64 spacing(const ckks_tuple *t, uint32_t batch) {
    const i64 bs = batch > 1 ? (i64)(t[1].data - t[0].data) : 0;
    for (uint32_t b = 0; b < batch; ++b)
        if (t[b].data != t[0].data + b * bs) return -1;
    return bs;
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

int ckks_encrypt_batch_workspace_size(const ckks_context *ctx, uint32_t level, uint32_t batch, size_t *bytes) {
    if (!ctx || !bytes || batch < 1) return CKKS_EINVAL;
    if (level < 1 || level > (uint32_t)ctx->c.L) return CKKS_ELEVEL;
    *bytes = enc_batch_ws(ctx->c, level, batch);
    return CKKS_OK;
}

int ckks_encrypt_batch(ckks_context *ctx, const int64_t *m, const int64_t *v, const int64_t *e0, const int64_t *e1,
                       uint32_t batch, const uint64_t *pk, uint32_t level, ckks_tuple *out, void *workspace,
                       size_t ws_bytes, void *stream) {
    if (!ctx || !m || !v || !e0 || !e1 || !pk || !out || !workspace || batch < 1) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (level < 1 || level > (uint32_t)C.L) return CKKS_ELEVEL;
    for (uint32_t b = 0; b < batch; ++b) {
        if (!out[b].data) return CKKS_EINVAL;
        if (out[b].poly_stride == 0) out[b].poly_stride = level;
        if (out[b].poly_stride < level || out[b].poly_stride != out[0].poly_stride) return CKKS_EINVAL;
    }
    const i64 os = spacing(out, batch);
    if (os < 0 || (batch > 1 && os == 0)) return CKKS_EINVAL;
    if (ws_bytes < enc_batch_ws(C, level, batch)) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t chunk = std::min<uint32_t>(16383u, 65535u / (4u * level));
    const i64 N = C.N, ps = (i64)out[0].poly_stride * N;
    u64 *W = (u64 *)workspace;
    cudaError_t err = cudaSuccess;
    for (uint32_t b0 = 0; b0 < batch && err == cudaSuccess; b0 += chunk) {
        const uint32_t cb = std::min(chunk, batch - b0);
        Src4 src{{(const i64 *)v + b0 * N, (const i64 *)e0 + b0 * N, (const i64 *)e1 + b0 * N,
                  (const i64 *)m + b0 * N}};
        count_kernel(C);
        signed4_kernel<<<dim3(blocks((i64)level * N), cb * 4), kThr, 0, st>>>(src, W, (int)level, C.N, C.d_mods);
        err = cudaGetLastError();
        if (err == cudaSuccess) {
            LimbView w{W, 4 * (i64)level * N, (i64)level * N};
            err = transform_plain(C, true, (int)cb, 4, (int)level, w, w, st);
        }
        if (err == cudaSuccess) {
            count_kernel(C);
            enc_batch_kernel<<<dim3(blocks((i64)level * N), cb), kThr, 0, st>>>(
                W, (const u64 *)pk, (i64)C.L * N, (u64 *)out[b0].data, os, ps, (int)level, C.N, C.d_mods, C.d_r2);
            err = cudaGetLastError();
        }
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    for (uint32_t b = 0; b < batch; ++b) {
        out[b].n_polys = 2;
        out[b].level = level;
        out[b].ntt_form = 1;
    }
    return CKKS_OK;
}

int ckks_encrypt(ckks_context *ctx, const int64_t *m, const int64_t *v, const int64_t *e0, const int64_t *e1,
                 const uint64_t *pk, uint32_t level, ckks_tuple *out, void *workspace, size_t ws_bytes,
                 void *stream) {
    return ckks_encrypt_batch(ctx, m, v, e0, e1, 1, pk, level, out, workspace, ws_bytes, stream);
}

int ckks_decrypt_batch_workspace_size(const ckks_context *ctx, uint32_t batch, size_t *bytes) {
    if (!ctx || !bytes || batch < 1) return CKKS_EINVAL;
    *bytes = dec_batch_ws(ctx->c, batch);
    return CKKS_OK;
}

int ckks_decrypt_batch(ckks_context *ctx, const ckks_tuple *ct, uint32_t batch, const int64_t *s, double *out,
                       void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !ct || !s || !out || !workspace || batch < 1 || batch > 32767) return CKKS_EINVAL;
    const Context &C = ctx->c;
    for (uint32_t b = 0; b < batch; ++b) {
        if (!ct[b].data || ct[b].n_polys != 2 || !ct[b].ntt_form || ct[b].level < 1 ||
            ct[b].level > (uint32_t)C.L || ct[b].poly_stride < ct[b].level || ct[b].level != ct[0].level ||
            ct[b].poly_stride != ct[0].poly_stride)
            return CKKS_EINVAL;
    }
    const i64 cs = spacing(ct, batch);
    if (cs < 0) return CKKS_EINVAL;
    if (ws_bytes < dec_batch_ws(C, batch)) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    const int limbs = ct[0].level >= 2 ? 2 : 1;
    const i64 N = C.N;
    u64 *S = (u64 *)workspace, *P = S + (size_t)(C.L + C.K) * N;
    cudaError_t err = launch_signed_to_res(C, (const long long *)s, S, st);
    if (err == cudaSuccess) err = ntt_limbs(C, S, limbs, st);
    if (err == cudaSuccess) {
        count_kernel(C);
        dec_batch_kernel<<<dim3(blocks((i64)limbs * N), batch), kThr, 0, st>>>(
            (const u64 *)ct[0].data, cs, (i64)ct[0].poly_stride * N, S, P, limbs, C.N, C.d_mods, C.d_r2);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) {
        LimbView v{P, (i64)limbs * N, (i64)limbs * N};
        err = transform_plain(C, false, (int)batch, 1, limbs, v, v, st);
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
        crt2_kernel<<<dim3(blocks(N), batch), kThr, 0, st>>>(P, out, limbs, C.N, q0, q1, inv, one_q1);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

int ckks_decrypt(ckks_context *ctx, const ckks_tuple *ct, const int64_t *s, double *out, void *workspace,
                 size_t ws_bytes, void *stream) {
    return ckks_decrypt_batch(ctx, ct, 1, s, out, workspace, ws_bytes, stream);
}

}  // extern "C"
