// Canonical-embedding encoding and decoding (Section II) on the device.
//
// Slot j sits at zeta_j = omega^(5^j mod 2N), omega = exp(i pi / N). Every odd
// power omega^(2k+1) is an evaluation point, and
//   m(omega^(2k+1)) = sum_i (m_i omega^i) exp(2 pi i i k / N),
// a length-N DFT of the twisted coefficients. So
//   decode: Z = DFT+(m_i omega^i);            z_j = Z[(5^j mod 2N - 1) / 2] / scale
//   encode: V[k_j] = scale z_j, V[k'_j] = conj(scale z_j) (2k'_j + 1 = 2N - 5^j),
//           w = DFT-(V);                       m_i = round(Re(omega^-i w_i) / N)
// The DFT is a four-step transform (N = N1 N2): length-N1 transforms down the
// columns with the exp(+-2 pi i n2 k1 / N) twiddle fused, then length-N2
// transforms along the rows, each in shared memory, in double precision.
#include <cmath>
#include <cstdint>

#include "../../include/ckks_mulk.h"
#include "internal.h"

using namespace ckks;


namespace {

constexpr int kThr = 256;
constexpr int kTC = 8;  // transforms per block

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cis_pi(double t) {  // exp(i pi t)
    double s, c;
    sincospi(t, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ uint32_t brv(uint32_t x, int bits) { return bits ? __brev(x) >> (32 - bits) : 0u; }

// 5^j mod 2N (2N <= 2^17: products fit in 64 bits)
__device__ __forceinline__ uint32_t pow5(uint32_t j, uint32_t two_n) {
    uint64_t x = 1, b = 5 % two_n;
    for (; j; j >>= 1, b = b * b % two_n)
        if (j & 1) x = x * b % two_n;
    return (uint32_t)x;
}

// T[j] = exp(i pi j / N), j < 2N (one table per call, in the workspace):
// exp(sign 2 pi i x / N) = T[2x] or its conjugate
__device__ __forceinline__ double2 root(const double2 *T, long long two_x, int sign) {
    const double2 w = T[two_x];
    return sign > 0 ? w : make_double2(w.x, -w.y);
}

// kTC radix-2 transforms of length 2^lg held in s[t * len + ...] in
// bit-reversed order; natural order on return. sign = +1 or -1.
__device__ void smem_fft(double2 *s, int lg, int sign, double2 *tw, const double2 *T, int log_n) {
    const int len = 1 << lg;
    for (int j = threadIdx.x; j < len / 2; j += blockDim.x) tw[j] = root(T, (2ll * j) << (log_n - lg), sign);
    __syncthreads();
    for (int h = 1; h < len; h <<= 1) {
        const int stride = len / (2 * h);
        for (int u = threadIdx.x; u < kTC * len / 2; u += blockDim.x) {
            const int t = u / (len / 2), b = u % (len / 2);
            const int grp = b / h, j = b % h;
            double2 *base = s + t * len + grp * 2 * h;
            const double2 w = tw[j * stride];
            const double2 x = base[j], y = cmul(base[j + h], w);
            base[j] = make_double2(x.x + y.x, x.y + y.y);
            base[j + h] = make_double2(x.x - y.x, x.y - y.y);
        }
        __syncthreads();
    }
}

// Step 1 (columns): for columns n2 = c0..c0+kTC-1,
// Y[k1][n2] = exp(sign 2 pi i n2 k1 / N) sum_n1 x[N2 n1 + n2] exp(sign 2 pi i n1 k1 / N1)
__global__ void __launch_bounds__(kThr) fft_cols_kernel(const double2 *x, double2 *y, int lg1, int lg2, int sign,
                                                        const double2 *T) {
    extern __shared__ double2 sm[];
    const int N1 = 1 << lg1, N2 = 1 << lg2, N = N1 * N2;
    const int tc = N2 < kTC ? N2 : kTC;
    double2 *s = sm, *tw = sm + kTC * N1;
    const int c0 = blockIdx.x * tc;
    const size_t off = (size_t)blockIdx.y * N;
    for (int u = threadIdx.x; u < tc * N1; u += blockDim.x) {
        const int n1 = u / tc, c = u % tc;
        s[c * N1 + brv(n1, lg1)] = x[off + (size_t)n1 * N2 + c0 + c];
    }
    for (int u = threadIdx.x + tc * N1; u < kTC * N1; u += blockDim.x) s[u] = make_double2(0, 0);
    __syncthreads();
    smem_fft(s, lg1, sign, tw, T, lg1 + lg2);
    for (int u = threadIdx.x; u < tc * N1; u += blockDim.x) {
        const int k1 = u / tc, c = u % tc;
        const int n2 = c0 + c;
        const long long e = ((long long)n2 * k1) % N;  // exact argument reduction
        y[off + (size_t)k1 * N2 + n2] = cmul(s[c * N1 + k1], root(T, 2 * e, sign));
    }
}

// Step 2 (rows): X[k1 + N1 k2] = sum_n2 Y[k1][n2] exp(sign 2 pi i n2 k2 / N2)
__global__ void __launch_bounds__(kThr) fft_rows_kernel(const double2 *y, double2 *X, int lg1, int lg2, int sign,
                                                        const double2 *T) {
    extern __shared__ double2 sm[];
    const int N1 = 1 << lg1, N2 = 1 << lg2, N = N1 * N2;
    const int tr = N1 < kTC ? N1 : kTC;
    double2 *s = sm, *tw = sm + kTC * N2;
    const int r0 = blockIdx.x * tr;
    const size_t off = (size_t)blockIdx.y * N;
    for (int u = threadIdx.x; u < tr * N2; u += blockDim.x) {
        const int r = u / N2, n2 = u % N2;
        s[r * N2 + brv(n2, lg2)] = y[off + (size_t)(r0 + r) * N2 + n2];
    }
    for (int u = threadIdx.x + tr * N2; u < kTC * N2; u += blockDim.x) s[u] = make_double2(0, 0);
    __syncthreads();
    smem_fft(s, lg2, sign, tw, T, lg1 + lg2);
    for (int u = threadIdx.x; u < tr * N2; u += blockDim.x) {
        const int k2 = u / tr, r = u % tr;
        X[off + (size_t)(r0 + r) + (size_t)N1 * k2] = s[r * N2 + k2];
    }
}

// decode, before the DFT: x_i = m_i omega^i
__global__ void twist_kernel(const double *m, double2 *x, int N, const double2 *T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const size_t o = (size_t)blockIdx.y * N + i;
    const double2 w = T[i];
    x[o] = make_double2(m[o] * w.x, m[o] * w.y);
}

// decode, after: z_j = Z[(5^j mod 2N - 1) / 2] / scale
__global__ void slots_kernel(const double2 *Z, double *z, int N, double inv_scale) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N / 2) return;
    const double2 v = Z[(size_t)blockIdx.y * N + (pow5(j, 2u * N) - 1) / 2];
    double *o = z + ((size_t)blockIdx.y * (N / 2) + j) * 2;
    o[0] = v.x * inv_scale;
    o[1] = v.y * inv_scale;
}

// encode, before: V[(5^j - 1)/2] = scale z_j, V[(2N - 5^j - 1)/2] = conj
__global__ void scatter_kernel(const double *z, double2 *V, int N, double scale) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N / 2) return;
    const double *zi = z + ((size_t)blockIdx.y * (N / 2) + j) * 2;
    const double re = zi[0] * scale, im = zi[1] * scale;
    const uint32_t e = pow5(j, 2u * N);
    const size_t off = (size_t)blockIdx.y * N;
    V[off + (e - 1) / 2] = make_double2(re, im);
    V[off + (2u * N - e - 1) / 2] = make_double2(re, -im);
}

// encode, after: m_i = round(Re(omega^-i w_i) / N)
__global__ void untwist_round_kernel(const double2 *w, long long *m, int N, const double2 *T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const size_t o = (size_t)blockIdx.y * N + i;
    const double2 c = make_double2(T[i].x, -T[i].y);
    const double re = w[o].x * c.x - w[o].y * c.y;
    m[o] = llrint(re / N);
}

// T[j] = exp(i pi j / N) for j < 2N
__global__ void roots_kernel(double2 *T, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < 2 * N) T[j] = cis_pi((double)j / N);
}

int geometry(int log_n, int &lg1, int &lg2) {
    lg1 = (log_n + 1) / 2;
    lg2 = log_n / 2;
    return 0;
}

cudaError_t dft(const Context &C, const double2 *in, double2 *tmp, double2 *out, int batch, int sign,
                const double2 *T, cudaStream_t st) {
    int lg1, lg2;
    geometry(C.log_n, lg1, lg2);
    const int N1 = 1 << lg1, N2 = 1 << lg2;
    const size_t sm1 = (size_t)(kTC * N1 + N1 / 2 + 1) * sizeof(double2);
    const size_t sm2 = (size_t)(kTC * N2 + N2 / 2 + 1) * sizeof(double2);
    const int tc = N2 < kTC ? N2 : kTC, tr = N1 < kTC ? N1 : kTC;
    count_kernel(C);
    fft_cols_kernel<<<dim3(N2 / tc, batch), kThr, sm1, st>>>(in, tmp, lg1, lg2, sign, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_kernel(C);
    fft_rows_kernel<<<dim3(N1 / tr, batch), kThr, sm2, st>>>(tmp, out, lg1, lg2, sign, T);
    return cudaGetLastError();
}

size_t embed_ws(const Context &C, uint32_t batch) { return (2 * (size_t)batch + 2) * C.N * sizeof(double2); }

// the roots table at the end of the workspace, filled on `st`
cudaError_t roots(const Context &C, double2 *T, cudaStream_t st) {
    count_kernel(C);
    roots_kernel<<<(2 * C.N + kThr - 1) / kThr, kThr, 0, st>>>(T, C.N);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int ckks_embed_workspace_size(const ckks_context *ctx, uint32_t batch, size_t *bytes) {
    if (!ctx || !bytes || batch < 1 || ctx->c.N < 4) return CKKS_EINVAL;
    *bytes = embed_ws(ctx->c, batch);
    return CKKS_OK;
}

int ckks_encode(ckks_context *ctx, const double *z, uint32_t batch, double scale, int64_t *m, void *workspace,
                size_t ws_bytes, void *stream) {
    if (!ctx || !z || !m || !workspace || batch < 1 || !(scale > 0) || ctx->c.N < 4 || batch > 65535)
        return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (ws_bytes < embed_ws(C, batch)) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    double2 *A = (double2 *)workspace;
    double2 *Bf = A + (size_t)batch * C.N;
    double2 *T = Bf + (size_t)batch * C.N;
    cudaError_t err = roots(C, T, st);
    if (err == cudaSuccess) {
        count_kernel(C);
        scatter_kernel<<<dim3((C.N / 2 + kThr - 1) / kThr, batch), kThr, 0, st>>>(z, A, C.N, scale);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = dft(C, A, Bf, A, (int)batch, -1, T, st);
    if (err == cudaSuccess) {
        count_kernel(C);
        untwist_round_kernel<<<dim3((C.N + kThr - 1) / kThr, batch), kThr, 0, st>>>(A, (long long *)m, C.N, T);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

int ckks_decode(ckks_context *ctx, const double *m, uint32_t batch, double scale, double *z, void *workspace,
                size_t ws_bytes, void *stream) {
    if (!ctx || !z || !m || !workspace || batch < 1 || !(scale > 0) || ctx->c.N < 4 || batch > 65535)
        return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (ws_bytes < embed_ws(C, batch)) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    double2 *A = (double2 *)workspace;
    double2 *Bf = A + (size_t)batch * C.N;
    double2 *T = Bf + (size_t)batch * C.N;
    cudaError_t err = roots(C, T, st);
    if (err == cudaSuccess) {
        count_kernel(C);
        twist_kernel<<<dim3((C.N + kThr - 1) / kThr, batch), kThr, 0, st>>>(m, A, C.N, T);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = dft(C, A, Bf, A, (int)batch, +1, T, st);
    if (err == cudaSuccess) {
        count_kernel(C);
        slots_kernel<<<dim3((C.N / 2 + kThr - 1) / kThr, batch), kThr, 0, st>>>(A, z, C.N, 1.0 / scale);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        const_cast<Context &>(C).sticky.store((int)err);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

}  // extern "C"
