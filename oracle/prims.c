/*
 * Oracle primitives: exact modular arithmetic on uint64 residues.
 *
 * TEST INFRASTRUCTURE ONLY. This file is part of the CPU oracle that the
 * tests and the benchmark's CPU-baseline leg use to check the CUDA path. The
 * product library never links or calls it.
 *
 * Every product is formed in unsigned __int128 and reduced with the C `%`
 * operator, so each routine is its own definition. Nothing here is blocked,
 * lazy-reduced or vectorised by hand.
 *
 *  or_ntt_definition  : A[i] = sum_j a_j psi^((2 brv(i) + 1) j) mod q
 *                       (negacyclic evaluation map, bit-reversed order;
 *                       the NTT of Section II, written as its definition)
 *  or_negacyclic_mul  : schoolbook product in Z_q[x]/(x^N + 1)
 *  or_ntt / or_intt   : the textbook iterative radix-2 transform for the
 *                       same map (Cooley-Tukey forward, Gentleman-Sande
 *                       inverse); used as a fast step at large N and pinned
 *                       to or_ntt_definition by the tests.
 */
#include <stdint.h>
#include <stddef.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
/* q < 2^63, so the sums below cannot wrap */
static u64 addmod(u64 a, u64 b, u64 q) { return (a % q + b % q) % q; }
static u64 submod(u64 a, u64 b, u64 q) { return (a % q + q - b % q) % q; }

static u64 powmod(u64 b, u64 e, u64 q) {
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

static u64 brv(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

static int log2u(size_t n) {
    int l = 0;
    while (((size_t)1 << l) < n) ++l;
    return l;
}

/* out[i] = a[i] * b[i] mod q */
void or_mulmod(const u64 *a, const u64 *b, u64 *out, size_t n, u64 q) {
    for (size_t i = 0; i < n; ++i) out[i] = mulmod(a[i] % q, b[i] % q, q);
}

/* out[i] = a[i] * c mod q (a[i] any uint64) */
void or_scalar_mulmod(const u64 *a, u64 c, u64 *out, size_t n, u64 q) {
    for (size_t i = 0; i < n; ++i) out[i] = mulmod(a[i] % q, c % q, q);
}

/* out[i] = (sum_j a[j][i] * c[j]) mod q, a is [m][n] */
void or_dot_const(const u64 *a, const u64 *c, size_t m, u64 *out, size_t n, u64 q) {
    for (size_t i = 0; i < n; ++i) {
        u64 acc = 0;
        for (size_t j = 0; j < m; ++j) acc = addmod(acc, mulmod(a[j * n + i] % q, c[j] % q, q), q);
        out[i] = acc;
    }
}

/* Definition of the transform: O(N^2). */
void or_ntt_definition(const u64 *a, u64 *out, size_t N, u64 q, u64 psi) {
    int lg = log2u(N);
    for (size_t i = 0; i < N; ++i) {
        u64 root = powmod(psi, 2 * brv(i, lg) + 1, q);
        u64 acc = 0, pw = 1;
        for (size_t j = 0; j < N; ++j) {
            acc = addmod(acc, mulmod(a[j], pw, q), q);
            pw = mulmod(pw, root, q);
        }
        out[i] = acc;
    }
}

/* Inverse of the definition: a_j = N^-1 sum_i A[i] psi^-((2 brv(i)+1) j). O(N^2). */
void or_intt_definition(const u64 *A, u64 *out, size_t N, u64 q, u64 psi) {
    int lg = log2u(N);
    u64 psi_inv = powmod(psi, q - 2, q);
    u64 n_inv = powmod((u64)N % q, q - 2, q);
    for (size_t j = 0; j < N; ++j) out[j] = 0;
    for (size_t i = 0; i < N; ++i) {
        u64 root = powmod(psi_inv, 2 * brv(i, lg) + 1, q);
        u64 pw = 1;
        for (size_t j = 0; j < N; ++j) {
            out[j] = addmod(out[j], mulmod(A[i], pw, q), q);
            pw = mulmod(pw, root, q);
        }
    }
    for (size_t j = 0; j < N; ++j) out[j] = mulmod(out[j], n_inv, q);
}

/* Schoolbook product in Z_q[x]/(x^N+1): c_i = sum_j a_j b_{i-j} (-1)^[j>i]. */
void or_negacyclic_mul(const u64 *a, const u64 *b, u64 *out, size_t N, u64 q) {
    for (size_t i = 0; i < N; ++i) {
        u64 acc = 0;
        for (size_t j = 0; j < N; ++j) {
            if (j <= i) acc = addmod(acc, mulmod(a[j], b[i - j], q), q);
            else acc = submod(acc, mulmod(a[j], b[N + i - j], q), q);
        }
        out[i] = acc;
    }
}

#include <stdlib.h>

/* table[e] = r^e for e in [0, N) */
static u64 *power_table(u64 r, size_t N, u64 q) {
    u64 *t = (u64 *)malloc(N * sizeof(u64));
    t[0] = 1 % q;
    for (size_t e = 1; e < N; ++e) t[e] = mulmod(t[e - 1], r, q);
    return t;
}

/* Textbook iterative forward transform, in place. The stage with m groups
 * uses psi^brv(m + i) for group i. */
void or_ntt(u64 *a, size_t N, u64 q, u64 psi) {
    int lg = log2u(N);
    u64 *pw = power_table(psi, N, q);
    for (size_t m = 1, t = N / 2; m < N; m *= 2, t /= 2) {
        for (size_t i = 0; i < m; ++i) {
            u64 w = pw[brv(m + i, lg)];
            for (size_t j = 2 * i * t; j < 2 * i * t + t; ++j) {
                u64 u = a[j], v = mulmod(a[j + t], w, q);
                a[j] = addmod(u, v, q);
                a[j + t] = submod(u, v, q);
            }
        }
    }
    free(pw);
}

/* Textbook iterative inverse transform, in place, including the N^-1 factor. */
void or_intt(u64 *a, size_t N, u64 q, u64 psi) {
    int lg = log2u(N);
    u64 psi_inv = powmod(psi, q - 2, q);
    u64 *pw = power_table(psi_inv, N, q);
    for (size_t m = N / 2, t = 1; m >= 1; m /= 2, t *= 2) {
        for (size_t i = 0; i < m; ++i) {
            u64 w = pw[brv(m + i, lg)];
            for (size_t j = 2 * i * t; j < 2 * i * t + t; ++j) {
                u64 u = a[j], v = a[j + t];
                a[j] = addmod(u, v, q);
                a[j + t] = mulmod(submod(u, v, q), w, q);
            }
        }
    }
    free(pw);
    u64 n_inv = powmod((u64)N % q, q - 2, q);
    for (size_t j = 0; j < N; ++j) a[j] = mulmod(a[j], n_inv, q);
}

/* Batched forms over [rows][N], one modulus per row (OpenMP over rows). */
void or_ntt_rows(u64 *a, size_t rows, size_t N, const u64 *q, const u64 *psi) {
#pragma omp parallel for schedule(dynamic)
    for (long r = 0; r < (long)rows; ++r) or_ntt(a + (size_t)r * N, N, q[r], psi[r]);
}

void or_intt_rows(u64 *a, size_t rows, size_t N, const u64 *q, const u64 *psi) {
#pragma omp parallel for schedule(dynamic)
    for (long r = 0; r < (long)rows; ++r) or_intt(a + (size_t)r * N, N, q[r], psi[r]);
}

void or_mulmod_rows(const u64 *a, const u64 *b, u64 *out, size_t rows, size_t N, const u64 *q) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < (long)rows; ++r)
        or_mulmod(a + (size_t)r * N, b + (size_t)r * N, out + (size_t)r * N, N, q[r]);
}

int or_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
