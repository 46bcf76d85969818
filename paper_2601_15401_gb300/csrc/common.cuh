// Device-side modular arithmetic and launch descriptors shared by the kernels.
//
// Residues are uint64 in [0, q) with every modulus q < 2^61, so lazy values up
// to 4q fit a 64-bit word. Three multiplications are used:
//   * Shoup (constant operand w with companion w' = floor(w 2^64 / q)):
//     x w - floor(x w' / 2^64) q lies in [0, 2q) for any x < 2^64 (Shoup's
//     precomputed-quotient method, as used in Harvey's NTT butterflies);
//   * Montgomery REDC with R = 2^64 for variable products and for 128-bit
//     dot products: for T = hi 2^64 + lo with hi < q,
//     m = lo q^-1 mod 2^64 gives T R^-1 = hi - floor(m q / 2^64) (mod q),
//     a value in (-q, q);
//   * plain modular add / sub.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned long long u64;
typedef long long i64;

#define CKKS_MAX_PRIMES 64
#define CKKS_MAX_TUPLE 13   // k <= 12 inputs give at most 13 polynomials

struct ModQ {
    u64 q;      // modulus
    u64 qinv;   // q^-1 mod 2^64 (Montgomery)
};

__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// x * w mod q in [0, 2q), w < q, wp = floor(w 2^64 / q), any x < 2^64.
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 wp, u64 q) {
    return x * w - mulhi64(x, wp) * q;
}

// The same for a modulus q = 1 (mod 2^32), q = qh 2^32 + 1: with
// h = floor(x w'/2^64), h q = h + h qh 2^32, so modulo 2^64 the quotient
// product needs only the low 32 bits of h qh (one 32-bit multiply instead of
// a 64 x 64-bit low product).
__device__ __forceinline__ u64 shoup_lazy_q1(u64 x, u64 w, u64 wp, uint32_t qh) {
    const u64 h = mulhi64(x, wp);
    const uint32_t t = (uint32_t)h * qh;
    return x * w - h - ((u64)t << 32);
}

__device__ __forceinline__ u64 reduce2(u64 x, u64 q) { return x >= q ? x - q : x; }

__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 wp, u64 q) {
    return reduce2(shoup_lazy(x, w, wp, q), q);
}

// [0, 4q) -> [0, q)
__device__ __forceinline__ u64 reduce4(u64 x, u64 q) {
    u64 q2 = q << 1;
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}

// Montgomery reduction of hi 2^64 + lo (hi < q): returns (hi 2^64 + lo) 2^-64 mod q.
__device__ __forceinline__ u64 redc(u64 hi, u64 lo, ModQ m) {
    u64 t = lo * m.qinv;
    u64 u = mulhi64(t, m.q);
    return hi >= u ? hi - u : hi + m.q - u;
}

// a b 2^-64 mod q for a, b < q.
__device__ __forceinline__ u64 mont_mul(u64 a, u64 b, ModQ m) {
    return redc(mulhi64(a, b), a * b, m);
}

// REDC for q = 1 (mod 2^32), q = qh 2^32 + 1: q^-1 = 1 - qh 2^32 (mod 2^64),
// so t = lo q^-1 needs one 32-bit product; with t = t1 2^32 + t0,
// t q = t1 qh 2^64 + (t0 qh + t1) 2^32 + t0 and the high word of t q is
// t1 qh + floor((t0 qh + t1) / 2^32): two 32 x 32-bit products instead of a
// 64 x 64-bit low product and a 64 x 64-bit high product.
__device__ __forceinline__ u64 redc_q1(u64 hi, u64 lo, u64 q) {
    const uint32_t qh = (uint32_t)(q >> 32);
    const u64 t = lo - ((u64)((uint32_t)lo * qh) << 32);
    const uint32_t t0 = (uint32_t)t, t1 = (uint32_t)(t >> 32);
    const u64 u = (u64)t1 * qh + (((u64)t0 * qh + t1) >> 32);
    return hi >= u ? hi - u : hi + q - u;
}

// The modular products in two forms selected at compile time: Q1 = true for
// contexts whose primes are all 1 (mod 2^32).
template <bool Q1>
__device__ __forceinline__ u64 shoup_lazy_t(u64 x, u64 w, u64 wp, u64 q) {
    if constexpr (Q1) return shoup_lazy_q1(x, w, wp, (uint32_t)(q >> 32));
    else return shoup_lazy(x, w, wp, q);
}

template <bool Q1>
__device__ __forceinline__ u64 shoup_t(u64 x, u64 w, u64 wp, u64 q) {
    return reduce2(shoup_lazy_t<Q1>(x, w, wp, q), q);
}

template <bool Q1>
__device__ __forceinline__ u64 redc_t(u64 hi, u64 lo, ModQ m) {
    if constexpr (Q1) return redc_q1(hi, lo, m.q);
    else return redc(hi, lo, m);
}

template <bool Q1>
__device__ __forceinline__ u64 mont_mul_t(u64 a, u64 b, ModQ m) {
    return redc_t<Q1>(mulhi64(a, b), a * b, m);
}

// 128-bit accumulator for dot products reduced once by REDC. Adding a product
// of two values below 2^61 and q keeps hi below q after the conditional
// subtraction of q 2^64 (which does not change the value mod q).
struct Acc128 {
    u64 hi, lo;
    __device__ __forceinline__ void zero() { hi = 0; lo = 0; }
    __device__ __forceinline__ void mac(u64 a, u64 b, u64 q) {
        u64 plo = a * b;
        u64 phi = mulhi64(a, b);
        lo += plo;
        hi += phi + (lo < plo ? 1ull : 0ull);
        hi = hi >= q ? hi - q : hi;
    }
    // add a 128-bit value below q * 2^64 (hi < q)
    __device__ __forceinline__ void add(u64 vhi, u64 vlo, u64 q) {
        lo += vlo;
        hi += vhi + (lo < vlo ? 1ull : 0ull);
        hi = hi >= q ? hi - q : hi;
        hi = hi >= q ? hi - q : hi;
    }
};

// Same accumulation without the per-term reduction: valid when the sum of
// the left operands' moduli is below 2^64 (checked at context creation for
// every BConv digit and for the P basis), which keeps hi < q.
struct Acc128Lazy {
    u64 hi, lo;
    __device__ __forceinline__ void zero() { hi = 0; lo = 0; }
    __device__ __forceinline__ void mac(u64 a, u64 b) {
        u64 plo = a * b;
        u64 phi = mulhi64(a, b);
        lo += plo;
        hi += phi + (lo < plo ? 1ull : 0ull);
    }
    // add the 128-bit value vhi 2^64 + vlo
    __device__ __forceinline__ void add(u64 vhi, u64 vlo) {
        lo += vlo;
        hi += vhi + (lo < vlo ? 1ull : 0ull);
    }
    // the same calls as Acc128 (the modulus is not needed)
    __device__ __forceinline__ void mac(u64 a, u64 b, u64) { mac(a, b); }
    __device__ __forceinline__ void add(u64 vhi, u64 vlo, u64) { add(vhi, vlo); }
};

// Shoup constant pair.
struct Shoup {
    u64 w, wp;
};

// Addressing of a set of limbs: limb (b, p, l) of a [batch][poly][limb][N]
// view lives at ptr + b * bstride + p * pstride + slot[l] * N.
struct LimbView {
    u64 *ptr;
    i64 bstride;   // elements
    i64 pstride;   // elements
};

// The limbs a launch works on: batch x polys x limbs, each limb l mapping to
// a storage slot and a prime index (Q primes first, then P primes).
struct LimbJobs {
    int n_batch, n_polys, n_limbs;
    uint8_t slot[CKKS_MAX_PRIMES];    // source slot of launch limb l
    uint8_t dslot[CKKS_MAX_PRIMES];   // destination slot of launch limb l
    uint8_t prime[CKKS_MAX_PRIMES];   // prime index of launch limb l
};

__device__ __forceinline__ void decode_job(const LimbJobs &J, int job, int &b, int &p, int &l) {
    l = job % J.n_limbs;
    int r = job / J.n_limbs;
    p = r % J.n_polys;
    b = r / J.n_polys;
}

__device__ __forceinline__ u64 *limb_ptr(const LimbView &v, int b, int p, int slot, int N) {
    return v.ptr + (i64)b * v.bstride + (i64)p * v.pstride + (i64)slot * N;
}
