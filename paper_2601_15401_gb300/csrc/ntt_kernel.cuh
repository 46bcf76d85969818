// Negacyclic NTT / INTT phase kernels over 64-bit NTT-friendly primes
// (device code; instantiated by ntt_uf.cu, ntt_ui.cu, ntt_tf.cu, ntt_ti.cu,
// the host logic is in ntt.cu).
//
// The transform is the evaluation map A[i] = sum_j a_j psi^((2 brv(i)+1) j)
// (bit-reversed order), computed with Cooley-Tukey butterflies forward and
// Gentleman-Sande butterflies inverse (Section II; Eq. 7 and Algorithm 1
// use it between the coefficient and the NTT domain).
//
// GPU structure. N = N1 * N2 points split into a 2-D array with element
// e = c + k N2. The forward transform's first log2 N1 stages only pair
// elements of the same column c; its last log2 N2 stages only pair elements
// of the same row block [b N2, (b+1) N2). So the transform runs as two
// launches (column phase, block phase), each CTA loading a tile of whole
// columns or whole blocks into shared memory, running its stages there and
// writing back. The inverse runs the block phase first. N <= 256 runs one
// block phase over the whole limb.
//
// Inside a phase the sub-transform of n = 2^LOGN points is done in passes of
// up to 4 stages: a thread holds 2^r points of one sub-problem in registers
// (radix-2^r), runs r butterfly stages on them and writes them back; passes
// are separated by __syncthreads. Butterflies are lazy (Harvey): forward
// values stay in [0, 4q), inverse values in [0, 2q).
//
// Twiddles: tw[prime][k] = (psi^brv(k), Shoup companion) for the forward,
// psi^-brv(k) for the inverse. The stage with m groups uses tw[m + i] for
// group i; in the block phase the global group index is b m_loc + i_loc and
// m = N1 m_loc, so the index is m_loc (N1 + b) + i_loc.
//
// Element-wise work is fused into the global <-> shared copies: the load side
// can add two limbs or form the rescale combination of Eq. 17; the store side
// can scale (N^-1 and BConv / ModDown constants), finish ModDown (Eq. 5 with
// Eq. 11/12) or finish Algorithm 1 (A' = g A - B).
//
// Template parameters LM / SM fix the load / store mode at compile time
// (-1: read from the launch's spec at run time). A fixed mode keeps only the
// pointers and constants that mode uses alive, which is what lets the
// specialised kernels fit three CTAs per SM. JOBS selects where a CTA finds
// its limb: from the launch's uniform batch x polynomial x limb description
// (LimbJobs), or from a device table of NttJob entries (limbs of different
// products, levels and tree nodes in one launch).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace ckks {

// ---------------------------------------------------------------------------
// butterflies
// ---------------------------------------------------------------------------
template <bool Q1>
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 q) {
    u64 q2 = q << 1;
    u64 x = X >= q2 ? X - q2 : X;
    u64 t = shoup_lazy_t<Q1>(Y, w.x, w.y, q);
    X = x + t;
    Y = x - t + q2;
}

template <bool Q1>
__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 q) {
    u64 q2 = q << 1;
    u64 s = X + Y;
    s = s >= q2 ? s - q2 : s;
    u64 d = X - Y + q2;
    Y = shoup_lazy_t<Q1>(d, w.x, w.y, q);
    X = s;
}

// ---------------------------------------------------------------------------
// pass plan: LOGN stages in ceil(LOGN/4) passes of near-equal length
// ---------------------------------------------------------------------------
#ifndef CKKS_NTT_RMAX
#define CKKS_NTT_RMAX 4
#endif
template <int LOGN, int P>
struct Pass {
    static constexpr int NP = (LOGN + CKKS_NTT_RMAX - 1) / CKKS_NTT_RMAX;
    static constexpr int base = LOGN / NP;
    static constexpr int extra = LOGN % NP;
    static constexpr int len = base + (P < extra ? 1 : 0);
    static constexpr int start = P * base + (P < extra ? P : extra);
};

// Shared-memory layouts of a tile (n_sub = 2^lsub sub-problems of n points).
//   columns: [n][n_sub] row-major (sub-problems side by side); threads run
//            over sub-problems fastest, so every pass reads whole 128-byte
//            row segments of global memory.
//   blocks:  [n_sub][n + n/16] with one pad word per 16; threads run over
//            point sets fastest.
template <bool COLS, int LOGN>
struct Layout {
    int lsub;
    __device__ __forceinline__ int off(int sp, int k) const {
        if (COLS) return (k << lsub) + sp;
        return sp * ((1 << LOGN) + (1 << LOGN >> 4)) + k + (k >> 4);
    }
    __device__ __forceinline__ void split(int s, int lsets, int &sp, int &set) const {
        if (COLS) { sp = s & ((1 << lsub) - 1); set = s >> lsub; }
        else { set = s & ((1 << lsets) - 1); sp = s >> lsets; }
    }
};

// ---------------------------------------------------------------------------
// fused element-wise load / store with per-CTA base pointers
// ---------------------------------------------------------------------------
struct LoadCtx {
    int mode;
    const u64 *a, *b;      // limb base pointers (b: T limbs / z limbs / second addend)
    const Shoup *g;        // LD_EQ17: g[0..mu-1], g[mu] = self
    int mu, with_self, K, N;
    const u64 *cK;         // LD_BCONVK
    ModQ m;
};

struct StoreCtx {
    int mode;
    u64 *dst;
    const u64 *aux, *aux2;
    Shoup c;
    int K, N;
    const u64 *cK;
    ModQ m;
};

// uniform launches: limb (b, p, l) of the launch's views
__device__ __forceinline__ LoadCtx make_load(const LoadSpec &L, const LimbJobs &J, int N, int b, int p, int l,
                                             int prime, ModQ m) {
    LoadCtx c;
    c.mode = L.mode;
    c.N = N;
    c.m = m;
    c.mu = L.mu;
    c.with_self = L.with_self;
    c.K = L.K;
    const int slot = J.slot[l];
    c.a = L.a.ptr ? limb_ptr(L.a, b, p, slot, N) : nullptr;
    c.b = nullptr;
    c.g = nullptr;
    c.cK = nullptr;
    if (L.mode == LD_ADD) c.b = limb_ptr(L.b, b, p, slot, N);
    if (L.mode == LD_EQ17 || L.mode == LD_BCONVK) c.b = L.b.ptr + (i64)b * L.b.bstride + (i64)p * L.b.pstride;
    if (L.mode == LD_EQ17) c.g = L.g + (i64)l * (L.mu + 1);
    if (L.mode == LD_BCONVK) c.cK = L.cK + (i64)prime * CKKS_MAX_PRIMES;
    return c;
}

__device__ __forceinline__ StoreCtx make_store(const StoreSpec &S, const LimbJobs &J, int N, int b, int p, int l,
                                               int prime, ModQ m) {
    StoreCtx c;
    c.mode = S.mode;
    c.N = N;
    c.m = m;
    c.K = S.K;
    const int ds = J.dslot[l];
    c.dst = limb_ptr(S.dst, b, p, ds, N);
    c.aux = nullptr;
    c.aux2 = nullptr;
    c.cK = nullptr;
    c.c = Shoup{0, 0};
    if (S.mode == ST_SCALE || S.mode == ST_MODDOWN || S.mode == ST_MRS) c.c = S.c[l * S.c_stride];
    if (S.mode == ST_MODDOWN) {
        c.aux = S.aux.ptr + (i64)b * S.aux.bstride + (i64)p * S.aux.pstride;
        c.cK = S.cK + (i64)prime * CKKS_MAX_PRIMES;
    }
    if (S.mode == ST_MRS || S.mode == ST_ADDSUB) c.aux = limb_ptr(S.aux, b, p, ds, N);
    if (S.mode == ST_ADDSUB) c.aux2 = limb_ptr(S.aux2, b, p, ds, N);
    return c;
}

// table launches: the limb's pointers come from its NttJob entry
__device__ __forceinline__ LoadCtx make_load(const LoadSpec &L, const NttJob &j, int N, ModQ m) {
    LoadCtx c;
    c.mode = L.mode;
    c.N = N;
    c.m = m;
    c.mu = j.mu;
    c.with_self = j.with_self;
    c.K = L.K;
    c.a = j.a;
    c.b = j.b;
    c.g = j.g;
    c.cK = L.mode == LD_BCONVK ? L.cK + (i64)j.prime * CKKS_MAX_PRIMES : nullptr;
    return c;
}

__device__ __forceinline__ StoreCtx make_store(const StoreSpec &S, const NttJob &j, int N, ModQ m) {
    StoreCtx c;
    c.mode = S.mode;
    c.N = N;
    c.m = m;
    c.K = S.K;
    c.dst = j.dst;
    c.aux = j.aux;
    c.aux2 = j.aux2;
    c.c = (S.mode == ST_SCALE || S.mode == ST_MODDOWN || S.mode == ST_MRS) ? *j.c : Shoup{0, 0};
    c.cK = S.mode == ST_MODDOWN ? S.cK + (i64)j.prime * CKKS_MAX_PRIMES : nullptr;
    return c;
}

template <int LM, bool Q1>
__device__ __forceinline__ u64 load_elem(const LoadCtx &c, int e) {
    const u64 q = c.m.q;
    const int mode = LM >= 0 ? LM : c.mode;
    switch (mode) {
    case LD_ADD:
        return add_mod(c.a[e], c.b[e], q);
    case LD_EQ17: {
        // sum_t g_t T_t (mod q); with the self term: g_self a - sum
        u64 s = 0;
        for (int t = 0; t < c.mu; ++t)
            s = add_mod(s, shoup_t<Q1>(c.b[(i64)t * c.N + e], c.g[t].w, c.g[t].wp, q), q);
        if (c.with_self) s = sub_mod(shoup_t<Q1>(c.a[e], c.g[c.mu].w, c.g[c.mu].wp, q), s, q);
        return s;
    }
    case LD_BCONVK: {
        Acc128Lazy acc;  // sum of the P primes < 2^64 (context check)
        acc.zero();
        for (int i = 0; i < c.K; ++i) acc.mac(c.b[(i64)i * c.N + e], c.cK[i]);
        return redc_t<Q1>(acc.hi, acc.lo, c.m);
    }
    default:
        return c.a[e];
    }
}

template <int SM, bool Q1>
__device__ __forceinline__ void store_elem(const StoreCtx &c, int e, u64 v, bool fwd) {
    const u64 q = c.m.q;
    const int mode = SM >= 0 ? SM : c.mode;
    switch (mode) {
    case ST_LAZY:
        c.dst[e] = v;
        break;
    case ST_SCALE:
        c.dst[e] = shoup_t<Q1>(v, c.c.w, c.c.wp, q);
        break;
    case ST_MODDOWN: {
        // c* = v N^-1 - sum_i z_i [p_i^-1 R]_q  (Eq. 5 with Eq. 11 / 12)
        u64 x = shoup_t<Q1>(v, c.c.w, c.c.wp, q);
        Acc128Lazy acc;  // sum of the P primes < 2^64 (context check)
        acc.zero();
        for (int i = 0; i < c.K; ++i) acc.mac(c.aux[(i64)i * c.N + e], c.cK[i]);
        c.dst[e] = sub_mod(x, redc_t<Q1>(acc.hi, acc.lo, c.m), q);
        break;
    }
    case ST_MRS:
        // Algorithm 1, last step: A' = g^{mu,L-1} A - B
        c.dst[e] = sub_mod(shoup_t<Q1>(c.aux[e], c.c.w, c.c.wp, q), fwd ? reduce4(v, q) : reduce2(v, q), q);
        break;
    case ST_ADDSUB:
        c.dst[e] = sub_mod(add_mod(c.aux[e], c.aux2[e], q), fwd ? reduce4(v, q) : reduce2(v, q), q);
        break;
    default:  // ST_REDUCE
        c.dst[e] = fwd ? reduce4(v, q) : reduce2(v, q);
        break;
    }
}

// Fused loads / stores that sum over several limbs (the Eq. 17 load, the
// ModDown store) issue the loads of several elements together.
#ifndef CKKS_NTT_EQ17_BY_TERM
#define CKKS_NTT_EQ17_BY_TERM 1
#endif
#ifndef CKKS_NTT_MODDOWN_GROUPS
#define CKKS_NTT_MODDOWN_GROUPS 1
#endif

// One pass of R stages starting at local stage E0 on every point set of the
// tile. GIN / GOUT: the pass reads / writes global memory (fused load /
// store) instead of shared memory.
template <int LOGN, int R, int E0, bool FWD, bool COLS, bool GIN, bool GOUT, int LM, int SM, bool Q1>
__device__ __forceinline__ void run_pass(u64 *sm, const Layout<COLS, LOGN> &lay, const ulonglong2 *tw, int tw_b0,
                                         int tw_bmul, u64 q, const LoadCtx &lc, const StoreCtx &sc, int t0,
                                         int log_n2) {
    constexpr int n = 1 << LOGN;
    constexpr int EL = 1 << R;
    constexpr int t_min = n >> (E0 + R);
    constexpr int t0s = n >> (E0 + 1);
    constexpr int lsets = LOGN - R;
    const int total = 1 << (lay.lsub + lsets);
    for (int s = threadIdx.x; s < total; s += blockDim.x) {
        int sp, set;
        lay.split(s, lsets, sp, set);
        const int o = set & (t_min - 1);
        const int g = set / t_min;
        const int base = g * 2 * t0s + o;
        u64 x[EL];
        if constexpr (CKKS_NTT_EQ17_BY_TERM && GIN && LM == LD_EQ17) {
            // Eq. 17 combination term by term: the EL loads of one term are
            // in flight together (the per-element loop over the terms had
            // one load in flight per thread)
            const u64 q = lc.m.q;
#pragma unroll
            for (int k = 0; k < EL; ++k) x[k] = 0;
            for (int t = 0; t < lc.mu; ++t) {
                const Shoup g = lc.g[t];
                const u64 *bt = lc.b + (i64)t * lc.N;
#pragma unroll
                for (int k = 0; k < EL; ++k) {
                    const int pt = base + k * t_min;
                    const int e = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                    x[k] = add_mod(x[k], shoup_t<Q1>(bt[e], g.w, g.wp, q), q);
                }
            }
            if (lc.with_self) {
                const Shoup g = lc.g[lc.mu];
#pragma unroll
                for (int k = 0; k < EL; ++k) {
                    const int pt = base + k * t_min;
                    const int e = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                    x[k] = sub_mod(shoup_t<Q1>(lc.a[e], g.w, g.wp, q), x[k], q);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < EL; ++k) {
                const int pt = base + k * t_min;
                if (GIN) {
                    const int e = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                    x[k] = load_elem<LM, Q1>(lc, e);
                } else {
                    x[k] = sm[lay.off(sp, pt)];
                }
            }
        }
        const int twb = tw_b0 + tw_bmul * sp;
        if (FWD) {
#pragma unroll
            for (int ep = 0; ep < R; ++ep) {
                const int h = EL >> (ep + 1);
                const int m = 1 << (E0 + ep);
#pragma unroll
                for (int k = 0; k < EL; ++k) {
                    if ((k & h) == 0) {
                        const int i = (g << ep) + (k >> (R - ep));
                        ct_bfly<Q1>(x[k], x[k + h], tw[m * twb + i], q);
                    }
                }
            }
        } else {
#pragma unroll
            for (int ep = R - 1; ep >= 0; --ep) {
                const int h = EL >> (ep + 1);
                const int m = 1 << (E0 + ep);
#pragma unroll
                for (int k = 0; k < EL; ++k) {
                    if ((k & h) == 0) {
                        const int i = (g << ep) + (k >> (R - ep));
                        gs_bfly<Q1>(x[k], x[k + h], tw[m * twb + i], q);
                    }
                }
            }
        }
        if constexpr (CKKS_NTT_MODDOWN_GROUPS && GOUT && SM == ST_MODDOWN) {
            // ModDown store (Eq. 5 with Eq. 11 / 12) four elements at a time,
            // their K z-limb loads in flight together
            const u64 q = sc.m.q;
            constexpr int G4 = EL >= 4 ? 4 : EL;
#pragma unroll
            for (int k0 = 0; k0 < EL; k0 += G4) {
                int e[G4];
                Acc128Lazy acc[G4];  // sum of the P primes < 2^64 (context check)
#pragma unroll
                for (int u = 0; u < G4; ++u) {
                    const int pt = base + (k0 + u) * t_min;
                    e[u] = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                    acc[u].zero();
                }
                for (int i = 0; i < sc.K; ++i) {
                    const u64 c = sc.cK[i];
                    const u64 *zi = sc.aux + (i64)i * sc.N;
                    u64 z[G4];
#pragma unroll
                    for (int u = 0; u < G4; ++u) z[u] = zi[e[u]];
#pragma unroll
                    for (int u = 0; u < G4; ++u) acc[u].mac(z[u], c);
                }
#pragma unroll
                for (int u = 0; u < G4; ++u)
                    sc.dst[e[u]] = sub_mod(shoup_t<Q1>(x[k0 + u], sc.c.w, sc.c.wp, q),
                                           redc_t<Q1>(acc[u].hi, acc[u].lo, sc.m), q);
            }
        } else {
#pragma unroll
            for (int k = 0; k < EL; ++k) {
                const int pt = base + k * t_min;
                if (GOUT) {
                    const int e = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                    store_elem<SM, Q1>(sc, e, x[k], FWD);
                } else {
                    sm[lay.off(sp, pt)] = x[k];
                }
            }
        }
    }
}

// Direct global access is used on a side whose pass reads / writes at
// least 8 consecutive words per sub-problem (always true for column tiles).
// CKKS_NTT_DIRECT_IN = 0 stages every tile through shared memory on the
// load side (batched loads), keeping direct global stores.
#ifndef CKKS_NTT_DIRECT_IN
#define CKKS_NTT_DIRECT_IN 1
#endif
template <int LOGN, bool COLS, int P>
struct PassAccess {
    static constexpr int t_min = (1 << LOGN) >> (Pass<LOGN, P>::start + Pass<LOGN, P>::len);
    static constexpr bool direct = COLS || t_min >= 8;
    static constexpr bool direct_in = direct && CKKS_NTT_DIRECT_IN;
};

template <int LOGN, bool FWD, bool COLS, int LM, int SM, bool Q1, int I>
__device__ __forceinline__ void run_passes(u64 *sm, const Layout<COLS, LOGN> &lay, const ulonglong2 *tw, int tw_b0,
                                           int tw_bmul, u64 q, const LoadCtx &lc, const StoreCtx &sc, int t0,
                                           int log_n2) {
    constexpr int NP = Pass<LOGN, 0>::NP;
    if constexpr (I < NP) {
        constexpr int PP = FWD ? I : NP - 1 - I;
        constexpr bool first = I == 0, last = I == NP - 1;
        constexpr bool gin = first && PassAccess<LOGN, COLS, PP>::direct_in;
        constexpr bool gout = last && PassAccess<LOGN, COLS, PP>::direct;
        run_pass<LOGN, Pass<LOGN, PP>::len, Pass<LOGN, PP>::start, FWD, COLS, gin, gout, LM, SM, Q1>(
            sm, lay, tw, tw_b0, tw_bmul, q, lc, sc, t0, log_n2);
        if (!last || !gout) __syncthreads();
        run_passes<LOGN, FWD, COLS, LM, SM, Q1, I + 1>(sm, lay, tw, tw_b0, tw_bmul, q, lc, sc, t0, log_n2);
    }
}

// 1: the column phases read their twiddles (the same n - 1 for every
// column) from a copy in shared memory, 4 KB behind the tile: forward column
// phase 55.0 vs 60.1 ms per bench step with them read from L1 / L2
#ifndef CKKS_NTT_COL_TW_SMEM
#define CKKS_NTT_COL_TW_SMEM 1
#endif

// Staged stores that read an aux limb gather eight elements at a time.
#ifndef CKKS_NTT_STORE_BATCH
#define CKKS_NTT_STORE_BATCH 1
#endif

// One tile (CTA) of one limb: tile index `tile` of the phase.
template <int LOGN, bool FWD, bool COLS, int LM, int SM, bool Q1>
__device__ __forceinline__ void phase_tile(u64 *sm, const NttPhase &P, const ulonglong2 *tw, u64 q,
                                           const LoadCtx &lc, const StoreCtx &sc, int tile) {
    constexpr int n = 1 << LOGN;
    constexpr int NP = Pass<LOGN, 0>::NP;
    const int lsub = P.log_sub;
    const int n_sub = 1 << lsub;
    Layout<COLS, LOGN> lay{lsub};
    const int t0 = tile << lsub;  // first column (COLS) or block (!COLS)
    constexpr int PF = FWD ? 0 : NP - 1;
    constexpr int PL = FWD ? NP - 1 : 0;
    constexpr bool gin = PassAccess<LOGN, COLS, PF>::direct_in;
    constexpr bool gout = PassAccess<LOGN, COLS, PL>::direct;
    const int total = n_sub << LOGN;
    // twiddle base: columns -> 1; blocks -> N1 + block
    const int tw_b0 = COLS ? 1 : P.N1 + t0;
    const int tw_bmul = COLS ? 0 : 1;
    if constexpr (COLS && CKKS_NTT_COL_TW_SMEM) {
        // the column phase's n - 1 twiddles (the same for every column) copied
        // once per CTA into shared memory behind the tile
        ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(sm + total);
        for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
        __syncthreads();
        tw = tws;
    }
    if (!gin) {
        // coalesced global -> shared with the fused load, eight loads in
        // flight per thread before their shared-memory stores
        constexpr int U = 8;
        for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
            u64 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = base + u * blockDim.x;
                if (idx < total) {
                    int sp, k, e;
                    if (COLS) { k = idx >> lsub; sp = idx & (n_sub - 1); e = t0 + sp + (k << P.log_n2); }
                    else { sp = idx >> LOGN; k = idx & (n - 1); e = ((t0 + sp) << LOGN) + k; }
                    v[u] = load_elem<LM, Q1>(lc, e);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = base + u * blockDim.x;
                if (idx < total) {
                    int sp, k;
                    if (COLS) { k = idx >> lsub; sp = idx & (n_sub - 1); }
                    else { sp = idx >> LOGN; k = idx & (n - 1); }
                    sm[lay.off(sp, k)] = v[u];
                }
            }
        }
        __syncthreads();
    }
    run_passes<LOGN, FWD, COLS, LM, SM, Q1, 0>(sm, lay, tw, tw_b0, tw_bmul, q, lc, sc, t0, P.log_n2);
    if (!gout) {
        // shared -> global with the fused store (coalesced)
        if constexpr (CKKS_NTT_STORE_BATCH && (SM == ST_MRS || SM == ST_ADDSUB)) {
            // the store reads an aux limb: gather eight elements and their
            // aux words first, so that eight loads are in flight per thread
            constexpr int U = 8;
            for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
                u64 v[U], a[U], a2[U];
                int e[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int idx = base + u * blockDim.x;
                    e[u] = -1;
                    if (idx < total) {
                        int sp, k;
                        if (COLS) { k = idx >> lsub; sp = idx & (n_sub - 1); e[u] = t0 + sp + (k << P.log_n2); }
                        else { sp = idx >> LOGN; k = idx & (n - 1); e[u] = ((t0 + sp) << LOGN) + k; }
                        v[u] = sm[lay.off(sp, k)];
                        a[u] = sc.aux[e[u]];
                        if (SM == ST_ADDSUB) a2[u] = sc.aux2[e[u]];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (e[u] < 0) continue;
                    const u64 q = sc.m.q;
                    const u64 r = FWD ? reduce4(v[u], q) : reduce2(v[u], q);
                    if (SM == ST_MRS) sc.dst[e[u]] = sub_mod(shoup_t<Q1>(a[u], sc.c.w, sc.c.wp, q), r, q);
                    else sc.dst[e[u]] = sub_mod(add_mod(a[u], a2[u], q), r, q);
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
                int sp, k, e;
                if (COLS) { k = idx >> lsub; sp = idx & (n_sub - 1); e = t0 + sp + (k << P.log_n2); }
                else { sp = idx >> LOGN; k = idx & (n - 1); e = ((t0 + sp) << LOGN) + k; }
                store_elem<SM, Q1>(sc, e, sm[lay.off(sp, k)], FWD);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the phase kernels: grid (tiles, limbs) for uniform launches, one
// flattened dimension (limb * tiles + tile) for table launches
// ---------------------------------------------------------------------------
template <int LOGN, bool FWD, bool COLS, int LM, int SM, int MINB, bool Q1>
__global__ void __launch_bounds__(256, MINB) ntt_phase_kernel(NttPhase P, LimbJobs J, LoadSpec L, StoreSpec S) {
    extern __shared__ u64 sm[];
    int b, p, l;
    decode_job(J, blockIdx.y, b, p, l);
    const int prime = J.prime[l];
    const ModQ m = P.mods[prime];
    const ulonglong2 *tw = (FWD ? P.tw_fwd : P.tw_inv) + (i64)prime * P.N;
    const LoadCtx lc = make_load(L, J, P.N, b, p, l, prime, m);
    const StoreCtx sc = make_store(S, J, P.N, b, p, l, prime, m);
    phase_tile<LOGN, FWD, COLS, LM, SM, Q1>(sm, P, tw, m.q, lc, sc, blockIdx.x);
}

template <int LOGN, bool FWD, bool COLS, int LM, int SM, int MINB, bool Q1>
__global__ void __launch_bounds__(256, MINB) ntt_phase_table_kernel(NttPhase P, const NttJob *jobs, int tiles,
                                                                    LoadSpec L, StoreSpec S) {
    extern __shared__ u64 sm[];
    const int job = blockIdx.x / tiles;
    const int tile = blockIdx.x - job * tiles;
    const NttJob j = jobs[job];
    const ModQ m = P.mods[j.prime];
    const ulonglong2 *tw = (FWD ? P.tw_fwd : P.tw_inv) + (i64)j.prime * P.N;
    const LoadCtx lc = make_load(L, j, P.N, m);
    const StoreCtx sc = make_store(S, j, P.N, m);
    phase_tile<LOGN, FWD, COLS, LM, SM, Q1>(sm, P, tw, m.q, lc, sc, tile);
}

// ---------------------------------------------------------------------------
// host-side launch of one instantiation
// ---------------------------------------------------------------------------
struct PhaseLaunch {
    int tiles, threads;
    size_t smem;
    cudaStream_t st;
};

#ifndef CKKS_NTT_MINB
#define CKKS_NTT_MINB 2         // run-time modes: 128 registers, two CTAs per SM
#endif
#ifndef CKKS_NTT_FAST_MINB
#define CKKS_NTT_FAST_MINB 3    // fixed modes: 80 registers, three CTAs per SM
#endif
#ifndef CKKS_NTT_EQ17_MINB
#define CKKS_NTT_EQ17_MINB 3    // the Eq. 17 load spills a little at 80 registers; three CTAs per SM
                                // still run the phase 9 % faster than two at 128
#endif

template <typename K>
static inline cudaError_t allow_smem(K kern, size_t smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <int LOGN, bool FWD, bool COLS, int LM, int SM, int MINB, bool Q1>
static inline cudaError_t launch_uniform(const NttPhase &P, const LimbJobs &J, const LoadSpec &L,
                                         const StoreSpec &S, const PhaseLaunch &G) {
    auto kern = ntt_phase_kernel<LOGN, FWD, COLS, LM, SM, MINB, Q1>;
    cudaError_t e = allow_smem(kern, G.smem);
    if (e != cudaSuccess) return e;
    dim3 grid(G.tiles, J.n_batch * J.n_polys * J.n_limbs);
    kern<<<grid, G.threads, G.smem, G.st>>>(P, J, L, S);
    return cudaGetLastError();
}

template <int LOGN, bool FWD, bool COLS, int LM, int SM, int MINB, bool Q1>
static inline cudaError_t launch_table(const NttPhase &P, const NttJob *jobs, int n_jobs, const LoadSpec &L,
                                       const StoreSpec &S, const PhaseLaunch &G) {
    auto kern = ntt_phase_table_kernel<LOGN, FWD, COLS, LM, SM, MINB, Q1>;
    cudaError_t e = allow_smem(kern, G.smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)n_jobs * G.tiles;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, G.threads, G.smem, G.st>>>(P, jobs, G.tiles, L, S);
    return cudaGetLastError();
}

// Dispatch of one direction (FWD) and job source (TABLE) over the phase
// geometry (cols, log2 n) and the modes. dispatch_fast launches the
// specialised kernel for the mode combinations of the hot path at n = 128 /
// 256 (N = 2^14 .. 2^16), with the modular products in the form Q1 selects,
// and sets `found`; dispatch_generic launches the run-time-mode kernel (the
// general products, valid for every prime).
#define CKKS_LAUNCH(LG, CO, LMv, SMv, MB, Q)                                                         \
    do {                                                                                             \
        if constexpr (TABLE) return launch_table<LG, FWD, CO, LMv, SMv, MB, Q>(P, jobs, n_jobs, L, S, G); \
        else return launch_uniform<LG, FWD, CO, LMv, SMv, MB, Q>(P, *J, L, S, G);                    \
    } while (0)

template <bool FWD, bool TABLE, bool Q1>
static inline cudaError_t dispatch_fast(bool cols, int logn, const NttPhase &P, const LimbJobs *J,
                                        const NttJob *jobs, int n_jobs, const LoadSpec &L, const StoreSpec &S,
                                        const PhaseLaunch &G, bool &found) {
    found = true;
    // specialised: the phase that fuses a mode has the plain mode on its other side
#define CKKS_FAST(LG)                                                                              \
    if (logn == LG) {                                                                              \
        if constexpr (FWD) {                                                                       \
            if (cols && S.mode == ST_LAZY) {                                                       \
                if (L.mode == LD_PLAIN) CKKS_LAUNCH(LG, true, LD_PLAIN, ST_LAZY, CKKS_NTT_FAST_MINB, Q1); \
                if (L.mode == LD_EQ17) CKKS_LAUNCH(LG, true, LD_EQ17, ST_LAZY, CKKS_NTT_EQ17_MINB, Q1);   \
            }                                                                                      \
            if (!cols && L.mode == LD_PLAIN) {                                                     \
                if (S.mode == ST_REDUCE) CKKS_LAUNCH(LG, false, LD_PLAIN, ST_REDUCE, CKKS_NTT_FAST_MINB, Q1); \
                if (S.mode == ST_MRS) CKKS_LAUNCH(LG, false, LD_PLAIN, ST_MRS, CKKS_NTT_FAST_MINB, Q1);   \
            }                                                                                      \
        } else {                                                                                   \
            if (!cols && S.mode == ST_LAZY) {                                                      \
                if (L.mode == LD_PLAIN) CKKS_LAUNCH(LG, false, LD_PLAIN, ST_LAZY, CKKS_NTT_FAST_MINB, Q1); \
                if (L.mode == LD_ADD) CKKS_LAUNCH(LG, false, LD_ADD, ST_LAZY, CKKS_NTT_FAST_MINB, Q1);    \
            }                                                                                      \
            if (cols && L.mode == LD_PLAIN) {                                                      \
                if (S.mode == ST_SCALE) CKKS_LAUNCH(LG, true, LD_PLAIN, ST_SCALE, CKKS_NTT_FAST_MINB, Q1); \
                if (S.mode == ST_MODDOWN) CKKS_LAUNCH(LG, true, LD_PLAIN, ST_MODDOWN, CKKS_NTT_FAST_MINB, Q1); \
            }                                                                                      \
        }                                                                                          \
    }
    CKKS_FAST(7)
    CKKS_FAST(8)
#undef CKKS_FAST
    found = false;
    return cudaSuccess;
}

template <bool FWD, bool TABLE>
static inline cudaError_t dispatch_generic(bool cols, int logn, const NttPhase &P, const LimbJobs *J,
                                           const NttJob *jobs, int n_jobs, const LoadSpec &L, const StoreSpec &S,
                                           const PhaseLaunch &G) {
#define CKKS_GENERIC(LG)                                                          \
    case LG:                                                                      \
        if (cols) CKKS_LAUNCH(LG, true, -1, -1, CKKS_NTT_MINB, false);            \
        CKKS_LAUNCH(LG, false, -1, -1, CKKS_NTT_MINB, false)
    switch (logn) {
        CKKS_GENERIC(1);
        CKKS_GENERIC(2);
        CKKS_GENERIC(3);
        CKKS_GENERIC(4);
        CKKS_GENERIC(5);
        CKKS_GENERIC(6);
        CKKS_GENERIC(7);
        CKKS_GENERIC(8);
    default:
        return cudaErrorInvalidValue;
    }
#undef CKKS_GENERIC
}
#undef CKKS_LAUNCH

// general products: the specialised kernel if one matches, else the generic one
template <bool FWD, bool TABLE>
static inline cudaError_t dispatch_phase(bool cols, int logn, const NttPhase &P, const LimbJobs *J,
                                         const NttJob *jobs, int n_jobs, const LoadSpec &L, const StoreSpec &S,
                                         const PhaseLaunch &G) {
    bool found;
    const cudaError_t e = dispatch_fast<FWD, TABLE, false>(cols, logn, P, J, jobs, n_jobs, L, S, G, found);
    if (found) return e;
    return dispatch_generic<FWD, TABLE>(cols, logn, P, J, jobs, n_jobs, L, S, G);
}

// ntt_uf.cu / ntt_ui.cu / ntt_tf.cu / ntt_ti.cu: general products;
// ntt_uf1.cu / ntt_ui1.cu / ntt_tf1.cu / ntt_ti1.cu: the specialised kernels
// with the products for primes = 1 (mod 2^32) (`found` false when none
// matches: the caller then takes the general dispatch)
cudaError_t ntt_dispatch_q1_uniform_fwd(bool cols, int logn, const NttPhase &P, const LimbJobs &J,
                                        const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G, bool &found);
cudaError_t ntt_dispatch_q1_uniform_inv(bool cols, int logn, const NttPhase &P, const LimbJobs &J,
                                        const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G, bool &found);
cudaError_t ntt_dispatch_q1_table_fwd(bool cols, int logn, const NttPhase &P, const NttJob *jobs, int n_jobs,
                                      const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G, bool &found);
cudaError_t ntt_dispatch_q1_table_inv(bool cols, int logn, const NttPhase &P, const NttJob *jobs, int n_jobs,
                                      const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G, bool &found);
cudaError_t ntt_dispatch_uniform_fwd(bool cols, int logn, const NttPhase &P, const LimbJobs &J, const LoadSpec &L,
                                     const StoreSpec &S, const PhaseLaunch &G);
cudaError_t ntt_dispatch_uniform_inv(bool cols, int logn, const NttPhase &P, const LimbJobs &J, const LoadSpec &L,
                                     const StoreSpec &S, const PhaseLaunch &G);
cudaError_t ntt_dispatch_table_fwd(bool cols, int logn, const NttPhase &P, const NttJob *jobs, int n_jobs,
                                   const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G);
cudaError_t ntt_dispatch_table_inv(bool cols, int logn, const NttPhase &P, const NttJob *jobs, int n_jobs,
                                   const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G);

}  // namespace ckks
