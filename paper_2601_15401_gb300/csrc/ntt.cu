// Negacyclic NTT / INTT over 64-bit NTT-friendly primes.
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
#include "common.cuh"
#include "internal.h"

namespace ckks {

// ---------------------------------------------------------------------------
// butterflies
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 q) {
    u64 q2 = q << 1;
    u64 x = X >= q2 ? X - q2 : X;
    u64 t = shoup_lazy(Y, w.x, w.y, q);
    X = x + t;
    Y = x - t + q2;
}

__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 q) {
    u64 q2 = q << 1;
    u64 s = X + Y;
    s = s >= q2 ? s - q2 : s;
    u64 d = X - Y + q2;
    Y = shoup_lazy(d, w.x, w.y, q);
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

__device__ __forceinline__ u64 load_elem(const LoadCtx &c, int e) {
    const u64 q = c.m.q;
    switch (c.mode) {
    case LD_ADD:
        return add_mod(c.a[e], c.b[e], q);
    case LD_EQ17: {
        // sum_t g_t T_t (mod q); with the self term: g_self a - sum
        u64 s = 0;
        for (int t = 0; t < c.mu; ++t) s = add_mod(s, shoup(c.b[(i64)t * c.N + e], c.g[t].w, c.g[t].wp, q), q);
        if (c.with_self) s = sub_mod(shoup(c.a[e], c.g[c.mu].w, c.g[c.mu].wp, q), s, q);
        return s;
    }
    case LD_BCONVK: {
        Acc128Lazy acc;  // sum of the P primes < 2^64 (context check)
        acc.zero();
        for (int i = 0; i < c.K; ++i) acc.mac(c.b[(i64)i * c.N + e], c.cK[i]);
        return redc(acc.hi, acc.lo, c.m);
    }
    default:
        return c.a[e];
    }
}

__device__ __forceinline__ void store_elem(const StoreCtx &c, int e, u64 v, bool fwd) {
    const u64 q = c.m.q;
    switch (c.mode) {
    case ST_LAZY:
        c.dst[e] = v;
        break;
    case ST_SCALE:
        c.dst[e] = shoup(v, c.c.w, c.c.wp, q);
        break;
    case ST_MODDOWN: {
        // c* = v N^-1 - sum_i z_i [p_i^-1 R]_q  (Eq. 5 with Eq. 11 / 12)
        u64 x = shoup(v, c.c.w, c.c.wp, q);
        Acc128Lazy acc;  // sum of the P primes < 2^64 (context check)
        acc.zero();
        for (int i = 0; i < c.K; ++i) acc.mac(c.aux[(i64)i * c.N + e], c.cK[i]);
        c.dst[e] = sub_mod(x, redc(acc.hi, acc.lo, c.m), q);
        break;
    }
    case ST_MRS:
        // Algorithm 1, last step: A' = g^{mu,L-1} A - B
        c.dst[e] = sub_mod(shoup(c.aux[e], c.c.w, c.c.wp, q), fwd ? reduce4(v, q) : reduce2(v, q), q);
        break;
    case ST_ADDSUB:
        c.dst[e] = sub_mod(add_mod(c.aux[e], c.aux2[e], q), fwd ? reduce4(v, q) : reduce2(v, q), q);
        break;
    default:  // ST_REDUCE
        c.dst[e] = fwd ? reduce4(v, q) : reduce2(v, q);
        break;
    }
}

// One pass of R stages starting at local stage E0 on every point set of the
// tile. SRC/DST: 0 = shared memory, 1 = global (fused load / store).
template <int LOGN, int R, int E0, bool FWD, bool COLS, bool GIN, bool GOUT>
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
#pragma unroll
        for (int k = 0; k < EL; ++k) {
            const int pt = base + k * t_min;
            if (GIN) {
                const int e = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                x[k] = load_elem(lc, e);
            } else {
                x[k] = sm[lay.off(sp, pt)];
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
                        ct_bfly(x[k], x[k + h], tw[m * twb + i], q);
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
                        gs_bfly(x[k], x[k + h], tw[m * twb + i], q);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < EL; ++k) {
            const int pt = base + k * t_min;
            if (GOUT) {
                const int e = COLS ? t0 + sp + (pt << log_n2) : ((t0 + sp) << LOGN) + pt;
                store_elem(sc, e, x[k], FWD);
            } else {
                sm[lay.off(sp, pt)] = x[k];
            }
        }
    }
}

// Direct global access is used on a side whose pass reads / writes at
// least 8 consecutive words per sub-problem (always true for column tiles).
template <int LOGN, bool COLS, int P>
struct PassAccess {
    static constexpr int t_min = (1 << LOGN) >> (Pass<LOGN, P>::start + Pass<LOGN, P>::len);
    static constexpr bool direct = COLS || t_min >= 8;
};

template <int LOGN, bool FWD, bool COLS, int I>
__device__ __forceinline__ void run_passes(u64 *sm, const Layout<COLS, LOGN> &lay, const ulonglong2 *tw, int tw_b0,
                                           int tw_bmul, u64 q, const LoadCtx &lc, const StoreCtx &sc, int t0,
                                           int log_n2) {
    constexpr int NP = Pass<LOGN, 0>::NP;
    if constexpr (I < NP) {
        constexpr int PP = FWD ? I : NP - 1 - I;
        constexpr bool first = I == 0, last = I == NP - 1;
        constexpr bool gin = first && PassAccess<LOGN, COLS, PP>::direct;
        constexpr bool gout = last && PassAccess<LOGN, COLS, PP>::direct;
        run_pass<LOGN, Pass<LOGN, PP>::len, Pass<LOGN, PP>::start, FWD, COLS, gin, gout>(
            sm, lay, tw, tw_b0, tw_bmul, q, lc, sc, t0, log_n2);
        if (!last || !gout) __syncthreads();
        run_passes<LOGN, FWD, COLS, I + 1>(sm, lay, tw, tw_b0, tw_bmul, q, lc, sc, t0, log_n2);
    }
}

// ---------------------------------------------------------------------------
// the phase kernel
// ---------------------------------------------------------------------------
template <int LOGN, bool FWD, bool COLS>
#ifndef CKKS_NTT_MINB
#define CKKS_NTT_MINB 2
#endif
__global__ void __launch_bounds__(256, CKKS_NTT_MINB) ntt_phase_kernel(NttPhase P, LimbJobs J, LoadSpec L, StoreSpec S) {
    extern __shared__ u64 sm[];
    constexpr int n = 1 << LOGN;
    constexpr int NP = Pass<LOGN, 0>::NP;
    int b, p, l;
    decode_job(J, blockIdx.y, b, p, l);
    const int prime = J.prime[l];
    const ModQ m = P.mods[prime];
    const u64 q = m.q;
    const ulonglong2 *tw = (FWD ? P.tw_fwd : P.tw_inv) + (i64)prime * P.N;
    const int lsub = P.log_sub;
    const int n_sub = 1 << lsub;
    Layout<COLS, LOGN> lay{lsub};
    const int t0 = blockIdx.x << lsub;  // first column (COLS) or block (!COLS)
    const LoadCtx lc = make_load(L, J, P.N, b, p, l, prime, m);
    const StoreCtx sc = make_store(S, J, P.N, b, p, l, prime, m);
    constexpr int PF = FWD ? 0 : NP - 1;
    constexpr int PL = FWD ? NP - 1 : 0;
    constexpr bool gin = PassAccess<LOGN, COLS, PF>::direct;
    constexpr bool gout = PassAccess<LOGN, COLS, PL>::direct;
    const int total = n_sub << LOGN;
    if (!gin) {
        // coalesced global -> shared with the fused load
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int sp, k, e;
            if (COLS) { k = idx >> lsub; sp = idx & (n_sub - 1); e = t0 + sp + (k << P.log_n2); }
            else { sp = idx >> LOGN; k = idx & (n - 1); e = ((t0 + sp) << LOGN) + k; }
            sm[lay.off(sp, k)] = load_elem(lc, e);
        }
        __syncthreads();
    }
    // twiddle base: columns -> 1; blocks -> N1 + block
    const int tw_b0 = COLS ? 1 : P.N1 + t0;
    const int tw_bmul = COLS ? 0 : 1;
    run_passes<LOGN, FWD, COLS, 0>(sm, lay, tw, tw_b0, tw_bmul, q, lc, sc, t0, P.log_n2);
    if (!gout) {
        // shared -> global with the fused store (coalesced)
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int sp, k, e;
            if (COLS) { k = idx >> lsub; sp = idx & (n_sub - 1); e = t0 + sp + (k << P.log_n2); }
            else { sp = idx >> LOGN; k = idx & (n - 1); e = ((t0 + sp) << LOGN) + k; }
            store_elem(sc, e, sm[lay.off(sp, k)], FWD);
        }
    }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
template <int LOGN, bool FWD, bool COLS>
static cudaError_t launch_phase_t(const NttPhase &P, const LimbJobs &J, const LoadSpec &L, const StoreSpec &S,
                                  int tiles, int threads, size_t smem, cudaStream_t st) {
    auto kern = ntt_phase_kernel<LOGN, FWD, COLS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int jobs = J.n_batch * J.n_polys * J.n_limbs;
    dim3 grid(tiles, jobs);
    kern<<<grid, threads, smem, st>>>(P, J, L, S);
    return cudaGetLastError();
}

template <bool FWD, bool COLS>
static cudaError_t launch_phase_log(int logn, const NttPhase &P, const LimbJobs &J, const LoadSpec &L,
                                    const StoreSpec &S, int tiles, int threads, size_t smem, cudaStream_t st) {
    switch (logn) {
    case 1: return launch_phase_t<1, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 2: return launch_phase_t<2, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 3: return launch_phase_t<3, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 4: return launch_phase_t<4, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 5: return launch_phase_t<5, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 6: return launch_phase_t<6, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 7: return launch_phase_t<7, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    case 8: return launch_phase_t<8, FWD, COLS>(P, J, L, S, tiles, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// Geometry of the two phases for a given log N.
void ntt_geometry(int logN, int &log_n1, int &log_n2) {
    if (logN <= 8) { log_n1 = 0; log_n2 = logN; }
    else { log_n1 = logN / 2; log_n2 = logN - log_n1; }
}


// One phase. phase 0 = the first phase executed (forward: columns; inverse:
// blocks), phase 1 = the second. With log_n1 == 0 there is only phase 1 work
// done as a single block phase over the whole limb.
cudaError_t launch_ntt_phase(const Context &C, bool fwd, bool cols, const LimbJobs &J, const LoadSpec &L,
                             const StoreSpec &S, cudaStream_t st) {
    int log_n1, log_n2;
    ntt_geometry(C.log_n, log_n1, log_n2);
    NttPhase P;
    P.N = C.N;
    P.N1 = 1 << log_n1;
    P.N2 = 1 << log_n2;
    P.mods = C.d_mods;
    P.tw_fwd = C.d_tw_fwd;
    P.tw_inv = C.d_tw_inv;
    int logn, tiles, n_sub;
    size_t smem;
    if (cols) {
        logn = log_n1;
        int n = 1 << logn;
        n_sub = C.tune_ntt_tile_cols / n;
        if (n_sub > P.N2) n_sub = P.N2;
        tiles = P.N2 / n_sub;
        smem = (size_t)n * n_sub * sizeof(u64);
    } else {
        logn = log_n2;
        int n = 1 << logn;
        n_sub = C.tune_ntt_tile_blocks / n;
        if (n_sub < 1) n_sub = 1;
        if (n_sub > P.N1) n_sub = P.N1;
        tiles = P.N1 / n_sub;
        smem = (size_t)n_sub * (n + n / 16) * sizeof(u64);
    }
    P.sub_per_tile = n_sub;
    P.log_sub = 0;
    while ((1 << P.log_sub) < n_sub) ++P.log_sub;
    P.log_n2 = log_n2;
    int per_sub = (1 << logn) >= (1 << CKKS_NTT_RMAX) ? (1 << logn) >> CKKS_NTT_RMAX : 1;  // point sets per sub-problem
    int threads = ((n_sub * per_sub + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    count_op(C, fwd ? OP_NTT_PHASE : OP_INTT_PHASE);
    count_kernel(C);
    // algorithmic bytes: every launch limb read and written once, plus the
    // extra limbs its fused load / store touch
    const double limb = (double)C.N * sizeof(u64);
    const double jobs_d = (double)J.n_batch * J.n_polys * J.n_limbs;
    const double bp = (double)J.n_batch * J.n_polys;
    double bytes = 2.0 * jobs_d * limb;
    if (L.mode == LD_ADD) bytes += jobs_d * limb;
    if (L.mode == LD_EQ17) bytes += bp * L.mu * limb;
    if (L.mode == LD_BCONVK) bytes += bp * L.K * limb - jobs_d * limb;
    if (S.mode == ST_MODDOWN) bytes += bp * S.K * limb;
    if (S.mode == ST_MRS) bytes += jobs_d * limb;
    if (S.mode == ST_ADDSUB) bytes += 2.0 * jobs_d * limb;
    // integer work: one Shoup product per butterfly (log2 n stages of N / 2
    // per limb) plus the Shoup products of the fused load / store
    double ops = jobs_d * (double)C.N * 0.5 * logn;
    if (L.mode == LD_EQ17) ops += jobs_d * (double)C.N * (L.mu + L.with_self);
    if (S.mode == ST_SCALE || S.mode == ST_MODDOWN || S.mode == ST_MRS) ops += jobs_d * (double)C.N;
    ProfScope ps(C, fwd ? (cols ? KC_NTT_FWD_COLS : KC_NTT_FWD_BLOCKS) : (cols ? KC_NTT_INV_COLS : KC_NTT_INV_BLOCKS),
                 bytes, st, ops);
    if (fwd) {
        return cols ? launch_phase_log<true, true>(logn, P, J, L, S, tiles, threads, smem, st)
                    : launch_phase_log<true, false>(logn, P, J, L, S, tiles, threads, smem, st);
    }
    return cols ? launch_phase_log<false, true>(logn, P, J, L, S, tiles, threads, smem, st)
                : launch_phase_log<false, false>(logn, P, J, L, S, tiles, threads, smem, st);
}

// Full transform src -> dst with fused first load / last store. The first
// phase writes its lazy intermediate into dst (in place for the second).
cudaError_t ntt_transform(const Context &C, bool fwd, const LimbJobs &J, const LoadSpec &L, const StoreSpec &S,
                          const StoreSpec *mid, cudaStream_t st) {
    int log_n1, log_n2;
    ntt_geometry(C.log_n, log_n1, log_n2);
    count_op(C, fwd ? OP_LIMB_NTT : OP_LIMB_INTT, (unsigned long long)J.n_batch * J.n_polys * J.n_limbs);
    if (log_n1 == 0) return launch_ntt_phase(C, fwd, false, J, L, S, st);
    // first phase: forward -> columns, inverse -> blocks
    StoreSpec s1;
    if (mid) s1 = *mid;
    else { s1 = StoreSpec{}; s1.mode = ST_LAZY; s1.dst = S.dst; }
    cudaError_t e = launch_ntt_phase(C, fwd, fwd, J, L, s1, st);
    if (e != cudaSuccess) return e;
    // second phase reads the intermediate from s1.dst at the destination slots
    LimbJobs J2 = J;
    for (int i = 0; i < J.n_limbs; ++i) J2.slot[i] = J.dslot[i];
    LoadSpec l2{};
    l2.mode = LD_PLAIN;
    l2.a = s1.dst;
    return launch_ntt_phase(C, fwd, !fwd, J2, l2, S, st);
}

}  // namespace ckks
