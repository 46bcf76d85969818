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
template <int LOGN, int P>
struct Pass {
    static constexpr int NP = (LOGN + 3) / 4;
    static constexpr int base = LOGN / NP;
    static constexpr int extra = LOGN % NP;
    static constexpr int len = base + (P < extra ? 1 : 0);
    static constexpr int start = P * base + (P < extra ? P : extra);
};

// Shared-memory layouts of a tile.
//   columns: [n][C] row-major (C sub-problems side by side); thread index
//            runs over sub-problems fastest.
//   blocks:  [B][n + n/16] with one pad word per 16; thread index runs over
//            point sets fastest.
template <bool COLS>
struct Layout {
    int n_sub, n;
    __device__ __forceinline__ int off(int sp, int k) const {
        if (COLS) return k * n_sub + sp;
        return sp * (n + (n >> 4)) + k + (k >> 4);
    }
    __device__ __forceinline__ void split(int s, int sets, int &sp, int &set) const {
        if (COLS) { sp = s % n_sub; set = s / n_sub; }
        else { set = s % sets; sp = s / sets; }
    }
};

template <int LOGN, int R, int E0, bool FWD, bool COLS>
__device__ __forceinline__ void run_pass(u64 *sm, const Layout<COLS> &lay, const ulonglong2 *tw,
                                         int tw_b0, int tw_bmul, u64 q) {
    constexpr int n = 1 << LOGN;
    constexpr int EL = 1 << R;
    constexpr int t_min = n >> (E0 + R);
    constexpr int t0 = n >> (E0 + 1);
    constexpr int sets = n >> R;
    const int total = lay.n_sub * sets;
    for (int s = threadIdx.x; s < total; s += blockDim.x) {
        int sp, set;
        lay.split(s, sets, sp, set);
        const int o = set % t_min;
        const int g = set / t_min;
        const int base = g * 2 * t0 + o;
        u64 x[EL];
#pragma unroll
        for (int k = 0; k < EL; ++k) x[k] = sm[lay.off(sp, base + k * t_min)];
        // twiddle index m_loc * twb + i_loc with twb = tw_b0 + tw_bmul * sp
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
        for (int k = 0; k < EL; ++k) sm[lay.off(sp, base + k * t_min)] = x[k];
    }
}

template <int LOGN, bool FWD, bool COLS, int P>
__device__ __forceinline__ void run_passes(u64 *sm, const Layout<COLS> &lay, const ulonglong2 *tw,
                                           int tw_b0, int tw_bmul, u64 q) {
    constexpr int NP = Pass<LOGN, 0>::NP;
    if constexpr (P < NP) {
        constexpr int PP = FWD ? P : NP - 1 - P;
        run_pass<LOGN, Pass<LOGN, PP>::len, Pass<LOGN, PP>::start, FWD, COLS>(sm, lay, tw, tw_b0, tw_bmul, q);
        __syncthreads();
        run_passes<LOGN, FWD, COLS, P + 1>(sm, lay, tw, tw_b0, tw_bmul, q);
    }
}

// ---------------------------------------------------------------------------
// fused element-wise load / store
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 load_elem(const LoadSpec &L, const LimbJobs &J, int N, int b, int p, int l,
                                         int prime, u64 q, int e) {
    const int slot = J.slot[l];
    switch (L.mode) {
    case LD_ADD: {
        u64 x = limb_ptr(L.a, b, p, slot, N)[e];
        u64 y = limb_ptr(L.b, b, p, slot, N)[e];
        return add_mod(x, y, q);
    }
    case LD_EQ17: {
        // sum_t g_t T_t (mod q); with the self term: g_self a - sum
        const Shoup *g = L.g + (i64)l * (L.mu + 1);
        const u64 *T = L.b.ptr + (i64)b * L.b.bstride + (i64)p * L.b.pstride + e;
        u64 s = 0;
        for (int t = 0; t < L.mu; ++t) s = add_mod(s, shoup(T[(i64)t * N], g[t].w, g[t].wp, q), q);
        if (L.with_self) {
            u64 a = limb_ptr(L.a, b, p, slot, N)[e];
            s = sub_mod(shoup(a, g[L.mu].w, g[L.mu].wp, q), s, q);
        }
        return s;
    }
    case LD_BCONVK: {
        ModQ m = L.mods[prime];
        const u64 *cK = L.cK + (i64)prime * CKKS_MAX_PRIMES;
        const u64 *z = L.b.ptr + (i64)b * L.b.bstride + (i64)p * L.b.pstride + e;
        Acc128 acc;
        acc.zero();
        for (int i = 0; i < L.K; ++i) acc.mac(z[(i64)i * N], cK[i], q);
        return redc(acc.hi, acc.lo, m);
    }
    default:
        return limb_ptr(L.a, b, p, slot, N)[e];
    }
}

__device__ __forceinline__ void store_elem(const StoreSpec &S, const LimbJobs &J, int N, int b, int p, int l,
                                           int prime, u64 q, int e, u64 v, bool fwd) {
    u64 *dst = limb_ptr(S.dst, b, p, J.dslot[l], N) + e;
    switch (S.mode) {
    case ST_LAZY:
        *dst = v;
        break;
    case ST_SCALE: {
        Shoup c = S.c[l * S.c_stride];
        *dst = shoup(v, c.w, c.wp, q);
        break;
    }
    case ST_MODDOWN: {
        // c* = v N^-1 - sum_i z_i [p_i^-1 R]_q  (Eq. 5 with Eq. 11/12)
        Shoup c = S.c[l * S.c_stride];
        u64 x = shoup(v, c.w, c.wp, q);
        ModQ m = S.mods[prime];
        const u64 *cK = S.cK + (i64)prime * CKKS_MAX_PRIMES;
        const u64 *z = S.aux.ptr + (i64)b * S.aux.bstride + (i64)p * S.aux.pstride + e;
        Acc128 acc;
        acc.zero();
        for (int i = 0; i < S.K; ++i) acc.mac(z[(i64)i * N], cK[i], q);
        *dst = sub_mod(x, redc(acc.hi, acc.lo, m), q);
        break;
    }
    case ST_MRS: {
        // Algorithm 1, last step: A' = g^{mu,L-1} A - B (A read from aux)
        Shoup c = S.c[l * S.c_stride];
        u64 a = limb_ptr(S.aux, b, p, J.dslot[l], N)[e];
        *dst = sub_mod(shoup(a, c.w, c.wp, q), fwd ? reduce4(v, q) : reduce2(v, q), q);
        break;
    }
    case ST_ADDSUB: {
        u64 a = limb_ptr(S.aux, b, p, J.dslot[l], N)[e];
        u64 c = limb_ptr(S.aux2, b, p, J.dslot[l], N)[e];
        *dst = sub_mod(add_mod(a, c, q), fwd ? reduce4(v, q) : reduce2(v, q), q);
        break;
    }
    default:  // ST_REDUCE
        *dst = fwd ? reduce4(v, q) : reduce2(v, q);
        break;
    }
}

// ---------------------------------------------------------------------------
// the phase kernel
// ---------------------------------------------------------------------------
template <int LOGN, bool FWD, bool COLS>
__global__ void __launch_bounds__(256) ntt_phase_kernel(NttPhase P, LimbJobs J, LoadSpec L, StoreSpec S) {
    extern __shared__ u64 sm[];
    constexpr int n = 1 << LOGN;
    int b, p, l;
    decode_job(J, blockIdx.y, b, p, l);
    const int prime = J.prime[l];
    const u64 q = P.mods[prime].q;
    const ulonglong2 *tw = (FWD ? P.tw_fwd : P.tw_inv) + (i64)prime * P.N;
    const int n_sub = P.sub_per_tile;
    Layout<COLS> lay{n_sub, n};
    const int t0 = blockIdx.x * n_sub;  // first column (COLS) or block (!COLS)
    const int total = n_sub * n;
    // global -> shared with the fused load
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int sp, k, e;
        if (COLS) { k = idx / n_sub; sp = idx % n_sub; e = t0 + sp + k * P.N2; }
        else { sp = idx / n; k = idx % n; e = (t0 + sp) * n + k; }
        sm[lay.off(sp, k)] = load_elem(L, J, P.N, b, p, l, prime, q, e);
    }
    __syncthreads();
    // twiddle base: columns -> 1; blocks -> N1 + block
    const int tw_b0 = COLS ? 1 : P.N1 + t0;
    const int tw_bmul = COLS ? 0 : 1;
    run_passes<LOGN, FWD, COLS, 0>(sm, lay, tw, tw_b0, tw_bmul, q);
    // shared -> global with the fused store
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int sp, k, e;
        if (COLS) { k = idx / n_sub; sp = idx % n_sub; e = t0 + sp + k * P.N2; }
        else { sp = idx / n; k = idx % n; e = (t0 + sp) * n + k; }
        store_elem(S, J, P.N, b, p, l, prime, q, e, sm[lay.off(sp, k)], FWD);
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

static constexpr int kTileElems = 4096;

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
        n_sub = kTileElems / n;
        if (n_sub > P.N2) n_sub = P.N2;
        tiles = P.N2 / n_sub;
        smem = (size_t)n * n_sub * sizeof(u64);
    } else {
        logn = log_n2;
        int n = 1 << logn;
        n_sub = kTileElems / n;
        if (n_sub < 1) n_sub = 1;
        if (n_sub > P.N1) n_sub = P.N1;
        tiles = P.N1 / n_sub;
        smem = (size_t)n_sub * (n + n / 16) * sizeof(u64);
    }
    P.sub_per_tile = n_sub;
    int per_sub = (1 << logn) >= 16 ? (1 << logn) / 16 : 1;  // radix-16 point sets per sub-problem
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
    ProfScope ps(C, fwd ? (cols ? KC_NTT_FWD_COLS : KC_NTT_FWD_BLOCKS) : (cols ? KC_NTT_INV_COLS : KC_NTT_INV_BLOCKS),
                 bytes, st);
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
