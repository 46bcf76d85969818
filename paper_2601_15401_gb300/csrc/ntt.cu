// Host side of the negacyclic NTT / INTT (the kernels and their design are
// described in ntt_kernel.cuh): phase geometry, algorithmic byte and Shoup
// product counts for the timing hook, and the two-phase transform with fused
// first load / last store.
#include "common.cuh"
#include "internal.h"
#include "ntt_kernel.cuh"

namespace ckks {

// Geometry of the two phases for a given log N.
void ntt_geometry(int logN, int &log_n1, int &log_n2) {
    if (logN <= 8) { log_n1 = 0; log_n2 = logN; }
    else { log_n1 = logN / 2; log_n2 = logN - log_n1; }
}

// Tile shape of one phase: sub-problems per CTA from the context's tile
// tunables, CTAs per limb, threads and shared memory per CTA.
static int phase_geometry(const Context &C, bool cols, NttPhase &P, PhaseLaunch &G) {
    int log_n1, log_n2;
    ntt_geometry(C.log_n, log_n1, log_n2);
    P.N = C.N;
    P.N1 = 1 << log_n1;
    P.N2 = 1 << log_n2;
    P.mods = C.d_mods;
    P.tw_fwd = C.d_tw_fwd;
    P.tw_inv = C.d_tw_inv;
    int logn, n_sub;
    if (cols) {
        logn = log_n1;
        int n = 1 << logn;
        n_sub = C.tune_ntt_tile_cols / n;
        if (n_sub > P.N2) n_sub = P.N2;
        G.tiles = P.N2 / n_sub;
        G.smem = (size_t)n * n_sub * sizeof(u64) + (CKKS_NTT_COL_TW_SMEM ? (size_t)n * sizeof(ulonglong2) : 0);
    } else {
        logn = log_n2;
        int n = 1 << logn;
        n_sub = C.tune_ntt_tile_blocks / n;
        if (n_sub < 1) n_sub = 1;
        if (n_sub > P.N1) n_sub = P.N1;
        G.tiles = P.N1 / n_sub;
        G.smem = (size_t)n_sub * (n + n / 16) * sizeof(u64);
    }
    P.sub_per_tile = n_sub;
    P.log_sub = 0;
    while ((1 << P.log_sub) < n_sub) ++P.log_sub;
    P.log_n2 = log_n2;
    int per_sub = (1 << logn) >= (1 << CKKS_NTT_RMAX) ? (1 << logn) >> CKKS_NTT_RMAX : 1;  // point sets per sub-problem
    int threads = ((n_sub * per_sub + 31) / 32) * 32;
    G.threads = threads > 256 ? 256 : threads;
    return logn;
}

// One phase. phase 0 = the first phase executed (forward: columns; inverse:
// blocks), phase 1 = the second. With log_n1 == 0 there is only phase 1 work
// done as a single block phase over the whole limb.
cudaError_t launch_ntt_phase(const Context &C, bool fwd, bool cols, const LimbJobs &J, const LoadSpec &L,
                             const StoreSpec &S, cudaStream_t st) {
    NttPhase P;
    PhaseLaunch G;
    const int logn = phase_geometry(C, cols, P, G);
    G.st = st;
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
    if (C.q1()) {
        bool found;
        const cudaError_t e = fwd ? ntt_dispatch_q1_uniform_fwd(cols, logn, P, J, L, S, G, found)
                                  : ntt_dispatch_q1_uniform_inv(cols, logn, P, J, L, S, G, found);
        if (found) return e;
    }
    return fwd ? ntt_dispatch_uniform_fwd(cols, logn, P, J, L, S, G)
               : ntt_dispatch_uniform_inv(cols, logn, P, J, L, S, G);
}

// One phase over a device table of limbs (cross-shape launches). The caller
// counts the algorithmic bytes and Shoup products (they depend on the
// table's entries).
cudaError_t launch_ntt_phase_table(const Context &C, bool fwd, bool cols, const NttJob *jobs, int n_jobs,
                                   const LoadSpec &L, const StoreSpec &S, double alg_bytes, double ops,
                                   cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    NttPhase P;
    PhaseLaunch G;
    const int logn = phase_geometry(C, cols, P, G);
    G.st = st;
    count_op(C, fwd ? OP_NTT_PHASE : OP_INTT_PHASE);
    count_kernel(C);
    ProfScope ps(C, fwd ? (cols ? KC_NTT_FWD_COLS : KC_NTT_FWD_BLOCKS) : (cols ? KC_NTT_INV_COLS : KC_NTT_INV_BLOCKS),
                 alg_bytes, st, ops);
    if (C.q1()) {
        bool found;
        const cudaError_t e = fwd ? ntt_dispatch_q1_table_fwd(cols, logn, P, jobs, n_jobs, L, S, G, found)
                                  : ntt_dispatch_q1_table_inv(cols, logn, P, jobs, n_jobs, L, S, G, found);
        if (found) return e;
    }
    return fwd ? ntt_dispatch_table_fwd(cols, logn, P, jobs, n_jobs, L, S, G)
               : ntt_dispatch_table_inv(cols, logn, P, jobs, n_jobs, L, S, G);
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
