// Internal declarations of the CKKS multi-input multiplication library.
#pragma once
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "common.cuh"

namespace ckks {

// LD_PLAIN   a
// LD_ADD     a + b
// LD_EQ17    sum_t g_t T_t, or g_self a - sum_t g_t T_t (Eq. 17)
// LD_BCONVK  sum_i z_i [p_i^-1]_q (scaled BConv of Eq. 12; z = b)
enum LoadMode { LD_PLAIN = 0, LD_ADD = 1, LD_EQ17 = 2, LD_BCONVK = 3 };
// ST_REDUCE  canonical value
// ST_LAZY    lazy value (between the two phases)
// ST_SCALE   v * c (Shoup constant per launch limb)
// ST_MODDOWN v * c - sum_i z_i [p_i^-1]_q  (Eq. 5 with Eq. 11 / 12; z = aux)
// ST_MRS     g A - v   (last step of Algorithm 1; A = aux)
// ST_ADDSUB  aux + aux2 - v (prior ModDown finished in the NTT domain)
enum StoreMode { ST_REDUCE = 0, ST_LAZY = 1, ST_SCALE = 2, ST_MODDOWN = 3, ST_MRS = 4, ST_ADDSUB = 5 };

enum OpCounter {
    OP_NTT_PHASE = 0,
    OP_INTT_PHASE,
    OP_LIMB_NTT,     // limb forward transforms
    OP_LIMB_INTT,    // limb inverse transforms
    OP_BCONV,        // basis conversions (one per source digit / ModDown poly)
    OP_KERNELS,      // every kernel launch
    OP_COUNT
};

struct NttPhase {
    int N, N1, N2;
    int sub_per_tile, log_sub, log_n2;
    const ModQ *mods;
    const ulonglong2 *tw_fwd;
    const ulonglong2 *tw_inv;
};

struct LoadSpec {
    int mode;
    LimbView a, b;
    const Shoup *g;     // LD_EQ17: [limb][mu + 1] Shoup constants
    int mu;
    int with_self;
    const ModQ *mods;   // LD_BCONVK
    const u64 *cK;      // LD_BCONVK: [prime][64] Montgomery constants
    int K;
};

struct StoreSpec {
    int mode;
    LimbView dst, aux, aux2;
    const Shoup *c;     // per launch-limb Shoup constant, c[l * c_stride]
    int c_stride;
    const ModQ *mods;   // ST_MODDOWN
    const u64 *cK;      // ST_MODDOWN: [prime][64] Montgomery constants
    int K;
};

// One limb of an NTT phase launch whose limbs come from a device table
// (cross-shape launches): every pointer is the limb's own; the load and
// store modes and the per-prime constant tables stay per launch (LoadSpec /
// StoreSpec).
struct NttJob {
    const u64 *a;       // load: input limb (LD_PLAIN, first addend of LD_ADD, self term of LD_EQ17)
    const u64 *b;       // load: LD_ADD second addend; LD_EQ17 / LD_BCONVK first of the limbs N apart
    u64 *dst;           // store: output limb
    const u64 *aux;     // store: ST_MRS A limb; ST_MODDOWN first z limb (limbs N apart); ST_ADDSUB first addend
    const u64 *aux2;    // store: ST_ADDSUB second addend
    const Shoup *g;     // LD_EQ17: g[0..mu-1], g[mu] = self
    const Shoup *c;     // ST_SCALE / ST_MODDOWN / ST_MRS constant
    int prime;          // prime index (Q primes first, then P primes)
    int mu;             // LD_EQ17
    int with_self;      // LD_EQ17
    int pad;
};

// Kernel classes of the timing hook.
enum KernelClass {
    KC_NTT_FWD_COLS = 0,
    KC_NTT_FWD_BLOCKS,
    KC_NTT_INV_BLOCKS,
    KC_NTT_INV_COLS,
    KC_TENSOR,
    KC_BCONV,
    KC_MAC,
    KC_RSCHAIN,
    KC_KEYS,
    KC_AUTOMORPHISM,
    KC_COUNT
};

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes;
    double ops;   // integer work units of the launch (see ProfScope)
};

struct Profiler {
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
};

// Level-dependent constant tables live in one device allocation; offsets are
// host-side.
struct Context {
    int device = 0;
    int log_n = 0, N = 0, L = 0, K = 0, dnum = 0, alpha = 0;
    std::vector<u64> primes;  // q_0..q_{L-1}, p_0..p_{K-1}
    // host copies used to build per-call constants
    std::vector<Shoup> h_ninv;
    // device tables
    ModQ *d_mods = nullptr;           // [L+K]
    ulonglong2 *d_tw_fwd = nullptr;   // [L+K][N]
    ulonglong2 *d_tw_inv = nullptr;   // [L+K][N]
    Shoup *d_ninv = nullptr;          // [L+K]   N^-1
    Shoup *d_one = nullptr;           // [L+K]   (1, floor(2^64/q)): x mod q for any x
    Shoup *d_pscale = nullptr;        // [K]     N^-1 [phat_i^-1]_{p_i}
    u64 *d_cK = nullptr;              // [L+K][64]: row j < L: [p_i^-1 R]_{q_j}
    u64 *d_r2 = nullptr;              // [L+K]   R^2 mod q
    Shoup *d_rfix = nullptr;          // [L+K][16] R^(e-1) mod q (Shoup), e >= 1
    u64 *d_keyfold = nullptr;         // [L+K]   Q limbs: P^-1 R^2, P limbs: R^2 (mod prime)
    Shoup *d_invq = nullptr;          // [64][64] inv(prime i) mod prime j
    Shoup *d_bconv_pre = nullptr;     // [L+1][L] level, limb: N^-1 [(Q_beta/q_j)^-1]_{q_j}
    u64 *d_bconv_c = nullptr;         // [L+1][dnum][alpha][L+K] Montgomery [(Q_beta/q_j) mod x] R
    Shoup *d_g = nullptr;             // Eq. 16 tables, offsets g_off[level][mu]
    std::vector<std::vector<size_t>> g_off;
    unsigned long long *d_check = nullptr;  // [2] residue-check counter (zero between calls)
    Shoup *d_pgadget = nullptr;       // [dnum][L+K] P G_beta mod x (Q limbs), 0 for P limbs
    void *d_block = nullptr;          // one allocation holding all tables
    std::atomic<unsigned long long> counters[OP_COUNT];
    std::atomic<int> sticky{0};
    Profiler prof;
    // launch tunables
    int tune_ntt_tile_cols = 4096;    // elements per CTA tile, column phases
    int tune_ntt_tile_blocks = 4096;  // elements per CTA tile, block phases
    int tune_bconv_threads = 256;
    int tune_mac_threads = 256;
    // forms of the rescaling (same results; for measuring the paper's
    // reformulations): see multi_rs and run_mul_k in engine.cu
    int tune_inner_rescale = 0;
    int tune_root_rescale = 0;
    // key switching: 0 = one ModDown over the summed keys (Eq. 15), 1 = one
    // ModDown per key, summed afterwards (the form before Eq. 15)
    int tune_moddown = 0;
    // debugging aids: 1 = count residues >= q in the inputs and after every
    // stage of a k-input product (the call then synchronises and fails with
    // CKKS_ECHECK on a violation); 1 = NVTX ranges per tree node and stage
    int tune_check_residues = 0;
    int tune_nvtx = 0;
    // tensor products of tree nodes whose children are all multi-term tuples
    // and whose shape is one of the compiled ones (rns.cu, kFixedShapes) run
    // exactly unrolled kernels for that shape; 0 = the bounded generic kernels
    int tune_tensor_fixed = 1;
    // every prime (Q and P) is 1 (mod 2^32): the kernels can then take the
    // cheaper forms of the Shoup product and of REDC (shoup_lazy_q1,
    // redc_q1); set at creation. tune_q1 = 0 keeps the general forms.
    bool primes_q1 = false;
    int tune_q1 = 1;
    bool q1() const { return primes_q1 && tune_q1 != 0; }
};

// Records CUDA events around one launch on its stream when the hook is on;
// `bytes` is the launch's algorithmic traffic (each input and output limb
// counted once); `ops` its integer work: for NTT phases the Shoup products
// (one per butterfly plus the fused load / store scalings), for BConv and
// the key MAC the 64 x 64 -> 128-bit multiply-accumulates, 0 where not
// counted.
struct ProfScope {
    Context *C;
    int cls;
    double bytes;
    double ops;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    ProfScope(const Context &c, int k, double by, cudaStream_t s, double ops = 0.0);
    ~ProfScope();
};

struct Plan;

// counters (host side, counted when work is enqueued)
inline void count_op(const Context &C, int op, unsigned long long n = 1) {
    const_cast<Context &>(C).counters[op].fetch_add(n, std::memory_order_relaxed);
}
inline void count_kernel(const Context &C) { count_op(C, OP_KERNELS, 1); }

// ntt.cu
void ntt_geometry(int logN, int &log_n1, int &log_n2);
// phase launch over a device table of NttJob (ntt_launch.cu); jobs: device
// array of n_jobs entries
cudaError_t launch_ntt_phase_table(const Context &C, bool fwd, bool cols, const NttJob *jobs, int n_jobs,
                                   const LoadSpec &L, const StoreSpec &S, double alg_bytes, double ops,
                                   cudaStream_t st);
cudaError_t launch_ntt_phase(const Context &C, bool fwd, bool cols, const LimbJobs &J, const LoadSpec &L,
                             const StoreSpec &S, cudaStream_t st);
cudaError_t ntt_transform(const Context &C, bool fwd, const LimbJobs &J, const LoadSpec &L, const StoreSpec &S,
                          const StoreSpec *mid, cudaStream_t st);

}  // namespace ckks

// The opaque handle of the C ABI (include/ckks_mulk.h): one definition for
// every translation unit that unwraps it.
struct ckks_context {
    ckks::Context c;
};

// The evaluation-key set and the plan handles of the C ABI.
struct ckks_evk_set {
    ckks_context *ctx;
    u64 *keys;
    uint32_t t_max;
    unsigned long long sum;  // checksum of the prepared keys, taken at creation
};
