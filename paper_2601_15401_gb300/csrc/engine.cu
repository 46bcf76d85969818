// Host orchestration of the k-input multiplication (Section V) and of the
// standard 2-input multiplication used as the comparator (Section II).
//
// Every step works on a whole batch of independent products in one launch:
// a tuple view is (pointer of batch element 0, batch stride, poly stride).
//
// Inner node (m children, mu = m - 1):
//   tensor product (Eq. 13) -> D [r+1][l]
//   Algorithm 1 in place: INTT of the mu top limbs (with N^-1), the rescale
//   chain among them, then one fused NTT per remaining limb whose load forms
//   b = sum_t g_t a_t (Eq. 17) and whose store forms A' = g A - B.
// Root (n + 1 = size of D):
//   INTT of d_2..d_n with the BConv prescale [(Q_beta/q_j)^-1] in the epilogue
//   ModUp BConv (Eq. 4) of every digit into Q_l u P, NTT of the new limbs
//   key inner product over all t and digits (Eq. 15, combined), keys holding
//   P^-1 on their Q rows (Eq. 12)
//   ModDown: INTT of the P limbs with [phat_i^-1] N^-1 in the epilogue, then
//   one INTT of (D_l + acc_l) per Q limb whose epilogue subtracts the scaled
//   BConv (Eq. 11 merged form + Eq. 12) -> c*_l, coefficient domain
//   relocated rescale (Section IV): the rescale chain among the mu top limbs
//   of c*, then one NTT per surviving limb with the Eq. 17 combination
//   (with the self term) fused into its load -> output, NTT domain.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <cmath>

#include "engine.h"
#include "internal.h"
#include "plan.h"
#include "rns.h"

namespace ckks {

// ---------------------------------------------------------------------------
// workspace bump allocator (dry run computes the size)
// ---------------------------------------------------------------------------
struct Ws {
    char *base;
    size_t off = 0;
    size_t cap;
    bool dry;
    u64 *take(size_t elems) {
        size_t bytes = (elems * sizeof(u64) + 255) / 256 * 256;
        u64 *p = dry ? nullptr : (u64 *)(base + off);
        off += bytes;
        return p;
    }
};

static LimbView view(u64 *ptr, i64 bstride, i64 pstride) {
    LimbView v;
    v.ptr = ptr;
    v.bstride = bstride;
    v.pstride = pstride;
    return v;
}

static LimbView offset(LimbView v, i64 elems) {
    v.ptr = v.ptr ? v.ptr + elems : nullptr;
    return v;
}

static LimbJobs jobs(int B, int polys, int nl) {
    LimbJobs J;
    J.n_batch = B;
    J.n_polys = polys;
    J.n_limbs = nl;
    for (int i = 0; i < CKKS_MAX_PRIMES; ++i) {
        J.slot[i] = 0;
        J.dslot[i] = 0;
        J.prime[i] = 0;
    }
    for (int i = 0; i < nl; ++i) {
        J.slot[i] = (uint8_t)i;
        J.dslot[i] = (uint8_t)i;
        J.prime[i] = (uint8_t)i;
    }
    return J;
}

#define TRY(x)                                   \
    do {                                         \
        cudaError_t _e = (x);                    \
        if (_e != cudaSuccess) return _e;        \
    } while (0)

// ---------------------------------------------------------------------------
// building blocks
// ---------------------------------------------------------------------------
// Plain transform of limbs [0, level) of every poly: in -> out.
cudaError_t transform_plain(const Context &C, bool fwd, int B, int polys, int level, LimbView in, LimbView out,
                            cudaStream_t st) {
    if (!in.ptr) return cudaSuccess;
    LimbJobs J = jobs(B, polys, level);
    LoadSpec L{};
    L.mode = LD_PLAIN;
    L.a = in;
    StoreSpec S{};
    S.dst = out;
    if (fwd) {
        S.mode = ST_REDUCE;
    } else {
        S.mode = ST_SCALE;
        S.c = C.d_ninv;
        S.c_stride = 1;
    }
    return ntt_transform(C, fwd, J, L, S, nullptr, st);
}

// Algorithm 1 on `polys` polynomials: in (level limbs, NTT) -> out (level - mu).
static cudaError_t multi_rs_alg1(const Context &C, Ws &ws, int B, int polys, int level, int mu, LimbView in,
                                 LimbView out, cudaStream_t st) {
    const int N = C.N;
    u64 *a = ws.take((size_t)B * polys * mu * N);
    u64 *bb = ws.take((size_t)B * polys * (level - mu) * N);
    if (ws.dry) return cudaSuccess;
    LimbView av = view(a, (i64)polys * mu * N, (i64)mu * N);
    // 1. INTT of the mu top limbs (N^-1 in the epilogue)
    {
        LimbJobs J = jobs(B, polys, mu);
        for (int l = 0; l < mu; ++l) {
            J.slot[l] = (uint8_t)(level - mu + l);
            J.dslot[l] = (uint8_t)l;
            J.prime[l] = (uint8_t)(level - mu + l);
        }
        LoadSpec L{};
        L.mode = LD_PLAIN;
        L.a = in;
        StoreSpec S{};
        S.mode = ST_SCALE;
        S.dst = av;
        S.c = C.d_ninv + (level - mu);
        S.c_stride = 1;
        TRY(ntt_transform(C, false, J, L, S, nullptr, st));
    }
    // 2. rescale chain among the top limbs
    {
        RsChainArgs R;
        R.n_batch = B;
        R.n_polys = polys;
        R.N = N;
        R.level = level;
        R.mu = mu;
        R.v = av;
        R.mods = C.d_mods;
        R.one = C.d_one;
        R.invq = C.d_invq;
        TRY(launch_rschain(C, R, st));
    }
    // 3. B = NTT(sum_t g_t a_t), A' = g_self A - B
    {
        LimbJobs J = jobs(B, polys, level - mu);
        const Shoup *g = C.d_g + C.g_off[level][mu];
        LoadSpec L{};
        L.mode = LD_EQ17;
        L.b = av;
        L.g = g;
        L.mu = mu;
        L.with_self = 0;
        StoreSpec mid{};
        mid.mode = ST_LAZY;
        mid.dst = view(bb, (i64)polys * (level - mu) * N, (i64)(level - mu) * N);
        StoreSpec S{};
        S.mode = ST_MRS;
        S.dst = out;
        S.aux = in;
        S.c = g + mu;
        S.c_stride = mu + 1;
        TRY(ntt_transform(C, true, J, L, S, &mid, st));
    }
    return cudaSuccess;
}

static cudaError_t root_rescale(const Context &C, int B, int level, int mu, LimbView cstar, LimbView out,
                                cudaStream_t st);

// Rescaling of a tuple by mu primes in the NTT domain, in the form the
// context's "inner_rescale" setting selects (all forms give the same
// residues, Section V-B):
//   0  Algorithm 1: mu INTT + (level - mu) NTT per polynomial;
//   1  mu single rescales of Eq. 7, one after the other;
//   2  INTT of every limb, the mu rescales of Eq. 6 in the coefficient
//      domain (combined as in Eq. 17), NTT of the survivors: level INTT +
//      (level - mu) NTT per polynomial (Table IV's baseline).
cudaError_t multi_rs(const Context &C, Ws &ws, int B, int polys, int level, int mu, LimbView in, LimbView out,
                     cudaStream_t st) {
    if (C.tune_inner_rescale == 1 && mu > 1) {
        TRY(multi_rs_alg1(C, ws, B, polys, level, 1, in, out, st));
        for (int j = 1; j < mu; ++j) TRY(multi_rs_alg1(C, ws, B, polys, level - j, 1, out, out, st));
        return cudaSuccess;
    }
    if (C.tune_inner_rescale == 2) {
        const int N = C.N;
        u64 *a = ws.take((size_t)B * polys * level * N);
        if (ws.dry) return cudaSuccess;
        LimbView av = view(a, (i64)polys * level * N, (i64)level * N);
        TRY(transform_plain(C, false, B, polys, level, in, av, st));
        LimbView top = offset(av, (i64)(level - mu) * N);
        RsChainArgs R;
        R.n_batch = B;
        R.n_polys = polys;
        R.N = N;
        R.level = level;
        R.mu = mu;
        R.v = top;
        R.mods = C.d_mods;
        R.one = C.d_one;
        R.invq = C.d_invq;
        TRY(launch_rschain(C, R, st));
        LimbJobs J = jobs(B, polys, level - mu);
        const Shoup *g = C.d_g + C.g_off[level][mu];
        LoadSpec L{};
        L.mode = LD_EQ17;
        L.a = av;
        L.b = top;
        L.g = g;
        L.mu = mu;
        L.with_self = 1;
        StoreSpec S{};
        S.mode = ST_REDUCE;
        S.dst = out;
        return ntt_transform(C, true, J, L, S, nullptr, st);
    }
    return multi_rs_alg1(C, ws, B, polys, level, mu, in, out, st);
}

// Relinearisation up to the coefficient-domain c* (or the NTT-domain C* of
// the prior arrangement when ntt_moddown is set).
// D: [B][n+1][level], NTT domain. cstar: [B][2][level] output view.
static cudaError_t relin_core(const Context &C, Ws &ws, int B, int n, int level, LimbView D, const u64 *keys,
                              int t_max_keys, bool ntt_moddown, LimbView cstar, cudaStream_t st) {
    const int N = C.N, K = C.K, A = C.alpha;
    const int nd = (level + A - 1) / A;
    const int ext_l = level + K;
    u64 *y = ws.take((size_t)B * (n - 1) * level * N);
    u64 *ext = ws.take((size_t)B * (n - 1) * nd * ext_l * N);
    u64 *acc = ws.take((size_t)B * 2 * ext_l * N);
    u64 *z = ws.take((size_t)B * 2 * K * N);
    if (ws.dry) return cudaSuccess;
    (void)t_max_keys;
    LimbView yv = view(y, (i64)(n - 1) * level * N, (i64)level * N);
    LimbView ev = view(ext, (i64)(n - 1) * nd * ext_l * N, (i64)ext_l * N);
    LimbView av = view(acc, (i64)2 * ext_l * N, (i64)ext_l * N);
    LimbView zv = view(z, (i64)2 * K * N, (i64)K * N);
    // 1. INTT of d_2..d_n with the BConv prescale
    {
        LimbJobs J = jobs(B, n - 1, level);
        LoadSpec L{};
        L.mode = LD_PLAIN;
        L.a = offset(D, 2 * D.pstride);
        StoreSpec S{};
        S.mode = ST_SCALE;
        S.dst = yv;
        S.c = C.d_bconv_pre + (size_t)level * C.L;
        S.c_stride = 1;
        TRY(ntt_transform(C, false, J, L, S, nullptr, st));
    }
    // 2. ModUp BConv of every digit (Eq. 4)
    {
        BconvArgs Bc;
        Bc.n_batch = B;
        Bc.N = N;
        Bc.level = level;
        Bc.L = C.L;
        Bc.K = K;
        Bc.alpha = A;
        Bc.n_digits = nd;
        Bc.n_t = n - 1;
        Bc.n_primes = C.L + K;
        Bc.y = yv;
        Bc.ext = ev;
        Bc.consts = C.d_bconv_c + (size_t)level * C.dnum * A * (C.L + K);
        Bc.mods = C.d_mods;
        TRY(launch_bconv(C, Bc, st));
    }
    // 3. NTT of the converted limbs, one launch pair per digit
    for (int beta = 0; beta < nd; ++beta) {
        const int d0 = beta * A, d1 = std::min(level, d0 + A);
        const int nt = level - (d1 - d0) + K;
        LimbJobs J = jobs(B, n - 1, nt);
        int l = 0;
        for (int x = 0; x < level; ++x) {
            if (x >= d0 && x < d1) continue;
            J.slot[l] = J.dslot[l] = (uint8_t)x;
            J.prime[l] = (uint8_t)x;
            ++l;
        }
        for (int i = 0; i < K; ++i, ++l) {
            J.slot[l] = J.dslot[l] = (uint8_t)(level + i);
            J.prime[l] = (uint8_t)(C.L + i);
        }
        LimbView v = view(ext + (size_t)beta * ext_l * N, ev.bstride, (i64)nd * ext_l * N);
        LoadSpec L{};
        L.mode = LD_PLAIN;
        L.a = v;
        StoreSpec S{};
        S.mode = ST_REDUCE;
        S.dst = v;
        TRY(ntt_transform(C, true, J, L, S, nullptr, st));
    }
    // 4-6. key inner product and ModDown. Combined form (Eq. 15): one MAC
    // over every ek_t, one ModDown. Separate form (before Eq. 15, kept for
    // measuring the saving): per ek_t its own MAC and ModDown, summed.
    const bool separate = C.tune_moddown == 1 && n > 2;
    const int t_lo = 2, t_hi = separate ? n : 2;
    for (int t = t_lo; t <= t_hi; ++t) {
        const int t_first = separate ? t : 2, t_last = separate ? t : n;
        const bool first = t == t_lo;
        // 4. key inner product over ek_{t_first..t_last}
        {
            MacArgs M;
            M.n_batch = B;
            M.N = N;
            M.level = level;
            M.L = C.L;
            M.K = K;
            M.alpha = A;
            M.n_digits = nd;
            M.key_digits = C.dnum;
            M.n = 2 + (t_last - t_first);
            M.d = offset(D, (i64)(t_first - 2) * D.pstride);
            M.ext = offset(ev, (i64)(t_first - 2) * nd * ev.pstride);
            M.ext.pstride = ev.pstride;
            M.acc = av;
            M.keys = keys + (size_t)(t_first - 2) * C.dnum * 2 * (C.L + K) * N;
            M.key_pstride = (i64)(C.L + K) * N;
            M.mods = C.d_mods;
            TRY(launch_mac(C, M, st));
        }
        // 5. ModDown, P part: z_i = [phat_i^-1 INTT(acc_i)]_{p_i}
        {
            LimbJobs J = jobs(B, 2, K);
            for (int i = 0; i < K; ++i) {
                J.slot[i] = (uint8_t)(level + i);
                J.dslot[i] = (uint8_t)i;
                J.prime[i] = (uint8_t)(C.L + i);
            }
            LoadSpec L{};
            L.mode = LD_PLAIN;
            L.a = av;
            StoreSpec S{};
            S.mode = ST_SCALE;
            S.dst = zv;
            S.c = C.d_pscale;
            S.c_stride = 1;
            TRY(ntt_transform(C, false, J, L, S, nullptr, st));
            count_op(C, OP_BCONV, 2ull * B);
        }
        // 6. ModDown, Q part
        if (!ntt_moddown) {
            // c* = INTT(D_l + P^-1 acc_l) - scBConv(z)   (Eq. 11 merged, Eq. 12);
            // later keys of the separate form: INTT(P^-1 acc_l) - scBConv(z)
            // into the free y buffer, then added to c*
            LimbView tmp = view(y, yv.bstride, (i64)level * N);
            LimbJobs J = jobs(B, 2, level);
            LoadSpec L{};
            L.mode = first ? LD_ADD : LD_PLAIN;
            L.a = first ? D : av;
            L.b = av;
            StoreSpec S{};
            S.mode = ST_MODDOWN;
            S.dst = first ? cstar : tmp;
            S.aux = zv;
            S.c = C.d_ninv;
            S.c_stride = 1;
            S.mods = C.d_mods;
            S.cK = C.d_cK;
            S.K = K;
            TRY(ntt_transform(C, false, J, L, S, nullptr, st));
            if (!first) TRY(launch_add_limbs(C, cstar, tmp, B, 2, level, st));
        } else {
            // prior arrangement: C* = D_l + P^-1 acc_l - NTT(scBConv(z)); later
            // keys of the separate form add to C* in place
            LimbJobs J = jobs(B, 2, level);
            LoadSpec L{};
            L.mode = LD_BCONVK;
            L.b = zv;
            L.mods = C.d_mods;
            L.cK = C.d_cK;
            L.K = K;
            StoreSpec S{};
            S.mode = ST_ADDSUB;
            S.dst = cstar;
            S.aux = first ? D : cstar;
            S.aux2 = av;
            // the first phase's intermediate must not overwrite C* while C*
            // is also the addend: stage it in the free y buffer
            StoreSpec mid{};
            mid.mode = ST_LAZY;
            mid.dst = view(y, yv.bstride, (i64)level * N);
            TRY(ntt_transform(C, true, J, L, S, first ? nullptr : &mid, st));
        }
    }
    return cudaSuccess;
}

// Relocated root rescale: chain among the mu top limbs of c* (coefficient
// domain), then NTT with the Eq. 17 combination in the load.
static cudaError_t root_rescale(const Context &C, int B, int level, int mu, LimbView cstar, LimbView out,
                                cudaStream_t st) {
    const int N = C.N;
    LimbView top = offset(cstar, (i64)(level - mu) * N);
    RsChainArgs R;
    R.n_batch = B;
    R.n_polys = 2;
    R.N = N;
    R.level = level;
    R.mu = mu;
    R.v = top;
    R.mods = C.d_mods;
    R.one = C.d_one;
    R.invq = C.d_invq;
    TRY(launch_rschain(C, R, st));
    LimbJobs J = jobs(B, 2, level - mu);
    const Shoup *g = C.d_g + C.g_off[level][mu];
    LoadSpec L{};
    L.mode = LD_EQ17;
    L.a = cstar;
    L.b = top;
    L.g = g;
    L.mu = mu;
    L.with_self = 1;
    StoreSpec S{};
    S.mode = ST_REDUCE;
    S.dst = out;
    return ntt_transform(C, true, J, L, S, nullptr, st);
}

// ---------------------------------------------------------------------------
// k-input multiply over a plan
// ---------------------------------------------------------------------------
// NVTX range around the enqueueing of one stage (tunable "nvtx")
struct NvtxRange {
    bool on;
    NvtxRange(const Context &C, const char *name) : on(C.tune_nvtx != 0) {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxRange() {
        if (on) nvtxRangePop();
    }
};

// tunable "check_residues": count residues >= q of a stage's output
#define CHECK_STAGE(v, polys, lvl)                                                        \
    do {                                                                                  \
        if (C.tune_check_residues && !ws.dry) {                                          \
            err = launch_range_check(C, (v), B, (polys), (lvl), st);                      \
            if (err != cudaSuccess) return -5;                                            \
        }                                                                                 \
    } while (0)

int run_mul_k(const Context &C, const Plan &P, int level, int B, const LimbView *in, LimbView out, const u64 *keys,
              int t_max, Ws &ws, cudaStream_t st, cudaError_t &err) {
    std::vector<int> lin, lout, polys;
    plan_levels(P, level, lin, lout, polys);
    const int N = C.N;
    std::vector<LimbView> node_out(P.nodes.size());
    err = cudaSuccess;
    for (int u = 0; u < P.k; ++u) CHECK_STAGE(in[u], 2, level);
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        const PlanNode &nd = P.nodes[i];
        const int lv = lin[i];
        int np = 1;
        TensorArgs T;
        T.n_batch = B;
        T.level = lv;
        T.N = N;
        T.m = (int)nd.children.size();
        T.mods = C.d_mods;
        T.rfix = C.d_rfix;
        for (int c = 0; c < T.m; ++c) {
            int ch = nd.children[c];
            T.child[c] = ch >= 0 ? node_out[ch] : in[-1 - ch];
            T.child_polys[c] = ch >= 0 ? polys[ch] : 2;
            np += T.child_polys[c] - 1;
        }
        u64 *d = ws.take((size_t)B * np * lv * N);
        LimbView dv = view(d, (i64)np * lv * N, (i64)lv * N);
        T.out = dv;
        if (!ws.dry) {
            NvtxRange r(C, nd.root ? "root: tensor product" : "node: tensor product");
            err = launch_tensor(C, T, st);
            if (err != cudaSuccess) return -5;
        }
        CHECK_STAGE(dv, np, lv);
        if (!nd.root) {
            NvtxRange r(C, "node: multi-level rescale (Algorithm 1)");
            err = multi_rs(C, ws, B, np, lv, nd.mu, dv, dv, st);
            if (err != cudaSuccess) return -5;
            node_out[i] = dv;  // level lv - mu, poly stride lv
            CHECK_STAGE(dv, np, lv - nd.mu);
        } else {
            const int n = np - 1;
            if (n > t_max) return -3;
            u64 *cs = ws.take((size_t)B * 2 * lv * N);
            LimbView cv = view(cs, (i64)2 * lv * N, (i64)lv * N);
            if (C.tune_root_rescale == 1) {
                // prior arrangement: ModDown finished in the NTT domain, then
                // mu_root rescales of Eq. 7
                err = relin_core(C, ws, B, n, lv, dv, keys, t_max, true, cv, st);
                if (err != cudaSuccess) return -5;
                err = multi_rs_alg1(C, ws, B, 2, lv, 1, cv, nd.mu == 1 ? out : cv, st);
                if (err != cudaSuccess) return -5;
                for (int j = 1; j < nd.mu; ++j) {
                    err = multi_rs_alg1(C, ws, B, 2, lv - j, 1, cv, j == nd.mu - 1 ? out : cv, st);
                    if (err != cudaSuccess) return -5;
                }
            } else {
                {
                    NvtxRange r(C, "root: relinearisation (ModUp, key MAC, ModDown)");
                    err = relin_core(C, ws, B, n, lv, dv, keys, t_max, false, cv, st);
                    if (err != cudaSuccess) return -5;
                }
                CHECK_STAGE(cv, 2, lv);
                if (!ws.dry) {
                    NvtxRange r(C, "root: relocated rescale");
                    err = root_rescale(C, B, lv, nd.mu, cv, out, st);
                    if (err != cudaSuccess) return -5;
                }
            }
            CHECK_STAGE(out, 2, lv - nd.mu);
        }
    }
    return 0;
}

// Output scale of a plan: the product of the children's scales at every
// node, divided by each prime a rescale removes.
double plan_scale(const Context &C, const Plan &P, int level, const double *scales) {
    std::vector<int> lin, lout, polys;
    plan_levels(P, level, lin, lout, polys);
    std::vector<double> sc(P.nodes.size(), 1.0);
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        double s = 1.0;
        for (int c : P.nodes[i].children) s *= c >= 0 ? sc[c] : scales[-1 - c];
        for (int j = 0; j < P.nodes[i].mu; ++j) s /= (double)C.primes[lin[i] - 1 - j];
        sc[i] = s;
    }
    return sc.back();
}

size_t relin_ws_bytes(const Context &C, int n, int level, int B) {
    Ws ws{nullptr, 0, 0, true};
    LimbView d{};
    relin_core(C, ws, B, n, level, d, nullptr, n, false, d, 0);
    ws.take((size_t)B * 2 * level * C.N);  // c* scratch for NTT-domain output
    return ws.off;
}

int run_relin(const Context &C, int B, int n, int level, LimbView D, const u64 *keys, bool out_ntt, LimbView out,
              Ws &ws, cudaStream_t st, cudaError_t &err) {
    if (!out_ntt) {
        err = relin_core(C, ws, B, n, level, D, keys, n, false, out, st);
        ws.take((size_t)B * 2 * level * C.N);
        return err == cudaSuccess ? 0 : -5;
    }
    err = relin_core(C, ws, B, n, level, D, keys, n, false, out, st);
    u64 *tmp = ws.take((size_t)B * 2 * level * C.N);
    (void)tmp;
    if (err != cudaSuccess) return -5;
    if (!ws.dry) {
        err = transform_plain(C, true, B, 2, level, out, out, st);
        if (err != cudaSuccess) return -5;
    }
    return 0;
}

// Rotation (Galois automorphism sigma_g) with key switching back to s:
// D = (sigma c0, 0, sigma c1), then the relinearisation steps with the one
// Galois key in the place of ek_2 and ModDown finished in the NTT domain:
// out = (sigma c0 + [P^-1 sigma(c1) gk_0], [P^-1 sigma(c1) gk_1]).
static int run_rotate(const Context &C, int B, int level, uint32_t g, LimbView in, LimbView out, const u64 *keys,
                      Ws &ws, cudaStream_t st, cudaError_t &err) {
    const int N = C.N;
    u64 *d = ws.take((size_t)B * 3 * level * N);
    LimbView dv = view(d, (i64)3 * level * N, (i64)level * N);
    err = cudaSuccess;
    if (!ws.dry) {
        AutoMap map{};
        map.n_out = 3;
        map.src[0] = 0;
        map.src[1] = -1;
        map.src[2] = 1;
        err = launch_automorphism(C, in, dv, map, B, level, g, st);
        if (err != cudaSuccess) return -5;
    }
    err = relin_core(C, ws, B, 2, level, dv, keys, 2, true, out, st);
    return err == cudaSuccess ? 0 : -5;
}

size_t rotate_ws_bytes(const Context &C, int level, int B) {
    Ws ws{nullptr, 0, 0, true};
    LimbView v{};
    cudaError_t err;
    run_rotate(C, B, level, 1, v, v, nullptr, ws, 0, err);
    return ws.off;
}

int run_rotate_ws(const Context &C, int B, int level, uint32_t g, LimbView in, LimbView out, const u64 *keys,
                  void *wsp, size_t bytes, cudaStream_t st, cudaError_t &err) {
    Ws ws{(char *)wsp, 0, bytes, false};
    return run_rotate(C, B, level, g, in, out, keys, ws, st, err);
}

size_t rescale_ws_bytes(const Context &C, int polys, int level, int mu, int B) {
    Ws ws{nullptr, 0, 0, true};
    LimbView v{};
    multi_rs(C, ws, B, polys, level, mu, v, v, 0);
    return ws.off;
}

// Algorithm 1 whatever the context's "inner_rescale" setting: the
// allocation-free entry point sizes its fixed scratch for this form.
size_t rescale_alg1_ws_bytes(const Context &C, int polys, int level, int mu, int B) {
    Ws ws{nullptr, 0, 0, true};
    LimbView v{};
    multi_rs_alg1(C, ws, B, polys, level, mu, v, v, 0);
    return ws.off;
}

int run_rescale_alg1_ws(const Context &C, int B, int polys, int level, int mu, LimbView in, LimbView out, void *wsp,
                        size_t bytes, cudaStream_t st, cudaError_t &err) {
    Ws ws{(char *)wsp, 0, bytes, false};
    err = multi_rs_alg1(C, ws, B, polys, level, mu, in, out, st);
    return err == cudaSuccess ? 0 : -5;
}

int run_rescale(const Context &C, int B, int polys, int level, int mu, LimbView in, LimbView out, Ws &ws,
                cudaStream_t st, cudaError_t &err) {
    err = multi_rs(C, ws, B, polys, level, mu, in, out, st);
    return err == cudaSuccess ? 0 : -5;
}

// Standard 2-input multiply (Eq. 1-7): tensor, relinearisation with the
// ModDown finished in the NTT domain, one RS in the NTT domain.
int run_mul2(const Context &C, int level, int B, LimbView a, LimbView b, LimbView out, const u64 *keys, Ws &ws,
             cudaStream_t st, cudaError_t &err) {
    const int N = C.N;
    u64 *d = ws.take((size_t)B * 3 * level * N);
    LimbView dv = view(d, (i64)3 * level * N, (i64)level * N);
    u64 *cs = ws.take((size_t)B * 2 * level * N);
    LimbView cv = view(cs, (i64)2 * level * N, (i64)level * N);
    err = cudaSuccess;
    if (!ws.dry) {
        TensorArgs T;
        T.n_batch = B;
        T.level = level;
        T.N = N;
        T.m = 2;
        T.mods = C.d_mods;
        T.rfix = C.d_rfix;
        T.child[0] = a;
        T.child[1] = b;
        T.child_polys[0] = T.child_polys[1] = 2;
        T.out = dv;
        err = launch_tensor(C, T, st);
        if (err != cudaSuccess) return -5;
    }
    err = relin_core(C, ws, B, 2, level, dv, keys, 2, true, cv, st);
    if (err != cudaSuccess) return -5;
    err = multi_rs(C, ws, B, 2, level, 1, cv, out, st);
    return err == cudaSuccess ? 0 : -5;
}

size_t mul_k_ws_bytes(const Context &C, const Plan &P, int level, int B) {
    Ws ws{nullptr, 0, 0, true};
    std::vector<LimbView> in(P.k);
    LimbView out{};
    cudaError_t err;
    run_mul_k(C, P, level, B, in.data(), out, nullptr, P.k, ws, 0, err);
    return ws.off;
}

size_t mul2_ws_bytes(const Context &C, int level, int B) {
    Ws ws{nullptr, 0, 0, true};
    LimbView v{};
    cudaError_t err;
    run_mul2(C, level, B, v, v, v, nullptr, ws, 0, err);
    return ws.off;
}

int run_mul_k_ws(const Context &C, const Plan &P, int level, int B, const LimbView *in, LimbView out,
                 const u64 *keys, int t_max, void *wsp, size_t bytes, cudaStream_t st, cudaError_t &err) {
    Ws ws{(char *)wsp, 0, bytes, false};
    return run_mul_k(C, P, level, B, in, out, keys, t_max, ws, st, err);
}

int run_relin_ws(const Context &C, int B, int n, int level, LimbView D, const u64 *keys, bool out_ntt, LimbView out,
                 void *wsp, size_t bytes, cudaStream_t st, cudaError_t &err) {
    Ws ws{(char *)wsp, 0, bytes, false};
    return run_relin(C, B, n, level, D, keys, out_ntt, out, ws, st, err);
}

int run_rescale_ws(const Context &C, int B, int polys, int level, int mu, LimbView in, LimbView out, void *wsp,
                   size_t bytes, cudaStream_t st, cudaError_t &err) {
    Ws ws{(char *)wsp, 0, bytes, false};
    return run_rescale(C, B, polys, level, mu, in, out, ws, st, err);
}

int run_mul2_ws(const Context &C, int level, int B, LimbView a, LimbView b, LimbView out, const u64 *keys,
                void *wsp, size_t bytes, cudaStream_t st, cudaError_t &err) {
    Ws ws{(char *)wsp, 0, bytes, false};
    return run_mul2(C, level, B, a, b, out, keys, ws, st, err);
}

cudaError_t run_tensor(const Context &C, int B, int level, int m, const LimbView *in, const int *polys,
                       LimbView out, cudaStream_t st) {
    TensorArgs T;
    T.n_batch = B;
    T.level = level;
    T.N = C.N;
    T.m = m;
    T.mods = C.d_mods;
    T.rfix = C.d_rfix;
    for (int c = 0; c < m; ++c) {
        T.child[c] = in[c];
        T.child_polys[c] = polys[c];
    }
    T.out = out;
    return launch_tensor(C, T, st);
}

}  // namespace ckks
