// Cross-shape batches ("waves"): many k-input products of one context with
// different k, partition trees and input levels, run as one sequence of
// stage launches whose work comes from device job tables.
//
// Every product follows the evaluation of Section V exactly as
// ckks_mul_k does (so its residues are the same): inner nodes take the
// tensor product (Eq. 13) and Algorithm 1 (INTT of the mu top limbs, the
// rescale chain, one NTT per surviving limb with Eq. 17 in its load and
// A' = g A - B in its store); the root takes the tensor product, ModUp of
// d_2..d_n (INTT with the BConv prescale, Eq. 4, NTT), the key MAC of Eq. 15,
// ModDown with Eq. 11 / 12 and the relocated rescale of Section IV. What
// changes is the schedule: inner nodes of every product are grouped by
// height (a node's children always have a smaller height), and each stage
// of a group (tensor, INTT, rescale chain, NTT, BConv, MAC, ...) is one
// launch over all products whose tree has work there. A batch of any mix of
// k and levels therefore takes a bounded number of launches: heights x 6 +
// 14, plus per round one tensor launch per tuple-size class and one per node
// shape with a fixed kernel (tensor_fixed.cu), plus one when the key MAC has
// both paired and single products.
//
// Memory: two caller buffers, the job tables (written on the first run with
// that pair of buffers, by one host-to-device copy on the run's stream) and
// every product's own scratch (the same per-product layout as ckks_mul_k with
// batch 1). Waves that run one after the other on a stream can share one
// scratch buffer while each keeps its own (small) table buffer. Nothing is
// allocated on the device by the library; the host staging buffer for the
// tables belongs to the wave.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/ckks_mulk.h"
#include "engine.h"
#include "internal.h"
#include "plan.h"
#include "rns.h"

using namespace ckks;

namespace {

struct WaveProduct {
    int k = 0;
    const Plan *plan = nullptr;
    int level = 0;
    std::vector<const u64 *> in;   // limb 0 of polynomial 0 of each input
    std::vector<i64> in_ps;        // polynomial stride of each input (elements)
    u64 *out = nullptr;
    i64 out_ps = 0;
    std::vector<double> scales;
};

enum StageKind { SK_TENSOR, SK_NTT, SK_RSCHAIN, SK_BCONV, SK_MAC };

// One launch of the wave: its kind, launch-wide parameters and where its
// table lives in the table region.
struct Stage {
    int kind = SK_NTT;
    bool fwd = true, cols = true;
    LoadSpec L{};
    StoreSpec S{};
    int maxt = 0, max_level = 0, max_polys = 0;
    bool vec2 = true;  // tensor: every entry 16-byte aligned with even strides
    bool fixed = false;  // tensor: every entry has a fixed-shape kernel
    struct FixedRun {    // tensor, fixed: entries [first, first + count) have shape `code`
        int code, first, count, max_level;
        double bytes, ops;
    };
    std::vector<FixedRun> runs;
    int n_pairs = 0;   // key MAC: targets[0 .. n_pairs) pair two products
    std::vector<NttJob> ntt;
    std::vector<TensorJob> tensor;
    std::vector<RsJob> rs;
    std::vector<BconvJob> bconv;
    std::vector<MacJob> mac;
    std::vector<MacTarget> targets;
    size_t off = 0, off2 = 0;  // byte offsets of the table(s)
    double bytes = 0, ops = 0;
    unsigned long long limb_transforms = 0;
    int count() const {
        switch (kind) {
        case SK_TENSOR: return (int)tensor.size();
        case SK_RSCHAIN: return (int)rs.size();
        case SK_BCONV: return (int)bconv.size();
        case SK_MAC: return (int)targets.size();
        default: return (int)ntt.size();
        }
    }
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct ckks_wave {
    ckks_context *ctx = nullptr;
    const ckks_evk_set *evk = nullptr;
    std::vector<WaveProduct> items;
    std::vector<ckks_tuple *> outs;
    size_t scratch_bytes = 0;     // every product's scratch
    size_t table_bytes = 0;       // upper bound of the tables (sized by a dry build)
    // state of the last build
    void *bound_tables = nullptr, *bound_scratch = nullptr;
    std::vector<Stage> stages;
    void *staging = nullptr;      // pinned host copy of the tables
    size_t staging_bytes = 0;
    cudaEvent_t uploaded = nullptr;
    int heights = 0;
};

namespace {

// Per-product scratch, carved in the order of ckks_mul_k's workspace.
struct Bump {
    char *base;
    size_t off;
    u64 *take(size_t elems) {
        size_t bytes = align256(elems * sizeof(u64));
        u64 *p = base ? (u64 *)(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

// Stage lists of one build, addressed by (round, step): rounds 0..H-1 are
// the inner-node heights, round H is the root.
struct Builder {
    const Context &C;
    const u64 *keys;
    int H;
    std::map<std::pair<int, int>, Stage> st;

    Stage &at(int round, int step, int kind) {
        Stage &s = st[{round, step}];
        s.kind = kind;
        return s;
    }
    int prime_of_slot(int x, int level) const { return x < level ? x : C.L + (x - level); }

    // both phases of one transform: phase-1 entry, phase-2 entry
    void ntt_pair(int round, int step, bool fwd, const NttJob &p1, const NttJob &p2, const LoadSpec &L1,
                  const StoreSpec &S1, const LoadSpec &L2, const StoreSpec &S2, double bytes1, double bytes2,
                  double ops1, double ops2) {
        Stage &a = at(round, step, SK_NTT);
        a.fwd = fwd;
        a.cols = fwd;  // forward starts with the column phase, inverse with the block phase
        a.L = L1;
        a.S = S1;
        a.ntt.push_back(p1);
        a.bytes += bytes1;
        a.ops += ops1;
        a.limb_transforms += 1;
        Stage &b = at(round, step + 1, SK_NTT);
        b.fwd = fwd;
        b.cols = !fwd;
        b.L = L2;
        b.S = S2;
        b.ntt.push_back(p2);
        b.bytes += bytes2;
        b.ops += ops2;
    }
};

int node_heights(const Plan &P, std::vector<int> &h) {
    h.assign(P.nodes.size(), 0);
    int hmax = 0;
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        int m = 0;
        for (int c : P.nodes[i].children)
            if (c >= 0) m = std::max(m, h[c]);
        h[i] = m + 1;
        if (!P.nodes[i].root) hmax = std::max(hmax, h[i]);
    }
    return hmax;
}

NttJob njob(const u64 *a, u64 *dst, int prime) {
    NttJob j{};
    j.a = a;
    j.dst = dst;
    j.prime = prime;
    return j;
}

// Emits every stage entry of one product into the builder (or, with a null
// scratch base, only sizes its scratch).
void build_product(Builder &B, const WaveProduct &w, Bump &ws) {
    const Context &C = B.C;
    const Plan &P = *w.plan;
    const int N = C.N, K = C.K, A = C.alpha, logN = C.log_n;
    int log_n1, log_n2;
    ntt_geometry(logN, log_n1, log_n2);
    const double limb = (double)N * sizeof(u64);
    const double bf1 = (double)N * 0.5 * log_n1, bf2 = (double)N * 0.5 * log_n2;  // butterflies per limb and phase
    std::vector<int> lin, lout, polys, height;
    plan_levels(P, w.level, lin, lout, polys);
    node_heights(P, height);
    std::vector<u64 *> node_out(P.nodes.size(), nullptr);
    std::vector<i64> node_ps(P.nodes.size(), 0);
    const bool emit = ws.base != nullptr;
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        const PlanNode &nd = P.nodes[i];
        const int lv = lin[i];
        int np = 1;
        TensorJob T{};
        T.m = (int)nd.children.size();
        T.level = lv;
        int maxt = 0, in_polys = 0;
        for (int c = 0; c < T.m; ++c) {
            const int ch = nd.children[c];
            T.child[c] = ch >= 0 ? node_out[ch] : w.in[-1 - ch];
            T.cstride[c] = ch >= 0 ? node_ps[ch] : w.in_ps[-1 - ch];
            T.cpolys[c] = ch >= 0 ? polys[ch] : 2;
            np += T.cpolys[c] - 1;
            in_polys += T.cpolys[c];
            maxt = std::max(maxt, T.cpolys[c]);
        }
        maxt = std::max(maxt, np);
        u64 *d = ws.take((size_t)np * lv * N);
        const i64 dps = (i64)lv * N;
        T.out = d;
        T.ostride = dps;
        const int round = nd.root ? B.H : height[i] - 1;
        // tuple-size class of the tensor launch (its instantiation); class 6:
        // shapes with fixed kernels (children sorted by size)
        int cls = maxt <= 3 ? 0 : maxt <= 4 ? 1 : maxt <= 5 ? 2 : maxt <= 7 ? 3 : maxt <= 9 ? 4 : 5;
        // children sorted by size, largest first (the smallest, last, takes
        // the R^(m-1) correction)
        if (tensor_sort_children(T) >= 0 && C.tune_tensor_fixed) cls = 6;
        if (emit) {
            Stage &s = B.at(round, cls, SK_TENSOR);
            s.fixed = cls == 6;
            s.tensor.push_back(T);
            s.vec2 = s.vec2 && tensor_job_vec2(T);
            s.maxt = std::max(s.maxt, maxt);
            s.max_level = std::max(s.max_level, lv);
            s.bytes += (double)(in_polys + np) * lv * limb;
            s.ops += (double)lv * N * tensor_products_per_coeff(T.cpolys, T.m);
        }
        if (!nd.root) {
            // Algorithm 1 in place on D (np polynomials, level lv, mu = nd.mu)
            const int mu = nd.mu;
            u64 *a = ws.take((size_t)np * mu * N);
            u64 *bb = ws.take((size_t)np * (lv - mu) * N);
            if (emit) {
                const Shoup *g = C.d_g + C.g_off[lv][mu];
                LoadSpec Lp{};
                Lp.mode = LD_PLAIN;
                StoreSpec Sl{};
                Sl.mode = ST_LAZY;
                StoreSpec Ss{};
                Ss.mode = ST_SCALE;
                for (int p = 0; p < np; ++p)
                    for (int l = 0; l < mu; ++l) {
                        // 1. INTT of the top limbs, N^-1 in the store
                        const int prime = lv - mu + l;
                        u64 *al = a + ((i64)p * mu + l) * N;
                        NttJob j1 = njob(d + p * dps + (i64)prime * N, al, prime);
                        NttJob j2 = njob(al, al, prime);
                        j2.c = C.d_ninv + prime;
                        B.ntt_pair(round, 10, false, j1, j2, Lp, Sl, Lp, Ss, 2 * limb, 2 * limb, bf2, bf1 + N);
                    }
                if (mu >= 2) {
                    Stage &s = B.at(round, 12, SK_RSCHAIN);
                    RsJob r{a, (i64)mu * N, np, lv, mu, 0};
                    s.rs.push_back(r);
                    s.max_polys = std::max(s.max_polys, np);
                    s.bytes += 2.0 * np * mu * limb;
                }
                LoadSpec Le{};
                Le.mode = LD_EQ17;
                StoreSpec Sm{};
                Sm.mode = ST_MRS;
                for (int p = 0; p < np; ++p)
                    for (int l = 0; l < lv - mu; ++l) {
                        // 3. B = NTT(sum_t g_t a_t) (lazy into bb), A' = g_self A - B
                        u64 *bl = bb + ((i64)p * (lv - mu) + l) * N;
                        NttJob j1{};
                        j1.b = a + (i64)p * mu * N;
                        j1.g = g + (i64)l * (mu + 1);
                        j1.mu = mu;
                        j1.with_self = 0;
                        j1.dst = bl;
                        j1.prime = l;
                        NttJob j2 = njob(bl, d + p * dps + (i64)l * N, l);
                        j2.aux = d + p * dps + (i64)l * N;
                        j2.c = g + (i64)l * (mu + 1) + mu;
                        B.ntt_pair(round, 13, true, j1, j2, Le, Sl, Lp, Sm, limb + (double)mu * limb / (lv - mu),
                                   3 * limb, bf1 + (double)N * mu, bf2 + N);
                    }
            }
            node_out[i] = d;
            node_ps[i] = dps;
            continue;
        }
        // ---- root: relinearisation (ModUp, key MAC, ModDown) and relocated rescale
        const int n = np - 1, mu = nd.mu;
        u64 *cs = ws.take((size_t)2 * lv * N);
        const int ndig = (lv + A - 1) / A;
        const int ext_l = lv + K;
        u64 *y = ws.take((size_t)(n - 1) * lv * N);
        u64 *ext = ws.take((size_t)(n - 1) * ndig * ext_l * N);
        u64 *acc = ws.take((size_t)2 * ext_l * N);
        u64 *z = ws.take((size_t)2 * K * N);
        if (!emit) continue;
        const i64 cps = (i64)lv * N, yps = (i64)lv * N, eps = (i64)ext_l * N, aps = (i64)ext_l * N, zps = (i64)K * N;
        LoadSpec Lp{};
        Lp.mode = LD_PLAIN;
        StoreSpec Sl{};
        Sl.mode = ST_LAZY;
        StoreSpec Ss{};
        Ss.mode = ST_SCALE;
        StoreSpec Sr{};
        Sr.mode = ST_REDUCE;
        // 1. INTT of d_2..d_n with the BConv prescale in the store
        for (int t = 2; t <= n; ++t)
            for (int l = 0; l < lv; ++l) {
                u64 *yl = y + (i64)(t - 2) * yps + (i64)l * N;
                NttJob j1 = njob(d + t * dps + (i64)l * N, yl, l);
                NttJob j2 = njob(yl, yl, l);
                j2.c = C.d_bconv_pre + (size_t)lv * C.L + l;
                B.ntt_pair(B.H, 10, false, j1, j2, Lp, Sl, Lp, Ss, 2 * limb, 2 * limb, bf2, bf1 + N);
            }
        // 2. ModUp BConv of every (d_t, digit) (Eq. 4)
        {
            Stage &s = B.at(B.H, 12, SK_BCONV);
            for (int t = 2; t <= n; ++t)
                for (int beta = 0; beta < ndig; ++beta) {
                    BconvJob J{};
                    J.y = y + (i64)(t - 2) * yps;
                    J.ext = ext + (i64)((t - 2) * ndig + beta) * eps;
                    J.consts = C.d_bconv_c + ((size_t)lv * C.dnum + beta) * A * (C.L + K);
                    J.level = lv;
                    J.beta = beta;
                    s.bconv.push_back(J);
                    const int na = std::min(lv, (beta + 1) * A) - beta * A;
                    s.bytes += (double)(ext_l - na) * limb;
                    s.ops += (double)na * (lv - na + K) * N;
                }
            s.bytes += (double)(n - 1) * lv * limb;
        }
        // 3. NTT of the converted limbs
        for (int t = 2; t <= n; ++t)
            for (int beta = 0; beta < ndig; ++beta) {
                const int d0 = beta * A, d1 = std::min(lv, d0 + A);
                u64 *e0 = ext + (i64)((t - 2) * ndig + beta) * eps;
                for (int x = 0; x < ext_l; ++x) {
                    if (x >= d0 && x < d1) continue;
                    const int prime = B.prime_of_slot(x, lv);
                    u64 *el = e0 + (i64)x * N;
                    B.ntt_pair(B.H, 13, true, njob(el, el, prime), njob(el, el, prime), Lp, Sl, Lp, Sr, 2 * limb,
                               2 * limb, bf1, bf2);
                }
            }
        // 4. key MAC over every ek_t and digit (Eq. 15, combined)
        {
            Stage &s = B.at(B.H, 15, SK_MAC);
            MacJob M{};
            M.d = d;
            M.dstride = dps;
            M.ext = ext;
            M.estride = eps;
            M.acc = acc;
            M.astride = aps;
            M.level = lv;
            M.n = n;
            M.nd = ndig;
            const int job = (int)s.mac.size();
            s.mac.push_back(M);
            for (int x = 0; x < ext_l; ++x) s.targets.push_back(MacTarget{job, x, -1, 0});
            const double terms = (double)(n - 1) * ndig;
            s.bytes += (terms + 2.0) * ext_l * limb;
            s.ops += 2.0 * terms * ext_l * N;
        }
        // 5. ModDown, P part: z_i = [phat_i^-1 INTT(acc_i)]_{p_i}
        for (int p = 0; p < 2; ++p)
            for (int i = 0; i < K; ++i) {
                u64 *zl = z + p * zps + (i64)i * N;
                NttJob j1 = njob(acc + p * aps + (i64)(lv + i) * N, zl, C.L + i);
                NttJob j2 = njob(zl, zl, C.L + i);
                j2.c = C.d_pscale + i;
                B.ntt_pair(B.H, 16, false, j1, j2, Lp, Sl, Lp, Ss, 2 * limb, 2 * limb, bf2, bf1 + N);
            }
        // 6. ModDown, Q part: c* = INTT(D_l + P^-1 acc_l) - scBConv(z)  (Eq. 11, 12)
        {
            LoadSpec La{};
            La.mode = LD_ADD;
            StoreSpec Sd{};
            Sd.mode = ST_MODDOWN;
            Sd.mods = C.d_mods;
            Sd.cK = C.d_cK;
            Sd.K = K;
            for (int p = 0; p < 2; ++p)
                for (int l = 0; l < lv; ++l) {
                    u64 *cl = cs + p * cps + (i64)l * N;
                    NttJob j1 = njob(d + p * dps + (i64)l * N, cl, l);
                    j1.b = acc + p * aps + (i64)l * N;
                    NttJob j2 = njob(cl, cl, l);
                    j2.aux = z + p * zps;
                    j2.c = C.d_ninv + l;
                    B.ntt_pair(B.H, 18, false, j1, j2, La, Sl, Lp, Sd, 3 * limb, 2 * limb + (double)K * limb / lv, bf2,
                               bf1 + N);
                }
        }
        // 7. relocated rescale: chain among the mu top limbs of c*, then NTT
        //    with the Eq. 17 combination (self term included) in the load
        if (mu >= 2) {
            Stage &s = B.at(B.H, 20, SK_RSCHAIN);
            RsJob r{cs + (i64)(lv - mu) * N, cps, 2, lv, mu, 0};
            s.rs.push_back(r);
            s.max_polys = std::max(s.max_polys, 2);
            s.bytes += 2.0 * 2 * mu * limb;
        }
        {
            const Shoup *g = C.d_g + C.g_off[lv][mu];
            LoadSpec Le{};
            Le.mode = LD_EQ17;
            for (int p = 0; p < 2; ++p)
                for (int l = 0; l < lv - mu; ++l) {
                    u64 *ol = w.out + p * w.out_ps + (i64)l * N;
                    NttJob j1{};
                    j1.a = cs + p * cps + (i64)l * N;
                    j1.b = cs + p * cps + (i64)(lv - mu) * N;
                    j1.g = g + (i64)l * (mu + 1);
                    j1.mu = mu;
                    j1.with_self = 1;
                    j1.dst = ol;
                    j1.prime = l;
                    B.ntt_pair(B.H, 21, true, j1, njob(ol, ol, l), Le, Sl, Lp, Sr,
                               2 * limb + (double)mu * limb / (lv - mu), 2 * limb, bf1 + (double)N * (mu + 1), bf2);
                }
        }
    }
}

template <class T>
size_t put(std::vector<char> &buf, const std::vector<T> &v) {
    const size_t off = align256(buf.size());
    buf.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

// Builds the stage list and the job tables of a wave whose products' scratch
// starts at device address `scratch`.
int build(ckks_wave &W, char *scratch, std::vector<char> &tables) {
    const Context &C = W.ctx->c;
    int H = 0;
    for (const WaveProduct &w : W.items) {
        std::vector<int> h;
        H = std::max(H, node_heights(*w.plan, h));
    }
    Builder B{C, W.evk->keys, H, {}};
    Bump bump{scratch, 0};
    for (const WaveProduct &w : W.items) build_product(B, w, bump);
    W.stages.clear();
    tables.clear();
    for (auto &kv : B.st) {
        Stage &s = kv.second;
        if (s.count() == 0) continue;
        if (s.kind == SK_NTT) s.off = put(tables, s.ntt);
        if (s.kind == SK_TENSOR && s.fixed) {
            // one launch per shape: entries grouped by shape code
            // (the entries' children were sorted when they were built)
            auto code_of = [](const TensorJob &T) {
                return tensor_fixed_code(T.m, T.cpolys[0], T.cpolys[1], T.m > 2 ? T.cpolys[2] : 0);
            };
            std::stable_sort(s.tensor.begin(), s.tensor.end(),
                             [&](const TensorJob &a, const TensorJob &b) { return code_of(a) < code_of(b); });
            s.runs.clear();
            const double limb = (double)C.N * sizeof(u64);
            for (int i = 0; i < (int)s.tensor.size(); ++i) {
                const TensorJob &T = s.tensor[i];
                const int code = code_of(T);
                if (s.runs.empty() || s.runs.back().code != code) s.runs.push_back({code, i, 0, 0, 0.0, 0.0});
                Stage::FixedRun &r = s.runs.back();
                int in_polys = 0;
                for (int c = 0; c < T.m; ++c) in_polys += T.cpolys[c];
                r.count += 1;
                r.max_level = std::max(r.max_level, T.level);
                r.bytes += (double)(2 * in_polys - T.m + 1) * T.level * limb;
                r.ops += (double)T.level * C.N * tensor_products_per_coeff(T.cpolys, T.m);
            }
        }
        if (s.kind == SK_TENSOR) s.off = put(tables, s.tensor);
        if (s.kind == SK_RSCHAIN) s.off = put(tables, s.rs);
        if (s.kind == SK_BCONV) s.off = put(tables, s.bconv);
        if (s.kind == SK_MAC) {
            // two products of the same shape (level, n, digits) share the key
            // loads of a limb x: pair their targets, pairs first; each part
            // ordered by prime, so that neighbouring blocks share key rows
            std::vector<MacTarget> pairs, singles;
            {
                std::map<std::tuple<int, int, int, int>, int> open;  // (level, n, nd, x) -> unpaired target
                for (const MacTarget &t : s.targets) {
                    const MacJob &J = s.mac[t.job];
                    const auto key = std::make_tuple(J.level, J.n, J.nd, t.x);
                    if (!CKKS_MAC_PAIR) {
                        singles.push_back(t);
                        continue;
                    }
                    auto it = open.find(key);
                    if (it != open.end()) {
                        pairs.push_back(MacTarget{it->second, t.x, t.job, 0});
                        open.erase(it);
                    } else {
                        open[key] = t.job;
                    }
                }
                for (const auto &kv : open) singles.push_back(MacTarget{kv.second, std::get<3>(kv.first), -1, 0});
            }
            auto by_prime = [&](const MacTarget &a, const MacTarget &b) {
                return B.prime_of_slot(a.x, s.mac[a.job].level) < B.prime_of_slot(b.x, s.mac[b.job].level);
            };
            std::stable_sort(pairs.begin(), pairs.end(), by_prime);
            std::stable_sort(singles.begin(), singles.end(), by_prime);
            s.n_pairs = (int)pairs.size();
            s.targets = pairs;
            s.targets.insert(s.targets.end(), singles.begin(), singles.end());
            s.off = put(tables, s.mac);
            s.off2 = put(tables, s.targets);
        }
        W.stages.push_back(std::move(s));
    }
    W.heights = H;
    if (align256(tables.size()) > W.table_bytes) return CKKS_ENOMEM;
    return CKKS_OK;
}

cudaError_t enqueue(ckks_wave &W, char *ws /* the job tables */, cudaStream_t st) {
    const Context &C = W.ctx->c;
    for (const Stage &s : W.stages) {
        cudaError_t e = cudaSuccess;
        const int n = s.count();
        switch (s.kind) {
        case SK_NTT:
            if (s.fwd == s.cols) count_op(C, s.fwd ? OP_LIMB_NTT : OP_LIMB_INTT, s.limb_transforms);
            e = launch_ntt_phase_table(C, s.fwd, s.cols, (const NttJob *)(ws + s.off), n, s.L, s.S, s.bytes, s.ops,
                                       st);
            break;
        case SK_TENSOR:
            if (s.fixed) {
                for (const Stage::FixedRun &r : s.runs) {
                    e = launch_tensor_fixed_table(C, (const TensorJob *)(ws + s.off) + r.first, r.count, r.code,
                                                  r.max_level, r.bytes, r.ops, st);
                    if (e != cudaSuccess) break;
                }
            } else
                e = launch_tensor_table(C, (const TensorJob *)(ws + s.off), n, s.maxt, s.max_level, s.vec2, s.bytes,
                                        s.ops, st);
            break;
        case SK_RSCHAIN:
            e = launch_rschain_table(C, (const RsJob *)(ws + s.off), n, s.max_polys, s.bytes, st);
            break;
        case SK_BCONV:
            e = launch_bconv_table(C, (const BconvJob *)(ws + s.off), n, s.bytes, s.ops, st);
            break;
        case SK_MAC:
            e = launch_mac_table(C, (const MacJob *)(ws + s.off), (const MacTarget *)(ws + s.off2), s.n_pairs, n,
                                 W.evk->keys, s.bytes, s.ops, st);
            break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int ckks_wave_create(ckks_context *ctx, const ckks_wave_item *items, uint32_t n, const ckks_evk_set *evk,
                     ckks_wave **out) {
    if (!out) return CKKS_EINVAL;
    *out = nullptr;
    if (!ctx || !items || n < 1 || !evk || evk->ctx != ctx) return CKKS_EINVAL;
    const Context &C = ctx->c;
    int log_n1, log_n2;
    ntt_geometry(C.log_n, log_n1, log_n2);
    if (log_n1 == 0) return CKKS_EINVAL;  // ring degrees of one-phase transforms (N <= 256) are not supported
    ckks_wave *W = new (std::nothrow) ckks_wave();
    if (!W) return CKKS_ENOMEM;
    W->ctx = ctx;
    W->evk = evk;
    for (uint32_t i = 0; i < n; ++i) {
        const ckks_wave_item &it = items[i];
        int rc = CKKS_OK;
        if (!it.ct || !it.plan || !it.out || !it.out->data || (int)it.k != it.plan->p.k) rc = CKKS_EINVAL;
        const uint32_t level = rc == CKKS_OK ? it.ct[0].level : 0;
        for (uint32_t u = 0; rc == CKKS_OK && u < it.k; ++u) {
            const ckks_tuple &t = it.ct[u];
            if (!t.data || t.n_polys != 2 || t.ntt_form != 1 || t.level != level || t.level < 1 ||
                t.level > (uint32_t)C.L || t.poly_stride < t.level)
                rc = CKKS_EINVAL;
        }
        if (rc == CKKS_OK && (int)level <= it.plan->p.depth) rc = CKKS_ELEVEL;
        if (rc == CKKS_OK && evk->t_max < it.k) rc = CKKS_EKEY;
        const uint32_t ol = level - (rc == CKKS_OK ? it.plan->p.depth : 0);
        if (rc == CKKS_OK) {
            if (it.out->poly_stride == 0) it.out->poly_stride = ol;
            if (it.out->poly_stride < ol) rc = CKKS_EINVAL;
        }
        if (rc != CKKS_OK) {
            delete W;
            return rc;
        }
        WaveProduct w;
        w.k = (int)it.k;
        w.plan = &it.plan->p;
        w.level = (int)level;
        for (uint32_t u = 0; u < it.k; ++u) {
            w.in.push_back((const u64 *)it.ct[u].data);
            w.in_ps.push_back((i64)it.ct[u].poly_stride * C.N);
            w.scales.push_back(it.ct[u].scale);
        }
        w.out = (u64 *)it.out->data;
        w.out_ps = (i64)it.out->poly_stride * C.N;
        W->items.push_back(w);
        W->outs.push_back(it.out);
    }
    // two products cannot write one output
    std::vector<const u64 *> o;
    for (const WaveProduct &w : W->items) o.push_back(w.out);
    std::sort(o.begin(), o.end());
    if (std::adjacent_find(o.begin(), o.end()) != o.end()) {
        delete W;
        return CKKS_EINVAL;
    }
    // sizes: a dry build with a fake base measures the tables and the scratch
    Bump sizing{nullptr, 0};
    {
        int H = 0;
        for (const WaveProduct &w : W->items) {
            std::vector<int> h;
            H = std::max(H, node_heights(*w.plan, h));
        }
        Builder B{C, evk->keys, H, {}};
        for (const WaveProduct &w : W->items) build_product(B, w, sizing);
    }
    W->scratch_bytes = sizing.off;
    W->table_bytes = (size_t)1 << 30;  // provisional: measured below
    std::vector<char> tables;
    int rc = build(*W, (char *)(size_t)4096, tables);
    W->table_bytes = align256(tables.size());
    W->stages.clear();
    if (rc != CKKS_OK) {
        delete W;
        return rc;
    }
    *out = W;
    return CKKS_OK;
}

int ckks_wave_workspace_size(const ckks_wave *w, size_t *table_bytes, size_t *scratch_bytes) {
    if (!w || !table_bytes || !scratch_bytes) return CKKS_EINVAL;
    *table_bytes = w->table_bytes;
    *scratch_bytes = w->scratch_bytes;
    return CKKS_OK;
}

int ckks_wave_describe(const ckks_wave *w, uint32_t *n_launches, uint32_t *heights) {
    if (!w || !n_launches || !heights) return CKKS_EINVAL;
    // one launch per stage, except: a fixed-shape tensor stage launches once
    // per shape, the key MAC once for paired and once for single products
    uint32_t n = 0;
    for (const Stage &s : w->stages) {
        if (s.kind == SK_TENSOR && s.fixed) n += (uint32_t)s.runs.size();
        else if (s.kind == SK_MAC) n += (s.n_pairs > 0 ? 1u : 0u) + (s.count() > s.n_pairs ? 1u : 0u);
        else n += 1;
    }
    *n_launches = n;
    *heights = (uint32_t)w->heights;
    return CKKS_OK;
}

int ckks_wave_run(ckks_wave *w, void *tables, size_t table_bytes, void *scratch, size_t scratch_bytes,
                  void *stream) {
    if (!w || !tables || !scratch) return CKKS_EINVAL;
    if (table_bytes < w->table_bytes || scratch_bytes < w->scratch_bytes) return CKKS_ENOMEM;
    if ((size_t)tables % 256 || (size_t)scratch % 256) return CKKS_EINVAL;
    ckks_context *ctx = w->ctx;
    const Context &C = ctx->c;
    if (C.sticky.load() != 0) return CKKS_ECUDA;
    cudaSetDevice(C.device);
    cudaStream_t st = (cudaStream_t)stream;
    if (w->bound_tables != tables || w->bound_scratch != scratch) {
        std::vector<char> host;
        int rc = build(*w, (char *)scratch, host);
        if (rc != CKKS_OK) return rc;
        cudaError_t e = cudaSuccess;
        if (w->uploaded) e = cudaEventSynchronize(w->uploaded);  // the previous copy has left the staging buffer
        if (e == cudaSuccess && w->staging_bytes < host.size()) {
            if (w->staging) cudaFreeHost(w->staging);
            w->staging = nullptr;
            w->staging_bytes = 0;
            e = cudaMallocHost(&w->staging, host.size());
            if (e == cudaSuccess) w->staging_bytes = host.size();
        }
        if (e == cudaSuccess && !w->uploaded) e = cudaEventCreateWithFlags(&w->uploaded, cudaEventDisableTiming);
        if (e == cudaSuccess && !host.empty()) {
            memcpy(w->staging, host.data(), host.size());
            e = cudaMemcpyAsync(tables, w->staging, host.size(), cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(w->uploaded, st);
        if (e != cudaSuccess) {
            ctx->c.sticky.store((int)e);
            return CKKS_ECUDA;
        }
        w->bound_tables = tables;
        w->bound_scratch = scratch;
    }
    cudaError_t e = enqueue(*w, (char *)tables, st);
    if (e != cudaSuccess) {
        ctx->c.sticky.store((int)e);
        return CKKS_ECUDA;
    }
    for (size_t i = 0; i < w->items.size(); ++i) {
        const WaveProduct &p = w->items[i];
        ckks_tuple *o = w->outs[i];
        o->n_polys = 2;
        o->level = (uint32_t)(p.level - p.plan->depth);
        o->ntt_form = 1;
        o->scale = plan_scale(C, *p.plan, p.level, p.scales.data());
    }
    return CKKS_OK;
}

void ckks_wave_destroy(ckks_wave *w) {
    if (!w) return;
    if (w->uploaded) {
        cudaEventSynchronize(w->uploaded);
        cudaEventDestroy(w->uploaded);
    }
    if (w->staging) cudaFreeHost(w->staging);
    delete w;
}

}  // extern "C"
