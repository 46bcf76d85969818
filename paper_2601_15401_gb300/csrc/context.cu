// Context creation: parameter checks and the constant tables of the method.
//
// Host arithmetic uses unsigned __int128. Tables (all per prime index x,
// Q primes first):
//   twiddles      psi^brv(k) and psi^-brv(k) with Shoup companions (NTT)
//   N^-1          Shoup constants (INTT)
//   ModUp BConv   per level and digit: N^-1 [(Q_beta/q_j)^-1]_{q_j} (applied
//                 in the INTT epilogue) and [(Q_beta/q_j) mod x] R (Eq. 4)
//   ModDown       N^-1 [phat_i^-1]_{p_i} and [p_i^-1]_{q_j} R (Eq. 5, 12)
//   key fold      P^-1 R^2 mod q_j, R^2 mod p_i (Eq. 12: P^-1 inside the key)
//   rescale       q_i^-1 mod q_j, and g^{mu,t}_eta of Eq. 16 per level, mu
//   gadget        P G_beta mod q_x (G_beta = 1 on its digit, 0 elsewhere)
#include <cstring>
#include <new>

#include "internal.h"

namespace ckks {

typedef unsigned __int128 u128;

static u64 h_mul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 h_pow(u64 b, u64 e, u64 q) {
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = h_mul(r, b, q);
        b = h_mul(b, b, q);
        e >>= 1;
    }
    return r;
}
static u64 h_inv(u64 a, u64 q) { return h_pow(a % q, q - 2, q); }
static Shoup h_shoup(u64 w, u64 q) {
    Shoup s;
    s.w = w % q;
    s.wp = (u64)(((u128)s.w << 64) / q);
    return s;
}
static u64 h_mont_qinv(u64 q) {
    u64 x = q;  // Newton iteration for q^-1 mod 2^64 (q odd)
    for (int i = 0; i < 6; ++i) x *= 2 - q * x;
    return x;
}
static u64 h_R(u64 q) { return (u64)(((u128)1 << 64) % q); }

static bool h_is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : bases) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; ++r; }
    for (u64 a : bases) {
        u64 x = h_pow(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; ++i) {
            x = h_mul(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

static unsigned brv(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// Smallest primitive 2N-th root of unity mod q.
static u64 h_min_psi(u64 q, int N) {
    u64 r = 0;
    for (u64 g = 2; g < 1000000; ++g) {
        r = h_pow(g, (q - 1) / (2 * (u64)N), q);
        if (h_pow(r, (u64)N, q) == q - 1) break;
        r = 0;
    }
    if (!r) return 0;
    u64 r2 = h_mul(r, r, q), best = r, cur = r;
    for (int i = 1; i < N; ++i) {
        cur = h_mul(cur, r2, q);
        if (cur < best) best = cur;
    }
    return best;
}

int context_build(Context &C, const uint32_t log_n, const uint32_t L, const uint32_t K, const uint32_t dnum,
                  const u64 *q, const u64 *p, int device) {
    if (log_n < 4 || log_n > 16 || L < 1 || dnum < 1 || dnum > L || L + K > CKKS_MAX_PRIMES || K < 1) return -1;
    C.device = device;
    C.log_n = (int)log_n;
    C.N = 1 << log_n;
    C.L = (int)L;
    C.K = (int)K;
    C.dnum = (int)dnum;
    C.alpha = (int)((L + dnum - 1) / dnum);
    if (C.alpha > 16) return -1;  // BConv keeps a digit in registers
    C.primes.assign(q, q + L);
    C.primes.insert(C.primes.end(), p, p + K);
    const int NP = C.L + C.K;
    const int N = C.N;
    for (int i = 0; i < NP; ++i) {
        u64 x = C.primes[i];
        if (x >= (1ull << 61) || !h_is_prime(x) || (x - 1) % (2 * (u64)N) != 0) return -1;
        for (int j = 0; j < i; ++j)
            if (C.primes[j] == x) return -1;
    }
    C.primes_q1 = true;
    for (int i = 0; i < NP; ++i) C.primes_q1 = C.primes_q1 && (C.primes[i] & 0xffffffffull) == 1;
    // BConv sums of products stay below hi < q only if sum of source primes < 2^64
    // (see Acc128); check every digit and the P basis.
    {
        u128 s = 0;
        for (int i = 0; i < C.K; ++i) s += p[i];
        if (s >> 64) return -1;
        for (int b = 0; b < C.dnum; ++b) {
            u128 t = 0;
            for (int j = b * C.alpha; j < std::min(C.L, (b + 1) * C.alpha); ++j) t += q[j];
            if (t >> 64) return -1;
        }
    }

    // ---- host tables
    std::vector<ModQ> mods(NP);
    std::vector<ulonglong2> twf((size_t)NP * N), twi((size_t)NP * N);
    std::vector<Shoup> ninv(NP), one(NP);
    std::vector<u64> r2(NP), keyfold(NP);
    std::vector<Shoup> rfix((size_t)NP * 16);
    std::vector<u64> cK((size_t)NP * CKKS_MAX_PRIMES, 0);
    std::vector<Shoup> invq((size_t)CKKS_MAX_PRIMES * CKKS_MAX_PRIMES);
    std::vector<Shoup> pscale(C.K);
    std::vector<Shoup> pgadget((size_t)C.dnum * NP);
    std::vector<u64> powt(N);
    for (int x = 0; x < NP; ++x) {
        const u64 m = C.primes[x];
        mods[x].q = m;
        mods[x].qinv = h_mont_qinv(m);
        const u64 psi = h_min_psi(m, N);
        if (!psi) return -1;
        // forward: psi^brv(k); inverse: psi^-brv(k)
        powt[0] = 1;
        for (int e = 1; e < N; ++e) powt[e] = h_mul(powt[e - 1], psi, m);
        for (int k = 0; k < N; ++k) {
            u64 w = powt[brv(k, C.log_n)];
            Shoup s = h_shoup(w, m);
            twf[(size_t)x * N + k] = make_ulonglong2(s.w, s.wp);
        }
        const u64 psi_inv = h_inv(psi, m);
        powt[0] = 1;
        for (int e = 1; e < N; ++e) powt[e] = h_mul(powt[e - 1], psi_inv, m);
        for (int k = 0; k < N; ++k) {
            u64 w = powt[brv(k, C.log_n)];
            Shoup s = h_shoup(w, m);
            twi[(size_t)x * N + k] = make_ulonglong2(s.w, s.wp);
        }
        ninv[x] = h_shoup(h_inv((u64)N % m, m), m);
        one[x] = h_shoup(1, m);
        const u64 R = h_R(m);
        r2[x] = h_mul(R, R, m);
        // rfix[e] = R^(e-1) mod q as a Shoup constant (e >= 1): the factor a
        // product of e tuples (e - 1 Montgomery products) is short of
        rfix[(size_t)x * 16] = h_shoup(1 % m, m);
        u64 acc = 1 % m;
        for (int e = 1; e < 16; ++e) {
            rfix[(size_t)x * 16 + e] = h_shoup(acc, m);
            acc = h_mul(acc, R, m);
        }
        u64 Pm = 1 % m;
        for (int i = 0; i < C.K; ++i) Pm = h_mul(Pm, p[i] % m, m);
        keyfold[x] = x < C.L ? h_mul(h_inv(Pm, m), r2[x], m) : r2[x];
        if (x < C.L) {
            for (int i = 0; i < C.K; ++i) cK[(size_t)x * CKKS_MAX_PRIMES + i] = h_mul(h_inv(p[i] % m, m), R, m);
            for (int b = 0; b < C.dnum; ++b) {
                bool in_digit = x / C.alpha == b;
                pgadget[(size_t)b * NP + x] = h_shoup(in_digit ? Pm : 0, m);
            }
        } else {
            for (int b = 0; b < C.dnum; ++b) pgadget[(size_t)b * NP + x] = h_shoup(0, m);
        }
    }
    for (int i = 0; i < NP; ++i)
        for (int j = 0; j < NP; ++j)
            invq[(size_t)i * CKKS_MAX_PRIMES + j] = i == j ? Shoup{0, 0} : h_shoup(h_inv(C.primes[i] % C.primes[j], C.primes[j]), C.primes[j]);
    for (int i = 0; i < C.K; ++i) {
        u64 pi = p[i];
        u64 phat = 1 % pi;
        for (int i2 = 0; i2 < C.K; ++i2)
            if (i2 != i) phat = h_mul(phat, p[i2] % pi, pi);
        pscale[i] = h_shoup(h_mul(h_inv(phat, pi), h_inv((u64)N % pi, pi), pi), pi);
    }
    // ModUp: for each level l (1..L) and digit beta at that level
    const int A = C.alpha;
    std::vector<Shoup> bpre((size_t)(C.L + 1) * C.L, Shoup{0, 0});
    std::vector<u64> bcon((size_t)(C.L + 1) * C.dnum * A * NP, 0);
    for (int lv = 1; lv <= C.L; ++lv) {
        for (int b = 0; b * A < lv; ++b) {
            const int d0 = b * A, d1 = std::min(lv, (b + 1) * A);
            for (int j = d0; j < d1; ++j) {
                const u64 qj = q[j];
                // (Q_beta / q_j) mod q_j and mod every x
                u64 hat_j = 1 % qj;
                for (int j2 = d0; j2 < d1; ++j2)
                    if (j2 != j) hat_j = h_mul(hat_j, q[j2] % qj, qj);
                bpre[(size_t)lv * C.L + j] = h_shoup(h_mul(h_inv(hat_j, qj), h_inv((u64)N % qj, qj), qj), qj);
                for (int x = 0; x < NP; ++x) {
                    const u64 m = C.primes[x];
                    u64 hx = 1 % m;
                    for (int j2 = d0; j2 < d1; ++j2)
                        if (j2 != j) hx = h_mul(hx, q[j2] % m, m);
                    bcon[(((size_t)lv * C.dnum + b) * A + (j - d0)) * NP + x] = h_mul(hx, h_R(m), m);
                }
            }
        }
    }
    // Eq. 16 tables: level lv, mu in [1, lv-1]; rows eta < lv - mu,
    // entries t' < mu -> g^{mu, lv-mu+t'}_eta, entry mu -> g^{mu, lv-1}_eta
    C.g_off.assign(C.L + 1, std::vector<size_t>(C.L + 1, 0));
    std::vector<Shoup> gt;
    for (int lv = 2; lv <= C.L; ++lv) {
        for (int mu = 1; mu < lv; ++mu) {
            C.g_off[lv][mu] = gt.size();
            for (int eta = 0; eta < lv - mu; ++eta) {
                const u64 qe = q[eta];
                // prefix products of inverses q_{lv-mu}^-1 ... q_t^-1
                u64 g = 1 % qe;
                std::vector<Shoup> row(mu + 1);
                for (int t = lv - mu; t < lv; ++t) {
                    g = h_mul(g, h_inv(q[t] % qe, qe), qe);
                    row[t - (lv - mu)] = h_shoup(g, qe);
                }
                row[mu] = h_shoup(g, qe);  // t = lv - 1
                gt.insert(gt.end(), row.begin(), row.end());
            }
        }
    }
    if (gt.empty()) gt.push_back(Shoup{0, 0});
    C.h_ninv = ninv;

    // ---- one device allocation
    struct Piece {
        const void *src;
        size_t bytes;
        void **dst;
    };
    static const unsigned long long zero_words[2] = {0, 0};  // integrity-check counter
    std::vector<Piece> pieces = {
        {mods.data(), mods.size() * sizeof(ModQ), (void **)&C.d_mods},
        {twf.data(), twf.size() * sizeof(ulonglong2), (void **)&C.d_tw_fwd},
        {twi.data(), twi.size() * sizeof(ulonglong2), (void **)&C.d_tw_inv},
        {ninv.data(), ninv.size() * sizeof(Shoup), (void **)&C.d_ninv},
        {one.data(), one.size() * sizeof(Shoup), (void **)&C.d_one},
        {pscale.data(), pscale.size() * sizeof(Shoup), (void **)&C.d_pscale},
        {cK.data(), cK.size() * sizeof(u64), (void **)&C.d_cK},
        {r2.data(), r2.size() * sizeof(u64), (void **)&C.d_r2},
        {rfix.data(), rfix.size() * sizeof(Shoup), (void **)&C.d_rfix},
        {keyfold.data(), keyfold.size() * sizeof(u64), (void **)&C.d_keyfold},
        {invq.data(), invq.size() * sizeof(Shoup), (void **)&C.d_invq},
        {bpre.data(), bpre.size() * sizeof(Shoup), (void **)&C.d_bconv_pre},
        {bcon.data(), bcon.size() * sizeof(u64), (void **)&C.d_bconv_c},
        {gt.data(), gt.size() * sizeof(Shoup), (void **)&C.d_g},
        {pgadget.data(), pgadget.size() * sizeof(Shoup), (void **)&C.d_pgadget},
        {zero_words, sizeof(zero_words), (void **)&C.d_check},
    };
    size_t total = 0;
    for (auto &pc : pieces) total += (pc.bytes + 255) / 256 * 256;
    if (cudaSetDevice(device) != cudaSuccess) return -5;
    void *blk = nullptr;
    if (cudaMalloc(&blk, total) != cudaSuccess) return -5;
    C.d_block = blk;
    size_t off = 0;
    for (auto &pc : pieces) {
        *pc.dst = (char *)blk + off;
        if (cudaMemcpy(*pc.dst, pc.src, pc.bytes, cudaMemcpyHostToDevice) != cudaSuccess) return -5;
        off += (pc.bytes + 255) / 256 * 256;
    }
    for (int i = 0; i < OP_COUNT; ++i) C.counters[i] = 0;
    return 0;
}

void profiler_release(Context &C);

void context_release(Context &C) {
    profiler_release(C);
    if (C.d_block) {
        cudaSetDevice(C.device);
        cudaFree(C.d_block);
        C.d_block = nullptr;
    }
}

}  // namespace ckks

namespace ckks {

ProfScope::ProfScope(const Context &c, int k, double by, cudaStream_t s, double op)
    : C(const_cast<Context *>(&c)), cls(k), bytes(by), ops(op), st(s) {
    Profiler &P = C->prof;
    if (!P.on) return;
    if (P.used + 2 > P.pool.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            P.pool.push_back(e);
        }
    }
    cudaEvent_t a = P.pool[P.used++];
    b = P.pool[P.used++];
    cudaEventRecord(a, st);
    P.recs.push_back(ProfRec{cls, a, b, bytes, ops});
}

ProfScope::~ProfScope() {
    if (b) cudaEventRecord(b, st);
}

void profiler_release(Context &C) {
    for (cudaEvent_t e : C.prof.pool) cudaEventDestroy(e);
    C.prof.pool.clear();
    C.prof.recs.clear();
    C.prof.used = 0;
}

}  // namespace ckks
