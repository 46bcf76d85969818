"""The paper's RNS-CKKS multiplication, written step by step (test
infrastructure only; see the package docstring).

Conventions
  * A tuple is a numpy uint64 array [n_polys][level][N]; limb j is modulo
    q_j. "NTT domain" arrays hold the evaluation map of `ring.ntt_definition`.
  * Evaluation-key limbs are ordered Q first (q_0..q_{L-1}) then P
    (p_0..p_{K-1}); Eq. 2 lists the P limbs first, only the storage order
    differs.
  * rs (Eq. 6) subtracts the top residue taken as an integer in [0, q_top):
    the result is floor(x / q_top) of the CRT value x, no rounding offset.
  * BConv is the fast conversion of Eq. 4 as an exact integer function, with
    no correction of its u * Q overflow term.
  * With dnum > 1 digits, digit beta covers q_{beta*alpha} .. q_{(beta+1)*alpha - 1}
    (truncated at the current level) and the key's Q limbs carry
    P * G_beta * s^t, G_beta = Qhat_beta * [Qhat_beta^-1]_{Q_beta},
    Qhat_beta = Q_L / Q_beta. For dnum = 1, G = 1 and this is Eq. 2/9/14.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import plan as _plan
from . import ring


def prod(xs) -> int:
    r = 1
    for x in xs:
        r *= int(x)
    return r


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
class Ctx:
    """Oracle view of the parameters (synth.Params or anything with
    log_n, q, p, dnum)."""

    def __init__(self, params):
        self.N = 1 << params.log_n
        self.q = [int(x) for x in params.q]
        self.p = [int(x) for x in params.p]
        self.L = len(self.q)
        self.K = len(self.p)
        self.dnum = params.dnum
        self.alpha = -(-self.L // self.dnum)
        self.P = prod(self.p)

    def digits(self, level: int) -> list[list[int]]:
        """Prime indices of each digit at this level (Q limbs only)."""
        return [list(range(b * self.alpha, min(level, (b + 1) * self.alpha)))
                for b in range(-(-level // self.alpha))]

    def gadget(self, beta: int) -> int:
        """G_beta over the full chain Q_L."""
        idx = range(beta * self.alpha, min(self.L, (beta + 1) * self.alpha))
        Qb = prod(self.q[j] for j in idx)
        Qhat = prod(self.q) // Qb
        return Qhat * pow(Qhat % Qb, -1, Qb)


# ---------------------------------------------------------------------------
# transforms on tuples
# ---------------------------------------------------------------------------
def ntt_poly(a: np.ndarray, primes) -> np.ndarray:
    return ring.ntt_rows(a, primes)


def intt_poly(A: np.ndarray, primes) -> np.ndarray:
    return ring.intt_rows(A, primes)


# ---------------------------------------------------------------------------
# Eq. 13: tensor product of child tuples (NTT domain, coefficient-wise)
# ---------------------------------------------------------------------------
def tensor_product(ctx: Ctx, children: list[np.ndarray]) -> np.ndarray:
    """d_t = sum over l_1..l_m with sum t of prod_u c^u_{l_u}. The children are
    tuples (polynomials in s); the product is their polynomial product in s,
    taken one child at a time. Every child must be at the same level."""
    level = children[0].shape[1]
    primes = ctx.q[:level]
    out = children[0]
    for c in children[1:]:
        assert c.shape[1] == level
        n_out = out.shape[0] + c.shape[0] - 1
        nxt = np.zeros((n_out, level, ctx.N), dtype=np.uint64)
        for a in range(out.shape[0]):
            for b in range(c.shape[0]):
                nxt[a + b] = ring.addmod_rows(nxt[a + b], ring.mulmod_rows(out[a], c[b], primes), primes)
        out = nxt
    return out


# ---------------------------------------------------------------------------
# Eq. 6 / Eq. 7 / Algorithm 1: rescaling
# ---------------------------------------------------------------------------
def rs(ctx: Ctx, a: np.ndarray) -> np.ndarray:
    """Eq. 6 on one polynomial in the coefficient domain, [l][N] -> [l-1][N]:
    divide by the top prime q_{l-1}."""
    l = a.shape[0]
    qt = ctx.q[l - 1]
    top = a[l - 1]
    out = np.empty((l - 1, ctx.N), dtype=np.uint64)
    for j in range(l - 1):
        qj = ctx.q[j]
        out[j] = ring.smul(ring.submod(a[j], top % np.uint64(qj), qj), ring.inv(qt, qj), qj)
    return out


def RS(ctx: Ctx, A: np.ndarray) -> np.ndarray:
    """Eq. 7: one rescale in the NTT domain (INTT of the top limb, NTT of it
    into every remaining modulus)."""
    l = A.shape[0]
    qt = ctx.q[l - 1]
    top = ring.intt(A[l - 1], qt)
    out = np.empty((l - 1, ctx.N), dtype=np.uint64)
    for j in range(l - 1):
        qj = ctx.q[j]
        T = ring.ntt(top % np.uint64(qj), qj)
        out[j] = ring.smul(ring.submod(A[j], T, qj), ring.inv(qt, qj), qj)
    return out


def g_const(ctx: Ctx, level: int, u: int, t: int, eta: int) -> int:
    """Eq. 16: g^{u,t}_eta = q_{L-u}^-1 q_{L-u+1}^-1 ... q_t^-1 mod q_eta, with
    L the current level."""
    qe = ctx.q[eta]
    g = 1
    for i in range(level - u, t + 1):
        g = g * ring.inv(ctx.q[i], qe) % qe
    return g


def multi_rs_alg1(ctx: Ctx, A: np.ndarray, mu: int) -> np.ndarray:
    """Algorithm 1 on one polynomial, NTT domain [L][N] -> [L-mu][N]."""
    L = A.shape[0]
    assert 1 <= mu < L
    # step 1: INTT of the mu top limbs
    a = {}
    for u in range(L - mu, L):
        a[(u, 0)] = ring.intt(A[u], ctx.q[u])
    # step 2: rescale the top limbs among themselves (Eq. 6), u = 1..mu-1
    for u in range(1, mu):
        top = a[(L - u, u - 1)]
        qtop = ctx.q[L - u]
        for t in range(L - mu, L - u):
            qt = ctx.q[t]
            a[(t, u)] = ring.smul(ring.submod(a[(t, u - 1)], top % np.uint64(qt), qt),
                                  ring.inv(qtop, qt), qt)
    # step 3: combine and transform back
    out = np.empty((L - mu, ctx.N), dtype=np.uint64)
    for eta in range(L - mu):
        qe = ctx.q[eta]
        b = np.zeros(ctx.N, dtype=np.uint64)
        for t in range(L - mu, L):
            b = ring.addmod(b, ring.smul(a[(t, L - 1 - t)] % np.uint64(qe),
                                         g_const(ctx, L, mu, t, eta), qe), qe)
        B = ring.ntt(b, qe)
        out[eta] = ring.submod(ring.smul(A[eta], g_const(ctx, L, mu, L - 1, eta), qe), B, qe)
    return out


def multi_rs_sequential(ctx: Ctx, A: np.ndarray, mu: int) -> np.ndarray:
    """The same mu rescales done plainly: INTT of every limb, mu times Eq. 6,
    NTT of the survivors (the 2L - mu transform alternative of Section V-B)."""
    L = A.shape[0]
    a = intt_poly(A, ctx.q[:L])
    for _ in range(mu):
        a = rs(ctx, a)
    return ntt_poly(a, ctx.q[:L - mu])


# ---------------------------------------------------------------------------
# Eq. 4: basis conversion; ModUp; Eq. 5: ModDown
# ---------------------------------------------------------------------------
def bconv(y: np.ndarray, src: list[int], dst: list[int]) -> np.ndarray:
    """Eq. 4 (coefficient domain): sum_j [y_j * qhat_j^-1]_{q_j} * qhat_j mod x,
    qhat_j = (prod src) / q_j, for each destination modulus x. Computed with
    residues; `bconv_bigint` is the same integer S written with big ints."""
    Qs = prod(src)
    ys = np.stack([ring.smul(y[j], ring.inv(Qs // qj, qj), qj) for j, qj in enumerate(src)])
    out = np.empty((len(dst), y.shape[1]), dtype=np.uint64)
    for i, x in enumerate(dst):
        out[i] = ring.dot_const(ys, [(Qs // qj) % x for qj in src], x)
    return out


def bconv_bigint(y: np.ndarray, src: list[int]) -> list[int]:
    """The integer S = sum_j [y_j qhat_j^-1]_{q_j} qhat_j of Eq. 4, per
    coefficient, as Python ints (S is in [0, |src| * prod(src)))."""
    Qs = prod(src)
    out = []
    for c in range(y.shape[1]):
        S = 0
        for j, qj in enumerate(src):
            qh = Qs // qj
            S += (int(y[j, c]) * pow(qh % qj, -1, qj) % qj) * qh
        out.append(S)
    return out


def modup(ctx: Ctx, D: np.ndarray, level: int, digit: list[int]) -> np.ndarray:
    """Raise one digit of D (NTT domain, [level][N]) to Q_level * P:
    INTT, Eq. 4 BConv to every other modulus, NTT. Returns [level + K][N]
    (Q limbs then P limbs), NTT domain. The digit's own limbs are D's."""
    src = [ctx.q[j] for j in digit]
    y = intt_poly(D[digit], src)
    others_q = [j for j in range(level) if j not in digit]
    dst = [ctx.q[j] for j in others_q] + ctx.p
    conv = ntt_poly(bconv(y, src, dst), dst)
    out = np.empty((level + ctx.K, ctx.N), dtype=np.uint64)
    for i, j in enumerate(others_q):
        out[j] = conv[i]
    for j in digit:
        out[j] = D[j]
    out[level:] = conv[len(others_q):]
    return out


def moddown_coef(ctx: Ctx, c_tilde: np.ndarray, level: int) -> np.ndarray:
    """Eq. 5 in the coefficient domain: c_tilde is [level + K][N] (Q then P
    limbs); returns [P^-1 (c_tilde^{(Q_j)} - BConv(c_tilde^{(P)}, p, q_j))]_{q_j}."""
    R = bconv(c_tilde[level:], ctx.p, ctx.q[:level])
    out = np.empty((level, ctx.N), dtype=np.uint64)
    for j in range(level):
        qj = ctx.q[j]
        out[j] = ring.smul(ring.submod(c_tilde[j], R[j], qj), ring.inv(ctx.P % qj, qj), qj)
    return out


def key_primes(ctx: Ctx, level: int) -> list[int]:
    return ctx.q[:level] + ctx.p


def key_rows(ctx: Ctx, level: int) -> list[int]:
    """Rows of a stored key ([L + K][N]) used at this level."""
    return list(range(level)) + list(range(ctx.L, ctx.L + ctx.K))


# ---------------------------------------------------------------------------
# Eq. 2 / 9 / 14: evaluation keys
# ---------------------------------------------------------------------------
def secret_ntt(ctx: Ctx, s: np.ndarray) -> np.ndarray:
    primes = ctx.q + ctx.p
    return ntt_poly(np.stack([ring.from_signed(s, x) for x in primes]), primes)


def keygen(ctx: Ctx, s: np.ndarray, a: np.ndarray, e: np.ndarray, t: int, beta: int, S=None, St=None):
    """ek_{t,beta} = (-a s + e + [Q limb] P G_beta s^t, a), NTT domain, all
    L + K limbs. s and e are small signed coefficient vectors; a is given in
    the NTT domain. S = NTT(s) and St = NTT(s)^t may be passed in."""
    primes = ctx.q + ctx.p
    if S is None:
        S = secret_ntt(ctx, s)
    E = ntt_poly(np.stack([ring.from_signed(e, x) for x in primes]), primes)
    if St is None:
        St = S.copy()
        for _ in range(t - 1):
            St = ring.mulmod_rows(St, S, primes)
    G = ctx.gadget(beta)
    ek0 = np.empty_like(a)
    for x, m in enumerate(primes):
        v = ring.submod(E[x], ring.mulmod(a[x], S[x], m), m)
        if x < ctx.L:
            v = ring.addmod(v, ring.smul(St[x], ctx.P * G % m, m), m)
        ek0[x] = v
    return ek0, a.copy()


def keygen_all(ctx: Ctx, km, t_max: int):
    """keys[t-2][beta] = (ek0, ek1) for t = 2..t_max from synth.KeyMaterial."""
    primes = ctx.q + ctx.p
    S = secret_ntt(ctx, km.s)
    St = S.copy()
    out = []
    for t in range(2, t_max + 1):
        St = ring.mulmod_rows(St, S, primes)
        out.append([keygen(ctx, km.s, km.a[t - 2][b], km.e[t - 2][b], t, b, S, St) for b in range(ctx.dnum)])
    return out


# ---------------------------------------------------------------------------
# Eq. 15: relinearisation with one combined ModDown per output polynomial
# ---------------------------------------------------------------------------
def relin_accumulate(ctx: Ctx, d: np.ndarray, keys, level: int, ts=None) -> np.ndarray:
    """acc_l = sum_{t >= 2} sum_beta ModUp_beta(d_t) * ek_{t,beta,l}
    (NTT domain, [2][level + K][N]) -- the sum taken before the single
    ModDown (Section III, combined form). `ts` restricts the sum to some t."""
    n = d.shape[0] - 1
    kp = key_primes(ctx, level)
    rows = key_rows(ctx, level)
    acc = np.zeros((2, level + ctx.K, ctx.N), dtype=np.uint64)
    for t in (range(2, n + 1) if ts is None else ts):
        for beta, digit in enumerate(ctx.digits(level)):
            ext = modup(ctx, d[t], level, digit)
            for l in range(2):
                ek = keys[t - 2][beta][l][rows]
                acc[l] = ring.addmod_rows(acc[l], ring.mulmod_rows(ext, ek, kp), kp)
    return acc


def _moddowns(ctx: Ctx, d: np.ndarray, keys, level: int, separate: bool) -> np.ndarray:
    """ModDown (Eq. 5) of the key products, coefficient domain [2][level][N].
    Combined (Eq. 15): one ModDown of the sum over t. Separate (the form the
    paper replaces): one ModDown per ek_t, the results summed."""
    n = d.shape[0] - 1
    kp = key_primes(ctx, level)
    qs = ctx.q[:level]
    groups = [[t] for t in range(2, n + 1)] if separate else [None]
    out = np.zeros((2, level, ctx.N), dtype=np.uint64)
    for ts in groups:
        acc = relin_accumulate(ctx, d, keys, level, ts)
        for l in range(2):
            out[l] = ring.addmod_rows(out[l], moddown_coef(ctx, intt_poly(acc[l], kp), level), qs)
    return out


def relin_coef(ctx: Ctx, d: np.ndarray, keys, level: int, separate: bool = False) -> np.ndarray:
    """c* = (d_0, d_1) + sum_t ceil(P^-1 d_t ek_t) in the coefficient domain
    ([2][level][N]): ModDown (Eq. 5) of the accumulated product, added to
    INTT(d_0), INTT(d_1)."""
    c_hat = _moddowns(ctx, d, keys, level, separate)
    qs = ctx.q[:level]
    return np.stack([ring.addmod_rows(intt_poly(d[l], qs), c_hat[l], qs) for l in range(2)])


def relin_ntt(ctx: Ctx, d: np.ndarray, keys, level: int, separate: bool = False) -> np.ndarray:
    """The same relinearisation in the prior (standard) arrangement: ModDown
    transformed back to the NTT domain and added to D_0, D_1 there."""
    c_hat = _moddowns(ctx, d, keys, level, separate)
    qs = ctx.q[:level]
    return np.stack([ring.addmod_rows(d[l], ntt_poly(c_hat[l], qs), qs) for l in range(2)])


# ---------------------------------------------------------------------------
# Section V: k-input multiplication over a partition tree
# ---------------------------------------------------------------------------
@dataclass
class Tup:
    data: np.ndarray    # [n_polys][level][N], NTT domain
    scale: float

    @property
    def level(self) -> int:
        return self.data.shape[1]


def align(children: list[Tup]) -> list[Tup]:
    """Drop top limbs so that every child sits at the lowest child level."""
    lv = min(c.level for c in children)
    return [Tup(c.data[:, :lv].copy(), c.scale) for c in children]


def eval_node(ctx: Ctx, node: _plan.Node, leaves: list, keys, pos: list, root: bool,
              rescale: str = "sequential", separate: bool = False) -> Tup:
    if node.is_leaf:
        ct = leaves[pos[0]]
        pos[0] += 1
        return ct
    kids = align([eval_node(ctx, c, leaves, keys, pos, False, rescale) for c in node.children])
    D = tensor_product(ctx, [k.data for k in kids])
    scale = math.prod(k.scale for k in kids)
    level = kids[0].level
    mu = len(node.children) - 1
    if root:
        cstar = relin_coef(ctx, D, keys, level, separate)
        for _ in range(mu):
            cstar = np.stack([rs(ctx, cstar[l]) for l in range(2)])
        out_level = level - mu
        out = np.stack([ntt_poly(cstar[l], ctx.q[:out_level]) for l in range(2)])
    else:
        f = multi_rs_sequential if rescale == "sequential" else multi_rs_alg1
        out = np.stack([f(ctx, D[i], mu) for i in range(D.shape[0])])
    for j in range(mu):
        scale /= ctx.q[level - 1 - j]
    return Tup(out, scale)


def mul_k(ctx: Ctx, cts: list[Tup], keys, partition: str | None = None,
          rescale: str = "sequential", separate_moddown: bool = False) -> Tup:
    """k-input product: tensor products and multi-rescales at the inner nodes
    (bottom-up), relinearisation at the root (Eq. 15), then the root's
    m - 1 rescales in the coefficient domain and one NTT (relocated
    rescale, Section IV). `separate_moddown` takes one ModDown per ek_t
    instead of Eq. 15's single one."""
    k = len(cts)
    part = partition or _plan.TABLE_II[k]
    root = _plan.parse(part, k)
    if not _plan.valid(root, k):
        raise ValueError(f"partition {part} breaks the depth rule")
    return eval_node(ctx, root, cts, keys, [0], True, rescale, separate_moddown)


def mul2_standard(ctx: Ctx, a: Tup, b: Tup, keys) -> Tup:
    """The 2-input multiply of Section II as printed: PM (Eq. 1), relin with
    ModDown back to the NTT domain (Eq. 3-5), RS in the NTT domain (Eq. 7)."""
    a, b = align([a, b])
    D = tensor_product(ctx, [a.data, b.data])
    level = a.level
    C = relin_ntt(ctx, D, keys, level)
    out = np.stack([RS(ctx, C[l]) for l in range(2)])
    return Tup(out, a.scale * b.scale / ctx.q[level - 1])


def mul_chain(ctx: Ctx, cts: list[Tup], keys) -> Tup:
    """k inputs through a binary tree of standard 2-input multiplies (the
    baseline column of Table II)."""
    def go(node, pos):
        if node.is_leaf:
            ct = cts[pos[0]]
            pos[0] += 1
            return ct
        x = go(node.children[0], pos)
        y = go(node.children[1], pos)
        return mul2_standard(ctx, x, y, keys)
    return go(_plan.binary_partition(len(cts)), [0])


# ---------------------------------------------------------------------------
# Section II: encoding, encryption, decryption (fixtures and gates)
# ---------------------------------------------------------------------------
def _roots(N: int) -> np.ndarray:
    """zeta_j = exp(i pi 5^j / N), j < N/2: the slots' evaluation points."""
    M = 2 * N
    e = np.array([pow(5, j, M) for j in range(N // 2)], dtype=np.float64)
    return np.exp(1j * np.pi * e / N)


def encode(N: int, z: np.ndarray, scale: float) -> list[int]:
    """Integer coefficients m with m(zeta_j) ~ scale * z_j (canonical
    embedding; m_i = (2/N) Re sum_j scale z_j conj(zeta_j)^i, rounded)."""
    zeta = _roots(N)
    i = np.arange(N)
    V = np.conj(zeta)[:, None] ** i[None, :]
    m = (2.0 / N) * np.real((scale * z)[:, None] * V).sum(axis=0)
    return [int(round(x)) for x in m]


def decode(N: int, m: list[int], scale: float) -> np.ndarray:
    zeta = _roots(N)
    i = np.arange(N)
    mf = np.array([x / scale for x in m], dtype=np.float64)
    return (zeta[:, None] ** i[None, :] * mf[None, :]).sum(axis=1)


def decode_slot(N: int, m, scale: float, j: int) -> complex:
    """One slot, z_j = sum_i m_i zeta_j^i / scale, with the exponent of
    zeta_j^i = omega^(5^j i) reduced mod 2N in integers (no power error)."""
    e = pow(5, j, 2 * N)
    i = np.arange(N, dtype=np.int64)
    ang = np.pi * ((e * i) % (2 * N)).astype(np.float64) / N
    mf = np.array([float(x) for x in m], dtype=np.float64) / scale
    return complex(np.sum(mf * np.cos(ang)), np.sum(mf * np.sin(ang)))


def encode_coef(N: int, z: np.ndarray, scale: float, i: int) -> float:
    """One coefficient before rounding: (2/N) Re sum_j scale z_j zeta_j^-i,
    exponents reduced mod 2N in integers."""
    e = np.array([pow(5, j, 2 * N) for j in range(N // 2)], dtype=np.int64)
    ang = -np.pi * ((e * i) % (2 * N)).astype(np.float64) / N
    return float((2.0 / N) * np.sum(scale * (z.real * np.cos(ang) - z.imag * np.sin(ang))))


def public_key(ctx: Ctx, s, a, e):
    """pk = (-a s + e, a) on the Q limbs, NTT domain (a given NTT domain)."""
    S = ntt_poly(np.stack([ring.from_signed(s, x) for x in ctx.q]), ctx.q)
    E = ntt_poly(np.stack([ring.from_signed(e, x) for x in ctx.q]), ctx.q)
    return ring.submod_rows(E, ring.mulmod_rows(a, S, ctx.q), ctx.q), a.copy()


def encrypt(ctx: Ctx, m: list[int], pk, v, e0, e1) -> np.ndarray:
    """(v pk_0 + e_0 + m, v pk_1 + e_1), NTT domain, all L limbs."""
    q = ctx.q

    def lift(x):
        return ntt_poly(np.stack([np.array([int(c) % qj for c in x], dtype=np.uint64) for qj in q]), q)

    V, E0, E1, M = lift(v), lift(e0), lift(e1), lift(m)
    c0 = ring.addmod_rows(ring.addmod_rows(ring.mulmod_rows(V, pk[0], q), E0, q), M, q)
    c1 = ring.addmod_rows(ring.mulmod_rows(V, pk[1], q), E1, q)
    return np.stack([c0, c1])


def crt_centered(limbs: np.ndarray, primes) -> list[int]:
    """Big-int CRT of [l][N] residues, centred in (-Q/2, Q/2]."""
    Q = prod(primes)
    coefs = [0] * limbs.shape[1]
    for j, qj in enumerate(primes):
        qh = Q // qj
        w = qh * pow(qh % qj, -1, qj)
        row = limbs[j]
        for c in range(limbs.shape[1]):
            coefs[c] += int(row[c]) * w
    out = []
    for x in coefs:
        x %= Q
        out.append(x - Q if x > Q // 2 else x)
    return out


def decrypt(ctx: Ctx, ct: np.ndarray, s) -> list[int]:
    """c_0 + c_1 s over every limb of the ciphertext's level (schoolbook
    product in the coefficient domain), lifted by CRT and centred."""
    level = ct.shape[1]
    primes = ctx.q[:level]
    c = np.stack([intt_poly(ct[l], primes) for l in range(2)])
    rows = []
    for j, qj in enumerate(primes):
        sj = ring.from_signed(s, qj)
        rows.append(ring.addmod(c[0][j], ring.negacyclic_mul(c[1][j], sj, qj), qj))
    return crt_centered(np.stack(rows), primes)


# ---------------------------------------------------------------------------
# Galois automorphisms and slot rotation (Section II's encoding; key switch
# as in Eq. 3-5 with the key of sigma_g(s))
# ---------------------------------------------------------------------------
def galois_element(r: int, N: int) -> int:
    """g = 5^r mod 2N: sigma_g moves slot j + r of the encoding to slot j."""
    return pow(5, r % (N // 2), 2 * N)


def automorphism_coef(a, g: int, q: int) -> np.ndarray:
    """a(X^g) mod (X^N + 1, q) from its definition: X^i -> X^(g i), and
    X^(N + j) = -X^j. `a` holds residues mod q."""
    N = len(a)
    out = np.zeros(N, dtype=np.uint64)
    for i in range(N):
        j = (g * i) % (2 * N)
        v = int(a[i]) % q
        if j < N:
            out[j] = (int(out[j]) + v) % q
        else:
            out[j - N] = (int(out[j - N]) - v) % q
    return out


def automorphism_signed(s, g: int) -> np.ndarray:
    """The same map on a signed integer polynomial (the secret)."""
    N = len(s)
    out = np.zeros(N, dtype=np.int64)
    for i in range(N):
        j = (g * i) % (2 * N)
        if j < N:
            out[j] += int(s[i])
        else:
            out[j - N] -= int(s[i])
    return out


def automorphism_ntt(A: np.ndarray, g: int, primes) -> np.ndarray:
    """sigma_g of an NTT-domain [limbs][N] array: back to coefficients,
    the definition, forward again."""
    a = intt_poly(A, primes)
    return ntt_poly(np.stack([automorphism_coef(a[j], g, qj) for j, qj in enumerate(primes)]), primes)


def galois_keygen(ctx: Ctx, km_s, a, e, g: int):
    """gk[beta] = (-a s + e + [Q limb] P G_beta sigma_g(s), a): the
    evaluation-key construction with sigma_g(s) in place of s^t. a: [dnum]
    NTT-domain [L + K][N]; e: [dnum] signed [N]."""
    S = secret_ntt(ctx, km_s)
    Sg = secret_ntt(ctx, automorphism_signed(km_s, g))
    return [keygen(ctx, km_s, a[b], e[b], 2, b, S, Sg) for b in range(ctx.dnum)]


def rotate(ctx: Ctx, ct: Tup, g: int, gkey) -> Tup:
    """(sigma c_0, sigma c_1) switched back to s: the relinearisation of
    (sigma c_0, 0, sigma c_1) with the Galois key in the place of ek_2,
    ModDown finished in the NTT domain."""
    level = ct.level
    primes = ctx.q[:level]
    c0 = automorphism_ntt(ct.data[0], g, primes)
    c1 = automorphism_ntt(ct.data[1], g, primes)
    d = np.stack([c0, np.zeros_like(c0), c1])
    return Tup(relin_ntt(ctx, d, [gkey], level), ct.scale)
