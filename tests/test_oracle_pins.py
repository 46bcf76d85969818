"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an independent big-integer computation, an invariant proved in the
paper, or a table the paper prints. No test here needs a GPU.
"""
import math

import numpy as np
import pytest

import synth
from oracle import ckks, plan, ring

PRIMES = [synth.prime_chain(50, 1)[0], synth.prime_chain(45, 1)[0], synth.prime_chain(60, 1)[0]]


def rand_res(g, q, n):
    return g.integers(0, q, size=n, dtype=np.uint64)


# --------------------------------------------------------------------------
# modular primitives and the transform (Section II)
# --------------------------------------------------------------------------
def test_mulmod_matches_python_ints():
    g = synth.rng(99)
    for q in PRIMES:
        a, b = rand_res(g, q, 257), rand_res(g, q, 257)
        got = ring.mulmod(a, b, q)
        assert [int(x) for x in got] == [int(x) * int(y) % q for x, y in zip(a, b)]


@pytest.mark.parametrize("log_n", [2, 3, 5, 8])
def test_psi_is_smallest_primitive_root(log_n):
    N = 1 << log_n
    q = PRIMES[0]
    psi = ring.psi_of(q, N)
    assert pow(psi, N, q) == q - 1
    # brute force over all primitive 2N-th roots: psi0^(odd)
    for g in range(2, 200):
        r = pow(g, (q - 1) // (2 * N), q)
        if pow(r, N, q) == q - 1:
            break
    assert pow(r, N, q) == q - 1
    roots = {pow(r, e, q) for e in range(1, 2 * N, 2)}
    assert psi == min(roots)


def test_ntt_closed_forms():
    """NTT(1) = all ones; NTT(x) at slot i = psi^(2 brv(i) + 1)."""
    N, q = 16, PRIMES[1]
    psi = ring.psi_of(q, N)
    one = np.zeros(N, dtype=np.uint64)
    one[0] = 1
    assert np.all(ring.ntt_definition(one, q) == 1)
    x = np.zeros(N, dtype=np.uint64)
    x[1] = 1
    want = [pow(psi, 2 * ring.brv(i, 4) + 1, q) for i in range(N)]
    assert [int(v) for v in ring.ntt_definition(x, q)] == want
    assert [int(v) for v in ring.ntt(x, q)] == want


@pytest.mark.parametrize("log_n", [3, 4, 6, 8, 10])
def test_fast_ntt_equals_definition(log_n):
    g = synth.rng(98, log_n)
    N = 1 << log_n
    for q in PRIMES:
        a = rand_res(g, q, N)
        A = ring.ntt_definition(a, q)
        assert np.array_equal(ring.ntt(a, q), A)
        assert np.array_equal(ring.intt_definition(A, q), a)
        assert np.array_equal(ring.intt(A, q), a)


def test_schoolbook_closed_form_and_convolution_theorem():
    N, q = 32, PRIMES[0]
    # x^i * x^j = x^(i+j) if i+j < N else -x^(i+j-N)
    for i, j in [(3, 5), (20, 17), (31, 1), (0, 31)]:
        a = np.zeros(N, dtype=np.uint64)
        b = np.zeros(N, dtype=np.uint64)
        a[i] = 1
        b[j] = 1
        c = ring.negacyclic_mul(a, b, q)
        want = np.zeros(N, dtype=np.uint64)
        if i + j < N:
            want[i + j] = 1
        else:
            want[i + j - N] = q - 1
        assert np.array_equal(c, want)
    g = synth.rng(97)
    a, b = rand_res(g, q, N), rand_res(g, q, N)
    # independent big-int product reduced by x^N + 1
    full = [0] * (2 * N)
    for i in range(N):
        for j in range(N):
            full[i + j] += int(a[i]) * int(b[j])
    want = [(full[i] - full[i + N]) % q for i in range(N)]
    assert [int(v) for v in ring.negacyclic_mul(a, b, q)] == want
    assert np.array_equal(ring.intt(ring.mulmod(ring.ntt(a, q), ring.ntt(b, q), q), q),
                          ring.negacyclic_mul(a, b, q))


# --------------------------------------------------------------------------
# rescaling: Eq. 6, Eq. 7, Algorithm 1 / Eq. 17
# --------------------------------------------------------------------------
def _ctx(log_n=4, L=6, K=2, dnum=3):
    return ckks.Ctx(synth.make_params(log_n, [50] * L, K, dnum))


def test_rs_is_floor_division():
    """Eq. 6 with the top residue taken in [0, q_top) divides the CRT value
    exactly: CRT(rs(x)) = floor(CRT(x) / q_top)."""
    ctx = _ctx()
    g = synth.rng(96)
    for level in (2, 4, 6):
        a = synth.uniform_residues(g, ctx.q[:level], ctx.N)
        X = [x % ckks.prod(ctx.q[:level]) for x in ckks.crt_centered(a, ctx.q[:level])]
        r = ckks.rs(ctx, a)
        Y = [y % ckks.prod(ctx.q[:level - 1]) for y in ckks.crt_centered(r, ctx.q[:level - 1])]
        assert Y == [x // ctx.q[level - 1] for x in X]


def test_multi_rs_alg1_equals_sequential_and_floor():
    """Algorithm 1 equals mu sequential rescales (proved by induction in
    Section V-B) for every mu in [1, L-1], and both equal
    floor(X / (q_{L-1} ... q_{L-mu}))."""
    ctx = _ctx(L=6)
    g = synth.rng(95)
    L = 6
    A = synth.uniform_residues(g, ctx.q, ctx.N)
    a = ckks.intt_poly(A, ctx.q)
    X = [x % ckks.prod(ctx.q) for x in ckks.crt_centered(a, ctx.q)]
    for mu in range(1, L):
        seq = ckks.multi_rs_sequential(ctx, A, mu)
        assert np.array_equal(ckks.multi_rs_alg1(ctx, A, mu), seq)
        div = ckks.prod(ctx.q[L - mu:])
        got = ckks.intt_poly(seq, ctx.q[:L - mu])
        Y = [y % ckks.prod(ctx.q[:L - mu]) for y in ckks.crt_centered(got, ctx.q[:L - mu])]
        assert Y == [x // div for x in X]


def test_g_constants_eq16():
    ctx = _ctx(L=6)
    L = 6
    for mu in range(1, L):
        for t in range(L - mu, L):
            for eta in range(L - mu):
                g = ckks.g_const(ctx, L, mu, t, eta)
                want = pow(ckks.prod(ctx.q[L - mu:t + 1]), -1, ctx.q[eta])
                assert g == want


def test_RS_eq7_equals_coefficient_rs():
    ctx = _ctx()
    g = synth.rng(94)
    A = synth.uniform_residues(g, ctx.q, ctx.N)
    want = ckks.ntt_poly(ckks.rs(ctx, ckks.intt_poly(A, ctx.q)), ctx.q[:-1])
    assert np.array_equal(ckks.RS(ctx, A), want)


# --------------------------------------------------------------------------
# basis conversion (Eq. 4) and ModDown (Eq. 5)
# --------------------------------------------------------------------------
def test_bconv_matches_bigint_and_overflow_bound():
    ctx = _ctx(L=6, K=3)
    g = synth.rng(93)
    src = ctx.q[:3]
    dst = ctx.q[3:] + ctx.p
    y = synth.uniform_residues(g, src, ctx.N)
    conv = ckks.bconv(y, src, dst)
    S = ckks.bconv_bigint(y, src)
    Qs = ckks.prod(src)
    X = [x % Qs for x in ckks.crt_centered(y, src)]
    for c in range(ctx.N):
        for i, x in enumerate(dst):
            assert int(conv[i, c]) == S[c] % x
        u, r = divmod(S[c] - X[c], Qs)
        assert r == 0 and 0 <= u < len(src)


def test_moddown_is_floor_division_up_to_K():
    """Eq. 5 returns floor(X / P) - u with 0 <= u < K (the BConv overflow)."""
    ctx = _ctx(L=4, K=3)
    g = synth.rng(92)
    level = 4
    primes = ctx.q[:level] + ctx.p
    c = synth.uniform_residues(g, primes, ctx.N)
    PQ = ckks.prod(primes)
    X = [x % PQ for x in ckks.crt_centered(c, primes)]
    out = ckks.moddown_coef(ctx, c, level)
    Q = ckks.prod(ctx.q[:level])
    Y = [y % Q for y in ckks.crt_centered(out, ctx.q[:level])]
    for x, y in zip(X, Y):
        assert ((x // ctx.P) - y) % Q < ctx.K


# --------------------------------------------------------------------------
# keys (Eq. 2, 9, 14) and relinearisation (Eq. 15)
# --------------------------------------------------------------------------
def test_gadget_residues():
    ctx = _ctx(L=6, dnum=3)
    for beta in range(3):
        G = ctx.gadget(beta)
        for j, qj in enumerate(ctx.q):
            assert G % qj == (1 if j // ctx.alpha == beta else 0)


def test_keygen_decrypts_to_P_G_s_t():
    """ek_0 + ek_1 s = e + P G_beta s^t on Q limbs, = e on P limbs
    (schoolbook products in the coefficient domain)."""
    ctx = _ctx(log_n=4, L=4, K=2, dnum=2)
    params = synth.make_params(4, [50] * 4, 2, 2)
    km = synth.key_material(params, 3, 7)
    primes = ctx.q + ctx.p
    for t in (2, 3):
        for beta in range(2):
            ek0, ek1 = ckks.keygen(ctx, km.s, km.a[t - 2][beta], km.e[t - 2][beta], t, beta)
            c0 = ckks.intt_poly(ek0, primes)
            c1 = ckks.intt_poly(ek1, primes)
            G = ctx.gadget(beta)
            for x, m in enumerate(primes):
                s = ring.from_signed(km.s, m)
                lhs = ring.addmod(c0[x], ring.negacyclic_mul(c1[x], s, m), m)
                rhs = ring.from_signed(km.e[t - 2][beta], m)
                if x < ctx.L:
                    st = s.copy()
                    for _ in range(t - 1):
                        st = ring.negacyclic_mul(st, s, m)
                    rhs = ring.addmod(rhs, ring.smul(st, ctx.P * G % m, m), m)
                assert np.array_equal(lhs, rhs)


def _signed_poly_mul(a, b, N):
    full = [0] * (2 * N)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                full[i + j] += x * y
    return [full[i] - full[i + N] for i in range(N)]


def test_relin_decrypts_to_sum_d_t_s_t():
    """Dec(relin(d)) - sum_t d_t s^t is small: the key-switch noise only
    (big integers, coefficient domain)."""
    params = synth.make_params(5, [50] * 4, 1, 4)  # alpha = 1
    ctx = ckks.Ctx(params)
    km = synth.key_material(params, 4, 8)
    keys = ckks.keygen_all(ctx, km, 4)
    g = synth.rng(91)
    level, n = 4, 4
    d = np.stack([synth.uniform_residues(g, ctx.q[:level], ctx.N) for _ in range(n + 1)])
    c = ckks.relin_coef(ctx, d, keys, level)
    got = ckks.crt_centered(ring.addmod_rows(
        c[0], np.stack([ring.negacyclic_mul(c[1][j], ring.from_signed(km.s, qj), qj)
                        for j, qj in enumerate(ctx.q[:level])]), ctx.q[:level]), ctx.q[:level])
    # sum_t d_t s^t with big ints
    Q = ckks.prod(ctx.q[:level])
    dc = [ckks.crt_centered(ckks.intt_poly(d[t], ctx.q[:level]), ctx.q[:level]) for t in range(n + 1)]
    s = [int(x) for x in km.s]
    want = list(dc[0])
    st = [1] + [0] * (ctx.N - 1)
    for t in range(1, n + 1):
        st = _signed_poly_mul(st, s, ctx.N)
        prod_t = _signed_poly_mul(dc[t], st, ctx.N)
        want = [w + p for w, p in zip(want, prod_t)]
    diff = [((a - b + Q // 2) % Q) - Q // 2 for a, b in zip(got, want)]
    qmax = max(ctx.q)
    bound = (n - 1) * ctx.dnum * ctx.N * qmax * synth.ERR_CLIP // ctx.P + (ctx.N + 1) * (ctx.K + 1)
    assert max(abs(x) for x in diff) <= bound


# --------------------------------------------------------------------------
# products: decode gate, special cases, relocation
# --------------------------------------------------------------------------
def _encrypted_inputs(params, k, config, Delta):
    ctx = ckks.Ctx(params)
    km = synth.key_material(params, k, config)
    keys = ckks.keygen_all(ctx, km, k)
    pa, pe = synth.public_key_draw(params, config)
    pk = ckks.public_key(ctx, km.s, pa, pe)
    cts, zs = [], []
    for i in range(k):
        d = synth.encryption_draw(params, config, i)
        m = ckks.encode(params.N, d.z, Delta)
        cts.append(ckks.Tup(ckks.encrypt(ctx, m, pk, d.v, d.e0, d.e1), Delta))
        zs.append(d.z)
    return ctx, km, keys, cts, zs


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_product_decodes_to_fp64_product(k):
    """k-input product decrypts and decodes to the FP64 product of the slot
    vectors within 2^-20 (scale ~ prime size, alpha = 1 digits)."""
    params = synth.make_params(9, [50] * 6, 1, 6)
    ctx, km, keys, cts, zs = _encrypted_inputs(params, k, 11, 2.0 ** 50)
    out = ckks.mul_k(ctx, cts, keys)
    assert out.level == 6 - math.ceil(math.log2(k))
    z = ckks.decode(params.N, ckks.decrypt(ctx, out.data, km.s), out.scale)
    ref = np.prod(np.stack(zs), axis=0)
    assert np.abs(z - ref).max() <= 2.0 ** -20
    ch = ckks.mul_chain(ctx, cts, keys)
    zc = ckks.decode(params.N, ckks.decrypt(ctx, ch.data, km.s), ch.scale)
    assert np.abs(zc - ref).max() <= 2.0 ** -20


def test_k2_equals_standard_two_input_multiply():
    """With partition (1,1) the relocated 2-input path equals the printed one
    (Eq. 1-7) bit for bit."""
    params = synth.make_params(5, [50] * 4, 2, 2)
    ctx = ckks.Ctx(params)
    km = synth.key_material(params, 2, 12)
    keys = ckks.keygen_all(ctx, km, 2)
    a = ckks.Tup(synth.uniform_tuple(params, 2, 4, 12, 0), 1.0)
    b = ckks.Tup(synth.uniform_tuple(params, 2, 4, 12, 1), 1.0)
    x = ckks.mul_k(ctx, [a, b], keys, "(1,1)")
    y = ckks.mul2_standard(ctx, a, b, keys)
    assert np.array_equal(x.data, y.data)


def test_relocated_3input_equals_prior_arrangement():
    """Section IV: the improved 3-input multiply (coefficient-domain rs and
    RS*) equals the prior one (ModDown back to the NTT domain, then Eq. 7
    twice) bit for bit."""
    params = synth.make_params(5, [50] * 5, 2, 2)
    ctx = ckks.Ctx(params)
    km = synth.key_material(params, 3, 13)
    keys = ckks.keygen_all(ctx, km, 3)
    cts = [ckks.Tup(synth.uniform_tuple(params, 2, 5, 13, i), 1.0) for i in range(3)]
    x = ckks.mul_k(ctx, cts, keys, "(1,1,1)")
    D = ckks.tensor_product(ctx, [c.data for c in cts])
    C = ckks.relin_ntt(ctx, D, keys, 5)
    prior = np.stack([ckks.RS(ctx, ckks.RS(ctx, C[l])) for l in range(2)])
    assert np.array_equal(x.data, prior)


def test_separate_moddowns_differ_by_wrap_count():
    """One ModDown per ek_t (the form before Eq. 15) against one ModDown of
    the sum: ModDown is linear except that each [.]_{p_i} of Eq. 5 wraps
    once per extra addend at most, and every wrap adds p_i (P / p_i) = P
    before the division by P. So separate - combined = -W in every limb,
    the same integer W in [0, K (n - 2)] for each coefficient."""
    params = synth.make_params(5, [50] * 5, 3, 2)  # K = 3
    ctx = ckks.Ctx(params)
    n = 5
    km = synth.key_material(params, n, 17)
    keys = ckks.keygen_all(ctx, km, n)
    g = synth.rng(97)
    level = 5
    d = np.stack([synth.uniform_residues(g, ctx.q[:level], ctx.N) for _ in range(n + 1)])
    comb = ckks.relin_coef(ctx, d, keys, level)
    sep = ckks.relin_coef(ctx, d, keys, level, separate=True)
    assert not np.array_equal(comb, sep)  # wraps do happen at these sizes
    for l in range(2):
        W = None
        for j, qj in enumerate(ctx.q[:level]):
            w = (comb[l][j].astype(object) - sep[l][j].astype(object)) % qj
            W = w if W is None else W
            assert np.array_equal(w, W)
        assert max(W) <= ctx.K * (n - 2)
    # and the NTT-domain arrangement is the same function
    sep_ntt = ckks.relin_ntt(ctx, d, keys, level, separate=True)
    assert np.array_equal(sep_ntt, np.stack([ckks.ntt_poly(sep[l], ctx.q[:level]) for l in range(2)]))


def test_inner_node_rescale_forms_agree():
    params = synth.make_params(4, [50] * 6, 2, 3)
    ctx = ckks.Ctx(params)
    km = synth.key_material(params, 7, 14)
    keys = ckks.keygen_all(ctx, km, 7)
    cts = [ckks.Tup(synth.uniform_tuple(params, 2, 6, 14, i), 1.0) for i in range(7)]
    a = ckks.mul_k(ctx, cts, keys, "(4,3)|(2,2)", rescale="sequential")
    b = ckks.mul_k(ctx, cts, keys, "(4,3)|(2,2)", rescale="alg1")
    assert np.array_equal(a.data, b.data)


def test_tensor_product_matches_schoolbook_definition():
    """Eq. 13 in the NTT domain equals the coefficient-domain sum of
    schoolbook products over all index choices."""
    ctx = _ctx(log_n=3, L=2)
    g = synth.rng(90)
    cts = [synth.uniform_residues(g, ctx.q[:2], ctx.N).reshape(1, 2, ctx.N) for _ in range(6)]
    cts = [np.concatenate([cts[2 * i], cts[2 * i + 1]]) for i in range(3)]
    D = ckks.tensor_product(ctx, cts)
    for j, qj in enumerate(ctx.q[:2]):
        coef = [[ring.intt(c[l][j], qj) for l in range(2)] for c in cts]
        for t in range(4):
            acc = np.zeros(ctx.N, dtype=np.uint64)
            for l1 in range(2):
                for l2 in range(2):
                    for l3 in range(2):
                        if l1 + l2 + l3 == t:
                            p = ring.negacyclic_mul(ring.negacyclic_mul(coef[0][l1], coef[1][l2], qj),
                                                    coef[2][l3], qj)
                            acc = ring.addmod(acc, p, qj)
            assert np.array_equal(ring.intt(D[t][j], qj), acc)


def test_encode_decode_roundtrip_and_slot_product():
    N = 64
    g = synth.rng(89)
    z1, z2 = synth.unit_disk_slots(g, N // 2), synth.unit_disk_slots(g, N // 2)
    D = 2.0 ** 30
    m1, m2 = ckks.encode(N, z1, D), ckks.encode(N, z2, D)
    assert np.abs(ckks.decode(N, m1, D) - z1).max() < 1e-7
    prodm = _signed_poly_mul(m1, m2, N)
    assert np.abs(ckks.decode(N, prodm, D * D) - z1 * z2).max() < 1e-6


# --------------------------------------------------------------------------
# partitions (Section V-C, Table II)
# --------------------------------------------------------------------------
def _golden_table_ii():
    """Rows of tests/golden/table2_partitions.txt: k -> (baseline RS units,
    proposed RS units, proposed partition or None)."""
    import os
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_partitions.txt")
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        k, base, prop, part = int(line[0]), int(line[1]), int(line[2]), line[3]
        rows[k] = (base, prop, None if part == "-" else part)
    return rows


TABLE_II_ROWS = _golden_table_ii()


@pytest.mark.parametrize("k", sorted(k for k in TABLE_II_ROWS if k <= 12))
def test_table_ii_rescale_units(k):
    base, prop, part = TABLE_II_ROWS[k]
    assert plan.TABLE_II[k] == part
    root = plan.parse(part, k)
    assert plan.valid(root, k)
    assert plan.rs_units(root) == prop
    assert plan.rs_units(plan.binary_partition(k)) == base
    assert plan.min_rs_units(k) == prop


def test_17_input_example():
    base, prop, _ = TABLE_II_ROWS[17]
    b = plan.binary_partition(17)
    assert plan.rs_units(b) == base == 79
    assert plan.rs_units(b.children[0]) - 17 == 62 or plan.rs_units(plan.binary_partition(16)) == 62
    assert plan.min_rs_units(17) == prop == 41


def test_6_input_depth_rule():
    assert plan.valid(plan.parse("(2,2,2)", 6), 6)
    assert not plan.valid(plan.parse("(5,1)|(3,2)", 6), 6)


# --------------------------------------------------------------------------
# Galois automorphisms and rotation
# --------------------------------------------------------------------------
def test_automorphism_closed_forms_and_homomorphism():
    """sigma_g(X) = X^g (with X^N = -1), sigma_1 = id, sigma_g sigma_h =
    sigma_{gh mod 2N}, and sigma_g(a b) = sigma_g(a) sigma_g(b)."""
    N, q = 32, synth.prime_chain(50, 1)[0]
    g0 = synth.rng(301)
    x = np.zeros(N, dtype=np.uint64)
    x[1] = 1
    for g in (3, 5, 2 * N - 1, 41):
        y = ckks.automorphism_coef(x, g, q)
        want = np.zeros(N, dtype=np.uint64)
        if g < N:
            want[g] = 1
        else:
            want[g - N] = q - 1
        assert np.array_equal(y, want)
    a = synth.uniform_residues(g0, [q], N)[0]
    b = synth.uniform_residues(g0, [q], N)[0]
    assert np.array_equal(ckks.automorphism_coef(a, 1, q), a)
    for g, h in ((5, 25), (3, 2 * N - 1), (7, 9)):
        lhs = ckks.automorphism_coef(ckks.automorphism_coef(a, h, q), g, q)
        assert np.array_equal(lhs, ckks.automorphism_coef(a, g * h % (2 * N), q))
        ab = ring.negacyclic_mul(a, b, q)
        assert np.array_equal(ckks.automorphism_coef(ab, g, q),
                              ring.negacyclic_mul(ckks.automorphism_coef(a, g, q), ckks.automorphism_coef(b, g, q), q))
    # the signed form agrees with the residue form
    s = synth.ternary_secret(g0, N)
    assert np.array_equal(ring.from_signed(ckks.automorphism_signed(s, 5), q),
                          ckks.automorphism_coef(ring.from_signed(s, q), 5, q))
    # in the NTT domain sigma_g permutes the limb, the same way for every prime
    primes = synth.prime_chain(50, 2)
    A = synth.uniform_residues(g0, primes, N)
    B = ckks.automorphism_ntt(A, 5, primes)
    perms = []
    for j in range(2):
        pos = {int(v): i for i, v in enumerate(A[j])}
        perms.append([pos[int(v)] for v in B[j]])
    assert perms[0] == perms[1] and sorted(perms[0]) == list(range(N))


@pytest.mark.parametrize("r", [1, 3, -2, "conj"])
def test_rotation_decodes_to_rotated_slots(r):
    """Decrypt(rotate(Enc(z))) decodes to z rotated by r (g = 5^r) or to
    conj(z) (g = 2N - 1), within 2^-20 (alpha = 1 digits, scale 2^50)."""
    params = synth.make_params(8, [50] * 4, 1, 4)
    ctx, km, keys, cts, zs = _encrypted_inputs(params, 2, 31, 2.0 ** 50)
    N = params.N
    g = 2 * N - 1 if r == "conj" else ckks.galois_element(r, N)
    a, e = synth.galois_key_draw(params, 31, g)
    gk = ckks.galois_keygen(ctx, km.s, a, e, g)
    out = ckks.rotate(ctx, cts[0], g, gk)
    assert out.level == cts[0].level
    z = ckks.decode(N, ckks.decrypt(ctx, out.data, km.s), out.scale)
    want = np.conj(zs[0]) if r == "conj" else np.roll(zs[0], -r)
    assert np.abs(z - want).max() <= 2.0 ** -20
    # the key of another element does not decrypt
    g_bad = ckks.galois_element(r + 1 if r != "conj" else 1, N)
    bad = ckks.rotate(ctx, cts[0], g, ckks.galois_keygen(ctx, km.s, a, e, g_bad))
    zb = ckks.decode(N, ckks.decrypt(ctx, bad.data, km.s), bad.scale)
    assert np.abs(zb - want).max() > 1.0


def test_embedding_closed_forms():
    """Canonical embedding: m = scale (constant 1) has every slot 1; m =
    scale X has slot j = zeta_j; encoding inverts both; the per-slot and
    per-coefficient forms agree with the vector forms."""
    N, scale = 64, 2.0 ** 20
    one = [int(scale)] + [0] * (N - 1)
    x = [0, int(scale)] + [0] * (N - 2)
    zeta = np.exp(1j * np.pi * np.array([pow(5, j, 2 * N) for j in range(N // 2)]) / N)
    assert np.allclose(ckks.decode(N, one, scale), 1.0, atol=1e-12)
    assert np.allclose(ckks.decode(N, x, scale), zeta, atol=1e-12)
    assert ckks.encode(N, np.ones(N // 2, dtype=complex), scale) == one
    assert ckks.encode(N, zeta, scale) == x
    for j in (0, 5, N // 2 - 1):
        assert abs(ckks.decode_slot(N, x, scale, j) - zeta[j]) < 1e-12
    z = synth.unit_disk_slots(synth.rng(302), N // 2)
    m = ckks.encode(N, z, scale)
    for i in (0, 1, 17, N - 1):
        assert abs(ckks.encode_coef(N, z, scale, i) - m[i]) <= 0.5 + 1e-6
    dz = ckks.decode(N, m, scale)
    for j in (0, 3, N // 2 - 1):
        assert abs(ckks.decode_slot(N, m, scale, j) - dz[j]) < 1e-9
