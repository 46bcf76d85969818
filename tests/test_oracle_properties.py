"""Property tests of the oracle over random seeds and shapes (hypothesis):
the identities the paper proves or relies on, checked on inputs the fixed
pins do not cover. CPU only; skipped where hypothesis is not installed."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import synth  # noqa: E402
from oracle import ckks, ring  # noqa: E402

PRIMES = synth.prime_chain(50, 8)
P60 = synth.prime_chain(60, 3, exclude=PRIMES)
SETTINGS = settings(max_examples=25, deadline=None)


def _ctx(log_n, L, K, dnum):
    return ckks.Ctx(synth.make_params(log_n, [50] * L, K, dnum))


@SETTINGS
@given(log_n=st.integers(2, 7), j=st.integers(0, 7), seed=st.integers(0, 2 ** 32))
def test_ntt_intt_identity_and_definition(log_n, j, seed):
    """INTT(NTT(a)) = a, and the fast transform equals the O(N^2) definition."""
    N, q = 1 << log_n, PRIMES[j]
    a = synth.uniform_residues(synth.rng(seed), [q], N)[0]
    A = ring.ntt(a, q)
    assert np.array_equal(ring.intt(A, q), a)
    assert np.array_equal(A, ring.ntt_definition(a, q))


@SETTINGS
@given(log_n=st.integers(2, 6), seed=st.integers(0, 2 ** 32))
def test_convolution_theorem(log_n, seed):
    """NTT(a * b) = NTT(a) . NTT(b) for the negacyclic product."""
    N, q = 1 << log_n, PRIMES[seed % 8]
    g = synth.rng(seed)
    a, b = synth.uniform_residues(g, [q, q], N)
    lhs = ring.ntt(ring.negacyclic_mul(a, b, q), q)
    assert np.array_equal(lhs, ring.mulmod(ring.ntt(a, q), ring.ntt(b, q), q))


@SETTINGS
@given(L=st.integers(2, 7), data=st.data())
def test_alg1_equals_sequential_rescales(L, data):
    """Algorithm 1 with mu combined rescales equals mu rescales of Eq. 7
    (Section V-B), at any level and mu."""
    mu = data.draw(st.integers(1, L - 1))
    seed = data.draw(st.integers(0, 2 ** 32))
    ctx = _ctx(3, L, 2, 1)
    A = synth.uniform_residues(synth.rng(seed), ctx.q, ctx.N)
    assert np.array_equal(ckks.multi_rs_alg1(ctx, A, mu), ckks.multi_rs_sequential(ctx, A, mu))


@SETTINGS
@given(n_src=st.integers(1, 4), seed=st.integers(0, 2 ** 32))
def test_bconv_is_the_integer_sum(n_src, seed):
    """Eq. 4 computed residue-wise equals the big-integer sum S reduced
    mod every target, and S = X + u Q_src with 0 <= u < #sources."""
    src, dst = PRIMES[:n_src], PRIMES[n_src:] + P60
    y = synth.uniform_residues(synth.rng(seed), src, 8)
    conv = ckks.bconv(y, src, dst)
    S = ckks.bconv_bigint(y, src)
    Qs = ckks.prod(src)
    X = [x % Qs for x in ckks.crt_centered(y, src)]
    for c in range(8):
        assert all(int(conv[i, c]) == S[c] % x for i, x in enumerate(dst))
        u, r = divmod(S[c] - X[c], Qs)
        assert r == 0 and 0 <= u < n_src


@SETTINGS
@given(L=st.integers(1, 5), K=st.integers(1, 3), seed=st.integers(0, 2 ** 32))
def test_moddown_floor_within_K(L, K, seed):
    """Eq. 5 gives floor(X / P) - u with 0 <= u < K."""
    ctx = _ctx(3, L, K, 1)
    primes = ctx.q[:L] + ctx.p
    c = synth.uniform_residues(synth.rng(seed), primes, ctx.N)
    PQ = ckks.prod(primes)
    X = [x % PQ for x in ckks.crt_centered(c, primes)]
    out = ckks.moddown_coef(ctx, c, L)
    Q = ckks.prod(ctx.q[:L])
    Y = [y % Q for y in ckks.crt_centered(out, ctx.q[:L])]
    assert all(((x // ctx.P) - y) % Q < K for x, y in zip(X, Y))


@SETTINGS
@given(m=st.integers(2, 4), seed=st.integers(0, 2 ** 32))
def test_tensor_product_matches_polynomial_product_in_s(m, seed):
    """Eq. 13: evaluating every child tuple at a random point s and
    multiplying equals evaluating the tensor product at s (NTT domain,
    coefficient-wise in each limb)."""
    ctx = _ctx(3, 2, 1, 1)
    g = synth.rng(seed)
    kids = [np.stack([synth.uniform_residues(g, ctx.q[:2], ctx.N) for _ in range(int(g.integers(2, 4)))])
            for _ in range(m)]
    D = ckks.tensor_product(ctx, kids)
    s = synth.uniform_residues(g, ctx.q[:2], ctx.N)

    def ev(tup):
        acc = np.zeros_like(s)
        for i in range(tup.shape[0] - 1, -1, -1):   # Horner in s
            acc = ring.addmod_rows(ring.mulmod_rows(acc, s, ctx.q[:2]), tup[i], ctx.q[:2])
        return acc
    want = ev(kids[0])
    for c in kids[1:]:
        want = ring.mulmod_rows(want, ev(c), ctx.q[:2])
    assert np.array_equal(ev(D), want)
