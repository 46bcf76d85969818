"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
residue for residue, on the same seeded inputs. Integer work, so the bar is
bit-exact equality everywhere."""
import math

import numpy as np
import pytest

import synth
from oracle import ckks as O
from oracle import ring

from gpu_common import Setup, dev, host, oracle_tuple

pytestmark = pytest.mark.gpu


def _setup(log_n, L, K, dnum, t_max, config, **kw):
    return Setup(synth.make_params(log_n, [50] * L, K, dnum), t_max, config, **kw)


# ---------------------------------------------------------------------------
# transforms (Section II evaluation map)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log_n", [4, 5, 8, 9, 10, 12, 14, 16])
def test_ntt_intt_parity(log_n):
    import paper_2601_15401_gb300 as G
    params = synth.make_params(log_n, [50, 45, 60], 1, 1)
    ctx = G.Context.from_params(params)
    g = synth.rng(200, log_n)
    primes = list(params.q)
    a = np.stack([synth.uniform_residues(g, primes, params.N) for _ in range(2)])
    t = G.Tuple.wrap(dev(a), ntt_form=0)
    ctx.ntt(t)
    got = host(t.data)
    for p in range(2):
        assert np.array_equal(got[p], ring.ntt_rows(a[p], primes))
    A = np.stack([synth.uniform_residues(g, primes, params.N) for _ in range(2)])
    u = G.Tuple.wrap(dev(A))
    ctx.intt(u)
    got = host(u.data)
    for p in range(2):
        assert np.array_equal(got[p], ring.intt_rows(A[p], primes))
    # round trip on a strided view (level below the stride)
    w = G.Tuple(dev(a), 2, 2, 3, 0)
    ctx.ntt(w)
    ctx.intt(w)
    back = host(w.data)
    assert np.array_equal(back[:, :2], a[:, :2]) and np.array_equal(back[:, 2], a[:, 2])


# ---------------------------------------------------------------------------
# steps
# ---------------------------------------------------------------------------
def test_tensor_parity():
    import paper_2601_15401_gb300 as G
    params = synth.make_params(6, [50] * 4, 1, 2)
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    g = synth.rng(201)
    shapes = [2, 3, 2, 4]
    tups = [np.stack([synth.uniform_residues(g, params.q, params.N) for _ in range(s)]) for s in shapes]
    out = G.Tuple.wrap(dev(np.zeros((sum(shapes) - 3, 4, params.N), dtype=np.uint64)))
    ins = [G.Tuple.wrap(dev(t)) for t in tups]
    ins[1].level = 3  # a higher child drops its top limb (level alignment)
    ctx.tensor(ins, out)
    assert out.level == 3 and out.n_polys == sum(shapes) - 3
    want = O.tensor_product(octx, [t[:, :3] for t in tups])
    assert np.array_equal(host(out.data)[:, :3], want)


@pytest.mark.parametrize("mu", [1, 2, 3, 5])
def test_rescale_multi_parity(mu):
    import paper_2601_15401_gb300 as G
    params = synth.make_params(7, [50] * 6, 2, 3)
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    g = synth.rng(202, mu)
    A = np.stack([synth.uniform_residues(g, params.q, params.N) for _ in range(3)])
    t = G.Tuple.wrap(dev(A))
    out = G.Tuple.wrap(dev(np.zeros((3, 6 - mu, params.N), dtype=np.uint64)))
    ws = dev(np.zeros(ctx.rescale_workspace_size(3, 6, mu) // 8 + 1, dtype=np.uint64))
    ctx.rescale_multi(t, mu, out, ws)
    assert out.level == 6 - mu
    got = host(out.data)
    for p in range(3):
        assert np.array_equal(got[p], O.multi_rs_sequential(octx, A[p], mu))
    # in place
    ctx.rescale_multi(t, mu, t, ws)
    assert np.array_equal(host(t.data)[:, :6 - mu], got)


@pytest.mark.parametrize("n,level", [(2, 5), (3, 4), (5, 5)])
def test_relin_parity(n, level):
    import paper_2601_15401_gb300 as G
    S = _setup(6, 5, 2, 2, 5, 203)
    g = synth.rng(203, n)
    d = np.stack([synth.uniform_residues(g, S.params.q[:level], S.params.N) for _ in range(n + 1)])
    dt = G.Tuple.wrap(dev(d))
    ws = S.ws(S.ctx.relin_workspace_size(n, level))
    out = G.Tuple.wrap(dev(np.zeros((2, level, S.params.N), dtype=np.uint64)))
    S.ctx.relin(dt, S.evk, out, ws, out_ntt=False)
    assert np.array_equal(host(out.data), O.relin_coef(S.octx, d, S.okeys, level))
    S.ctx.relin(dt, S.evk, out, ws, out_ntt=True)
    assert np.array_equal(host(out.data), O.relin_ntt(S.octx, d, S.okeys, level))


def test_keygen_parity():
    S = _setup(6, 4, 2, 2, 4, 204, gpu_keygen=True)
    assert np.array_equal(host(S.gpu_plain_keys), S.plain_keys)


# ---------------------------------------------------------------------------
# the k-input multiply
# ---------------------------------------------------------------------------
def _inputs(S, k, level, config, index0=0):
    return [synth.uniform_tuple(S.params, 2, level, config, index0 + i) for i in range(k)]


def _run_mul_k(S, cts, level, partition=None):
    import paper_2601_15401_gb300 as G
    k = len(cts)
    depth = S.ctx.plan_describe(k, partition)["depth"]
    out = G.Tuple.wrap(dev(np.zeros((2, level - depth, S.params.N), dtype=np.uint64)))
    ws = S.ws(S.ctx.workspace_size(k, level, 1, partition))
    S.ctx.mul_k([G.Tuple.wrap(dev(c), scale=2.0 ** 30) for c in cts], S.evk, out, ws, partition=partition)
    return out


@pytest.fixture(scope="module")
def S12():
    # depth <= 4 for k <= 12; L = 7 leaves room for a lower input level
    return _setup(5, 7, 2, 3, 12, 205)


@pytest.mark.parametrize("k", range(2, 13))
def test_mul_k_parity_table_ii(S12, k):
    level = 7 if k > 8 else 6
    cts = _inputs(S12, k, level, 205, 10 * k)
    out = _run_mul_k(S12, cts, level)
    want = O.mul_k(S12.octx, [oracle_tuple(c, 2.0 ** 30) for c in cts], S12.okeys)
    assert out.level == want.level == level - math.ceil(math.log2(k))
    assert np.array_equal(host(out.data)[:, :out.level], want.data)
    assert out.scale == pytest.approx(want.scale, rel=1e-12)


@pytest.mark.parametrize("k,part", [(6, "(2,2,2)"), (5, "(3,2)"), (7, "(3,3,1)"), (4, "(2,2)"),
                                    (8, "(2,2,2,2)|(1,1),(1,1),(1,1),(1,1)"), (3, "(2,1)")])
def test_mul_k_other_partitions(S12, k, part):
    level = 6
    cts = _inputs(S12, k, level, 206, 10 * k)
    try:
        out = _run_mul_k(S12, cts, level, part)
    except Exception as e:  # partitions the depth rule rejects must be rejected by both sides
        with pytest.raises(ValueError):
            O.mul_k(S12.octx, [oracle_tuple(c) for c in cts], S12.okeys, part)
        assert "EINVAL" in str(e)
        return
    want = O.mul_k(S12.octx, [oracle_tuple(c) for c in cts], S12.okeys, part)
    assert np.array_equal(host(out.data)[:, :out.level], want.data)


def test_mul_k_minimum_level_and_ragged_digits(S12):
    # level 3 with alpha = 3: one full digit; k = 4 has depth 2 -> output level 1
    cts = _inputs(S12, 4, 3, 207)
    out = _run_mul_k(S12, cts, 3)
    want = O.mul_k(S12.octx, [oracle_tuple(c) for c in cts], S12.okeys)
    assert out.level == 1 and np.array_equal(host(out.data)[:, :1], want.data)
    # level 5: digits {0,1,2},{3,4} (ragged last digit)
    cts = _inputs(S12, 5, 5, 208)
    out = _run_mul_k(S12, cts, 5)
    want = O.mul_k(S12.octx, [oracle_tuple(c) for c in cts], S12.okeys)
    assert np.array_equal(host(out.data)[:, :out.level], want.data)


def test_mul2_parity_and_k2_equivalence(S12):
    import paper_2601_15401_gb300 as G
    cts = _inputs(S12, 2, 6, 209)
    a, b = [G.Tuple.wrap(dev(c)) for c in cts]
    out = G.Tuple.wrap(dev(np.zeros((2, 5, S12.params.N), dtype=np.uint64)))
    ws = S12.ws(S12.ctx.mul2_workspace_size(6))
    S12.ctx.mul2(a, b, S12.evk, out, ws)
    want = O.mul2_standard(S12.octx, oracle_tuple(cts[0]), oracle_tuple(cts[1]), S12.okeys)
    assert np.array_equal(host(out.data), want.data)
    k2 = _run_mul_k(S12, cts, 6, "(1,1)")
    assert np.array_equal(host(k2.data), host(out.data))


def test_batch_equals_alone(S12):
    import paper_2601_15401_gb300 as G
    T = __import__("torch")
    B, k, level = 4, 5, 6
    cts = [_inputs(S12, k, level, 210, 100 * b) for b in range(B)]
    big = dev(np.stack([np.stack(row) for row in cts]))  # [B][k][2][level][N]
    outs_t = T.zeros((B, 2, level - 3, S12.params.N), dtype=T.uint64, device="cuda")
    tup = [[G.Tuple(big[b, u], 2, level, level) for u in range(k)] for b in range(B)]
    outs = [G.Tuple(outs_t[b], 2, level - 3, level - 3) for b in range(B)]
    ws = S12.ws(S12.ctx.workspace_size(k, level, B))
    S12.ctx.mul_k_batch(tup, S12.evk, outs, ws)
    for b in range(B):
        alone = _run_mul_k(S12, cts[b], level)
        assert np.array_equal(host(outs_t[b]), host(alone.data))
    want = O.mul_k(S12.octx, [oracle_tuple(c) for c in cts[2]], S12.okeys)
    assert np.array_equal(host(outs_t[2]), want.data)


# ---------------------------------------------------------------------------
# Table V / Table IV operation counts
# ---------------------------------------------------------------------------
def test_op_counts_table_v():
    import paper_2601_15401_gb300 as G
    L = 6
    S = Setup(synth.make_params(5, [50] * L, L, 1), 3, 211)  # dnum = 1, K = L
    K = L
    cts = _inputs(S, 3, L, 211)
    S.ctx.counters(reset=True)
    _run_mul_k(S, cts, L, "(1,1,1)")
    c = S.ctx.counters(reset=True)
    assert c["limb_ntt"] == 2 * L + 2 * K - 4
    assert c["limb_intt"] == 4 * L + 2 * K
    # Table IV: one mu-rescale of a polynomial = mu INTT + (L - mu) NTT
    t = G.Tuple.wrap(dev(np.stack([synth.uniform_residues(synth.rng(1), S.params.q, S.params.N)])))
    for mu in (1, 2, 4):
        ws = S.ws(S.ctx.rescale_workspace_size(1, L, mu))
        S.ctx.rescale_multi(t, mu, G.Tuple.wrap(dev(np.zeros((1, L - mu, S.params.N), dtype=np.uint64))), ws)
        c = S.ctx.counters(reset=True)
        assert (c["limb_intt"], c["limb_ntt"]) == (mu, L - mu)


# ---------------------------------------------------------------------------
# error handling at the boundary
# ---------------------------------------------------------------------------
def test_error_codes(S12):
    import paper_2601_15401_gb300 as G
    cts = _inputs(S12, 4, 6, 212)
    tups = [G.Tuple.wrap(dev(c)) for c in cts]
    out = G.Tuple.wrap(dev(np.zeros((2, 4, S12.params.N), dtype=np.uint64)))
    need = S12.ctx.workspace_size(4, 6, 1)
    with pytest.raises(G.CkksError) as e:
        S12.ctx.mul_k(tups, S12.evk, out, S12.ws(need - 4096))
    assert e.value.code == -4
    with pytest.raises(G.CkksError) as e:
        S12.ctx.workspace_size(4, 2, 1)
    assert e.value.code == -2
    small_keys = dev(S12.plain_keys[:1])
    evk2 = S12.ctx.evk_set(2, small_keys)
    with pytest.raises(G.CkksError) as e:
        S12.ctx.mul_k(tups, evk2, out, S12.ws(need))
    assert e.value.code == -3
    tups[1].ntt_form = 0
    with pytest.raises(G.CkksError) as e:
        S12.ctx.mul_k(tups, S12.evk, out, S12.ws(need))
    assert e.value.code == -1
    S12.ctx.check()


# ---------------------------------------------------------------------------
# forms of the rescaling (same residues; Section IV and V-B)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("key,value", [("inner_rescale", 1), ("inner_rescale", 2), ("root_rescale", 1)])
@pytest.mark.parametrize("k", [3, 7, 9])
def test_rescale_forms_give_identical_products(S12, key, value, k):
    level = 7 if k > 8 else 6
    cts = _inputs(S12, k, level, 213, 10 * k)
    base = host(_run_mul_k(S12, cts, level).data)
    S12.ctx.tune_set(key, value)
    try:
        other = host(_run_mul_k(S12, cts, level).data)
    finally:
        S12.ctx.tune_set(key, 0)
    assert np.array_equal(other, base)


@pytest.mark.parametrize("root_rescale", [0, 1])
@pytest.mark.parametrize("k", [3, 5, 9])
def test_separate_moddowns_match_oracle(S12, k, root_rescale):
    """One ModDown per ek_t (the form Eq. 15 replaces), in both root
    arrangements, against the oracle's separate form."""
    level = 7 if k > 8 else 6
    cts = _inputs(S12, k, level, 216, 10 * k)
    S12.ctx.tune_set("moddown", 1)
    S12.ctx.tune_set("root_rescale", root_rescale)
    try:
        out = _run_mul_k(S12, cts, level)
    finally:
        S12.ctx.tune_set("moddown", 0)
        S12.ctx.tune_set("root_rescale", 0)
    want = O.mul_k(S12.octx, [oracle_tuple(c) for c in cts], S12.okeys, separate_moddown=True)
    assert np.array_equal(host(out.data)[:, :out.level], want.data)


def test_separate_moddowns_relin_parity_and_counts(S12):
    """ckks_relin in the separate form: residues and the (n - 2) extra
    ModDowns (K + level limb INTTs per polynomial each)."""
    import paper_2601_15401_gb300 as G
    n, level = 5, 6
    g = synth.rng(217)
    d = np.stack([synth.uniform_residues(g, S12.params.q[:level], S12.params.N) for _ in range(n + 1)])
    ws = S12.ws(S12.ctx.relin_workspace_size(n, level))
    counts = {}
    for mode in (0, 1):
        S12.ctx.tune_set("moddown", mode)
        try:
            out = G.Tuple.wrap(dev(np.zeros((2, level, S12.params.N), dtype=np.uint64)))
            S12.ctx.counters(reset=True)
            S12.ctx.relin(G.Tuple.wrap(dev(d)), S12.evk, out, ws, out_ntt=False)
            counts[mode] = S12.ctx.counters(reset=True)
        finally:
            S12.ctx.tune_set("moddown", 0)
        want = O.relin_coef(S12.octx, d, S12.okeys, level, separate=bool(mode))
        assert np.array_equal(host(out.data), want), mode
    extra = counts[1]["limb_intt"] - counts[0]["limb_intt"]
    assert extra == (n - 2) * 2 * (S12.params.K + level)
    assert counts[1]["limb_ntt"] == counts[0]["limb_ntt"]


def test_table_iv_counts_for_each_rescale_form():
    """Table IV: mu combined rescales cost mu INTT + (L - mu) NTT per
    polynomial (Algorithm 1); the baseline costs L INTT + (L - mu) NTT."""
    import paper_2601_15401_gb300 as G
    params = synth.make_params(5, [50] * 8, 2, 2)
    ctx = G.Context.from_params(params)
    L = 8
    t = G.Tuple.wrap(dev(np.stack([synth.uniform_residues(synth.rng(2), params.q, params.N)])))
    for mode, want in [(0, lambda mu: (mu, L - mu)), (2, lambda mu: (L, L - mu)),
                       (1, lambda mu: (mu, sum(L - 1 - j for j in range(mu))))]:
        ctx.tune_set("inner_rescale", mode)
        for mu in (1, 3):
            ws = dev(np.zeros(ctx.rescale_workspace_size(1, L, mu) // 8 + 1, dtype=np.uint64))
            ctx.counters(reset=True)
            ctx.rescale_multi(t, mu, G.Tuple.wrap(dev(np.zeros((1, L - mu, params.N), dtype=np.uint64))), ws)
            c = ctx.counters(reset=True)
            assert (c["limb_intt"], c["limb_ntt"]) == want(mu), (mode, mu)
    ctx.tune_set("inner_rescale", 0)


@pytest.mark.parametrize("log_n,k", [(9, 5), (11, 7), (13, 4), (15, 3)])
def test_mul_k_parity_two_phase_geometries(log_n, k):
    """Ring degrees whose transforms split unevenly (N1 != N2) and the
    serving mix's degrees, against the oracle."""
    S = _setup(log_n, 5, 2, 2, k, 214 + log_n)
    level = 5
    cts = _inputs(S, k, level, 214, 100 * log_n)
    out = _run_mul_k(S, cts, level)
    want = O.mul_k(S.octx, [oracle_tuple(c) for c in cts], S.okeys)
    assert np.array_equal(host(out.data)[:, :out.level], want.data)


def test_mul_k_k10_search_partition_matches_oracle(S12):
    """The partition the transform-count search prefers for k = 10."""
    import paper_2601_15401_gb300 as G
    part, _ = G.plan_optimize(10, "transforms", 24, 8, 8)
    cts = _inputs(S12, 10, 7, 215)
    out = _run_mul_k(S12, cts, 7, part)
    want = O.mul_k(S12.octx, [oracle_tuple(c) for c in cts], S12.okeys, part)
    assert np.array_equal(host(out.data)[:, :out.level], want.data)
