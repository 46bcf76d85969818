"""GPU parity on the workload configurations, including the full-size launch
that bench.py times (N = 2^16, L = 24, K = 8, dnum = 3, batch 16), and the
decryption gate (decoded product vs the FP64 product of the slots)."""
import math

import numpy as np
import pytest

import synth
from oracle import ckks as O

from gpu_common import Setup, dev, host, oracle_tuple

pytestmark = pytest.mark.gpu


def _encrypted(S, k, config, Delta):
    pa, pe = synth.public_key_draw(S.params, config)
    pk = O.public_key(S.octx, S.km.s, pa, pe)
    cts, zs = [], []
    for i in range(k):
        d = synth.encryption_draw(S.params, config, i)
        m = O.encode(S.params.N, d.z, Delta)
        cts.append(O.encrypt(S.octx, m, pk, d.v, d.e0, d.e1))
        zs.append(d.z)
    return cts, zs


def _gpu_mul_k(S, cts, scale, partition=None):
    import paper_2601_15401_gb300 as G
    k = len(cts)
    level = cts[0].shape[1]
    depth = S.ctx.plan_describe(k, partition)["depth"]
    out = G.Tuple.wrap(dev(np.zeros((2, level - depth, S.params.N), dtype=np.uint64)))
    ws = S.ws(S.ctx.workspace_size(k, level, 1, partition))
    S.ctx.mul_k([G.Tuple.wrap(dev(c), scale=scale) for c in cts], S.evk, out, ws, partition=partition)
    return out


def test_3input_small_config_bit_exact():
    """N = 2^10, 4 x 50-bit q, one 60-bit p, dnum = 1, scale 2^40, k = 3
    with partition (1,1,1): encrypted inputs, relinearised and rescaled output
    equal to the oracle's residue for residue."""
    S = Setup(synth.params_small(10, dnum=1), 3, 1)
    cts, _ = _encrypted(S, 3, 1, 2.0 ** 40)
    out = _gpu_mul_k(S, cts, 2.0 ** 40, "(1,1,1)")
    want = O.mul_k(S.octx, [oracle_tuple(c, 2.0 ** 40) for c in cts], S.okeys, "(1,1,1)")
    assert out.level == 2 and np.array_equal(host(out.data), want.data)
    assert out.scale == pytest.approx(want.scale)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_decode_gate(k):
    """GPU product, decrypted and decoded by the oracle, within 2^-20 of the
    FP64 product (scale ~ prime size, one-prime digits so that a single
    60-bit P suffices); the chained 2-input product passes the same gate."""
    import paper_2601_15401_gb300 as G
    params = synth.make_params(10, [50] * 6, 1, 6)
    S = Setup(params, k, 30 + k)
    Delta = 2.0 ** 50
    cts, zs = _encrypted(S, k, 30 + k, Delta)
    out = _gpu_mul_k(S, cts, Delta)
    z = O.decode(params.N, O.decrypt(S.octx, host(out.data), S.km.s), out.scale)
    ref = np.prod(np.stack(zs), axis=0)
    err_k = np.abs(z - ref).max()
    assert err_k <= 2.0 ** -20
    # chained standard 2-input multiplies along the binary tree, on the GPU
    T = __import__("torch")

    def mul2(a, b):
        lv = min(a.level, b.level)
        o = G.Tuple.wrap(T.zeros((2, lv - 1, params.N), dtype=T.uint64, device="cuda"))
        S.ctx.mul2(a, b, S.evk, o, S.ws(S.ctx.mul2_workspace_size(lv)))
        return o

    def tree(lo, n):
        if n == 1:
            return G.Tuple.wrap(dev(cts[lo]), scale=Delta)
        a = 1 if n == 2 else 1 << (n - 1).bit_length() - 1
        return mul2(tree(lo, a), tree(lo + a, n - a))

    ch = tree(0, k)
    zc = O.decode(params.N, O.decrypt(S.octx, host(ch.data)[:, :ch.level], S.km.s), ch.scale)
    assert np.abs(zc - ref).max() <= 2.0 ** -20


def test_mid_config_batch64():
    """N = 2^14, 12 primes (q_0 60-bit, 45-bit rest), K = 4, dnum = 3:
    64 independent 3-input products in one batched call; every batch
    element equals the oracle."""
    import paper_2601_15401_gb300 as G
    T = __import__("torch")
    params = synth.params_mid()
    S = Setup(params, 3, 2)
    B, k, L, N = 64, 3, params.L, params.N
    inp = synth.uniform_residues_torch(params.q, (B, k, 2), N, 0x2000, "cuda")
    out = T.zeros((B, 2, L - 2, N), dtype=T.uint64, device="cuda")
    tup = [[G.Tuple(inp[b, u], 2, L, L) for u in range(k)] for b in range(B)]
    outs = [G.Tuple(out[b], 2, L - 2, L - 2) for b in range(B)]
    ws = S.ws(S.ctx.workspace_size(k, L, B))
    S.ctx.mul_k_batch(tup, S.evk, outs, ws)
    got = host(out)
    src = host(inp)
    for b in range(B):
        want = O.mul_k(S.octx, [oracle_tuple(src[b, u]) for u in range(k)], S.okeys)
        assert np.array_equal(got[b], want.data)


@pytest.fixture(scope="module")
def S_large():
    return Setup(synth.params_large(), 12, 3)


@pytest.mark.parametrize("k", list(range(4, 13)))
def test_full_size_bench_launch(S_large, k):
    """The launch bench.py times, for every k of its step: N = 2^16, L = 24,
    K = 8, dnum = 3, batch 16, Table II partition. The last batch element
    equals the oracle."""
    import paper_2601_15401_gb300 as G
    T = __import__("torch")
    S = S_large
    params = S.params
    B, L, N = 16, params.L, params.N
    depth = S.ctx.plan_describe(k)["depth"]
    inp = synth.uniform_residues_torch(params.q, (B, k, 2), N, 1000 + k, "cuda")
    out = T.zeros((B, 2, L - depth, N), dtype=T.uint64, device="cuda")
    tup = [[G.Tuple(inp[b, u], 2, L, L) for u in range(k)] for b in range(B)]
    outs = [G.Tuple(out[b], 2, L - depth, L - depth) for b in range(B)]
    ws = S.ws(S.ctx.workspace_size(k, L, B))
    S.ctx.mul_k_batch(tup, S.evk, outs, ws)
    S.ctx.check()
    b = B - 1
    src = host(inp[b])
    want = O.mul_k(S.octx, [oracle_tuple(src[u]) for u in range(k)], S.okeys)
    assert want.level == L - math.ceil(math.log2(k))
    assert np.array_equal(host(out[b]), want.data)
