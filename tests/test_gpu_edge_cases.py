"""Degenerate and malformed calls through the C ABI: empty batches, k
outside 2..12, mixed levels, unevenly spaced batches, levels outside the
chain, malformed tuples. Each must return its documented error code and
leave the context usable (a valid call afterwards still matches)."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import dev, host

pytestmark = pytest.mark.gpu

EINVAL, ELEVEL, ENOMEM = -1, -2, -4


@pytest.fixture(scope="module")
def env():
    import paper_2601_15401_gb300 as G
    params = synth.make_params(6, [50] * 5, 2, 2)
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    km = synth.key_material(params, 4, 301)
    okeys = O.keygen_all(octx, km, 4)
    keys = dev(np.stack([np.stack([np.stack([k[0], k[1]]) for k in row]) for row in okeys]))
    evk = ctx.evk_set(4, keys)
    return G, params, ctx, octx, okeys, evk


def _tuples(G, arr):
    return [G.Tuple.wrap(a) for a in arr]


def test_plan_rejects_k_outside_range(env):
    G, params, ctx, *_ = env
    from paper_2601_15401_gb300._lib import lib
    h = ctypes.c_void_p()
    for k in (0, 1, 13, 100):
        assert lib().ckks_plan_create(ctx._h, k, None, ctypes.byref(h)) == EINVAL
    assert lib().ckks_plan_create(ctx._h, 4, b"(2,2", ctypes.byref(h)) == EINVAL


def test_mul_k_batch_rejections_then_valid_call(env):
    G, params, ctx, octx, okeys, evk = env
    from paper_2601_15401_gb300 import _Tuple
    from paper_2601_15401_gb300._lib import lib
    N, k, level = params.N, 3, 5
    x = dev(np.stack([synth.uniform_tuple(params, 2, level, 302, i) for i in range(2 * k)]).reshape(2, k, 2, level, N))
    out = torch.zeros((2, 2, level - 2, N), dtype=torch.uint64, device="cuda")
    ws = torch.empty(ctx.workspace_size(k, level, 2) // 8 + 1, dtype=torch.uint64, device="cuda")
    plan = ctx.plan(k)

    def call(cts, outs, batch, wsbytes=ws.numel() * 8):
        arr = (_Tuple * max(1, len(cts)))(*[c.c() for c in cts])
        oarr = (_Tuple * max(1, len(outs)))(*[o.c() for o in outs])
        return lib().ckks_mul_k_batch(ctx._h, arr, k, batch, evk._h, plan, oarr, ws.data_ptr(), wsbytes, None)

    good = [G.Tuple.wrap(x[b, u]) for b in range(2) for u in range(k)]
    outs = [G.Tuple.wrap(out[b]) for b in range(2)]
    assert call(good, outs, 0) == EINVAL                                  # empty batch
    mixed = list(good)
    mixed[1] = G.Tuple.wrap(x[0, 1], level=4)                               # one input at another level
    assert call(mixed, outs, 2) == EINVAL
    assert call(good, [outs[0], G.Tuple.wrap(out[1][:, :1])], 2) == EINVAL  # output strides differ
    skew = [G.Tuple.wrap(x[b, u]) for b in (0, 1, 0) for u in range(k)]   # element 2 off the stride
    assert call(skew, outs + outs[:1], 3) == EINVAL
    assert call(good, [outs[0], outs[0]], 2) == EINVAL                   # two elements, one output
    assert call(good, outs, 2, 1024) == ENOMEM
    low = [G.Tuple.wrap(x[b, u], level=2) for b in range(2) for u in range(k)]
    assert call(low, outs, 2) == ELEVEL                                   # level <= depth
    # the context still works: a valid batch matches the oracle
    ctx.mul_k_batch([good[:k], good[k:]], evk, outs, ws)
    for b in range(2):
        want = O.mul_k(octx, [O.Tup(host(x[b, u]), 1.0) for u in range(k)], okeys)
        assert np.array_equal(host(out[b])[:, :want.level], want.data)
    ctx.check()


def test_encrypt_decrypt_rejections(env):
    G, params, ctx, *_ = env
    N, L = params.N, params.L
    z = torch.zeros((1, N), dtype=torch.int64, device="cuda")
    pk = torch.zeros((2, L, N), dtype=torch.uint64, device="cuda")
    out = [G.Tuple.wrap(torch.zeros((2, L, N), dtype=torch.uint64, device="cuda"))]
    ws = torch.empty(ctx.encrypt_batch_workspace_size(L, 1) // 8 + 1, dtype=torch.uint64, device="cuda")
    for level, code in ((0, ELEVEL), (L + 1, ELEVEL)):
        with pytest.raises(G.CkksError) as e:
            ctx.encrypt_batch(z, z, z, z, pk, level, out, ws)
        assert e.value.code == code
    with pytest.raises(G.CkksError) as e:
        ctx.encrypt_batch(z, z, z, z, pk, L, out, ws[:2])
    assert e.value.code == ENOMEM
    three = G.Tuple.wrap(torch.zeros((3, L, N), dtype=torch.uint64, device="cuda"))
    dec = torch.empty((1, N), dtype=torch.float64, device="cuda")
    dws = torch.empty(ctx.decrypt_batch_workspace_size(1) // 8 + 1, dtype=torch.uint64, device="cuda")
    with pytest.raises(G.CkksError) as e:
        ctx.decrypt_batch([three], z[0], dec, dws)                        # not a ciphertext
    assert e.value.code == EINVAL
    ctx.check()


def test_workspace_and_size_queries_reject_bad_levels(env):
    G, params, ctx, *_ = env
    for call in (lambda: ctx.workspace_size(4, params.L + 1, 1), lambda: ctx.rotate_workspace_size(0),
                 lambda: ctx.mul2_workspace_size(1), lambda: ctx.encrypt_batch_workspace_size(0, 1)):
        with pytest.raises(G.CkksError) as e:
            call()
        assert e.value.code == ELEVEL


@pytest.mark.parametrize("log_n", [6, 14])
def test_inputs_at_odd_word_offsets(log_n):
    """Tuples that start 8 bytes past a 16-byte boundary (or have odd
    polynomial strides) are valid: the tensor kernels then read one
    coefficient per thread instead of two (16-byte loads need 16-byte
    alignment); the result equals the oracle's, in a single product and (N >
    256) in a cross-shape wave."""
    import paper_2601_15401_gb300 as G
    from gpu_common import Setup, oracle_tuple
    params = synth.make_params(log_n, [50] * 5, 2, 2, congruence=synth.Q1_CONGRUENCE)
    S = Setup(params, 3, 303)
    N, k, level = params.N, 3, 5
    arrs = [synth.uniform_tuple(params, 2, level, 304, u) for u in range(k)]
    want = O.mul_k(S.octx, [oracle_tuple(a) for a in arrs], S.okeys).data
    depth = S.ctx.plan_describe(k)["depth"]
    # one spare word in front of every tuple, so each starts at an odd word
    flat = [torch.zeros(1 + 2 * level * N, dtype=torch.uint64, device="cuda") for _ in range(k)]
    for f, a in zip(flat, arrs):
        f[1:].copy_(dev(a).reshape(-1))
    cts = [G.Tuple(f[1:].view(2, level, N), 2, level, level) for f in flat]
    assert all(c.data.data_ptr() % 16 == 8 for c in cts)
    out = G.Tuple.wrap(torch.zeros((2, level - depth, N), dtype=torch.uint64, device="cuda"))
    ws = S.ws(S.ctx.workspace_size(k, level, 1))
    S.ctx.mul_k(cts, S.evk, out, ws)
    S.ctx.check()
    assert np.array_equal(host(out.data), want)
    if N <= 256:
        return  # waves need the two-phase NTT (N > 256)
    out2 = G.Tuple.wrap(torch.zeros_like(out.data))
    w = G.Wave(S.ctx, [(cts, out2, None)], S.evk)
    w.run(*w.buffers())
    S.ctx.check()
    assert np.array_equal(host(out2.data), want)


def test_evk_set_rejects_unaligned_keys(env):
    """The key MAC reads the evaluation keys with 16-byte loads, so a key
    buffer that is not 16-byte aligned is refused before any launch."""
    G, params, ctx, octx, okeys, evk = env
    from paper_2601_15401_gb300._lib import lib
    plain = np.stack([np.stack([np.stack([k[0], k[1]]) for k in row]) for row in okeys])
    flat = torch.zeros(1 + plain.size, dtype=torch.uint64, device="cuda")
    flat[1:].copy_(dev(plain).reshape(-1))
    h = ctypes.c_void_p()
    assert flat[1:].data_ptr() % 16 == 8
    assert lib().ckks_evk_set_create(ctx._h, 4, ctypes.c_void_p(flat[1:].data_ptr()), None, ctypes.byref(h)) == EINVAL
    assert not h.value
    ctx.check()
