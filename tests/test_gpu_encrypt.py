"""Public key, encryption and decryption on the GPU (Section II) against the
oracle, and the whole round trip: encode (host), encrypt, k-input multiply,
decrypt (GPU), decode (host) within 2^-20 of the FP64 slot product."""
import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import paper_2601_15401_gb300 as G
    params = synth.make_params(10, [50] * 6, 1, 6)  # alpha = 1 digits for the decryption gate
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    km = synth.key_material(params, 5, 41)
    pa, pe = synth.public_key_draw(params, 41)
    ws = torch.empty(ctx.encrypt_workspace_size() // 8, dtype=torch.uint64, device="cuda")
    pk = torch.empty((2, params.L, params.N), dtype=torch.uint64, device="cuda")
    s = torch.from_numpy(km.s).cuda()
    ctx.public_key(s, dev(pa), torch.from_numpy(pe).cuda(), pk, ws)
    opk = O.public_key(octx, km.s, pa, pe)
    return G, params, ctx, octx, km, s, pk, opk, ws


def test_public_key_parity(env):
    G, params, ctx, octx, km, s, pk, opk, ws = env
    assert np.array_equal(host(pk), np.stack(opk))


@pytest.mark.parametrize("level", [6, 3])
def test_encrypt_parity(env, level):
    G, params, ctx, octx, km, s, pk, opk, ws = env
    d = synth.encryption_draw(params, 42, level)
    m = np.array(O.encode(params.N, d.z, 2.0 ** 50), dtype=np.int64)
    out = G.Tuple.wrap(torch.zeros((2, level, params.N), dtype=torch.uint64, device="cuda"))
    ctx.encrypt(*(torch.from_numpy(x).cuda() for x in (m, d.v, d.e0, d.e1)), pk, level, out, ws)
    want = O.encrypt(octx, [int(x) for x in m], opk, d.v, d.e0, d.e1)
    assert np.array_equal(host(out.data), want[:, :level])


@pytest.mark.parametrize("level", [1, 2, 5])
def test_decrypt_parity(env, level):
    G, params, ctx, octx, km, s, pk, opk, ws = env
    ct = synth.uniform_tuple(params, 2, level, 43, level)
    out = torch.empty(params.N, dtype=torch.float64, device="cuda")
    ctx.decrypt(G.Tuple.wrap(dev(ct)), s, out, ws)
    lv = min(level, 2)
    want = O.decrypt(octx, ct[:, :lv], km.s)  # exact centred integers over q_0 (q_1)
    np.testing.assert_allclose(out.cpu().numpy(), np.array([float(x) for x in want]), rtol=1e-15, atol=0)


def test_round_trip_encode_encrypt_multiply_decrypt_decode(env):
    G, params, ctx, octx, km, s, pk, opk, ws = env
    k, Delta = 4, 2.0 ** 50
    okeys = O.keygen_all(octx, km, k)
    plain = np.stack([np.stack([np.stack([a, b]) for a, b in row]) for row in okeys])
    evk = ctx.evk_set(k, dev(plain))
    cts, zs = [], []
    for i in range(k):
        d = synth.encryption_draw(params, 44, i)
        m = np.array(O.encode(params.N, d.z, Delta), dtype=np.int64)
        t = G.Tuple.wrap(torch.zeros((2, params.L, params.N), dtype=torch.uint64, device="cuda"), scale=Delta)
        ctx.encrypt(*(torch.from_numpy(x).cuda() for x in (m, d.v, d.e0, d.e1)), pk, params.L, t, ws)
        t.scale = Delta
        cts.append(t)
        zs.append(d.z)
    depth = ctx.plan_describe(k)["depth"]
    out = G.Tuple.wrap(torch.zeros((2, params.L - depth, params.N), dtype=torch.uint64, device="cuda"))
    mws = torch.empty(ctx.workspace_size(k, params.L) // 8 + 1, dtype=torch.uint64, device="cuda")
    ctx.mul_k(cts, evk, out, mws)
    dec = torch.empty(params.N, dtype=torch.float64, device="cuda")
    ctx.decrypt(out, s, dec, ws)
    z = O.decode(params.N, [float(x) for x in dec.cpu().numpy()], out.scale)
    assert np.abs(z - np.prod(np.stack(zs), axis=0)).max() <= 2.0 ** -20
