"""Canonical-embedding encoding and decoding on the GPU (Section II)
against the oracle's definitions, and the whole plaintext round trip on the
device: encode, encrypt, k-input multiply, decrypt, decode.

Tolerances, from the double-precision arithmetic: decoding sums N terms of
size |m_i| / scale <= 1 with a log2(N)-deep FFT, error below ~log2(N) N
2^-53 <= 2^-31 at N = 2^16; the oracle's per-slot sum (exact argument
reduction) is as accurate; both checked to 2^-30. Encoding: the value before
rounding carries ~log2(N) 2^-53 scale on either side, so GPU and oracle
integers agree to 0.5 + 2^-40 scale."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import dev

pytestmark = pytest.mark.gpu


def _ctx(log_n, L=2, K=1, dnum=1):
    import paper_2601_15401_gb300 as G
    params = synth.make_params(log_n, [50] * L, K, dnum)
    return G, params, G.Context.from_params(params)


def _slots(n, config, index, batch=1):
    return np.stack([synth.unit_disk_slots(synth.rng(config, index + b, stream=6), n) for b in range(batch)])


@pytest.mark.parametrize("log_n", [4, 5, 7, 10, 12, 16])
def test_decode_parity(log_n):
    G, params, ctx = _ctx(log_n)
    N, scale = params.N, 2.0 ** 40
    batch = 2
    rng = synth.rng(601, log_n)
    m = np.stack([rng.integers(-2 ** 40, 2 ** 40, N) for _ in range(batch)]).astype(np.float64)
    z = torch.empty((batch, N // 2), dtype=torch.complex128, device="cuda")
    ws = torch.empty(ctx.embed_workspace_size(batch) // 8, dtype=torch.uint64, device="cuda")
    ctx.decode(torch.from_numpy(m).cuda(), scale, z, ws)
    got = z.cpu().numpy()
    js = range(N // 2) if log_n <= 12 else list(range(8)) + list(range(N // 2 - 8, N // 2)) + [1234, 20000]
    for b in range(batch):
        mi = [int(x) for x in m[b]]
        for j in js:
            assert abs(got[b, j] - O.decode_slot(N, mi, scale, j)) <= 2.0 ** -30, (b, j)


@pytest.mark.parametrize("log_n,scale_bits", [(4, 30), (5, 40), (9, 40), (10, 40), (12, 50), (16, 40)])
def test_encode_parity(log_n, scale_bits):
    G, params, ctx = _ctx(log_n)
    N, scale = params.N, 2.0 ** scale_bits
    batch = 2
    zs = _slots(N // 2, 602, log_n, batch)
    m = torch.empty((batch, N), dtype=torch.int64, device="cuda")
    ws = torch.empty(ctx.embed_workspace_size(batch) // 8, dtype=torch.uint64, device="cuda")
    ctx.encode(torch.from_numpy(zs).cuda(), scale, m, ws)
    got = m.cpu().numpy()
    tol = 0.5 + 2.0 ** -40 * scale
    idx = range(N) if log_n <= 10 else list(range(16)) + list(range(N - 16, N)) + [N // 2 + 1, 33333 % N]
    for b in range(batch):
        if log_n <= 10:  # the vector form agrees exactly away from ties
            want = O.encode(N, zs[b], scale)
            assert np.abs(got[b] - np.array(want)).max() <= 1 + 2.0 ** -40 * scale
        for i in idx:
            assert abs(got[b, i] - O.encode_coef(N, zs[b], scale, i)) <= tol, (b, i)


def test_round_trip_full_size():
    """decode(encode(z)) = z up to the rounding of encode: each coefficient
    moves by <= 1/2, so each slot by <= (N/2) / scale."""
    G, params, ctx = _ctx(16, 24, 8, 3)
    N, scale, batch = params.N, 2.0 ** 40, 4
    zs = _slots(N // 2, 603, 0, batch)
    ws = torch.empty(ctx.embed_workspace_size(batch) // 8, dtype=torch.uint64, device="cuda")
    m = torch.empty((batch, N), dtype=torch.int64, device="cuda")
    ctx.encode(torch.from_numpy(zs).cuda(), scale, m, ws)
    z = torch.empty((batch, N // 2), dtype=torch.complex128, device="cuda")
    ctx.decode(m.to(torch.float64), scale, z, ws)
    assert np.abs(z.cpu().numpy() - zs).max() <= (N / 2) / scale + 2.0 ** -30


@pytest.mark.parametrize("k", [3, 4])
def test_plaintext_round_trip_on_device(k):
    """slots -> encode -> encrypt -> k-input product -> decrypt -> decode,
    every step on the GPU: the FP64 slot product within 2^-20."""
    import paper_2601_15401_gb300 as G
    params = synth.make_params(10, [50] * 6, 1, 6)  # alpha = 1 digits
    N, L = params.N, params.L
    ctx = G.Context.from_params(params)
    km = synth.key_material(params, k, 604)
    s = torch.from_numpy(km.s).cuda()
    a = np.stack([np.stack(r) for r in km.a])
    e = np.stack([np.stack(r) for r in km.e])
    keys = torch.empty((k - 1, params.dnum, 2, L + params.K, N), dtype=torch.uint64, device="cuda")
    kws = torch.empty(ctx.keygen_workspace_size() // 8, dtype=torch.uint64, device="cuda")
    ctx.keygen_evk(k, s, dev(a), torch.from_numpy(e).cuda(), keys, kws)
    evk = ctx.evk_set(k, keys)
    pa, pe = synth.public_key_draw(params, 604)
    ews = torch.empty(ctx.encrypt_workspace_size() // 8, dtype=torch.uint64, device="cuda")
    pk = torch.empty((2, L, N), dtype=torch.uint64, device="cuda")
    ctx.public_key(s, dev(pa), torch.from_numpy(pe).cuda(), pk, ews)
    scale = 2.0 ** 50
    zs = _slots(N // 2, 604, 0, k)
    mws = torch.empty(ctx.embed_workspace_size(k) // 8, dtype=torch.uint64, device="cuda")
    m = torch.empty((k, N), dtype=torch.int64, device="cuda")
    ctx.encode(torch.from_numpy(zs).cuda(), scale, m, mws)
    cts = []
    for i in range(k):
        d = synth.encryption_draw(params, 604, i)
        ct = G.Tuple.wrap(torch.zeros((2, L, N), dtype=torch.uint64, device="cuda"), scale=scale)
        ctx.encrypt(m[i].contiguous(), *(torch.from_numpy(x).cuda() for x in (d.v, d.e0, d.e1)), pk, L, ct, ews)
        ct.scale = scale
        cts.append(ct)
    depth = math.ceil(math.log2(k))
    out = G.Tuple.wrap(torch.zeros((2, L - depth, N), dtype=torch.uint64, device="cuda"))
    ws = torch.empty(ctx.workspace_size(k, L) // 8 + 1, dtype=torch.uint64, device="cuda")
    ctx.mul_k(cts, evk, out, ws)
    dec = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.decrypt(out, s, dec, ews)
    z = torch.empty((1, N // 2), dtype=torch.complex128, device="cuda")
    ctx.decode(dec, out.scale, z, mws)
    assert np.abs(z.cpu().numpy()[0] - np.prod(zs, axis=0)).max() <= 2.0 ** -20


def test_embed_errors():
    G, params, ctx = _ctx(6)
    N = params.N
    z = torch.zeros((1, N // 2), dtype=torch.complex128, device="cuda")
    m = torch.empty((1, N), dtype=torch.int64, device="cuda")
    ws = torch.empty(ctx.embed_workspace_size(1) // 8, dtype=torch.uint64, device="cuda")
    for scale, w, code in ((0.0, ws, -1), (-1.0, ws, -1), (1.0, ws[:4], -4)):
        with pytest.raises(G.CkksError) as e:
            ctx.encode(z, scale, m, w)
        assert e.value.code == code
