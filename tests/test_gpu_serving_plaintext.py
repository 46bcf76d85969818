"""Plaintext-in / plaintext-out serving on the GPU: requests carry slot
vectors; each batch runs encode, batched encryption, the k-input product,
batched decryption and decode in the library. Every result decodes to the
FP64 product of its slot vectors within 2^-20, and is the same alone as in
the mix (the encryption noise is seeded per request). Batched encryption
and decryption equal the oracle and the single calls."""
import copy

import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt_state():
    from paper_2601_15401_gb300 import serve as S
    # alpha = 4 primes (200 bits) per digit under P = 2^240: key-switch noise
    # far below the 2^-20 gate at scale 2^50
    contexts, _ = S.build_gpu_state((12,), L=8, K=4, dnum=2, t_max=6, pool_size=1)
    keys = S.build_plaintext_keys(contexts)
    return S, contexts, keys


def test_plaintext_serving_results_and_mix_equals_alone(pt_state):
    S, contexts, keys = pt_state
    be = S.PlaintextBackend(contexts, keys, n_streams=3, ws_bytes=1 << 30, keep_results=True)
    reqs = S.plaintext_requests(400.0, 0.1, 77, log_ns=(12,), L=8, k_range=(2, 6))
    assert len(reqs) >= 10
    alone_src = copy.deepcopy(reqs[:4])
    sched = S.Scheduler(be, 20 << 30, max_batch=4)
    S.run_open_loop(sched, reqs, timeout=300)
    assert len(sched.completed) == len(reqs) and not sched.failed
    for r in reqs:
        want = np.prod(r.slots, axis=0)
        assert np.abs(be.results[r.rid] - want).max() <= 2.0 ** -20, (r.rid, r.k, r.level)
    # the same requests one at a time
    be1 = S.PlaintextBackend(contexts, keys, n_streams=1, ws_bytes=1 << 30, keep_results=True)
    for r in alone_src:
        r.arrival = 0.0
    s1 = S.Scheduler(be1, 20 << 30, max_batch=1)
    S.run_open_loop(s1, alone_src, timeout=300)
    for r in alone_src:
        assert np.array_equal(be1.results[r.rid], be.results[r.rid]), r.rid


def test_encrypt_decrypt_batch_match_single_and_oracle():
    import paper_2601_15401_gb300 as G
    params = synth.make_params(10, [50] * 6, 1, 6)
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    km = synth.key_material(params, 2, 81)
    s = torch.from_numpy(km.s).cuda()
    pa, pe = synth.public_key_draw(params, 81)
    ws1 = torch.empty(ctx.encrypt_workspace_size() // 8, dtype=torch.uint64, device="cuda")
    pk = torch.empty((2, params.L, params.N), dtype=torch.uint64, device="cuda")
    ctx.public_key(s, dev(pa), torch.from_numpy(pe).cuda(), pk, ws1)
    opk = O.public_key(octx, km.s, pa, pe)
    N, B = params.N, 5
    for level in (6, 3, 1):
        draws = [synth.encryption_draw(params, 82, level * 10 + b) for b in range(B)]
        m = np.stack([np.array(O.encode(N, d.z, 2.0 ** 45), dtype=np.int64) for d in draws])
        cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in
                (m, np.stack([d.v for d in draws]), np.stack([d.e0 for d in draws]), np.stack([d.e1 for d in draws]))]
        out = torch.zeros((B, 2, level, N), dtype=torch.uint64, device="cuda")
        outs = [G.Tuple.wrap(out[b]) for b in range(B)]
        ws = torch.empty(ctx.encrypt_batch_workspace_size(level, B) // 8 + 1, dtype=torch.uint64, device="cuda")
        ctx.encrypt_batch(*cols, pk, level, outs, ws)
        got = host(out)
        for b, d in enumerate(draws):
            want = O.encrypt(octx, [int(x) for x in m[b]], opk, d.v, d.e0, d.e1)
            assert np.array_equal(got[b], want[:, :level]), (level, b)
        dec = torch.empty((B, N), dtype=torch.float64, device="cuda")
        dws = torch.empty(ctx.decrypt_batch_workspace_size(B) // 8 + 1, dtype=torch.uint64, device="cuda")
        ctx.decrypt_batch(outs, s, dec, dws)
        one = torch.empty(N, dtype=torch.float64, device="cuda")
        for b in range(B):
            ctx.decrypt(outs[b], s, one, ws1)
            assert torch.equal(one, dec[b])
            lv = min(level, 2)
            want = O.decrypt(octx, got[b][:, :lv], km.s)
            np.testing.assert_allclose(dec[b].cpu().numpy(), np.array([float(x) for x in want]), rtol=1e-15, atol=0)


@pytest.mark.slow
def test_encrypt_decrypt_batch_full_size():
    """N = 2^16, L = 24: batched encryption equals the oracle's on every
    residue; decryption equals c_0 + c_1 s formed from oracle steps (the
    product in the NTT domain, pinned by the convolution theorem, then the
    inverse transform and a two-prime CRT)."""
    import paper_2601_15401_gb300 as G
    from oracle import ring
    params = synth.params_large()
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    km = synth.key_material(params, 2, 91)
    s = torch.from_numpy(km.s).cuda()
    pa, pe = synth.public_key_draw(params, 91)
    ws1 = torch.empty(ctx.encrypt_workspace_size() // 8, dtype=torch.uint64, device="cuda")
    pk = torch.empty((2, params.L, params.N), dtype=torch.uint64, device="cuda")
    ctx.public_key(s, dev(pa), torch.from_numpy(pe).cuda(), pk, ws1)
    opk = O.public_key(octx, km.s, pa, pe)
    assert np.array_equal(host(pk), np.stack(opk))
    N, L = params.N, params.L
    d = synth.encryption_draw(params, 92, 0)
    m = synth.rng(93, 0).integers(-2 ** 40, 2 ** 40, N).astype(np.int64)   # any integer message
    cols = [torch.from_numpy(np.ascontiguousarray(x[None])).cuda() for x in (m, d.v, d.e0, d.e1)]
    out = torch.zeros((1, 2, L, N), dtype=torch.uint64, device="cuda")
    outs = [G.Tuple.wrap(out[0])]
    ws = torch.empty(ctx.encrypt_batch_workspace_size(L, 1) // 8 + 1, dtype=torch.uint64, device="cuda")
    ctx.encrypt_batch(*cols, pk, L, outs, ws)
    got = host(out)[0]
    want = O.encrypt(octx, [int(x) for x in m], opk, d.v, d.e0, d.e1)
    assert np.array_equal(got, want)
    dec = torch.empty((1, N), dtype=torch.float64, device="cuda")
    dws = torch.empty(ctx.decrypt_batch_workspace_size(1) // 8 + 1, dtype=torch.uint64, device="cuda")
    ctx.decrypt_batch(outs, s, dec, dws)
    q2 = octx.q[:2]
    S2 = O.ntt_poly(np.stack([ring.from_signed(km.s, qj) for qj in q2]), q2)
    P = O.intt_poly(ring.addmod_rows(got[0][:2], ring.mulmod_rows(got[1][:2], S2, q2), q2), q2)
    want_dec = O.crt_centered(P, q2)
    np.testing.assert_allclose(dec[0].cpu().numpy(), np.array([float(x) for x in want_dec]), rtol=1e-15, atol=0)
