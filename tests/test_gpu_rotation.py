"""Galois automorphisms, Galois keys and slot rotation on the GPU (through
the C ABI) against the oracle, residue for residue, plus the decryption
gate: a rotated ciphertext decodes to the rotated slot vector."""
import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import dev, host, oracle_tuple

pytestmark = pytest.mark.gpu


class Rot:
    """Context, oracle context and Galois keys of some elements."""

    def __init__(self, params, config, gs):
        import paper_2601_15401_gb300 as G
        self.G = G
        self.params = params
        self.ctx = G.Context.from_params(params)
        self.octx = O.Ctx(params)
        self.km = synth.key_material(params, 2, config)
        self.s = torch.from_numpy(self.km.s).cuda()
        ws = torch.empty(self.ctx.keygen_workspace_size() // 8, dtype=torch.uint64, device="cuda")
        self.gk, self.ogk, self.plain = {}, {}, {}
        NP = params.L + params.K
        for g in gs:
            a, e = synth.galois_key_draw(params, config, g)
            keys = torch.empty((params.dnum, 2, NP, params.N), dtype=torch.uint64, device="cuda")
            self.ctx.keygen_galois(g, self.s, dev(np.stack(a)), torch.from_numpy(np.stack(e)).cuda(), keys, ws)
            self.plain[g] = keys.clone()
            self.gk[g] = self.ctx.evk_set(2, keys)
            self.ogk[g] = O.galois_keygen(self.octx, self.km.s, a, e, g)
        torch.cuda.synchronize()

    def rotate(self, cts, g, level, inplace=False):
        G, N = self.G, self.params.N
        B = len(cts)
        x = dev(np.stack(cts))
        ins = [G.Tuple.wrap(x[b], scale=2.0 ** 40) for b in range(B)]
        if inplace:
            outs = ins
        else:
            y = torch.zeros((B, 2, level, N), dtype=torch.uint64, device="cuda")
            outs = [G.Tuple.wrap(y[b]) for b in range(B)]
        ws = torch.empty(self.ctx.rotate_workspace_size(level, B) // 8 + 1, dtype=torch.uint64, device="cuda")
        self.ctx.rotate_batch(ins, g, self.gk[g], outs, ws)
        return [host(o.data)[:, :level] for o in outs], outs


def _elements(N):
    return [O.galois_element(1, N), O.galois_element(5, N), O.galois_element(-1, N), 2 * N - 1]


@pytest.fixture(scope="module")
def R():
    params = synth.make_params(6, [50] * 5, 2, 2)  # alpha = 3: a full and a ragged digit
    return Rot(params, 501, _elements(params.N))


@pytest.mark.parametrize("log_n", [4, 6, 10, 12, 16])
def test_automorphism_parity(log_n):
    import paper_2601_15401_gb300 as G
    params = synth.make_params(log_n, [50] * 3, 1, 1)
    ctx = G.Context.from_params(params)
    N = params.N
    A = synth.uniform_tuple(params, 2, 3, 502, log_n)
    for g in (O.galois_element(1, N), O.galois_element(7, N), 2 * N - 1, 1):
        out = G.Tuple.wrap(torch.zeros((2, 3, N), dtype=torch.uint64, device="cuda"))
        ctx.automorphism(G.Tuple.wrap(dev(A)), g, out)
        got = host(out.data)
        if log_n >= 12:  # the oracle's coefficient loop is slow: two limbs
            for p, j in ((0, 0), (1, 2)):
                want = O.automorphism_ntt(A[p][j:j + 1], g, [params.q[j]])[0]
                assert np.array_equal(got[p][j], want), (g, p, j)
        else:
            want = np.stack([O.automorphism_ntt(A[p], g, params.q[:3]) for p in range(2)])
            assert np.array_equal(got, want), g


def test_galois_keygen_parity(R):
    for g, keys in R.plain.items():
        want = np.stack([np.stack([k[0], k[1]]) for k in R.ogk[g]])
        assert np.array_equal(host(keys), want), g


@pytest.mark.parametrize("level", [5, 4, 3, 1])
def test_rotate_parity(R, level):
    for g in R.gk:
        ct = synth.uniform_tuple(R.params, 2, level, 503, g)
        got, _ = R.rotate([ct], g, level)
        want = O.rotate(R.octx, oracle_tuple(ct), g, R.ogk[g])
        assert np.array_equal(got[0], want.data), (g, level)


def test_rotate_batch_equals_alone_and_in_place(R):
    g = O.galois_element(1, R.params.N)
    cts = [synth.uniform_tuple(R.params, 2, 5, 504, i) for i in range(5)]
    batch, _ = R.rotate(cts, g, 5)
    inplace, outs = R.rotate(cts, g, 5, inplace=True)
    for i, ct in enumerate(cts):
        alone, _ = R.rotate([ct], g, 5)
        assert np.array_equal(batch[i], alone[0]) and np.array_equal(inplace[i], alone[0])
    assert outs[0].scale == 2.0 ** 40 and outs[0].level == 5


def test_rotate_errors(R):
    import paper_2601_15401_gb300 as G
    N = R.params.N
    ct = R.G.Tuple.wrap(dev(synth.uniform_tuple(R.params, 2, 5, 505, 0)))
    out = R.G.Tuple.wrap(torch.zeros((2, 5, N), dtype=torch.uint64, device="cuda"))
    ws = torch.empty(R.ctx.rotate_workspace_size(5) // 8 + 1, dtype=torch.uint64, device="cuda")
    g = next(iter(R.gk))
    for bad in (2, 2 * N + 1, 0):
        with pytest.raises(G.CkksError) as e:
            R.ctx.rotate(ct, bad, R.gk[g], out, ws)
        assert e.value.code == -1
    with pytest.raises(G.CkksError) as e:
        R.ctx.rotate(ct, g, R.gk[g], out, ws[:8])
    assert e.value.code == -4
    with pytest.raises(G.CkksError) as e:
        R.ctx.automorphism(ct, g, ct)
    assert e.value.code == -1
    assert R.ctx.galois_element(0) == 1 and R.ctx.galois_element(N // 2) == 1
    assert R.ctx.galois_element(-1) * R.ctx.galois_element(1) % (2 * N) == 1


@pytest.mark.parametrize("r", [1, 7, -3, "conj"])
def test_rotation_decrypts_to_rotated_slots(r):
    """encode (host) -> encrypt, rotate, decrypt (GPU) -> decode (host):
    the slots rotated by r (or conjugated) within 2^-20."""
    params = synth.make_params(10, [50] * 4, 1, 4)  # alpha = 1
    N = params.N
    ctx_g = 2 * N - 1 if r == "conj" else O.galois_element(r, N)
    S = Rot(params, 506, [ctx_g])
    pa, pe = synth.public_key_draw(params, 506)
    ews = torch.empty(S.ctx.encrypt_workspace_size() // 8, dtype=torch.uint64, device="cuda")
    pk = torch.empty((2, params.L, N), dtype=torch.uint64, device="cuda")
    S.ctx.public_key(S.s, dev(pa), torch.from_numpy(pe).cuda(), pk, ews)
    d = synth.encryption_draw(params, 506, 0)
    m = np.array(O.encode(N, d.z, 2.0 ** 50), dtype=np.int64)
    ct = S.G.Tuple.wrap(torch.zeros((2, params.L, N), dtype=torch.uint64, device="cuda"))
    S.ctx.encrypt(*(torch.from_numpy(x).cuda() for x in (m, d.v, d.e0, d.e1)), pk, params.L, ct, ews)
    ct.scale = 2.0 ** 50
    out = S.G.Tuple.wrap(torch.zeros((2, params.L, N), dtype=torch.uint64, device="cuda"))
    ws = torch.empty(S.ctx.rotate_workspace_size(params.L) // 8 + 1, dtype=torch.uint64, device="cuda")
    S.ctx.rotate(ct, ctx_g, S.gk[ctx_g], out, ws)
    dec = torch.empty(N, dtype=torch.float64, device="cuda")
    S.ctx.decrypt(out, S.s, dec, ews)
    z = O.decode(N, [int(round(x)) for x in dec.cpu().numpy()], out.scale)
    want = np.conj(d.z) if r == "conj" else np.roll(d.z, -r)
    assert np.abs(z - want).max() <= 2.0 ** -20


@pytest.mark.slow
def test_rotate_full_size_sampled():
    """N = 2^16, L = 24, K = 8, dnum = 3, batch 4 at level 24: the last batch
    element against the oracle, every residue."""
    params = synth.params_large()
    g = O.galois_element(1, params.N)
    S = Rot(params, 507, [g])
    cts = [synth.uniform_tuple(params, 2, 24, 507, i) for i in range(4)]
    got, _ = S.rotate(cts, g, 24)
    want = O.rotate(S.octx, oracle_tuple(cts[3]), g, S.ogk[g])
    assert np.array_equal(got[3], want.data)
