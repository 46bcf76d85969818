"""Cross-shape batches (ckks_wave_*): k-input products of any mix of k,
partition and input level run as one set of stage launches over device job
tables. Every product must equal the oracle's evaluation (Section V: Table
II or given partitions, Algorithm 1 at inner nodes, combined key switching
of Eq. 15, relocated rescale) and ckks_mul_k on the same product alone,
residue for residue."""
import numpy as np
import pytest

import synth
from oracle import ckks as O

from gpu_common import Setup, dev, host, oracle_tuple

pytestmark = pytest.mark.gpu

PARTS = {5: "(2,2,1)", 6: "(2,2,2)", 10: "(6,4)|(3,3)", 12: "(4,4,4)|(2,2),(2,2),(2,2)"}


def _mix(S, n, seed, ks=range(2, 13), other_parts=True):
    """n products: k, level, partition drawn from seed; inputs uniform
    residues, some of them strided views of a wider tuple."""
    import torch

    import paper_2601_15401_gb300 as G
    g = np.random.default_rng(seed)
    L, N = S.params.L, S.params.N
    items = []
    for i in range(n):
        k = int(g.choice(list(ks)))
        part = PARTS.get(k) if other_parts and g.random() < 0.4 else None
        depth = S.ctx.plan_describe(k, part)["depth"]
        level = int(g.integers(depth + 1, L + 1))
        stride = level + int(g.integers(0, 2)) if level < L else level
        arrs, cts = [], []
        for u in range(k):
            a = synth.uniform_tuple(S.params, 2, stride, 900 + seed, 100 * i + u)
            arrs.append(a[:, :level])
            cts.append(G.Tuple(dev(a), 2, level, stride, 1, 2.0 ** 20))
        out = G.Tuple.wrap(torch.zeros((2, level - depth, N), dtype=torch.uint64, device="cuda"))
        items.append({"k": k, "part": part, "level": level, "arrs": arrs, "cts": cts, "out": out, "depth": depth})
    return items


def _alone(S, it):
    """ckks_mul_k on one product (the library's one-product path)."""
    import torch

    import paper_2601_15401_gb300 as G
    o = G.Tuple.wrap(torch.zeros_like(it["out"].data))
    ws = S.ws(S.ctx.workspace_size(it["k"], it["level"], 1, it["part"]))
    S.ctx.mul_k(it["cts"], S.evk, o, ws, partition=it["part"])
    return host(o.data), o.scale


def _run_wave(S, items):
    import torch

    import paper_2601_15401_gb300 as G
    w = G.Wave(S.ctx, [(it["cts"], it["out"], it["part"]) for it in items], S.evk)
    ws = w.buffers()
    w.run(*ws)
    S.ctx.check()
    return w, ws


@pytest.fixture(scope="module")
def S_small():
    return Setup(synth.make_params(10, [50] * 12, 2, 3), 12, 40)


def test_wave_mixed_small_matches_oracle_and_alone(S_small):
    """24 products, k = 2..12, levels depth+1..12, Table II and other
    partitions, N = 2^10: every product equals the oracle and ckks_mul_k."""
    S = S_small
    items = _mix(S, 24, 1)
    w, ws = _run_wave(S, items)
    d = w.describe()
    # per round at most 6 tuple-size classes and 13 fixed shapes of tensor
    # launches; the key MAC's paired and single launches
    assert d["launches"] <= 6 * d["heights"] + 15 + 19 * (d["heights"] + 1)
    for i, it in enumerate(items):
        got = host(it["out"].data)
        want = O.mul_k(S.octx, [oracle_tuple(a, 2.0 ** 20) for a in it["arrs"]], S.okeys, it["part"])
        assert it["out"].level == want.level == it["level"] - it["depth"]
        assert np.array_equal(got, want.data), f"item {i}: k={it['k']} level={it['level']} part={it['part']}"
        alone, scale = _alone(S, it)
        assert np.array_equal(got, alone), f"item {i} differs from ckks_mul_k alone"
        assert it["out"].scale == pytest.approx(scale)


def test_wave_rerun_and_new_workspace(S_small):
    """A second run with the same buffers reuses the tables; a run with
    other buffers rebuilds them; both give the same residues."""
    S = S_small
    items = _mix(S, 9, 2)
    w, ws = _run_wave(S, items)
    first = [host(it["out"].data) for it in items]
    for it in items:
        it["out"].data.zero_()
    w.run(*ws)
    again = [host(it["out"].data) for it in items]
    t2, s2 = w.buffers()
    for it in items:
        it["out"].data.zero_()
    w.run(t2[32:], s2[32:])  # other buffers (256-byte aligned offsets): the tables are rebuilt
    other = [host(it["out"].data) for it in items]
    S.ctx.check()
    for a, b, c in zip(first, again, other):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_wave_argument_errors(S_small):
    import torch

    import paper_2601_15401_gb300 as G
    S = S_small
    items = _mix(S, 3, 3, other_parts=False)
    # two products writing one output
    with pytest.raises(G.CkksError) as e:
        G.Wave(S.ctx, [(items[0]["cts"], items[0]["out"], None)] * 2, S.evk)
    assert e.value.code == -1
    # level too low for the partition depth
    low = [items[0]["cts"][0]] * 12
    low = [G.Tuple(c.data, 2, 3, c.poly_stride) for c in low]
    out = G.Tuple.wrap(torch.zeros((2, 2, S.params.N), dtype=torch.uint64, device="cuda"))
    with pytest.raises(G.CkksError) as e:
        G.Wave(S.ctx, [(low, out, None)], S.evk)
    assert e.value.code == -2
    # buffers too small
    w = G.Wave(S.ctx, [(it["cts"], it["out"], it["part"]) for it in items], S.evk)
    t, n = w.workspace_size()
    tb = torch.empty(t // 8 + 1, dtype=torch.uint64, device="cuda")
    sb = torch.empty(n // 8 - 64, dtype=torch.uint64, device="cuda")
    with pytest.raises(G.CkksError) as e:
        w.run(tb, sb)
    assert e.value.code == -4
    # waves run one after the other may share one scratch buffer
    other = _mix(S, 4, 4, other_parts=False)
    w2 = G.Wave(S.ctx, [(it["cts"], it["out"], it["part"]) for it in other], S.evk)
    shared = torch.empty(max(n, w2.workspace_size()[1]) // 8 + 1, dtype=torch.uint64, device="cuda")
    t2 = torch.empty(w2.workspace_size()[0] // 8 + 1, dtype=torch.uint64, device="cuda")
    w.run(tb, shared)
    w2.run(t2, shared)
    w.run(tb, shared)
    for it in items + other:
        alone, _ = _alone(S, it)
        assert np.array_equal(host(it["out"].data), alone)
    S.ctx.check()


def test_wave_rejects_one_phase_ring():
    import torch

    import paper_2601_15401_gb300 as G
    S = Setup(synth.make_params(8, [50] * 4, 1, 1), 3, 41)
    cts = [S.tuple(synth.uniform_tuple(S.params, 2, 4, 41, u)) for u in range(3)]
    out = G.Tuple.wrap(torch.zeros((2, 2, S.params.N), dtype=torch.uint64, device="cuda"))
    with pytest.raises(G.CkksError) as e:
        G.Wave(S.ctx, [(cts, out, None)], S.evk)
    assert e.value.code == -1


@pytest.mark.parametrize("log_n,congruence", [(14, synth.NTT_CONGRUENCE), (14, synth.Q1_CONGRUENCE),
                                               (16, synth.Q1_CONGRUENCE)])
def test_wave_full_parameter_set(log_n, congruence):
    """N = 2^14 / 2^16, L = 24, K = 8, dnum = 3: a mixed wave equals
    ckks_mul_k alone on every product and the oracle on two sampled ones;
    with primes = 1 (mod 2^17) (the general modular products) and = 1 (mod
    2^32) (the cheaper forms)."""
    S = Setup(synth.params_large(log_n, congruence=congruence), 12, 42)
    n = 16 if log_n == 14 else 7
    items = _mix(S, n, 10 + log_n, ks=[2, 3, 4, 5, 7, 8, 12], other_parts=False)
    _run_wave(S, items)
    for i, it in enumerate(items):
        alone, _ = _alone(S, it)
        assert np.array_equal(host(it["out"].data), alone), f"item {i}: k={it['k']} level={it['level']}"
    for i in (0, n - 1):
        it = items[i]
        want = O.mul_k(S.octx, [oracle_tuple(a, 2.0 ** 20) for a in it["arrs"]], S.okeys, it["part"])
        assert np.array_equal(host(it["out"].data), want.data), f"item {i}"
