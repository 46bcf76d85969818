"""The request-array entry point (uneven k, partitions, levels and batch
sizes in one call) and the single Eq. 7 rescale, against the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import Setup, dev, host, oracle_tuple

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return Setup(synth.make_params(5, [50] * 7, 2, 3), 12, 701)


def _group(S, k, batch, level, seed, part=None):
    import paper_2601_15401_gb300 as G
    x = dev(np.stack([synth.uniform_tuple(S.params, 2, level, seed, i) for i in range(batch * k)])
            .reshape(batch, k, 2, level, S.params.N))
    depth = S.ctx.plan_describe(k, part)["depth"]
    out = torch.zeros((batch, 2, level - depth, S.params.N), dtype=torch.uint64, device="cuda")
    cts = [[G.Tuple.wrap(x[b, u]) for u in range(k)] for b in range(batch)]
    outs = [G.Tuple.wrap(out[b]) for b in range(batch)]
    return (cts, outs, part), x, out


def test_uneven_requests_match_the_oracle(S):
    specs = [(3, 2, 6, 702, None), (5, 1, 7, 703, "(3,2)"), (4, 3, 5, 704, None), (12, 1, 7, 705, None),
             (2, 2, 3, 706, "(1,1)")]
    made = [_group(S, *sp) for sp in specs]
    groups = [m[0] for m in made]
    ws = S.ws(S.ctx.requests_workspace_size(groups, S.evk))
    assert S.ctx.mul_k_requests(groups, S.evk, ws) == len(groups)
    for (k, batch, level, seed, part), (_, x, out) in zip(specs, made):
        got = host(out)
        for b in range(batch):
            want = O.mul_k(S.octx, [oracle_tuple(host(x[b, u])) for u in range(k)], S.okeys, part)
            assert np.array_equal(got[b][:, :want.level], want.data), (k, b)


def test_requests_errors_report_progress(S):
    import paper_2601_15401_gb300 as G
    from paper_2601_15401_gb300._lib import lib
    g1, _, _ = _group(S, 3, 1, 6, 707)
    g2, _, _ = _group(S, 4, 1, 2, 708)        # level 2 <= depth 2: ELEVEL
    rr, keep = S.ctx._requests([g1, g2], S.evk)
    ws = S.ws(S.ctx.workspace_size(3, 6, 1))
    import ctypes
    done = ctypes.c_uint32(99)
    rc = lib().ckks_mul_k_requests(S.ctx._h, rr, 2, ctypes.byref(done), ws.data_ptr(), ws.numel() * 8, None)
    assert rc == -2 and done.value == 1
    with pytest.raises(G.CkksError) as e:
        S.ctx.mul_k_requests([g1], S.evk, ws[:16])
    assert e.value.code == -4
    S.ctx.check()


def test_single_rescale_is_eq7(S):
    import paper_2601_15401_gb300 as G
    a = synth.uniform_tuple(S.params, 3, 6, 709, 0)
    ws = S.ws(S.ctx.rescale_workspace_size(3, 6, 1))
    out = G.Tuple.wrap(dev(np.zeros((3, 5, S.params.N), dtype=np.uint64)))
    S.ctx.rescale(G.Tuple.wrap(dev(a), scale=2.0 ** 60), out, ws)
    assert out.level == 5
    for p in range(3):
        assert np.array_equal(host(out.data)[p], O.RS(S.octx, a[p]))
    assert out.scale == pytest.approx(2.0 ** 60 / S.params.q[5], rel=1e-15)
