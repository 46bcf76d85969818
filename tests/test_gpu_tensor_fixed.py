"""Tensor products of fixed node shapes (tensor_fixed.cu).

Nodes whose two or three children are all tuples of at least four terms run
kernels unrolled for their exact shape (children sorted by size); the
tunable "tensor_fixed" = 0 sends them to the kernels bounded by the largest
tuple size. One partition per compiled shape (a child over g inputs is a
tuple of g + 1 terms, so groups of 3..6 inputs give the 4..7-term children),
each within the depth rule of Section V-C. Both settings must give the
oracle's residues (Eq. 13 evaluated over the tree), through ckks_mul_k (one
launch per node), ckks_mul_k_batch and a cross-shape wave (table launches
grouped by shape)."""
import numpy as np
import pytest

import synth
from oracle import ckks as O

from gpu_common import Setup, dev, host, oracle_tuple

pytestmark = pytest.mark.gpu

# k, partition, sorted child tuple sizes of the node with a fixed kernel (each
# a valid tree with that root: tests/test_tensor_shapes_host.py)
CASES = [
    (6, "(3,3)", (4, 4)),
    (7, "(4,3)|(2,2)", (5, 4)),
    (8, "(4,4)|(2,2),(2,2)", (5, 5)),
    (9, "(5,4)|(3,2),(2,2)", (6, 5)),
    (10, "(5,5)|(3,2),(3,2)", (6, 6)),
    (9, "(6,3)|(3,3)", (7, 4)),
    (10, "(6,4)|(3,3),(2,2)", (7, 5)),
    (11, "(6,5)|(3,3),(3,2)", (7, 6)),
    (12, "(6,6)|(3,3),(3,3)", (7, 7)),
    (9, "(3,3,3)", (4, 4, 4)),
    (10, "(4,3,3)|(2,2)", (5, 4, 4)),
    (11, "(4,4,3)|(2,2),(2,2)", (5, 5, 4)),
    (12, "(4,4,4)|(2,2),(2,2),(2,2)", (5, 5, 5)),
]
LEVEL = 8


@pytest.fixture(scope="module")
def S():
    # N = 2^10: every node spans several 256-thread blocks per limb
    return Setup(synth.make_params(10, [50] * LEVEL, 2, 3), 12, 311)


def _inputs(S, k, seed):
    return [synth.uniform_tuple(S.params, 2, LEVEL, 311, seed + u) for u in range(k)]


@pytest.mark.parametrize("fixed", [1, 0])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_mul_k_fixed_shapes(S, case, fixed):
    import paper_2601_15401_gb300 as G
    k, part, _ = CASES[case]
    cts = _inputs(S, k, 50 * case)
    want = O.mul_k(S.octx, [oracle_tuple(c) for c in cts], S.okeys, part)
    depth = S.ctx.plan_describe(k, part)["depth"]
    S.ctx.tune_set("tensor_fixed", fixed)
    try:
        out = G.Tuple.wrap(dev(np.zeros((2, LEVEL - depth, S.params.N), dtype=np.uint64)))
        ws = S.ws(S.ctx.workspace_size(k, LEVEL, 1, part))
        S.ctx.mul_k([G.Tuple.wrap(dev(c)) for c in cts], S.evk, out, ws, partition=part)
        S.ctx.check()
    finally:
        S.ctx.tune_set("tensor_fixed", 1)
    assert out.level == want.level
    assert np.array_equal(host(out.data)[:, :out.level], want.data), f"k={k} {part} tensor_fixed={fixed}"


def test_mul_k_batch_fixed_shapes(S):
    """The batched call (one uniform launch per node for the whole batch)."""
    import torch

    import paper_2601_15401_gb300 as G
    k, part, _ = CASES[12]
    B = 3
    cts = [_inputs(S, k, 1000 + 20 * b) for b in range(B)]
    depth = S.ctx.plan_describe(k, part)["depth"]
    inp = dev(np.stack([np.stack(c) for c in cts]))
    out = torch.zeros((B, 2, LEVEL - depth, S.params.N), dtype=torch.uint64, device="cuda")
    tup = [[G.Tuple(inp[b, u], 2, LEVEL, LEVEL) for u in range(k)] for b in range(B)]
    outs = [G.Tuple(out[b], 2, LEVEL - depth, LEVEL - depth) for b in range(B)]
    ws = S.ws(S.ctx.workspace_size(k, LEVEL, B, part))
    S.ctx.mul_k_batch(tup, S.evk, outs, ws, partition=part)
    S.ctx.check()
    got = host(out)
    for b in range(B):
        want = O.mul_k(S.octx, [oracle_tuple(c) for c in cts[b]], S.okeys, part)
        assert np.array_equal(got[b], want.data), f"batch element {b}"


def test_wave_fixed_shapes(S):
    """Every case in one cross-shape wave: the fixed-shape nodes of the
    tensor stage are grouped into one launch per shape."""
    import torch

    import paper_2601_15401_gb300 as G
    items, wants = [], []
    for i, (k, part, _) in enumerate(CASES):
        cts = _inputs(S, k, 2000 + 50 * i)
        depth = S.ctx.plan_describe(k, part)["depth"]
        out = G.Tuple.wrap(torch.zeros((2, LEVEL - depth, S.params.N), dtype=torch.uint64, device="cuda"))
        items.append(([G.Tuple.wrap(dev(c)) for c in cts], out, part))
        wants.append(O.mul_k(S.octx, [oracle_tuple(c) for c in cts], S.okeys, part).data)
    W = G.Wave(S.ctx, items, S.evk)
    tables, scratch = W.buffers()
    W.run(tables, scratch)
    torch.cuda.synchronize()
    S.ctx.check()
    for i, (_, out, part) in enumerate(items):
        assert np.array_equal(host(out.data)[:, :out.level], wants[i]), CASES[i][:2]
