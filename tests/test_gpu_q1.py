"""The two forms of the modular products.

With every prime = 1 (mod 2^32) the kernels take cheaper forms of the Shoup
product and of Montgomery reduction (the quotient product and q^-1 reduce
to 32-bit multiplies); with other primes, or with the tunable "q1_forms" set
to 0, they take the general forms. Both must give the oracle's residues
(Section V: Table II partitions, Algorithm 1 at inner nodes, Eq. 15, the
relocated root rescale), and the same residues as each other, at the ring
degrees where the specialised NTT kernels run (N = 2^14 .. 2^16) and below
(N = 2^10: generic NTT kernels, the tensor / BConv / key-MAC kernels in the
cheaper form)."""
import numpy as np
import pytest

import synth
from oracle import ckks as O

from gpu_common import Setup, host, oracle_tuple

pytestmark = pytest.mark.gpu

BATCH = 2


def _product(S, k, seed):
    """Batched k-input product at the top level under both forms; returns
    (cheaper-form output, general-form output, oracle output of element 0)."""
    import torch

    import paper_2601_15401_gb300 as G
    params = S.params
    L, N = params.L, params.N
    depth = S.ctx.plan_describe(k)["depth"]
    inp = synth.uniform_residues_torch(params.q, (BATCH, k, 2), N, seed, "cuda")
    out = torch.zeros((BATCH, 2, L - depth, N), dtype=torch.uint64, device="cuda")
    tup = [[G.Tuple(inp[b, u], 2, L, L) for u in range(k)] for b in range(BATCH)]
    outs = [G.Tuple(out[b], 2, L - depth, L - depth) for b in range(BATCH)]
    ws = S.ws(S.ctx.workspace_size(k, L, BATCH))
    got = {}
    for form in (1, 0):
        S.ctx.tune_set("q1_forms", form)
        out.zero_()
        S.ctx.mul_k_batch(tup, S.evk, outs, ws)
        S.ctx.check()
        got[form] = host(out)
    S.ctx.tune_set("q1_forms", 1)
    src = host(inp[0])
    want = O.mul_k(S.octx, [oracle_tuple(src[u]) for u in range(k)], S.okeys).data
    return got[1], got[0], want


@pytest.mark.parametrize("log_n,ks", [(10, (2, 3, 5, 8, 12)), (14, (3, 12)), (16, (4, 9))])
def test_cheaper_forms_match_oracle_and_general_forms(log_n, ks):
    S = Setup(synth.params_large(log_n, congruence=synth.Q1_CONGRUENCE), max(ks), 7)
    for k in ks:
        cheap, general, want = _product(S, k, 0x9100 + 16 * log_n + k)
        assert np.array_equal(cheap[0], want), f"N=2^{log_n} k={k}: cheaper forms differ from the oracle"
        assert np.array_equal(cheap, general), f"N=2^{log_n} k={k}: the two forms differ"


@pytest.mark.parametrize("log_n,k", [(14, 7), (16, 12)])
def test_general_primes_full_parameter_set(log_n, k):
    """The default prime chain (= 1 mod 2^17 only): the specialised NTT
    kernels in the general form at the bench's parameter shape."""
    params = synth.params_large(log_n)
    assert any(x % synth.Q1_CONGRUENCE != 1 for x in params.q + params.p)
    S = Setup(params, k, 8)
    cheap, general, want = _product(S, k, 0x9200 + 16 * log_n + k)
    assert np.array_equal(general[0], want)
    assert np.array_equal(cheap, general)  # q1_forms has no effect on such primes
