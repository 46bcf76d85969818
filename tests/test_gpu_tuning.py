"""Parity of every launch shape the autotuner can choose.

The autotuner (executor.autotune) picks NTT column / block tile sizes and
BConv / key-MAC block sizes; these change the NTT's CTA tiling and
shared-memory layout and every kernel's grid. Each value of each tunable,
every (column, block) tile pair at N = 2^16, and the autotuner's own choice
at each N must give the oracle's residues for a batched k = 8 product
(Table II partition (4,4)|(2,2),(2,2): Algorithm 1 at inner nodes, the
relocated rescale at the root) at N = 2^14, 2^15 and 2^16, L = 24, K = 8,
dnum = 3, and the same residues as the library defaults on every batch
element."""
import itertools

import numpy as np
import pytest

import synth
from oracle import ckks as O

from gpu_common import Setup, host, oracle_tuple

pytestmark = pytest.mark.gpu

K_IN = 8
BATCH = 3


class _Case:
    def __init__(self, log_n):
        import torch

        import paper_2601_15401_gb300 as G
        from paper_2601_15401_gb300.executor import TUNE_DEFAULTS
        self.S = Setup(synth.params_large(log_n), K_IN, 3)
        params = self.S.params
        L, N = params.L, params.N
        self.depth = self.S.ctx.plan_describe(K_IN)["depth"]
        self.inp = synth.uniform_residues_torch(params.q, (BATCH, K_IN, 2), N, 0x7E00 + log_n, "cuda")
        self.out = torch.zeros((BATCH, 2, L - self.depth, N), dtype=torch.uint64, device="cuda")
        self.tup = [[G.Tuple(self.inp[b, u], 2, L, L) for u in range(K_IN)] for b in range(BATCH)]
        self.outs = [G.Tuple(self.out[b], 2, L - self.depth, L - self.depth) for b in range(BATCH)]
        self.ws = self.S.ws(self.S.ctx.workspace_size(K_IN, L, BATCH))
        src = host(self.inp[0])
        self.want0 = O.mul_k(self.S.octx, [oracle_tuple(src[u]) for u in range(K_IN)], self.S.okeys).data
        self.defaults = dict(TUNE_DEFAULTS)
        self.apply(self.defaults)
        self.reference = self.run()
        assert np.array_equal(self.reference[0], self.want0)

    def apply(self, choice):
        for n, v in choice.items():
            self.S.ctx.tune_set(n, v)

    def run(self):
        self.out.zero_()
        self.S.ctx.mul_k_batch(self.tup, self.S.evk, self.outs, self.ws)
        self.S.ctx.check()
        return host(self.out)

    def check(self, choice, what):
        self.apply(self.defaults)
        self.apply(choice)
        got = self.run()
        self.apply(self.defaults)
        assert np.array_equal(got[0], self.want0), f"{what}: batch element 0 differs from the oracle"
        assert np.array_equal(got, self.reference), f"{what}: differs from the library defaults"


_cases = {}


@pytest.fixture(scope="module", params=[14, 15, 16])
def case(request):
    if request.param not in _cases:
        _cases.clear()  # one parameter set resident at a time
        _cases[request.param] = _Case(request.param)
    return _cases[request.param]


def _space():
    from paper_2601_15401_gb300.executor import TUNE_SPACE
    return [(n, v) for n, vs in TUNE_SPACE.items() for v in vs]


@pytest.mark.parametrize("name,value", _space())
def test_each_tunable_value_matches_oracle(case, name, value):
    case.check({name: value}, f"{name}={value}")


def test_every_ntt_tile_pair_matches_oracle(case):
    from paper_2601_15401_gb300.executor import TUNE_SPACE
    for cols, blocks in itertools.product(TUNE_SPACE["ntt_tile_cols"], TUNE_SPACE["ntt_tile_blocks"]):
        case.check({"ntt_tile_cols": cols, "ntt_tile_blocks": blocks}, f"tiles {cols}/{blocks}")


def test_autotuner_choice_matches_oracle(case, tmp_path):
    """The autotuner on this GPU (fresh cache): its choice, applied as the
    bench applies it, gives the oracle's residues; a cached entry is reused
    only after the same equality check."""
    from paper_2601_15401_gb300.executor import autotune
    cache = str(tmp_path / "tune.json")
    entry = autotune(case.S.ctx, case.S.evk, k=K_IN, batch=2, reps=1, cache=cache)
    assert entry["rejected"] == []
    case.check(entry["choice"], f"autotuned {entry['choice']}")
    again = autotune(case.S.ctx, case.S.evk, k=K_IN, batch=2, reps=1, cache=cache)
    assert again["choice"] == entry["choice"]
    case.apply(case.defaults)
