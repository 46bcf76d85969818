"""Failure detection without a GPU fault: the residue-range check, the
checking mode of the k-input product (CKKS_ECHECK on a residue >= q in an
input or after any stage) and the checksum of resident evaluation keys
(a changed key word is reported). Faults are made on the host side, by
writing a bad value into a buffer the test owns."""
import numpy as np
import pytest
import torch

import synth
from oracle import ckks as O

from gpu_common import Setup, dev, host, oracle_tuple

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return Setup(synth.make_params(6, [50] * 6, 2, 2), 5, 401)


def _cts(S, k, level, seed):
    return [synth.uniform_tuple(S.params, 2, level, seed, i) for i in range(k)]


def _mul(S, arrs, level, check=False):
    import paper_2601_15401_gb300 as G
    k = len(arrs)
    depth = S.ctx.plan_describe(k)["depth"]
    out = G.Tuple.wrap(dev(np.zeros((2, level - depth, S.params.N), dtype=np.uint64)))
    ws = S.ws(S.ctx.workspace_size(k, level, 1))
    S.ctx.tune_set("check_residues", int(check))
    try:
        S.ctx.mul_k([G.Tuple.wrap(dev(a)) for a in arrs], S.evk, out, ws)
    finally:
        S.ctx.tune_set("check_residues", 0)
    return host(out.data)


def test_check_residues_counts_out_of_range(S):
    import paper_2601_15401_gb300 as G
    a = synth.uniform_tuple(S.params, 3, 6, 402, 0)
    t = G.Tuple.wrap(dev(a))
    assert S.ctx.check_residues(t) == 0
    q = S.params.q
    v = t.data.view(torch.int64)      # same bits; plain int64 element writes
    v[1, 2, 7] = q[2]                 # exactly q: out of range
    v[2, 5, 0] = q[5] + 12345
    v[0, 0, 3] = q[0] - 1             # in range
    assert S.ctx.check_residues(t) == 2
    assert S.ctx.check_residues(G.Tuple(t.data, 3, 2, 6)) == 0  # limbs 2, 5 not active at level 2


@pytest.mark.parametrize("k", [3, 5])
def test_checking_mode_passes_valid_products_unchanged(S, k):
    arrs = _cts(S, k, 6, 403 + k)
    plain = _mul(S, arrs, 6)
    checked = _mul(S, arrs, 6, check=True)
    assert np.array_equal(plain, checked)
    want = O.mul_k(S.octx, [oracle_tuple(a) for a in arrs], S.okeys)
    assert np.array_equal(checked[:, :want.level], want.data)


def test_checking_mode_reports_a_bad_input(S):
    import paper_2601_15401_gb300 as G
    arrs = _cts(S, 3, 6, 405)
    arrs[1][0, 3, 11] = S.params.q[3]
    with pytest.raises(G.CkksError) as e:
        _mul(S, arrs, 6, check=True)
    assert e.value.code == -8
    S.ctx.check()                      # the context stays usable
    arrs[1][0, 3, 11] = 0
    assert np.array_equal(_mul(S, arrs, 6, check=True), _mul(S, arrs, 6))


def test_evk_checksum_detects_a_changed_key_word(S):
    assert S.evk.verify()
    flat = S.evk.keys.view(torch.int64).view(-1)
    i = flat.numel() // 2 + 3
    old = flat[i].clone()
    flat[i] = old ^ 1
    assert not S.evk.verify()
    flat[i] = old
    assert S.evk.verify()


def test_nvtx_ranges_do_not_change_results(S):
    arrs = _cts(S, 4, 6, 406)
    base = _mul(S, arrs, 6)
    S.ctx.tune_set("nvtx", 1)
    try:
        ranged = _mul(S, arrs, 6)
    finally:
        S.ctx.tune_set("nvtx", 0)
    assert np.array_equal(base, ranged)
