"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/ckks_mulk.h declares, and its planner (host C++)
agrees with the partition rules of Section V-C and Table II."""
import ctypes
import os
import re

import pytest

from oracle import plan as oplan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2601_15401_gb300 import build as B
    B.build()
    from paper_2601_15401_gb300._lib import lib
    return lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ckks_mulk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|size_t|const char \*)\s*\*?\s*(ckks_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    from paper_2601_15401_gb300._lib import SIGNATURES
    assert set(names) == set(SIGNATURES)


def test_strerror(L):
    assert L.ckks_strerror(0) == b"ok"
    assert L.ckks_strerror(-4) == b"workspace too small"
    assert b"integrity" in L.ckks_strerror(-8)
    # every code the header defines has its own message
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "ckks_mulk.h")).read()
    codes = [int(v) for v in re.findall(r"#define CKKS_E\w+ \((-\d+)\)", hdr)]
    assert len(codes) >= 8
    for c in codes:
        assert L.ckks_strerror(c) != b"unknown error", c


def _describe(L, k, part):
    h = ctypes.c_void_p()
    rc = L.ckks_plan_create(None, k, part.encode() if part else None, ctypes.byref(h))
    if rc != 0:
        return rc, None
    d, r, n = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    assert L.ckks_plan_describe(h, ctypes.byref(d), ctypes.byref(r), ctypes.byref(n)) == 0
    L.ckks_plan_destroy(h)
    return 0, (d.value, r.value, n.value)


@pytest.mark.parametrize("k", range(2, 13))
def test_default_plans_match_table_ii(L, k):
    rc, (depth, rs, nodes) = _describe(L, k, None)
    assert rc == 0
    root = oplan.parse(oplan.TABLE_II[k], k)
    assert depth == root.depth() == (k - 1).bit_length()
    assert rs == oplan.rs_units(root)


def test_plan_rejections(L):
    assert _describe(L, 6, "(5,1)|(3,2)")[0] == -1      # depth rule (Section V-C)
    assert _describe(L, 6, "(2,2,2)")[0] == 0
    assert _describe(L, 4, "(1,1,1,1)")[0] == -1        # depth 3 > 2
    assert _describe(L, 5, "(2,2)")[0] == -1            # sizes do not add up
    assert _describe(L, 7, "(4,3)|(2,1)")[0] == -1      # no group of 3 split (2,1)? it is valid


@pytest.mark.parametrize("k", range(2, 13))
def test_partition_search_reaches_table_ii_minimum(L, k):
    import paper_2601_15401_gb300 as G
    text, cost = G.plan_optimize(k, "rs_units")
    root = oplan.parse(text, k)
    assert oplan.valid(root, k)
    assert cost == oplan.rs_units(root) == oplan.min_rs_units(k)


def test_transform_cost_matches_table_v_total():
    """Table V: the improved 3-input multiply at dnum = 1, K = L performs
    2L + 2K - 4 NTT and 4L + 2K INTT limb transforms."""
    import ctypes

    import paper_2601_15401_gb300 as G
    from paper_2601_15401_gb300._lib import lib
    for Lq in (4, 12, 24):
        h = ctypes.c_void_p()
        assert lib().ckks_plan_create(None, 3, b"(1,1,1)", ctypes.byref(h)) == 0
        c = ctypes.c_double()
        assert lib().ckks_plan_cost(h, 1, Lq, Lq, Lq, ctypes.byref(c)) == 0
        lib().ckks_plan_destroy(h)
        assert c.value == (2 * Lq + 2 * Lq - 4) + (4 * Lq + 2 * Lq)
    text, cost = G.plan_optimize(3, "transforms", 24, 24, 24)
    assert text == "(1,1,1)" and cost == 6 * 24 + 4 * 24 - 4


def test_transform_search_beats_or_ties_every_table_ii_tree(L):
    import ctypes

    import paper_2601_15401_gb300 as G
    from paper_2601_15401_gb300._lib import lib
    for k in range(2, 13):
        best_text, best = G.plan_optimize(k, "transforms", 24, 8, 8)
        h = ctypes.c_void_p()
        assert lib().ckks_plan_create(None, k, None, ctypes.byref(h)) == 0
        c = ctypes.c_double()
        assert lib().ckks_plan_cost(h, 1, 24, 8, 8, ctypes.byref(c)) == 0
        lib().ckks_plan_destroy(h)
        assert best <= c.value
        assert oplan.valid(oplan.parse(best_text, k), k)


def test_precision_criterion_minimises_inner_degree():
    """Criterion "precision": the chosen tree keeps the depth rule (the
    oracle's parser and checker), its cost carries the largest degree of a
    tuple rescaled below the root, that degree is never above Table II's,
    and it is strictly below it for k = 6 and k = 12."""
    import paper_2601_15401_gb300 as G
    from oracle import plan as P

    def inner_degree(text, k):
        worst = [0]

        def go(n, root):
            if n.is_leaf:
                return 1
            d = sum(go(c, False) for c in n.children)
            if not root:
                worst[0] = max(worst[0], d)
            return d
        go(P.parse(text, k), True)
        return worst[0]

    for k in range(2, 13):
        text, cost = G.plan_optimize(k, "precision", 24, 8, 8)
        assert P.valid(P.parse(text, k), k)
        d = inner_degree(text, k)
        assert int(cost // 1e6) == d
        assert d <= inner_degree(P.TABLE_II[k], k)
    assert inner_degree(G.plan_optimize(12, "precision", 24, 8, 8)[0], 12) == 4
    assert inner_degree(G.plan_optimize(6, "precision", 24, 8, 8)[0], 6) == 2


def test_workload_primes_and_peak_form_check(L):
    """The named workloads take the prime chain of the default reading (the
    largest primes below 2^b that are 1 mod 2^17), or with
    congruence=Q1_CONGRUENCE primes = 1 (mod 2^32), the form the kernels'
    cheaper modular products need (q = h 2^32 + 1 stays NTT-friendly for
    every N <= 2^31). The integer-peak entry point rejects the cheaper-form
    kinds for any other prime before it launches anything."""
    import synth
    for f in (synth.params_small, synth.params_mid, synth.params_large):
        chain, q1 = f(), f(congruence=synth.Q1_CONGRUENCE)
        for params, m in ((chain, synth.NTT_CONGRUENCE), (q1, synth.Q1_CONGRUENCE)):
            for x in params.q + params.p:
                assert x % m == 1 and synth.is_prime(x)
                assert (x - 1) % (2 * params.N) == 0
            assert len(set(params.q + params.p)) == params.L + params.K
        # the default chain is the largest such primes, so it is not the q1 one
        assert any(x % synth.Q1_CONGRUENCE != 1 for x in chain.q + chain.p)
        assert [x.bit_length() for x in chain.q] == [x.bit_length() for x in q1.q]
    general = synth.make_params(10, [50] * 4, 1, 1)
    chains = L.ckks_peak_chains()
    w = (ctypes.c_uint64 * chains)(*([1] * chains))
    q = general.q[0]
    assert q % synth.Q1_CONGRUENCE != 1
    for kind in (6, 7):
        assert L.ckks_peak_int(kind, q, w, w, 1, 32, 1, ctypes.c_void_p(8), None) == -1
