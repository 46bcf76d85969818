"""Which tree nodes the fixed-shape tensor kernels serve (host only).

A node over g inputs outputs a tuple of g + 1 terms, so a node whose
children cover (g_1, .., g_m) inputs multiplies tuples of g_i + 1 terms. The
library compiles kernels for two children of 4..7 terms and three of 4 or 5
terms, except two children of 6 and 4 terms, which it says no tree within
the depth rule of Section V-C contains for k <= 16. These tests check both
claims from the depth rule alone (a node with m children adds m - 1
rescales; a tree is valid when its deepest path has at most ceil(log2 k)),
and that every compiled shape is the root of the partition the GPU tests
use for it."""
import functools
import itertools
import math

from oracle import plan as OP

# sorted child term counts of the compiled shapes
FIXED = [(a, b) for a in range(4, 8) for b in range(4, a + 1) if (a, b) != (6, 4)] + \
    [(4, 4, 4), (5, 4, 4), (5, 5, 4), (5, 5, 5)]

# the partitions tests/test_gpu_tensor_fixed.py runs, one per shape
GPU_CASES = {
    (4, 4): (6, "(3,3)"), (5, 4): (7, "(4,3)|(2,2)"), (5, 5): (8, "(4,4)|(2,2),(2,2)"),
    (6, 5): (9, "(5,4)|(3,2),(2,2)"), (6, 6): (10, "(5,5)|(3,2),(3,2)"), (7, 4): (9, "(6,3)|(3,3)"),
    (7, 5): (10, "(6,4)|(3,3),(2,2)"), (7, 6): (11, "(6,5)|(3,3),(3,2)"), (7, 7): (12, "(6,6)|(3,3),(3,3)"),
    (4, 4, 4): (9, "(3,3,3)"), (5, 4, 4): (10, "(4,3,3)|(2,2)"), (5, 5, 4): (11, "(4,4,3)|(2,2),(2,2)"),
    (5, 5, 5): (12, "(4,4,4)|(2,2),(2,2),(2,2)"),
}


@functools.lru_cache(maxsize=None)
def min_depth(g: int) -> int:
    """Fewest rescales along the deepest path of any tree over g inputs."""
    if g == 1:
        return 0
    best = math.inf
    for m in range(2, g + 1):
        for parts in _compositions(g, m):
            best = min(best, (m - 1) + max(min_depth(p) for p in parts))
    return best


def _compositions(n: int, m: int):
    if m == 1:
        yield (n,)
        return
    for first in range(1, n - m + 2):
        for rest in _compositions(n - first, m - 1):
            yield (first,) + rest


def node_reachable(inputs: tuple, k_max: int) -> bool:
    """Some valid tree for some k <= k_max has a node whose children cover
    these input counts (each child at its least depth): the node as the
    root, or as one child of a two-child root (deeper ancestor chains only
    add rescales)."""
    own = (len(inputs) - 1) + max(min_depth(g) for g in inputs)
    g = sum(inputs)
    for k in range(g, k_max + 1):
        budget = math.ceil(math.log2(k))
        if k == g:
            if own <= budget:
                return True
            continue
        # below a root of two children (this node and a tree over the other
        # k - g inputs): the least depth any ancestor chain can add
        if 1 + max(own, min_depth(k - g)) <= budget:
            return True
    return False


def test_min_depth_small_cases():
    # (2,2) for 4, (3,2) / (2,2,1) for 5, (3,3) for 6, (4,4) for 8, 9 needs 4
    assert [min_depth(g) for g in range(1, 10)] == [0, 1, 2, 2, 3, 3, 3, 3, 4]
    assert all(min_depth(k) <= math.ceil(math.log2(k)) for k in range(2, 17))


def test_every_fixed_shape_occurs_in_a_valid_tree():
    for shape in FIXED:
        assert node_reachable(tuple(t - 1 for t in shape), 12), shape


def test_the_excluded_shape_occurs_in_no_valid_tree():
    # two children of 6 and 4 terms cover 5 and 3 inputs
    assert not node_reachable((5, 3), 16)
    # every other pair of multi-term children up to 7 terms does occur
    for a, b in itertools.product(range(4, 8), repeat=2):
        if a >= b and (a, b) != (6, 4):
            assert node_reachable((a - 1, b - 1), 12), (a, b)


def test_gpu_cases_are_valid_trees_with_that_root():
    assert sorted(GPU_CASES) == sorted(FIXED)
    for shape, (k, part) in GPU_CASES.items():
        root = OP.parse(part, k)
        assert OP.valid(root, k), part
        assert tuple(sorted((c.size + 1 for c in root.children), reverse=True)) == shape, part
