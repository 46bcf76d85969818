"""Input partitions of a k-input multiplication (Section V-C, Table II).

Test infrastructure only (see the package docstring).

A partition tree has the k input ciphertexts as leaves. A node that multiplies
m children rescales its product m - 1 times (one combined multi-rescale,
Algorithm 1) unless it is the root, whose rescale is deferred until after
relinearisation. Along any leaf-to-root path the rescales add up; the tree is
valid when the largest sum is at most ceil(log2 k) (the depth rule of
Section V-C).

Notation (Table II): layers separated by '|', groups within a layer by ','.
"(4,3)|(2,2)" splits 7 inputs into groups of 4 and 3; the next layer splits
the group of 4 into (2,2); the group of 3 is multiplied directly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache


@dataclass
class Node:
    size: int                      # number of input ciphertexts below
    children: list = field(default_factory=list)

    @property
    def is_leaf(self) -> bool:
        return self.size == 1 and not self.children

    def depth(self) -> int:
        """Rescales along the longest path below and at this node."""
        if self.is_leaf:
            return 0
        return (len(self.children) - 1) + max(c.depth() for c in self.children)


def _groups(text: str) -> list[list[int]]:
    out = []
    for part in text.replace(" ", "").split("),("):
        part = part.strip("()")
        out.append([int(x) for x in part.split(",") if x])
    return out


def parse(partition: str, k: int) -> Node:
    """Build the tree. Each sub-partition of a layer is given, left to right,
    to the next not-yet-split group of the layer above whose size equals the
    sub-partition's sum. Groups never split become nodes over that many leaves
    (a group of one is the input ciphertext itself)."""
    layers = [_groups(x) for x in partition.split("|")]
    if len(layers[0]) != 1:
        raise ValueError("first layer must be a single group list")
    root = Node(k, [Node(s) for s in layers[0][0]])
    if sum(layers[0][0]) != k or len(layers[0][0]) < 2:
        raise ValueError("first layer must split k into at least 2 groups")
    frontier = list(root.children)
    for layer in layers[1:]:
        nxt = []
        used = set()
        for sub in layer:
            for idx, g in enumerate(frontier):
                if idx not in used and g.size == sum(sub) and len(sub) >= 2:
                    used.add(idx)
                    g.children = [Node(s) for s in sub]
                    nxt.extend(g.children)
                    break
            else:
                raise ValueError(f"no group of size {sum(sub)} for {sub}")
        frontier = nxt
    _expand(root)
    return root


def _expand(node: Node):
    """An undivided group of size g >= 2 multiplies g leaves."""
    if node.size >= 2 and not node.children:
        node.children = [Node(1) for _ in range(node.size)]
    for c in node.children:
        _expand(c)


def valid(root: Node, k: int) -> bool:
    return root.depth() <= math.ceil(math.log2(k))


def rs_units(root: Node) -> int:
    """Rescale units below the root (Table II, first number): a non-root node
    over g inputs outputs g + 1 polynomials, each through one (multi-)rescale
    unit. The root adds two more (its two output polynomials), not counted."""
    def cost(n: Node) -> int:
        if n.is_leaf:
            return 0
        return (n.size + 1) + sum(cost(c) for c in n.children)
    return sum(cost(c) for c in root.children)


def binary_partition(k: int) -> Node:
    """The binary tree of 2-input multiplies of Table II's baseline column:
    split n into the largest power of two below n and the rest, recursively."""
    def build(n: int) -> Node:
        if n == 1:
            return Node(1)
        if n == 2:
            return Node(2, [Node(1), Node(1)])
        a = 1 << (n - 1).bit_length() - 1
        return Node(n, [build(a), build(n - a)])
    return build(k)


def _compositions(n: int, m: int, max_part: int):
    """Non-increasing partitions of n into exactly m parts, each <= max_part."""
    if m == 1:
        if 1 <= n <= max_part:
            yield (n,)
        return
    for first in range(min(n - (m - 1), max_part), 0, -1):
        for rest in _compositions(n - first, m - 1, first):
            yield (first,) + rest


@lru_cache(maxsize=None)
def _best_node(g: int, budget: int) -> int:
    """Fewest rescale units for a non-root node over g inputs whose depth must
    not exceed budget (infinite if impossible)."""
    if g == 1:
        return 0
    best = math.inf
    for m in range(2, g + 1):
        if m - 1 > budget:
            break
        for parts in _compositions(g, m, g):
            c = sum(_best_node(p, budget - (m - 1)) for p in parts)
            best = min(best, c)
    return (g + 1) + best if best < math.inf else math.inf


def min_rs_units(k: int) -> int:
    """Exhaustive minimum of rs_units over valid partitions of k inputs."""
    D = math.ceil(math.log2(k))
    best = math.inf
    for m in range(2, k + 1):
        if m - 1 > D:
            break
        for parts in _compositions(k, m, k):
            best = min(best, sum(_best_node(p, D - (m - 1)) for p in parts))
    return best


# Table II, "Proposed Optimized Partition" column (the default trees).
TABLE_II = {
    2: "(1,1)",
    3: "(1,1,1)",
    4: "(2,2)",
    5: "(2,2,1)",
    6: "(3,3)",
    7: "(4,3)|(2,2)",
    8: "(4,4)|(2,2),(2,2)",
    9: "(3,3,3)",
    10: "(3,3,4)|(2,2)",
    11: "(4,4,3)|(2,2),(2,2)",
    12: "(6,6)|(3,3),(3,3)",
}
