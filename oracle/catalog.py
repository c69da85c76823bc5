"""Treelet catalogue of the oracle (test infrastructure only).

Rooted treelet shapes on h <= 8 nodes, their bitstring encoding s_T, the
canonical decomposition T -> (T', T'') with its multiplicity beta_T, and the
unrooted shape of each rooting.

* s_T (Section 3.2.1): a DFS from the root writes
  1 for every edge walked away from the root and 0 for every edge walked
  back; the children of a node are visited in the order of their own
  encodings.  The worked example of Figure 1 (root with a two-child subtree
  and a leaf, s_T = 11010010) fixes the direction: the larger child string
  comes first, i.e. children are visited in *decreasing* lexicographic
  order.  Shape ids within a size are ranks of s_T read as a 2(h-1)-bit
  unsigned integer, most significant bit first, ascending.
* Decomposition (Eq. 1, and the merge of Section 3.2.1, which writes a 1,
  then s_T'', then s_T'): T'' is the subtree of the
  root's first (largest) child and T' is T with that subtree removed;
  beta_T is the number of root children whose subtree equals T''.
* Unrooted shapes: the code of an unrooted tree is the smallest s_T over all
  of its rootings; unrooted ids within a size ascend with that code.
* Round skipping (Section 3.3.2): level k uses a balanced decomposition in
  which both parts have at most k-2 nodes, so level k-1 is never needed;
  rooted k-shapes without one (every star rooting, every leaf rooting) are
  not counted.

Trees are handled as strings over {0,1} throughout; this is slow and plain
on purpose.
"""
from __future__ import annotations

from functools import lru_cache

MAX_K = 8


def _split_children(s: str) -> list[str]:
    """Split the encoding of a rooted tree into the encodings '1'+child+'0'
    of the root's child subtrees, in the order they appear."""
    out, depth, start = [], 0, 0
    for i, ch in enumerate(s):
        depth += 1 if ch == "1" else -1
        if depth == 0:
            out.append(s[start:i + 1])
            start = i + 1
    return out


def canonical_from_children(child_strings: list[str]) -> str:
    """Encoding of a root whose children have the given (canonical) encodings."""
    return "".join("1" + c + "0" for c in sorted(child_strings, reverse=True))


def encode(adj: dict[int, list[int]], root: int) -> str:
    """Canonical s_T of the tree given by an adjacency dict, rooted at root."""
    def rec(v: int, parent: int) -> str:
        return canonical_from_children([rec(u, v) for u in adj[v] if u != parent])
    return rec(root, -1)


def decode(s: str) -> dict[int, list[int]]:
    """Adjacency dict of the tree with encoding s; node 0 is the root and the
    other nodes are numbered in DFS order."""
    adj: dict[int, list[int]] = {0: []}
    stack, nxt = [0], 1
    for ch in s:
        if ch == "1":
            adj[nxt] = [stack[-1]]
            adj[stack[-1]].append(nxt)
            stack.append(nxt)
            nxt += 1
        else:
            stack.pop()
    return adj


@lru_cache(maxsize=None)
def rooted_shapes(h: int) -> tuple[str, ...]:
    """All rooted shapes on h nodes, as s_T strings, sorted by shape id."""
    if h == 1:
        return ("",)
    found = set()
    for s in rooted_shapes(h - 1):
        adj = decode(s)
        for v in list(adj):  # hang a new leaf under every node
            a2 = {x: list(y) for x, y in adj.items()}
            a2[h - 1] = [v]
            a2[v].append(h - 1)
            found.add(encode(a2, 0))
    return tuple(sorted(found, key=lambda x: int(x, 2)))


def shape_id(s: str) -> int:
    return rooted_shapes(len(s) // 2 + 1).index(s)


def decompose(s: str) -> tuple[str, str, int]:
    """(s_T', s_T'', beta_T) for a rooted shape with at least 2 nodes."""
    kids = _split_children(s)
    first = kids[0]
    beta = sum(1 for c in kids if c == first)
    return "".join(kids[1:]), first[1:-1], beta


def balanced_decompose(s: str, k: int):
    """Balanced decomposition used when round k-1 is skipped (Section 3.3.2):
    T'' is the subtree of the first root child, in the order the children
    appear in s_T, whose size is between 2 and k-2; T' is T without that
    subtree, and beta_T counts the root children whose subtree equals T''.
    Returns (s_T', s_T'', beta_T), or None when no root child qualifies --
    such rooted shapes are not counted at level k."""
    kids = _split_children(s)
    for c in kids:
        if 2 <= len(c) // 2 <= k - 2:
            rest = list(kids)
            rest.remove(c)
            return "".join(rest), c[1:-1], kids.count(c)
    return None


def balanced_rootings(code: int, h: int) -> int:
    """a_j: the number of nodes x of the unrooted h-tree with this code such
    that the tree rooted at x has a balanced decomposition (h = k)."""
    s = format(code, "0%db" % (2 * (h - 1))) if h > 1 else ""
    adj = decode(s)
    return sum(1 for x in adj if balanced_decompose(encode(adj, x), h) is not None)


def unrooted_code(s: str) -> int:
    adj = decode(s)
    return min(int(encode(adj, r), 2) if len(adj) > 1 else 0 for r in adj)


@lru_cache(maxsize=None)
def unrooted_shapes(h: int) -> tuple[int, ...]:
    """Sorted unrooted codes of the trees on h nodes."""
    return tuple(sorted({unrooted_code(s) for s in rooted_shapes(h)}))


def unrooted_id(s: str) -> int:
    return unrooted_shapes(len(s) // 2 + 1).index(unrooted_code(s))


def root_automorphisms(s: str) -> int:
    """Number of automorphisms of the rooted tree that fix the root."""
    kids = _split_children(s)
    out = 1
    for c in set(kids):
        mult = kids.count(c)
        f = 1
        for i in range(2, mult + 1):
            f *= i
        out *= f * root_automorphisms(c[1:-1]) ** mult
    return out


def tree_automorphisms(s: str) -> int:
    """Automorphisms of the unrooted tree (orbit-stabiliser over rootings)."""
    adj = decode(s)
    orbit = sum(1 for r in adj if encode(adj, r) == s)
    return root_automorphisms(s) * orbit


class Catalog:
    """Flattened catalogue for k colours: global shape ids run over sizes
    1..k, each size block in shape-id order."""

    def __init__(self, k: int, skip_round: bool = False):
        if not 1 <= k <= MAX_K:
            raise ValueError("k must be in 1..8")
        self.k = k
        self.skip_round = skip_round
        self.strings: list[str] = []
        self.size: list[int] = []
        self.local: list[int] = []
        self.first = [0] * (k + 2)
        for h in range(1, k + 1):
            self.first[h] = len(self.strings)
            for i, s in enumerate(rooted_shapes(h)):
                self.strings.append(s)
                self.size.append(h)
                self.local.append(i)
        self.first[k + 1] = len(self.strings)
        gid = {(self.size[g], self.strings[g]): g for g in range(len(self.strings))}
        self.left, self.right, self.beta, self.unrooted = [], [], [], []
        for g, s in enumerate(self.strings):
            h = self.size[g]
            self.unrooted.append(unrooted_id(s))
            if h == 1:
                self.left.append(-1)
                self.right.append(-1)
                self.beta.append(1)
                continue
            if skip_round and h == k:
                d = balanced_decompose(s, k)
                if d is None:  # not counted at level k: no decomposition
                    self.left.append(-1)
                    self.right.append(-1)
                    self.beta.append(1)
                    continue
                a, b, beta = d
            else:
                a, b, beta = decompose(s)
            self.left.append(gid[(len(a) // 2 + 1, a)])
            self.right.append(gid[(len(b) // 2 + 1, b)])
            self.beta.append(beta)

    def copies_divisor(self, h: int) -> list[int]:
        """Per unrooted shape of size h: how many rooted copies the level-h
        table holds for each copy of the tree -- h (one per node), or, at
        level k with round skipping, a_j (0 for the star, not counted)."""
        codes = unrooted_shapes(h)
        if self.skip_round and h == self.k:
            return [balanced_rootings(c, h) for c in codes]
        return [h] * len(codes)

    def r(self, h: int) -> int:
        return self.first[h + 1] - self.first[h]

    def n_unrooted(self, h: int) -> int:
        return len(unrooted_shapes(h))
