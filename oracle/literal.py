"""Literal quadratic oracle for tiny graphs (TEST INFRASTRUCTURE).

Applies the paper's definitions word for word, with no lemma in between:

* Sec. 2: a simple path is a vertex sequence v1..vk (k > 0) whose consecutive
  pairs are arcs and in which no vertex repeats unless v1 = vk (read as: the
  only coincidence allowed is first = last, so v1..v(k-1) are distinct and
  v2..vk are distinct).
* Def. 1 / Sec. 7.2: a prime path is a simple path that is not a proper
  subpath of any other simple path.

Every walk of up to n+1 vertices is generated, the simple ones kept, and each
is tested against every other for being a contiguous proper subsequence:
O(S^2 L) for S simple paths.  Only for graphs of a handful of vertices.
"""
from __future__ import annotations


def is_simple(seq) -> bool:
    k = len(seq)
    if k == 0:
        return False
    head, tail = seq[:-1], seq[1:]
    return len(set(head)) == len(head) and len(set(tail)) == len(tail)


def simple_paths(n, succ):
    """All simple paths as tuples; succ[v] is an iterable of successors."""
    out = []
    frontier = [(v,) for v in range(n)]
    while frontier:
        nxt = []
        for w in frontier:
            if is_simple(w):
                out.append(w)
                if len(w) <= n:
                    for x in succ[w[-1]]:
                        nxt.append(w + (x,))
        frontier = nxt
    return out


def is_proper_subpath(p, q) -> bool:
    lp, lq = len(p), len(q)
    if lp >= lq:
        return False
    return any(q[i:i + lp] == p for i in range(lq - lp + 1))


def prime_paths(n, succ):
    sp = simple_paths(n, succ)
    pps = [p for p in sp if not any(is_proper_subpath(p, q) for q in sp)]
    return sorted(set(pps))


def succ_lists(n, row_ptr, col):
    return [[int(x) for x in col[row_ptr[v]:row_ptr[v + 1]]] for v in range(n)]
