"""SCC-compositional route to the prime paths (TEST INFRASTRUCTURE).

A second, independent route to the PP set of a CFG, written from the
compositional method the paper outlines in Sec. 2.1 (Defs. 3-11 and the
worked example of Fig. 1/Fig. 2): (1) the strongly connected components
and their component graph (Def. 3, CCFG); (2) the PPs of every SCC
(SccInternalPPs, Def. 9); (3) path extraction per SCC: SccEntryExitPaths
(Def. 6), SccExitPaths (Def. 7) and SccEntryPaths (Def. 8); (4) merging
along the component DAG into the PPs that cross SCCs (CompletePPs Def. 2,
SccExitPPs Def. 10, SccEntryPPs Def. 11, and, in general CFGs, PPs that
start in one SCC and end in another).

Readings (the section describes the method through its worked example; its
extraction and merging algorithms are those of an earlier work it cites):
* A PP that leaves an SCC never returns to it (the component graph is a
  DAG), so a PP crossing SCCs C1 -> ... -> Cm is a concatenation
  x1 . y2 ... y(m-1) . zm of simple paths inside each SCC joined by arcs.
* Its inner parts y are entry-exit paths: any acyclic simple path of the
  SCC from an SccEntryVertex to an SccExitVertex (Def. 6; in the worked
  example <2> and <2,3,5>).
* Its first part x is an exit path whose first vertex has every predecessor
  (in G) on x: then no vertex can be prepended.  This is the maximality
  Def. 7 asks for, read so that the concatenation is a PP (on the worked
  example it gives exactly the four printed SccExitPaths).
* Its last part z is an entry path whose last vertex has every successor
  on z (the maximality of Def. 8; the two printed SccEntryPaths).
* The Start vertex and the End vertex form one-vertex SCCs whose only
  part is <Start> (no predecessors) or <End> (no successors).
* SccInternalPPs (Def. 9) are the PPs of the SCC's own subgraph that are
  cycles, or acyclic and neither start at an SccEntryVertex nor end at an
  SccExitVertex.
Every PP of G lies inside one SCC or crosses SCCs as above, and every such
concatenation is a PP of G (no vertex can be added at either end), so the
union equals the set of Def. 1.  Plain Python, for small graphs.
"""
from __future__ import annotations


def succ_lists(n, row_ptr, col):
    return [[int(x) for x in col[row_ptr[v]:row_ptr[v + 1]]] for v in range(n)]


def pred_lists(n, succ):
    pred = [[] for _ in range(n)]
    for u in range(n):
        for w in succ[u]:
            pred[w].append(u)
    return pred


def sccs(n, succ):
    """Tarjan's algorithm (iterative): component id of every vertex, ids in
    reverse topological order of the component graph."""
    index = [-1] * n
    low = [0] * n
    onstack = [False] * n
    comp = [-1] * n
    stack, counter, ncomp = [], 0, 0
    for root in range(n):
        if index[root] >= 0:
            continue
        work = [(root, 0)]
        while work:
            v, i = work.pop()
            if i == 0:
                index[v] = low[v] = counter
                counter += 1
                stack.append(v)
                onstack[v] = True
            recurse = False
            while i < len(succ[v]):
                w = succ[v][i]
                i += 1
                if index[w] < 0:
                    work.append((v, i))
                    work.append((w, 0))
                    recurse = True
                    break
                if onstack[w]:
                    low[v] = min(low[v], index[w])
            if recurse:
                continue
            if low[v] == index[v]:
                while True:
                    w = stack.pop()
                    onstack[w] = False
                    comp[w] = ncomp
                    if w == v:
                        break
                ncomp += 1
            if work:
                u = work[-1][0]
                low[u] = min(low[u], low[v])
    return comp, ncomp


def _simple_paths_within(vs, succ, comp, c):
    """Every simple path of the subgraph of SCC c (vertex set vs): acyclic
    paths and closed cycles, as tuples."""
    out = []
    for r in sorted(vs):
        stack = [(r,)]
        while stack:
            p = stack.pop()
            out.append(p)
            if len(p) >= 2 and p[0] == p[-1]:
                continue
            for w in reversed(succ[p[-1]]):
                if comp[w] != c:
                    continue
                if w == p[0] or w not in p:
                    stack.append(p + (w,))
    return out


def decompose(n, row_ptr, col):
    """The intermediate results of the compositional method, per SCC."""
    succ = succ_lists(n, row_ptr, col)
    pred = pred_lists(n, succ)
    comp, ncomp = sccs(n, succ)
    members = [[] for _ in range(ncomp)]
    for v in range(n):
        members[comp[v]].append(v)
    entry = [v for v in range(n) if any(comp[u] != comp[v] for u in pred[v])]
    exitv = [v for v in range(n) if any(comp[w] != comp[v] for w in succ[v])]
    is_entry, is_exit = set(entry), set(exitv)
    parts = []
    for c in range(ncomp):
        vs = members[c]
        paths = _simple_paths_within(vs, succ, comp, c)
        cyc = [p for p in paths if len(p) >= 2 and p[0] == p[-1]]
        acyc = [p for p in paths if not (len(p) >= 2 and p[0] == p[-1])]
        # PPs of the SCC's subgraph: simple paths with no simple one-vertex
        # extension inside the subgraph (Def. 1 on the subgraph)
        def extends(p):
            if len(p) >= 2 and p[0] == p[-1]:
                return False
            for w in succ[p[-1]]:
                if comp[w] == c and (w == p[0] or w not in p):
                    return True
            for u in pred[p[0]]:
                if comp[u] == c and (u == p[-1] or u not in p):
                    return True
            return False
        scc_pps = [p for p in paths if not extends(p)]
        internal = [p for p in scc_pps if (len(p) >= 2 and p[0] == p[-1])
                    or (p[0] not in is_entry and p[-1] not in is_exit)]
        entry_exit = [p for p in acyc if p[0] in is_entry and p[-1] in is_exit]
        exit_paths = [p for p in acyc if p[-1] in is_exit and all(u in p for u in pred[p[0]])]
        entry_paths = [p for p in acyc if p[0] in is_entry and all(w in p for w in succ[p[-1]])]
        parts.append({"vertices": vs, "internal": sorted(internal), "entry_exit": sorted(entry_exit),
                      "exit_paths": sorted(exit_paths), "entry_paths": sorted(entry_paths),
                      "cycles": len(cyc)})
    return {"succ": succ, "pred": pred, "comp": comp, "ncomp": ncomp, "entry": entry, "exit": exitv,
            "parts": parts}


def merge(d):
    """PPs crossing SCCs: an exit path, then entry-exit paths of the SCCs
    after it, then an entry path, consecutive parts joined by arcs."""
    succ, comp, parts = d["succ"], d["comp"], d["parts"]
    by_start = {}
    for c, pt in enumerate(parts):
        for p in pt["entry_exit"]:
            by_start.setdefault(("ee", p[0]), []).append(p)
        for p in pt["entry_paths"]:
            by_start.setdefault(("en", p[0]), []).append(p)
    out = []
    stack = [p for pt in parts for p in pt["exit_paths"]]
    while stack:
        q = stack.pop()
        x = q[-1]
        for y in succ[x]:
            if comp[y] == comp[x]:
                continue
            for z in by_start.get(("en", y), []):
                out.append(q + z)
            for z in by_start.get(("ee", y), []):
                stack.append(q + z)
    return sorted(out)


def prime_paths(n, row_ptr, col):
    """All PPs of the graph by the compositional route, canonical order."""
    d = decompose(n, row_ptr, col)
    internal = [p for pt in d["parts"] for p in pt["internal"]]
    return sorted(set(internal) | set(merge(d)))


def ccfg_prime_paths(d):
    """PPs of the component graph (a DAG) as component-id sequences: the
    maximal paths from a component without predecessors to one without
    successors."""
    comp, succ, nc = d["comp"], d["succ"], d["ncomp"]
    csucc = [set() for _ in range(nc)]
    cpred = [set() for _ in range(nc)]
    for u in range(len(succ)):
        for w in succ[u]:
            if comp[u] != comp[w]:
                csucc[comp[u]].add(comp[w])
                cpred[comp[w]].add(comp[u])
    out = []
    stack = [(c,) for c in range(nc) if not cpred[c]]
    while stack:
        p = stack.pop()
        nxt = sorted(csucc[p[-1]])
        if not nxt:
            out.append(p)
        for c in nxt:
            stack.append(p + (c,))
    return out
