"""The SCC-compositional route (Sec. 2.1, Defs. 3-11) as a second oracle.

Pinned against what the paper prints for its worked example (Fig. 1, the
CFG of binarySearch0): the CCFG's two PPs, the 11 SccInternalPPs, the
extracted SccEntryExitPaths, SccExitPaths and SccEntryPaths, and the
merged CompletePPs, SccExitPPs and SccEntryPPs, 19 PPs in all.  Then its
union must equal the direct oracle's PP set (Def. 1) on many graphs, and
the GPU's (gpu-marked test).
"""
import numpy as np
import pytest

import oracle
from oracle import compositional as C
from paper_2210_16998_gb300 import cfggen as G

from .helpers import wrap_digraph
from .test_oracle import fig1_cfg, load_fig1

START, END = 0, 10


def _sets(rows, kind):
    return sorted(p for k, p in rows if k == kind)


def test_worked_example_extraction_as_printed():
    cfg, rows = fig1_cfg()
    d = C.decompose(cfg.n, cfg.row_ptr, cfg.col)
    big = [pt for pt in d["parts"] if len(pt["vertices"]) > 1]
    assert len(big) == 1
    scc = big[0]
    assert sorted(scc["vertices"]) == [2, 3, 4, 5, 6, 8]
    # SccEntryVertex {2}, SccExitVertex {2, 5} (Defs. 4, 5; Fig. 2a)
    assert [v for v in d["entry"] if v in scc["vertices"]] == [2]
    assert [v for v in d["exit"] if v in scc["vertices"]] == [2, 5]
    # PP Generation paragraph: the 11 internal PPs
    assert scc["internal"] == _sets(rows, "internal")
    # Path extraction paragraph
    assert scc["entry_exit"] == [(2,), (2, 3, 5)]
    assert scc["exit_paths"] == sorted([(3, 5, 6, 8, 2), (3, 4, 8, 2), (4, 8, 2, 3, 5), (6, 8, 2, 3, 5)])
    assert scc["entry_paths"] == [(2, 3, 4, 8), (2, 3, 5, 6, 8)]
    # the CCFG's PPs <Start,1,SCC1,9,End> and <Start,1,SCC1,7,End>
    comp = d["comp"]
    named = {comp[START]: "Start", comp[1]: "1", comp[2]: "SCC1", comp[9]: "9", comp[7]: "7", comp[END]: "End"}
    got = sorted(tuple(named[c] for c in p) for p in C.ccfg_prime_paths(d))
    assert got == sorted([("Start", "1", "SCC1", "9", "End"), ("Start", "1", "SCC1", "7", "End")])


def test_worked_example_merging_as_printed():
    cfg, rows = fig1_cfg()
    d = C.decompose(cfg.n, cfg.row_ptr, cfg.col)
    merged = C.merge(d)
    complete = [p for p in merged if p[0] == START and p[-1] == END]
    exit_pps = [p for p in merged if p[0] != START and p[-1] == END]
    entry_pps = [p for p in merged if p[0] == START and p[-1] != END]
    assert complete == _sets(rows, "complete")
    assert exit_pps == _sets(rows, "exit")
    assert entry_pps == _sets(rows, "entry")
    assert len(merged) == 8
    # "19 PPs of all four types"
    assert C.prime_paths(cfg.n, cfg.row_ptr, cfg.col) == sorted(p for _, p in load_fig1())


def _entered_scc(i):
    """A random 6-vertex digraph entered by one arc and left by one arc at
    different vertices: SCCs whose entry vertex does not lie on every exit
    path, where the closed-end reading of Defs. 7/8 matters."""
    inner = G.random_digraph(6, 0.3, 900 + i, self_loops=False)
    n = inner.n + 2
    arcs = [(0, 1 + (i % 3)), (1 + ((i + 2) % 6), n - 1)]
    for u in range(inner.n):
        for w in inner.succ(u):
            arcs.append((u + 1, int(w) + 1))
    rp, col = G.csr_from_arcs(n, arcs)
    return G.CFG(n, rp, col, 0, n - 1, f"entered{i}")


def _graphs():
    yield "config1", G.config1_cfg()
    for i in range(40):
        yield f"entered{i}", _entered_scc(i)
    for k in (1, 3, 6):
        yield f"chain{k}", G.diamond_chain(k)
    for i in range(25):
        yield f"random{i}", G.random_cfg(G.BATCH_SEED0 + 100 + i, n_max=40)
    for i in range(10):
        yield f"wrapped{i}", wrap_digraph(G.random_digraph(6, 0.35, 500 + i, self_loops=(i % 2 == 0)))
    for n in (1, 3, 5):
        yield f"ring{n}", G.ring(n)
    for n in (2, 4):
        yield f"complete{n}", G.complete_digraph(n)


@pytest.mark.parametrize("name,cfg", list(_graphs()), ids=[g[0] for g in _graphs()])
def test_compositional_equals_direct_oracle(name, cfg):
    got = C.prime_paths(cfg.n, cfg.row_ptr, cfg.col)
    ref = oracle.run(cfg.n, cfg.row_ptr, cfg.col).pp_list()
    assert got == ref


def test_tarjan_matches_mutual_reachability():
    for i in range(10):
        cfg = G.random_cfg(G.BATCH_SEED0 + 300 + i, n_max=60)
        succ = C.succ_lists(cfg.n, cfg.row_ptr, cfg.col)
        comp, _ = C.sccs(cfg.n, succ)
        dist, _ = oracle.bfs_tables(cfg.n, cfg.row_ptr, cfg.col)
        reach = (dist >= 0) | np.eye(cfg.n, dtype=bool)
        same = reach & reach.T
        np.testing.assert_array_equal(same, np.equal.outer(comp, comp))


@pytest.mark.gpu
def test_gpu_prime_paths_equal_compositional_route():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_16998_gb300 import tpg

    tpg.load_library(build=True)
    for name, cfg in _graphs():
        if name.startswith(("ring", "complete", "wrapped")):
            continue  # not CFGs (entry/exit rules); covered by the direct-oracle tests
        with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
            with tpg.tpg_prime_paths(h) as pp:
                got = pp.to_lists()
        assert got == C.prime_paths(cfg.n, cfg.row_ptr, cfg.col), name


def test_literal_maximality_of_defs_7_8_would_lose_parity():
    """Read literally, Defs. 7/8 keep the exit (entry) paths that are not a
    proper subpath of another exit (entry) path; merging those is not the
    PP set in general (an entry vertex before the path's first vertex can
    still be prepended).  The closed-end reading above matches the direct
    oracle on every graph; the literal one differs on some of them."""
    differs = 0
    for i in range(40):
        cfg = _entered_scc(i)
        d = C.decompose(cfg.n, cfg.row_ptr, cfg.col)
        ent, ext = set(d["entry"]), set(d["exit"])

        def sub(p, q):
            return len(p) < len(q) and any(q[j:j + len(p)] == p for j in range(len(q) - len(p) + 1))

        for c, pt in enumerate(d["parts"]):
            acyc = [p for p in C._simple_paths_within(pt["vertices"], d["succ"], d["comp"], c)
                    if not (len(p) >= 2 and p[0] == p[-1])]
            ex = [p for p in acyc if p[-1] in ext and p[0] not in ent]
            en = [p for p in acyc if p[0] in ent and p[-1] not in ext]
            pt["exit_paths"] = [p for p in ex if not any(sub(p, q) for q in ex)]
            pt["entry_paths"] = [p for p in en if not any(sub(p, q) for q in en)]
        internal = [p for pt in d["parts"] for p in pt["internal"]]
        literal = sorted(set(internal) | set(C.merge(d)))
        if literal != oracle.run(cfg.n, cfg.row_ptr, cfg.col).pp_list():
            differs += 1
    assert differs > 0
