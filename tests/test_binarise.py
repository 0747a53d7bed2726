"""Switch binarisation (the out-degree-2 input restriction of Sec. 3)."""
import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G


def _paths_through_new(cfg, b):
    """every original arc v -> w, followed in the binarised graph through new
    vertices only, reaches w along exactly one path"""
    n = cfg.n
    for v in range(n):
        for w in cfg.succ(v):
            w = int(w)
            hits = 0
            stack = [int(x) for x in b.succ(v)]
            while stack:
                x = stack.pop()
                if x == w:
                    hits += 1
                elif x >= n:
                    stack += [int(y) for y in b.succ(x)]
            assert hits == 1, (v, w, hits)


@pytest.mark.parametrize("make", [G.config3_cfg, G.config1_cfg] +
                         [(lambda s=s: G.random_cfg(G.BATCH_SEED0 + s)) for s in range(10)])
def test_binarised_graph_shape(make):
    cfg = make()
    b = G.binarise_switches(cfg)
    deg = np.diff(cfg.row_ptr)
    assert b.n == cfg.n + int(np.maximum(deg - 2, 0).sum())
    assert b.m == cfg.m + int(np.maximum(deg - 2, 0).sum())
    assert np.diff(b.row_ptr).max() <= 2
    # original arcs of vertices of out-degree <= 2 are kept, new vertices
    # have in-degree 1 and out-degree 2
    for v in range(cfg.n):
        if deg[v] <= 2:
            assert list(b.succ(v)) == list(cfg.succ(v))
    indeg = np.bincount(b.col, minlength=b.n)
    assert np.all(indeg[cfg.n:] == 1) and np.all(np.diff(b.row_ptr)[cfg.n:] == 2)
    assert (b.entry, b.exit) == (cfg.entry, cfg.exit)
    _paths_through_new(cfg, b)


def test_binarise_is_identity_without_switches():
    for cfg in (G.diamond_chain(6), G.config1_cfg()):
        b = G.binarise_switches(cfg)
        assert b.n == cfg.n and np.array_equal(b.row_ptr, cfg.row_ptr) and np.array_equal(b.col, cfg.col)


@pytest.mark.parametrize("k", [3, 4, 6, 9])
def test_binarised_switch_star_keeps_its_k_pps(k):
    # entry -> s, s -> w1..wk, wi -> exit: a DAG whose PPs are its k
    # entry-exit paths, before and after binarisation (k - 2 new vertices)
    n = k + 3
    arcs = [(0, 1)] + [(1, 2 + i) for i in range(k)] + [(2 + i, n - 1) for i in range(k)]
    rp, col = G.csr_from_arcs(n, arcs)
    cfg = G.CFG(n, rp, col, 0, n - 1, f"star{k}")
    b = G.binarise_switches(cfg)
    assert b.n == n + k - 2
    for g in (cfg, b):
        res = oracle.run_cfg(g, test_paths=False)
        assert res.num_pp == k
        assert all(p[0] == 0 and p[-1] == n - 1 for p in res.pp_list())
