"""Longest-first touring (tpg_test_paths_greedy) against the oracle.

The CUDA result must equal the oracle's longest-first touring element by
element: single graphs of every shape the other parity tests use, graphs
large enough that a block runs many rounds and several warp counts, a batch
whose graphs are toured by different blocks, and the device-result and
empty cases.  The oracle's touring is pinned in test_oracle_greedy.py.
"""
import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg

from .helpers import assert_paths_equal, ring_with_tail, wrap_digraph
from .test_oracle import fig1_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tpg.load_library(build=True)


def greedy_gpu(cfg, location=tpg.TPG_RESULT_HOST):
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=location) as h:
        with tpg.tpg_test_paths_greedy(h) as gt:
            arrs = gt.host_arrays()
        st = tpg.tpg_get_stats(h)
    return arrs, st


CASES = [
    ("fig1", lambda: fig1_cfg()[0]),
    ("config1", G.config1_cfg),
    ("diamond-10", lambda: G.diamond_chain(10)),
    ("ring-tail-40", lambda: ring_with_tail(40)),
    ("while-ring-200", lambda: ring_with_tail(200)),
    ("two-vertices", lambda: G.CFG(2, *G.csr_from_arcs(2, [(0, 1)]), 0, 1, "edge")),
    ("complete-5-wrapped", lambda: wrap_digraph(G.complete_digraph(5))),
] + [(f"cfg-{s}", (lambda s=s: G.random_cfg(G.BATCH_SEED0 + s))) for s in (3, 21, 24, 25, 47, 54)] + [
    (f"digraph-{s}", (lambda s=s: wrap_digraph(G.random_digraph(7, 0.35, s, self_loops=True)))) for s in range(4)]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_touring_matches_oracle(name, make):
    cfg = make()
    ref = oracle.run_cfg(cfg, test_paths=False, greedy=True)
    (_, off, vert), st = greedy_gpu(cfg)
    assert_paths_equal(off, vert, ref.gtp_offsets, ref.gtp_vertices, f"{name} touring TPs")
    assert st["touring_test_paths"] == len(ref.gtp_offsets) - 1
    assert st["touring_sweeps"] >= 1


def test_touring_device_result_and_subset_of_one_per_pp_list():
    cfg = G.random_cfg(G.BATCH_SEED0 + 25)
    (_, off, vert), _ = greedy_gpu(cfg, location=tpg.TPG_RESULT_DEVICE)
    ref = oracle.run_cfg(cfg, test_paths=True, greedy=True)
    assert_paths_equal(off, vert, ref.gtp_offsets, ref.gtp_vertices, "device result")
    assert set(ref.gtp_list()) <= set(ref.tp_list())


def test_touring_batch_matches_oracle_per_graph():
    cfgs = [G.diamond_chain(4), fig1_cfg()[0], G.config1_cfg()] + [G.random_cfg(G.BATCH_SEED0 + i) for i in range(200)]
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        with tpg.tpg_test_paths_greedy(h) as gt:
            gp, off, vert = gt.host_arrays()
        # the one-per-PP list afterwards on the same handle is unchanged
        with tpg.tpg_test_paths(h) as tp:
            tgp, toff, tvert = tp.host_arrays()
    assert len(gp) == len(cfgs) + 1
    for g, c in enumerate(cfgs):
        ref = oracle.run_cfg(c, test_paths=True, greedy=True)
        lo, hi = int(gp[g]), int(gp[g + 1])
        o = off[lo:hi + 1]
        assert_paths_equal(o - o[0], vert[o[0]:o[-1]], ref.gtp_offsets, ref.gtp_vertices, f"graph {g}")
        lo, hi = int(tgp[g]), int(tgp[g + 1])
        o = toff[lo:hi + 1]
        assert_paths_equal(o - o[0], tvert[o[0]:o[-1]], ref.tp_offsets, ref.tp_vertices, f"graph {g} one-per-PP")


def test_touring_repeated_calls_are_identical():
    cfg = G.config3_cfg()
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        outs = []
        for _ in range(3):
            with tpg.tpg_test_paths_greedy(h) as gt:
                outs.append(gt.host_arrays())
    for a in outs[1:]:
        for x, y in zip(outs[0], a):
            np.testing.assert_array_equal(x, y)


def test_touring_reports_unreachable():
    # a PP that cannot reach the exit cannot be toured
    rp, col = G.csr_from_arcs(5, [(0, 1), (1, 2), (2, 1), (1, 4), (3, 3)])
    with tpg.tpg_load_cfg(5, rp, col, 0, 4) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_test_paths_greedy(h)
        assert e.value.code == tpg.TPG_EUNREACH


def _digests():
    import os

    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "touring_digests.txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, g0, n, T, V, d = line.split()
                rows[(name, int(g0))] = (int(n), int(T), int(V), d)
    return rows


def test_touring_full_batch_and_config3_match_oracle_digests():
    # the oracle's touring of all 4096 graphs and of the 120-vertex CFG takes
    # ~20 minutes single-threaded: its digests are stored (written by
    # golden/make_touring_digests.py, which calls only the oracle)
    import hashlib

    from .helpers import touring_digest_update

    rows = _digests()
    cfgs = G.batch_cfgs(4096, G.BATCH_SEED0)
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        with tpg.tpg_test_paths_greedy(h) as gt:
            gp, off, vert = gt.host_arrays()
    for (name, g0), (n, T, V, d) in sorted(rows.items()):
        if name != "batch4096":
            continue
        hsh = hashlib.sha256()
        tot_t = tot_v = 0
        for g in range(g0, g0 + n):
            lo, hi = int(gp[g]), int(gp[g + 1])
            o = off[lo:hi + 1]
            touring_digest_update(hsh, o - o[0], vert[o[0]:o[-1]])
            tot_t += hi - lo
            tot_v += int(o[-1] - o[0])
        assert (tot_t, tot_v) == (T, V), (g0, tot_t, tot_v, T, V)
        assert hsh.hexdigest()[:16] == d, f"graphs {g0}..{g0 + n - 1}"
    cfg = G.config3_cfg()
    (_, off, vert), st = greedy_gpu(cfg)
    n, T, V, d = rows[("config3", 0)]
    hsh = hashlib.sha256()
    touring_digest_update(hsh, off, vert)
    assert (len(off) - 1, int(off[-1])) == (T, V)
    assert hsh.hexdigest()[:16] == d
