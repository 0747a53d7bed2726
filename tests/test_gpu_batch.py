"""Batched handles (many CFGs in one persistent launch) vs the oracle."""
import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg

from .helpers import assert_paths_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tpg.load_library(build=True)


def run_batch(cfgs, location=tpg.TPG_RESULT_HOST):
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=location) as h:
        pp = tpg.tpg_prime_paths(h)
        ppa = pp.host_arrays()
        pp.free()
        tp = tpg.tpg_test_paths(h)
        tpa = tp.host_arrays()
        tp.free()
        st = tpg.tpg_get_stats(h)
    return ppa, tpa, st


def split(arrs, g):
    gp, off, vert = arrs
    lo, hi = int(gp[g]), int(gp[g + 1])
    o = off[lo:hi + 1]
    return o - o[0], vert[o[0]:o[-1]]


def test_small_mixed_batch():
    cfgs = [G.diamond_chain(3), G.config1_cfg(), G.diamond_chain(1)] + \
           [G.random_cfg(G.BATCH_SEED0 + i) for i in range(20)]
    ppa, tpa, st = run_batch(cfgs)
    assert len(ppa[0]) == len(cfgs) + 1
    total_simple = 0
    for g, c in enumerate(cfgs):
        ref = oracle.run_cfg(c)
        total_simple += ref.n_simple
        o, v = split(ppa, g)
        assert_paths_equal(o, v, ref.pp_offsets, ref.pp_vertices, f"graph {g} PP")
        o, v = split(tpa, g)
        assert_paths_equal(o, v, ref.tp_offsets, ref.tp_vertices, f"graph {g} TP")
    assert st["simple_paths"] == total_simple


def test_batch_single_graph_equals_plain():
    c = G.config3_cfg()
    ppa, tpa, _ = run_batch([c])
    ref = oracle.run_cfg(c)
    assert_paths_equal(ppa[1], ppa[2], ref.pp_offsets, ref.pp_vertices, "PP")
    assert_paths_equal(tpa[1], tpa[2], ref.tp_offsets, ref.tp_vertices, "TP")


def test_full_4096_batch_sampled():
    """The 4096-graph workload at full size: totals from the oracle's count
    mode for every graph, full sequences for a sample of graphs."""
    cfgs = G.batch_cfgs(4096)
    ppa, tpa, st = run_batch(cfgs, location=tpg.TPG_RESULT_DEVICE)
    gp = ppa[0]
    counts = np.diff(gp)
    ref_counts = []
    ref_simple = 0
    for c in cfgs:
        r = oracle.run_cfg(c, test_paths=False, want_paths=False)
        ref_counts.append(r.num_pp)
        ref_simple += r.n_simple
    np.testing.assert_array_equal(counts, np.asarray(ref_counts))
    assert st["simple_paths"] == ref_simple
    rng = G.SplitMix64(2024)
    sample = sorted({rng.randint(0, 4095) for _ in range(40)} | {int(np.argmax(counts))})
    for g in sample:
        ref = oracle.run_cfg(cfgs[g])
        o, v = split(ppa, g)
        assert_paths_equal(o, v, ref.pp_offsets, ref.pp_vertices, f"graph {g} PP")
        o, v = split(tpa, g)
        assert_paths_equal(o, v, ref.tp_offsets, ref.tp_vertices, f"graph {g} TP")
