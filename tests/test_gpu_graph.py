"""Graph mode: the whole hot path captured in one CUDA graph and replayed,
for one graph and for batches, against the oracle and the host-driven path."""
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


def split(arrs, g):
    gp, off, vert = arrs
    lo, hi = int(gp[g]), int(gp[g + 1])
    o = off[lo:hi + 1]
    return o - o[0], vert[o[0]:o[-1]]


def graph_run(h, times=2):
    outs = []
    for _ in range(times):
        pp, tp = tpg.tpg_graph_launch(h)
        outs.append((pp.host_arrays(), tp.host_arrays()))
        pp.free()
        tp.free()
    return outs


@pytest.mark.parametrize("make", [G.config1_cfg, G.config3_cfg, lambda: G.diamond_chain(12)],
                         ids=["structured-24", "structured-120", "diamond-chain-12"])
def test_graph_mode_single(make):
    cfg = make()
    ref = oracle.run_cfg(cfg)
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit,
                          location=tpg.TPG_RESULT_DEVICE) as h:
        tpg.tpg_graph_capture(h)
        for ppa, tpa in graph_run(h):
            assert_paths_equal(ppa[1], ppa[2], ref.pp_offsets, ref.pp_vertices, "graph PP")
            assert_paths_equal(tpa[1], tpa[2], ref.tp_offsets, ref.tp_vertices, "graph TP")
        st = tpg.tpg_get_stats(h)
        assert st["graph_launches"] == 2
        assert st["graph_fallbacks"] == 0, (st["graph_flags"], st["graph_enum_error"])


def test_graph_mode_batch_vs_oracle():
    cfgs = [G.random_cfg(G.BATCH_SEED0 + i) for i in range(48)] + [G.config1_cfg(), G.diamond_chain(4)]
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
        tpg.tpg_graph_capture(h)
        (ppa, tpa), = graph_run(h, 1)
        assert tpg.tpg_get_stats(h)["graph_fallbacks"] == 0
    for g, c in enumerate(cfgs):
        ref = oracle.run_cfg(c)
        o, v = split(ppa, g)
        assert_paths_equal(o, v, ref.pp_offsets, ref.pp_vertices, f"graph {g} PP")
        o, v = split(tpa, g)
        assert_paths_equal(o, v, ref.tp_offsets, ref.tp_vertices, f"graph {g} TP")


def test_graph_mode_small_capacity_falls_back_exactly():
    cfg = G.config3_cfg()
    ref = oracle.run_cfg(cfg)
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        tpg.tpg_set_capacity(h, 1000, 500, 100)
        tpg.tpg_set_output_capacity(h, 100, 1000, 1000, 1000)
        tpg.tpg_graph_capture(h)
        (ppa, tpa), (ppb, tpb) = graph_run(h, 2)
        st = tpg.tpg_get_stats(h)
    assert st["graph_fallbacks"] == 1
    for pa, ta in ((ppa, tpa), (ppb, tpb)):
        assert_paths_equal(pa[1], pa[2], ref.pp_offsets, ref.pp_vertices, "fallback PP")
        assert_paths_equal(ta[1], ta[2], ref.tp_offsets, ref.tp_vertices, "fallback TP")


def test_graph_mode_full_batch_equals_host_path():
    cfgs = G.batch_cfgs(4096)
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
        pp = tpg.tpg_prime_paths(h)
        ref_pp = pp.host_arrays()
        pp.free()
        tp = tpg.tpg_test_paths(h)
        ref_tp = tp.host_arrays()
        tp.free()
        tpg.tpg_graph_capture(h)
        (ppa, tpa), = graph_run(h, 1)
        assert tpg.tpg_get_stats(h)["graph_fallbacks"] == 0
    for a, b in zip(ppa, ref_pp):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(tpa, ref_tp):
        np.testing.assert_array_equal(a, b)
