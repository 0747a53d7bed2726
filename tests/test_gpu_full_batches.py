"""The two 4096-graph workloads compared in full, graph by graph, with the
CPU oracle: every prime path and every test path of every graph.

* The 4096-graph batch (graphs of 10-150 vertices, loop nesting 0-4, switch
  fan-out 2-6) through the host-driven batched calls and through a graph-mode
  replay (one persistent launch, whole pipeline in one CUDA graph).
* The held-out batch of the learned sizer (4096 graphs from disjoint seeds),
  pre-sized by a trained network and run as a graph-mode capture + replay.

The oracle runs graph by graph on the host (about half a minute for each
batch); each graph's lists are compared element by element.
"""
import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg

from .helpers import assert_paths_equal

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tpg.load_library(build=True)


def compare_all(cfgs, pp_arrays, tp_arrays, what):
    pgp, poff, pvert = pp_arrays
    tgp, toff, tvert = tp_arrays
    assert len(pgp) == len(cfgs) + 1 and len(tgp) == len(cfgs) + 1
    for g, c in enumerate(cfgs):
        ref = oracle.run_cfg(c, test_paths=True)
        lo, hi = int(pgp[g]), int(pgp[g + 1])
        o = poff[lo:hi + 1]
        assert_paths_equal(o - o[0], pvert[o[0]:o[-1]], ref.pp_offsets, ref.pp_vertices, f"{what} graph {g} PP")
        lo, hi = int(tgp[g]), int(tgp[g + 1])
        o = toff[lo:hi + 1]
        assert_paths_equal(o - o[0], tvert[o[0]:o[-1]], ref.tp_offsets, ref.tp_vertices, f"{what} graph {g} TP")


def test_batch4096_host_driven_and_graph_replay_vs_oracle():
    cfgs = G.batch_cfgs(4096)
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_HOST) as h:
        with tpg.tpg_prime_paths(h) as pp, tpg.tpg_test_paths(h) as tp:
            host_pp, host_tp = pp.host_arrays(), tp.host_arrays()
        tpg.tpg_graph_capture(h)
        for _ in range(2):
            a, b = tpg.tpg_graph_launch(h)
            with a, b:
                for x, y in zip(a.host_arrays() + b.host_arrays(), host_pp + host_tp):
                    np.testing.assert_array_equal(x, y)
        assert tpg.tpg_get_stats(h)["graph_fallbacks"] == 0
    compare_all(cfgs, host_pp, host_tp, "batch4096")


def test_sizer_heldout4096_presized_replay_vs_oracle():
    train = [G.random_cfg(G.TRAIN_SEED0 + i) for i in range(4096)]
    held = G.batch_cfgs(4096, G.HELDOUT_SEED0)
    with tpg.tpg_sizer_create(seed=1) as z:
        for b0 in range(0, len(train), 1024):
            ns, rp, col, ent, ext = G.concat_batch(train[b0:b0 + 1024])
            with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
                tpg.tpg_sizer_add_batch(z, h)
        tpg.tpg_sizer_train(z, 40, 3e-3)
        ns, rp, col, ent, ext = G.concat_batch(held)
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_HOST) as h:
            caps = tpg.tpg_sizer_presize(z, h, 1.25)
            assert np.all(caps > 0)
            tpg.tpg_graph_capture(h)
            a, b = tpg.tpg_graph_launch(h)
            with a, b:
                pp, tp = a.host_arrays(), b.host_arrays()
    compare_all(held, pp, tp, "held-out")
