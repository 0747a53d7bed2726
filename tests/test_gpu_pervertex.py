"""The paper-style per-vertex-list baseline (tpg_prime_paths_pervertex)
against the oracle: the same PP set, grouped by end vertex."""
import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg

from .helpers import ring_with_tail, wrap_digraph
from .test_oracle import fig1_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tpg.load_library(build=True)


def pervertex(cfg, location=tpg.TPG_RESULT_HOST):
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=location) as h:
        with tpg.tpg_prime_paths_pervertex(h) as pp:
            vp, off, vert = pp.host_arrays()
            ng = pp.num_graphs
        st = tpg.tpg_get_stats(h)
    return ng, vp, off, vert, st


CASES = [
    ("fig1", lambda: fig1_cfg()[0]),
    ("config1", G.config1_cfg),
    ("diamond-8", lambda: G.diamond_chain(8)),
    ("ring-tail-12", lambda: ring_with_tail(12)),
    ("two-vertices", lambda: G.CFG(2, *G.csr_from_arcs(2, [(0, 1)]), 0, 1, "edge")),
    ("binarised-cfg-3", lambda: G.binarise_switches(G.random_cfg(G.BATCH_SEED0 + 3))),
    ("binarised-cfg-25", lambda: G.binarise_switches(G.random_cfg(G.BATCH_SEED0 + 25))),
    ("binarised-digraph", lambda: G.binarise_switches(wrap_digraph(G.random_digraph(6, 0.3, 2, self_loops=True)))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_pervertex_baseline_matches_oracle(name, make):
    cfg = make()
    assert np.diff(cfg.row_ptr).max() <= 2
    ref = oracle.run_cfg(cfg, test_paths=False)
    ng, vp, off, vert, st = pervertex(cfg)
    assert ng == cfg.n and len(vp) == cfg.n + 1
    got = []
    for v in range(cfg.n):
        lens = []
        for i in range(int(vp[v]), int(vp[v + 1])):
            p = tuple(int(x) for x in vert[off[i]:off[i + 1]])
            assert p[-1] == v, (v, p)  # grouped by end vertex
            lens.append(len(p))
            got.append(p)
        assert lens == sorted(lens)
    assert sorted(got) == ref.pp_list()
    assert st["pervertex_paths"] == ref.n_simple
    assert st["pervertex_bytes"] > 0


def test_pervertex_device_result():
    cfg = G.diamond_chain(6)
    ng, vp, off, vert, _ = pervertex(cfg, location=tpg.TPG_RESULT_DEVICE)
    ref = oracle.run_cfg(cfg, test_paths=False)
    got = sorted(tuple(int(x) for x in vert[off[i]:off[i + 1]]) for i in range(len(off) - 1))
    assert got == ref.pp_list()


def test_pervertex_rejects_switches_and_batches():
    cfg = G.config3_cfg()  # switches of fan-out 6
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_prime_paths_pervertex(h)
        assert e.value.code == tpg.TPG_EINVAL
    ns, rp, col, ent, ext = G.concat_batch([G.diamond_chain(2), G.diamond_chain(3)])
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_prime_paths_pervertex(h)
        assert e.value.code == tpg.TPG_EINVAL
