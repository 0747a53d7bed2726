"""The compositional route on the GPU (tpg_prime_paths_compositional)
against the direct route, the oracle and the compositional oracle's
intermediate sets (oracle/compositional.py, pinned to the worked example of
Sec. 2.1)."""
import numpy as np
import pytest

import oracle
from oracle import compositional as C
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


CASES = [
    ("fig1", lambda: fig1_cfg()[0]),
    ("config1", G.config1_cfg),
    ("diamond-7", lambda: G.diamond_chain(7)),
    ("ring-tail-9", lambda: ring_with_tail(9)),
    ("self-loop", lambda: G.CFG(4, *G.csr_from_arcs(4, [(0, 1), (1, 1), (1, 2), (2, 1), (2, 3)]), 0, 3, "loop")),
    ("two-vertices", lambda: G.CFG(2, *G.csr_from_arcs(2, [(0, 1)]), 0, 1, "edge")),
    ("complete-5-wrapped", lambda: wrap_digraph(G.complete_digraph(5))),
] + [(f"cfg-{s}", (lambda s=s: G.random_cfg(G.BATCH_SEED0 + s))) for s in (3, 21, 24, 25, 30, 47)] + [
    (f"digraph-{s}", (lambda s=s: wrap_digraph(G.random_digraph(6, 0.4, s, self_loops=True)))) for s in range(5)]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_compositional_route_equals_direct_route_and_oracle(name, make):
    cfg = make()
    ref = oracle.run_cfg(cfg, test_paths=False)
    d = C.decompose(cfg.n, cfg.row_ptr, cfg.col)
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        with tpg.tpg_prime_paths_compositional(h) as cp:
            _, coff, cvert = cp.host_arrays()
        st = tpg.tpg_get_stats(h)
        with tpg.tpg_prime_paths(h) as pp:
            _, off, vert = pp.host_arrays()
    assert_paths_equal(coff, cvert, ref.pp_offsets, ref.pp_vertices, f"{name} compositional")
    assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, f"{name} direct")
    tot = {k: sum(len(pt[k]) for pt in d["parts"]) for k in ("entry_exit", "exit_paths", "entry_paths", "internal")}
    assert st["comp_entry_exit_paths"] == tot["entry_exit"]
    assert st["comp_exit_paths"] == tot["exit_paths"]
    assert st["comp_entry_paths"] == tot["entry_paths"]
    assert st["scc_internal_pps"] == tot["internal"]
    assert st["comp_crossing_pps"] == len(C.merge(d))


def test_worked_example_counts():
    # 11 internal PPs and 8 joined across SCCs (2 complete + 4 exit + 2
    # entry PPs of Sec. 2.1); 5 / 5 / 3 extracted paths over all SCCs, of
    # which the big SCC's are the printed 2 / 4 / 2
    cfg, _ = fig1_cfg()
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        with tpg.tpg_prime_paths_compositional(h) as cp:
            assert cp.num_paths == 19
        st = tpg.tpg_get_stats(h)
    assert (st["scc_internal_pps"], st["comp_crossing_pps"]) == (11, 8)
    assert (st["comp_entry_exit_paths"], st["comp_exit_paths"], st["comp_entry_paths"]) == (5, 5, 3)


def test_compositional_limits():
    ns, rp, col, ent, ext = G.concat_batch([G.diamond_chain(2), G.diamond_chain(3)])
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_prime_paths_compositional(h)
        assert e.value.code == tpg.TPG_EINVAL
    big = ring_with_tail(300)
    with tpg.tpg_load_cfg(big.n, big.row_ptr, big.col, big.entry, big.exit) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_prime_paths_compositional(h)
        assert e.value.code == tpg.TPG_ETOOBIG
