"""The per-SCC step of the compositional route on the GPU (tpg_scc_ids,
tpg_scc_internal_pps) against the compositional oracle
(oracle/compositional.py, pinned to the worked example of Sec. 2.1)."""
import numpy as np
import pytest

from oracle import compositional as C
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


def gpu_scc(cfg):
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        comp = tpg.tpg_scc_ids(h, cfg.n)
        with tpg.tpg_scc_internal_pps(h) as r:
            _, off, vert = r.host_arrays()
        st = tpg.tpg_get_stats(h)
    paths = [tuple(int(x) for x in vert[off[i]:off[i + 1]]) for i in range(len(off) - 1)]
    return comp, paths, st


def same_partition(a, b):
    # a[v] == a[u] iff b[v] == b[u]
    pairs = {}
    for x, y in zip(a, b):
        if pairs.setdefault(int(x), int(y)) != int(y):
            return False
    return len(set(pairs.values())) == len(pairs)


def test_worked_example_eleven_internal_pps():
    cfg, rows = fig1_cfg()
    comp, paths, st = gpu_scc(cfg)
    listed = sorted(p for kind, p in rows if kind == "internal")
    assert len(listed) == 11
    assert paths == listed
    assert st["scc_internal_pps"] == 11
    # the SCC {2, 3, 4, 5, 6, 8} and one-vertex SCCs elsewhere, named by their smallest vertex
    assert all(comp[v] == 2 for v in (2, 3, 4, 5, 6, 8))
    assert all(comp[v] == v for v in (0, 1, 7, 9, 10))


CASES = [
    ("config1", G.config1_cfg),
    ("diamond-6", lambda: G.diamond_chain(6)),
    ("ring-tail-9", lambda: ring_with_tail(9)),
] + [(f"cfg-{s}", (lambda s=s: G.random_cfg(G.BATCH_SEED0 + s))) for s in (3, 21, 24, 25, 30)] + [
    (f"digraph-{s}", (lambda s=s: wrap_digraph(G.random_digraph(6, 0.4, s, self_loops=True)))) for s in range(4)]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_internal_pps_match_compositional_oracle(name, make):
    cfg = make()
    d = C.decompose(cfg.n, cfg.row_ptr, cfg.col)
    ref = sorted(p for pt in d["parts"] for p in pt["internal"])
    comp, paths, _ = gpu_scc(cfg)
    assert same_partition(comp, d["comp"])
    assert all(comp[v] <= v for v in range(cfg.n))
    assert paths == ref


def test_scc_rejects_batches():
    ns, rp, col, ent, ext = G.concat_batch([G.diamond_chain(2), G.diamond_chain(3)])
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_scc_internal_pps(h)
        assert e.value.code == tpg.TPG_EINVAL
