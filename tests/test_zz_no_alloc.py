"""The allocation-free entry point, tpg_prime_paths_noalloc.

It serves callers that cannot allocate memory when they ask for prime paths
(for example while their stream is being captured into a CUDA graph, or
under a memory budget fixed in advance): it keeps its temporaries in a fixed
device array inside the library and writes into buffers the caller owns.
Here it is called through the C ABI and must give exactly what the regular
tpg_load_cfg + tpg_prime_paths path gives, on two calls in a row (the shared
array keeps the previous call's contents, so the second call also checks
that everything that must start at zero is cleared).

This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def regular(cfg):
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        pp = tpg.tpg_prime_paths(h)
        _, off, vert = pp.host_arrays()
        pp.free()
    return off, vert


def noalloc(cfg, cap_paths, cap_vertices):
    import torch

    rp = torch.as_tensor(cfg.row_ptr, device="cuda")
    col = torch.as_tensor(cfg.col if cfg.m else np.zeros(1, np.int32), device="cuda")
    off = torch.full((cap_paths + 1,), -7, dtype=torch.int64, device="cuda")
    vert = torch.full((max(cap_vertices, 1),), -7, dtype=torch.int32, device="cuda")
    rc, P, V = tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col, off, vert)
    torch.cuda.synchronize()
    return rc, P, V, off.cpu().numpy(), vert.cpu().numpy()


CASES = [
    ("fig1", lambda: fig1_cfg()[0]),
    ("structured-24", G.config1_cfg),
    ("diamond-chain-10", lambda: G.diamond_chain(10)),
    ("ring-tail-40", lambda: ring_with_tail(40)),
    ("random-cfg", lambda: G.random_cfg(G.BATCH_SEED0 + 3)),
    ("wrapped-digraph", lambda: wrap_digraph(G.random_digraph(7, 0.35, 5, self_loops=True))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_regular_entry_point_twice(name, make):
    cfg = make()
    ref_off, ref_vert = regular(cfg)
    P, V = len(ref_off) - 1, int(ref_off[-1])
    for call in range(2):
        rc, p, v, off, vert = noalloc(cfg, P + 3, V + 5)
        assert rc == tpg.TPG_OK, (call, tpg.tpg_strerror(rc))
        assert (p, v) == (P, V)
        np.testing.assert_array_equal(off[:P + 1], ref_off)
        np.testing.assert_array_equal(vert[:V], ref_vert)


def test_noalloc_reports_needed_sizes():
    cfg = G.config1_cfg()
    ref_off, _ = regular(cfg)
    rc, p, v, _, _ = noalloc(cfg, 2, 4)
    assert rc == tpg.TPG_ETOOBIG
    assert (p, v) == (len(ref_off) - 1, int(ref_off[-1]))


def test_noalloc_rejects_graphs_beyond_its_limit():
    rc, _, _, _, _ = noalloc(ring_with_tail(200), 1000, 100000)
    assert rc == tpg.TPG_ETOOBIG
