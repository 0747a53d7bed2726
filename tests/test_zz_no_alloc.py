"""The allocation-free entry point, tpg_prime_paths_noalloc.

It serves callers that cannot allocate device memory when they ask for prime
paths: code held to a device-memory budget fixed in advance, and host
frameworks that own every allocation and hand the library only the buffers
it reads and writes.  It keeps its temporaries in a fixed device array
inside the library and writes into buffers the caller owns.  Here it is
called through the C ABI and must give exactly what the regular
tpg_load_cfg + tpg_prime_paths path gives, and what the CPU oracle gives, on
two calls in a row (the shared array keeps the previous call's contents, so
the second call also checks that everything that must start at zero is
cleared).

This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg

from .helpers import ring_with_tail, wrap_digraph
from .test_oracle import fig1_cfg


@pytest.fixture(scope="module")
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


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_regular_entry_point_and_oracle_twice(_lib, name, make):
    cfg = make()
    ref_off, ref_vert = regular(cfg)
    orc = oracle.run(cfg.n, cfg.row_ptr, cfg.col, want_paths=True)
    np.testing.assert_array_equal(ref_off, orc.pp_offsets)
    np.testing.assert_array_equal(ref_vert, orc.pp_vertices)
    P, V = len(ref_off) - 1, int(ref_off[-1])
    for call in range(2):
        rc, p, v, off, vert = noalloc(cfg, P + 3, V + 5)
        assert rc == tpg.TPG_OK, (call, tpg.tpg_strerror(rc))
        assert (p, v) == (P, V)
        np.testing.assert_array_equal(off[:P + 1], orc.pp_offsets)
        np.testing.assert_array_equal(vert[:V], orc.pp_vertices)
        # nothing written past the sizes
        assert np.all(off[P + 1:] == -7) and np.all(vert[V:] == -7)


@pytest.mark.gpu
def test_noalloc_reports_needed_sizes(_lib):
    cfg = G.config1_cfg()
    ref_off, _ = regular(cfg)
    rc, p, v, _, _ = noalloc(cfg, 2, 4)
    assert rc == tpg.TPG_ETOOBIG
    assert (p, v) == (len(ref_off) - 1, int(ref_off[-1]))


@pytest.mark.gpu
def test_noalloc_rejects_graphs_beyond_its_limit(_lib):
    rc, _, _, _, _ = noalloc(ring_with_tail(200), 1000, 100000)
    assert rc == tpg.TPG_ETOOBIG


@pytest.mark.gpu
def test_noalloc_device_overflow_then_exact(_lib):
    # 58 vertices fit the vertex limit, but a level of 2^19 paths passes the
    # 2^18-per-level scratch: the frontier stops on the device (error word in
    # the shared array); the next call must still be exact
    big = G.diamond_chain(19)
    rc, _, _, _, _ = noalloc(big, 1 << 19, 39 << 19)
    assert rc == tpg.TPG_ETOOBIG
    cfg = G.config1_cfg()
    orc = oracle.run_cfg(cfg, test_paths=False)
    P, V = len(orc.pp_offsets) - 1, int(orc.pp_offsets[-1])
    rc, p, v, off, vert = noalloc(cfg, P, V)
    assert rc == tpg.TPG_OK and (p, v) == (P, V)
    np.testing.assert_array_equal(off, orc.pp_offsets)
    np.testing.assert_array_equal(vert, orc.pp_vertices)


def test_noalloc_binding_rejects_wrong_arguments_without_a_call():
    # dtype, device and size checks happen in the binding before any call
    torch = pytest.importorskip("torch")
    cfg = G.config1_cfg()
    rp = torch.as_tensor(cfg.row_ptr)
    col = torch.as_tensor(cfg.col)
    off = torch.zeros(100, dtype=torch.int64)
    vert = torch.zeros(1000, dtype=torch.int32)
    # host tensors are not device buffers
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col, off, vert)[0] == tpg.TPG_EINVAL
    # an int32 offsets buffer would be written as int64
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col, off.int(), vert)[0] == tpg.TPG_EINVAL
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp.long(), col, off, vert)[0] == tpg.TPG_EINVAL
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col, off, np.zeros(3, np.int32))[0] == tpg.TPG_EINVAL


@pytest.mark.gpu
def test_noalloc_binding_rejects_bad_device_buffers(_lib):
    import torch

    cfg = G.config1_cfg()
    rp = torch.as_tensor(cfg.row_ptr, device="cuda")
    col = torch.as_tensor(cfg.col, device="cuda")
    off = torch.zeros(100, dtype=torch.int64, device="cuda")
    vert = torch.zeros(1000, dtype=torch.int32, device="cuda")
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col, off.int(), vert)[0] == tpg.TPG_EINVAL
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp[:-1], col, off, vert)[0] == tpg.TPG_EINVAL
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col[:-1], off, vert)[0] == tpg.TPG_EINVAL
    assert tpg.tpg_prime_paths_noalloc(cfg.n, cfg.m, rp, col, off[::2], vert)[0] == tpg.TPG_EINVAL
