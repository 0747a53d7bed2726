"""Failure detection without a GPU fault.

(1) Every grid-wide barrier of the persistent frontier launch waits at most a
per-handle limit (tpg_set_wait_limit).  With a limit of 0 ns any wait at all
runs out: the blocks stop, the launch ends with its error flag set, the call
returns TPG_ETIMEOUT, and the same handle gives the exact result once the
limit is restored.  Nothing spins unbounded and no kernel faults.

(2) Device allocation failures are injected on the host: an allocator that
returns NULL after a given number of allocations.  Every failure point of a
load + prime paths + test paths sequence must give TPG_ENOMEM (or succeed
when the failure point is past the last allocation), hand back every block
it obtained, and leave the library usable.

(3) Capacity hints are hints: an allocator that refuses to hold more than
256 MiB at once, and arena capacities of hundreds of GiB, still give the
exact result (the hinted sizes are halved until they fit).
"""
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


@pytest.mark.parametrize("make", [lambda: G.diamond_chain(14), G.config3_cfg], ids=["chain14", "config3"])
def test_barrier_wait_limit_runs_out_then_handle_recovers(make):
    cfg = make()
    ref = oracle.run_cfg(cfg, test_paths=True)
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        tpg.tpg_set_wait_limit(h, 0)
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_prime_paths(h)
        assert e.value.code == tpg.TPG_ETIMEOUT
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_test_paths(h)
        assert e.value.code == tpg.TPG_ETIMEOUT
        tpg.tpg_set_wait_limit(h, -1)
        for _ in range(2):
            with tpg.tpg_prime_paths(h) as pp, tpg.tpg_test_paths(h) as tp:
                _, off, vert = pp.host_arrays()
                _, toff, tvert = tp.host_arrays()
            assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, "PPs after a timeout")
            assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, "TPs after a timeout")


class _FailingAllocator:
    """Device blocks from torch's caching allocator; NULL from the k-th on."""

    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.foreign = []  # releases of blocks this allocator never handed out

    def alloc(self, nbytes, stream):
        import torch

        self.calls += 1
        if self.fail_at is not None and self.calls > self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        self.live[p] = nbytes
        return p

    def release(self, ptr, stream):
        import torch

        if ptr not in self.live:
            self.foreign.append(ptr)  # (an exception would be lost inside the C callback)
            return
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(int(ptr))


def _run_sequence(cfg):
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        with tpg.tpg_prime_paths(h) as pp, tpg.tpg_test_paths(h) as tp:
            return pp.host_arrays()[1:], tp.host_arrays()[1:]


def test_allocation_failure_at_every_point_gives_enomem_and_no_leak():
    import torch

    cfg = G.config3_cfg()
    ref = oracle.run_cfg(cfg, test_paths=True)
    try:
        # count the allocations of a clean sequence first
        probe = _FailingAllocator(None)
        tpg.tpg_set_allocator(probe.alloc, probe.release)
        _run_sequence(cfg)
        tpg.tpg_release_cached_memory()
        total = probe.calls
        assert total > 5 and not probe.live and not probe.foreign
        for k in range(total + 1):
            fa = _FailingAllocator(k)
            tpg.tpg_set_allocator(fa.alloc, fa.release)
            try:
                (off, vert), (toff, tvert) = _run_sequence(cfg)
                assert k >= total, f"failure at allocation {k} went unnoticed"
                assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, f"PPs, fail_at={k}")
                assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, f"TPs, fail_at={k}")
            except tpg.TPGError as e:
                assert e.code == tpg.TPG_ENOMEM, (k, e)
                assert k < total
            torch.cuda.synchronize()
            tpg.tpg_release_cached_memory()
            assert not fa.live, f"fail_at={k}: {len(fa.live)} blocks not handed back"
            assert not fa.foreign, f"fail_at={k}: foreign blocks released"
    finally:
        tpg.tpg_set_allocator(None)
        tpg._install_torch_allocator()
    # the library still gives exact results with its usual allocator
    (off, vert), (toff, tvert) = _run_sequence(cfg)
    assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, "PPs after the sweep")
    assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, "TPs after the sweep")


class _CappedAllocator:
    """Device blocks from torch's caching allocator while the bytes held stay
    within `cap`; NULL for a request that would pass it."""

    def __init__(self, cap):
        self.cap = cap
        self.live = {}
        self.refused = 0

    def alloc(self, nbytes, stream):
        import torch

        if sum(self.live.values()) + nbytes > self.cap:
            self.refused += 1
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        self.live[p] = nbytes
        return p

    def release(self, ptr, stream):
        import torch

        if self.live.pop(ptr, None) is not None:
            torch.cuda.caching_allocator_delete(int(ptr))


def test_capacity_hints_beyond_memory_are_halved_and_stay_exact():
    import torch

    cfg = G.diamond_chain(14)
    ref = oracle.run_cfg(cfg, test_paths=True)
    cap = 1 << 28
    ca = _CappedAllocator(cap)
    try:
        tpg.tpg_set_allocator(ca.alloc, ca.release)
        with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
            # 512 GiB of arena, a 2^32-path frontier, 2^36 PP references
            tpg.tpg_set_capacity(h, 1 << 36, 1 << 32, 1 << 36)
            with tpg.tpg_prime_paths(h) as pp, tpg.tpg_test_paths(h) as tp:
                off, vert = pp.host_arrays()[1:]
                toff, tvert = tp.host_arrays()[1:]
            st = tpg.tpg_get_stats(h)
        assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, "PPs")
        assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, "TPs")
        assert ca.refused > 0
        assert 0 < st["arena_bytes_alloc"] <= cap
        torch.cuda.synchronize()
        tpg.tpg_release_cached_memory()
        assert not ca.live
    finally:
        tpg.tpg_set_allocator(None)
        tpg._install_torch_allocator()
