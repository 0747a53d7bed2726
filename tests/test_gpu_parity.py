"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Every comparison is bit-exact: the outputs are integer vertex sequences in
canonical order (offsets int64, vertices int32).
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


def gpu_run(cfg, location=tpg.TPG_RESULT_HOST, test_paths=True, capacity=None, shape=None):
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=location) as h:
        if capacity:
            tpg.tpg_set_capacity(h, *capacity)
        if shape:
            tpg.tpg_set_tile_shape(h, *shape)
        pp = tpg.tpg_prime_paths(h)
        ppa = pp.host_arrays()
        assert pp.num_vertices == int(ppa[1][-1])  # the count the library reports, read from offsets
        pp.free()
        tpa = None
        if test_paths:
            tp = tpg.tpg_test_paths(h)
            tpa = tp.host_arrays()
            assert tp.num_vertices == int(tpa[1][-1])
            tp.free()
        stats = tpg.tpg_get_stats(h)
    return ppa, tpa, stats


def check_cfg(cfg, test_paths=True, location=tpg.TPG_RESULT_HOST, capacity=None, shape=None, ref=None):
    ref = ref or oracle.run_cfg(cfg, test_paths=test_paths)
    (gp, off, vert), tpa, stats = gpu_run(cfg, location, test_paths, capacity, shape)
    assert list(gp) == [0, len(off) - 1]
    assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, f"{cfg.name} PP")
    assert stats["simple_paths"] == ref.n_simple
    if test_paths:
        tgp, toff, tvert = tpa
        assert list(tgp) == [0, len(toff) - 1]
        assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, f"{cfg.name} TP")
    return ref, stats


def test_fig1_worked_example():
    cfg, rows = fig1_cfg()
    ref, stats = check_cfg(cfg)
    assert stats["prime_paths"] == 19


def test_config1_structured_24():
    ref, stats = check_cfg(G.config1_cfg())
    assert stats["prime_paths"] == ref.num_pp


@pytest.mark.parametrize("k", [1, 2, 3, 7, 10])
def test_diamond_chain_small(k):
    ref, stats = check_cfg(G.diamond_chain(k))
    assert stats["prime_paths"] == 2 ** k


def test_diamond_chain_k22_full():
    """The 2^22-PP chain, compared in full and with its closed forms."""
    cfg = G.diamond_chain(22)
    ref, stats = check_cfg(cfg, test_paths=True)
    assert stats["prime_paths"] == 4_194_304
    assert stats["simple_paths"] == 67_108_695
    assert stats["pp_vertices"] == 4_194_304 * 45
    assert stats["peak_level_nodes"] == 8_388_608


def test_config3_cyclic_120():
    cfg = G.config3_cfg()
    ref, stats = check_cfg(cfg)
    assert stats["prime_paths"] == 1_086_398


@pytest.mark.parametrize("r", [29, 30, 31, 32, 33, 61, 62, 63, 64, 93, 94, 95, 126, 127, 128, 158, 190, 254, 255])
def test_bitset_word_boundaries(r):
    check_cfg(ring_with_tail(r))


@pytest.mark.parametrize("r", [300, 1000])
def test_wide_bitsets(r):
    check_cfg(ring_with_tail(r))


def test_max_vertices_ring():
    cfg = ring_with_tail(tpg.TPG_MAX_N - 2)
    assert cfg.n == tpg.TPG_MAX_N
    check_cfg(cfg, test_paths=False)


@pytest.mark.parametrize("seed", range(10))
def test_random_digraphs_wrapped(seed):
    rng = G.SplitMix64(1000 + seed)
    k = rng.randint(4, 9)
    inner = G.random_digraph(k, 0.35, 77 + seed, self_loops=(seed % 2 == 0))
    check_cfg(wrap_digraph(inner))


@pytest.mark.parametrize("seed", [G.BATCH_SEED0 + i for i in range(8)])
def test_batch_graphs_single(seed):
    check_cfg(G.random_cfg(seed))


def test_minimal_graph():
    rp, col = G.csr_from_arcs(2, [(0, 1)])
    ref, stats = check_cfg(G.CFG(2, rp, col, 0, 1, "edge"))
    assert stats["prime_paths"] == 1


def test_device_result_location():
    cfg = G.config3_cfg()
    ref = oracle.run_cfg(cfg)
    (gp, off, vert), (tgp, toff, tvert), _ = gpu_run(cfg, location=tpg.TPG_RESULT_DEVICE)
    assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, "device PP")
    assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, "device TP")


def test_device_load():
    import torch

    cfg = G.config1_cfg()
    ref = oracle.run_cfg(cfg)
    rp = torch.as_tensor(cfg.row_ptr, device="cuda")
    col = torch.as_tensor(cfg.col, device="cuda")
    with tpg.tpg_load_cfg_device(cfg.n, cfg.m, rp, col, cfg.entry, cfg.exit) as h:
        pp = tpg.tpg_prime_paths(h)
        gp, off, vert = pp.host_arrays()
        pp.free()
    assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, "device-load PP")


def test_device_load_rejects_bad_csr():
    import torch

    rp = torch.as_tensor(np.array([0, 1, 2], np.int32), device="cuda")
    col = torch.as_tensor(np.array([1, 0], np.int32), device="cuda")  # arc into the entry
    with pytest.raises(tpg.TPGError) as e:
        tpg.tpg_load_cfg_device(2, 2, rp, col, 0, 1)
    assert e.value.code == tpg.TPG_EINVAL


def _chain_csr(n):
    """0 -> 1 -> ... -> n-1: one PP, the whole chain."""
    rp = np.minimum(np.arange(n + 1), n - 1).astype(np.int32)
    col = np.arange(1, n, dtype=np.int32)
    return rp, col


# 6 vertices take the single-block preprocessing, 1500 the general one
@pytest.mark.parametrize("n", [6, 1500])
@pytest.mark.parametrize("bad", ["arc_into_entry", "vertex_out_of_range", "arc_out_of_exit", "row_ptr_start",
                                 "entry_is_exit", "unsorted_row"])
def test_device_load_rejects_bad_csr_on_both_preprocessing_paths(n, bad):
    import torch

    rp, col = _chain_csr(n)
    entry, exit = 0, n - 1
    if bad == "arc_into_entry":
        col[n // 2] = 0
    elif bad == "vertex_out_of_range":
        col[1] = n
    elif bad == "arc_out_of_exit":
        rp[n] = n
        col = np.append(col, 1).astype(np.int32)
    elif bad == "row_ptr_start":
        rp[0] = 1
    elif bad == "entry_is_exit":
        exit = 0
    elif bad == "unsorted_row":
        # vertex 1 gets arcs (3, 2): out of order
        rp = np.concatenate([[0, 1], np.arange(3, n + 1), [n]]).astype(np.int32)
        col = np.concatenate([[1, 3, 2], np.arange(3, n)]).astype(np.int32)
    m = int(rp[n])
    assert len(col) >= m
    with pytest.raises(tpg.TPGError) as e:
        tpg.tpg_load_cfg_device(n, m, torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"),
                                entry, exit)
    assert e.value.code == tpg.TPG_EINVAL


def _looped_chain(n):
    """0 -> 1 -> ... -> n-1 with a back arc i -> i-5 at every tenth vertex:
    loops give PPs off the entry-exit line, so TPs get prefixes and suffixes."""
    arcs = [(i, i + 1) for i in range(n - 1)] + [(i, i - 5) for i in range(10, n - 1, 10)]
    rp, col = G.csr_from_arcs(n, arcs)
    return G.CFG(n=n, row_ptr=rp, col=col, entry=0, exit=n - 1, name=f"looped_chain_{n}")


# 600 vertices take the single-block preprocessing, 1100 the general one
@pytest.mark.parametrize("n", [600, 1100])
def test_tours_on_both_preprocessing_paths(n):
    import torch

    cfg = _looped_chain(n)
    ref, _ = check_cfg(cfg)  # host load
    assert len(ref.tp_offsets) > 2 and len(ref.tp_vertices) > n
    rp = torch.as_tensor(cfg.row_ptr, device="cuda")
    col = torch.as_tensor(cfg.col, device="cuda")
    with tpg.tpg_load_cfg_device(cfg.n, cfg.m, rp, col, cfg.entry, cfg.exit) as h:
        tp = tpg.tpg_test_paths(h)
        _, toff, tvert = tp.host_arrays()
        tp.free()
    assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, f"{cfg.name} device-load TP")


@pytest.mark.parametrize("n", [6, 1000, 1025, 1500])
def test_device_load_chain_on_both_preprocessing_paths(n):
    import torch

    rp, col = _chain_csr(n)
    with tpg.tpg_load_cfg_device(n, n - 1, torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"),
                                 0, n - 1) as h:
        pp = tpg.tpg_prime_paths(h)
        tp = tpg.tpg_test_paths(h)
        _, off, vert = pp.host_arrays()
        _, toff, tvert = tp.host_arrays()
        pp.free()
        tp.free()
    assert list(off) == [0, n] and list(vert) == list(range(n))
    assert list(toff) == [0, n] and list(tvert) == list(range(n))


def test_unreachable_reports_error():
    rp, col = G.csr_from_arcs(4, [(0, 1), (1, 3), (2, 2)])
    with tpg.tpg_load_cfg(4, rp, col, 0, 3) as h:
        pp = tpg.tpg_prime_paths(h)
        assert pp.to_lists() == [(0, 1, 3), (2, 2)]
        pp.free()
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_test_paths(h)
        assert e.value.code == tpg.TPG_EUNREACH


def test_repeated_calls_are_identical():
    cfg = G.config3_cfg()
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        outs = []
        for _ in range(3):
            p = tpg.tpg_prime_paths(h)
            outs.append(p.host_arrays())
            p.free()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


@pytest.fixture(scope="module")
def config3_ref():
    return oracle.run_cfg(G.config3_cfg())


@pytest.mark.parametrize("caps", [(200, 130, 7), (5000, 700, 64), (100000, 4000, 100000)])
def test_tiny_arena_resumes_at_the_failing_level(caps, config3_ref):
    """Arena, frontier and PP capacities far below the need: the launch stops
    and resumes with new segments; the result must not change."""
    ref, stats = check_cfg(G.config3_cfg(), capacity=caps, ref=config3_ref)
    assert stats["attempts"] > 1
    assert stats["prime_paths"] == ref.num_pp


@pytest.mark.parametrize("shape", [(256, 1), (256, 2), (256, 4), (512, 1), (512, 2), (1024, 1)])
def test_every_tile_shape(shape, config3_ref):
    ref, stats = check_cfg(G.config3_cfg(), shape=shape, ref=config3_ref)
    assert (stats["tile_block"], stats["tile_items"]) == shape


@pytest.fixture(scope="module")
def chain20_ref():
    return oracle.run_cfg(G.diamond_chain(20))


@pytest.mark.parametrize("split", [1, 2, 3, 4])
@pytest.mark.parametrize("which", ["config3", "chain20"])
def test_every_work_split(split, which, config3_ref, chain20_ref):
    """Cutting each chunk into `split` work units changes which warp does
    what, never the result: C3's levels have one-tile chunks (later parts
    empty), the k=20 chain's largest levels chunks of over a hundred paths."""
    cfg, ref = (G.config3_cfg(), config3_ref) if which == "config3" else (G.diamond_chain(20), chain20_ref)
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        tpg.tpg_set_work_split(h, split)
        pp = tpg.tpg_prime_paths(h)
        _, off, vert = pp.host_arrays()
        pp.free()
        tp = tpg.tpg_test_paths(h)
        _, toff, tvert = tp.host_arrays()
        tp.free()
    assert_paths_equal(off, vert, ref.pp_offsets, ref.pp_vertices, f"{which} split {split} PP")
    assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, f"{which} split {split} TP")


def test_unsupported_work_split_rejected():
    cfg = G.config1_cfg()
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        for bad in (0, 5, -1):
            with pytest.raises(tpg.TPGError) as e:
                tpg.tpg_set_work_split(h, bad)
            assert e.value.code == tpg.TPG_EINVAL


def test_unsupported_tile_shape_rejected():
    cfg = G.config1_cfg()
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit) as h:
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_set_tile_shape(h, 512, 4)
        with pytest.raises(tpg.TPGError) as e:
            tpg.tpg_set_tile_shape(h, 128, 1)
        assert e.value.code == tpg.TPG_EINVAL


@pytest.mark.parametrize("location", [tpg.TPG_RESULT_HOST, tpg.TPG_RESULT_DEVICE])
def test_tp_list_shares_the_pp_list_when_every_tp_is_its_pp(location):
    """Every PP of a diamond chain runs entry -> exit, so its TP is itself: the
    TP result shares the PP result's storage, and either outlives the other."""
    cfg = G.diamond_chain(6)
    ref = oracle.run_cfg(cfg)
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=location) as h:
        pp = tpg.tpg_prime_paths(h)
        tp = tpg.tpg_test_paths(h)
        if location == tpg.TPG_RESULT_HOST:
            assert tp.vertices.ctypes.data == pp.vertices.ctypes.data
        else:
            assert tp.vertices.data_ptr() == pp.vertices.data_ptr()
        pp.free()
        _, toff, tvert = tp.host_arrays()
        assert_paths_equal(toff, tvert, ref.tp_offsets, ref.tp_vertices, "shared TP")
        tp.free()
    # a graph with prefixes and suffixes gets its own TP list
    cfg = G.config1_cfg()
    with tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=location) as h:
        pp = tpg.tpg_prime_paths(h)
        tp = tpg.tpg_test_paths(h)
        if location == tpg.TPG_RESULT_HOST:
            assert tp.vertices.ctypes.data != pp.vertices.ctypes.data
        pp.free()
        tp.free()
