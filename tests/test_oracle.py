"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these tests use the CUDA library.  Each pin is chosen so that a
plausible slip in the oracle (a missing left-extension test, a wrong cycle
rule, a wrong tie-break, an unsorted list) fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import oracle
from oracle import literal
from paper_2210_16998_gb300 import cfggen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_fig1():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_binarysearch0.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                rows.append((parts[0], tuple(int(x) for x in parts[1:])))
    return rows


def fig1_cfg():
    rows = load_fig1()
    arcs = {(a, b) for _, p in rows for a, b in zip(p, p[1:])}
    rp, col = G.csr_from_arcs(11, arcs)
    return G.CFG(11, rp, col, 0, 10, "fig1"), rows


# ---------------------------------------------------------------------------
# the paper's worked example (Sec. 2.1, Fig. 1)
# ---------------------------------------------------------------------------
def test_fig1_worked_example_19_pps():
    cfg, rows = fig1_cfg()
    assert cfg.m == 13
    res = oracle.run_cfg(cfg)
    listed = sorted(p for _, p in rows)
    assert res.pp_list() == listed
    assert res.num_pp == 19
    kinds = {}
    for k, _ in rows:
        kinds[k] = kinds.get(k, 0) + 1
    # 11 internal + 2 complete + 4 exit + 2 entry (Sec. 2.1, last sentence)
    assert kinds == {"internal": 11, "complete": 2, "exit": 4, "entry": 2}
    # Def. 1's example PP
    assert (2, 3, 4, 8, 2) in res.pp_list()


def test_fig1_literal_oracle_agrees():
    cfg, rows = fig1_cfg()
    lit = literal.prime_paths(cfg.n, literal.succ_lists(cfg.n, cfg.row_ptr, cfg.col))
    assert lit == sorted(p for _, p in rows)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_diamond_chain_closed_form_small(k):
    cfg = G.diamond_chain(k)
    res = oracle.run_cfg(cfg)
    pps = res.pp_list()
    assert len(pps) == 2 ** k
    assert all(len(p) == 2 * k + 1 and p[0] == 0 and p[-1] == 3 * k for p in pps)
    # simple paths of the chain: 16 * 2^k - 7k - 15
    assert res.n_simple == 16 * 2 ** k - 7 * k - 15
    # TPs = PPs (every PP already runs entry -> exit)
    assert res.tp_list() == pps
    if k <= 3:
        assert literal.prime_paths(cfg.n, literal.succ_lists(cfg.n, cfg.row_ptr, cfg.col)) == pps


def test_diamond_chain_k22_counts():
    cfg = G.diamond_chain(22)
    assert (cfg.n, cfg.m) == (67, 88)
    res = oracle.run_cfg(cfg, test_paths=False, want_paths=False)
    assert res.num_pp == 4_194_304
    assert res.pp_len_counts[45] == 4_194_304
    assert res.n_simple == 67_108_695 == 16 * 2 ** 22 - 7 * 22 - 15
    # peak level: 8,388,608 paths at 42..44 vertices
    assert res.len_counts.max() == 8_388_608
    assert int(np.nonzero(res.len_counts)[0].max()) == 45


@pytest.mark.parametrize("n", [1, 2, 3, 7, 32, 33])
def test_ring_rotations(n):
    cfg = G.ring(n)
    res = oracle.run_cfg(cfg, test_paths=False)
    pps = res.pp_list()
    assert len(pps) == n
    assert sorted(pps) == sorted(tuple((r + i) % n for i in range(n + 1)) for r in range(n))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_complete_digraph_cycles(n):
    cfg = G.complete_digraph(n)
    res = oracle.run_cfg(cfg, test_paths=False)
    expected = sum(math.factorial(n) // math.factorial(n - k) for k in range(2, n + 1))
    assert res.num_pp == expected
    assert all(p[0] == p[-1] for p in res.pp_list())


# ---------------------------------------------------------------------------
# per-root volumes (the sizer's labels and the count-only mode): closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 4, 9])
def test_diamond_chain_per_root_counts(k):
    # d_i = 3i, a_i = 3i+1, b_i = 3i+2.  From d_i a path ends at d_{i+j}
    # (2^j ways, j = 0..k-i) or at a or b of diamond i+j (2^{j+1} ways,
    # j = 0..k-i-1): 2^{k-i+2} - 3 paths.  From a_i or b_i: the one-vertex
    # path plus the single arc into d_{i+1} followed by any path from
    # d_{i+1}: 2^{k-i+1} - 2.  Only the 2^k entry-to-exit paths (2k+1
    # vertices each, all rooted at d_0) are prime.
    cfg = G.diamond_chain(k)
    res = oracle.run_cfg(cfg, test_paths=False, want_paths=False)
    paths = np.zeros(cfg.n, np.int64)
    for i in range(k + 1):
        paths[3 * i] = 2 ** (k - i + 2) - 3
    for i in range(k):
        paths[3 * i + 1] = paths[3 * i + 2] = 2 ** (k - i + 1) - 2
    np.testing.assert_array_equal(res.root_paths, paths)
    pps = np.zeros(cfg.n, np.int64)
    pps[0] = 2 ** k
    np.testing.assert_array_equal(res.root_pps, pps)
    np.testing.assert_array_equal(res.root_pp_ints, pps * (2 * k + 1))


@pytest.mark.parametrize("n", [1, 2, 5, 33])
def test_ring_per_root_counts(n):
    # from each root: n acyclic paths (1..n vertices) and the closed cycle;
    # the cycle (n+1 vertices) is the root's only PP
    res = oracle.run_cfg(G.ring(n), test_paths=False, want_paths=False)
    np.testing.assert_array_equal(res.root_paths, np.full(n, n + 1))
    np.testing.assert_array_equal(res.root_pps, np.ones(n))
    np.testing.assert_array_equal(res.root_pp_ints, np.full(n, n + 1))


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_complete_digraph_per_root_counts(n):
    # from r: (n-1)!/(n-j)! acyclic paths of j vertices (j = 1..n); each with
    # j >= 2 also closes a cycle of j+1 vertices, and those cycles are the
    # root's PPs (every acyclic path can still close, so none is prime)
    arr = [math.factorial(n - 1) // math.factorial(n - j) for j in range(1, n + 1)]
    cyc = arr[1:]
    res = oracle.run_cfg(G.complete_digraph(n), test_paths=False, want_paths=False)
    np.testing.assert_array_equal(res.root_paths, np.full(n, sum(arr) + sum(cyc)))
    np.testing.assert_array_equal(res.root_pps, np.full(n, sum(cyc)))
    np.testing.assert_array_equal(res.root_pp_ints, np.full(n, sum((j + 1) * c for j, c in zip(range(2, n + 1), cyc))))


@pytest.mark.parametrize("seed", range(8))
def test_per_root_counts_vs_literal(seed):
    # brute force: group the literal oracle's simple paths and PPs by first vertex
    cfg = G.random_digraph(6, 0.35, 1000 + seed, self_loops=(seed % 2 == 0))
    succ = literal.succ_lists(cfg.n, cfg.row_ptr, cfg.col)
    sp_all = literal.simple_paths(cfg.n, succ)
    pps = literal.prime_paths(cfg.n, succ)
    res = oracle.run(cfg.n, cfg.row_ptr, cfg.col, want_paths=False)
    np.testing.assert_array_equal(res.root_paths, np.bincount([p[0] for p in sp_all], minlength=cfg.n))
    np.testing.assert_array_equal(res.root_pps, np.bincount([p[0] for p in pps], minlength=cfg.n))
    np.testing.assert_array_equal(res.root_pp_ints,
                                  np.bincount([p[0] for p in pps], weights=[len(p) for p in pps],
                                              minlength=cfg.n).astype(np.int64))


def test_self_loop_and_isolated_vertex():
    # 0 -> 0 self-loop, 1 isolated: PPs are <0,0> and <1>
    rp, col = G.csr_from_arcs(2, [(0, 0)])
    res = oracle.run(2, rp, col)
    assert res.pp_list() == [(0, 0), (1,)]


# ---------------------------------------------------------------------------
# exhaustive / random agreement with the literal definition
# ---------------------------------------------------------------------------
def _all_digraphs(n, self_loops):
    pairs = [(u, v) for u in range(n) for v in range(n) if self_loops or u != v]
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


@pytest.mark.parametrize("n,self_loops", [(1, True), (2, True), (3, True), (4, False)])
def test_exhaustive_small_digraphs(n, self_loops):
    for arcs in _all_digraphs(n, self_loops):
        rp, col = G.csr_from_arcs(n, arcs)
        assert oracle.run(n, rp, col).pp_list() == \
            literal.prime_paths(n, literal.succ_lists(n, rp, col)), arcs


def test_n4_with_self_loops_sampled():
    pairs = [(u, v) for u in range(4) for v in range(4)]
    rng = G.SplitMix64(44)
    for _ in range(1500):
        mask = rng.next_u64() & 0xFFFF
        arcs = [pairs[i] for i in range(16) if mask >> i & 1]
        rp, col = G.csr_from_arcs(4, arcs)
        assert oracle.run(4, rp, col).pp_list() == \
            literal.prime_paths(4, literal.succ_lists(4, rp, col)), arcs


@pytest.mark.parametrize("seed", range(12))
def test_random_digraphs_vs_literal(seed):
    rng = G.SplitMix64(seed)
    n = rng.randint(5, 7)
    cfg = G.random_digraph(n, 0.3, seed * 7 + 1, self_loops=(seed % 3 == 0))
    assert oracle.run(cfg.n, cfg.row_ptr, cfg.col).pp_list() == \
        literal.prime_paths(cfg.n, literal.succ_lists(cfg.n, cfg.row_ptr, cfg.col))


# ---------------------------------------------------------------------------
# invariants (completeness, maximality, touring)
# ---------------------------------------------------------------------------
def _arcs(cfg):
    return {(u, int(w)) for u in range(cfg.n) for w in cfg.succ(u)}


def _pred_lists(cfg):
    pred = [[] for _ in range(cfg.n)]
    for u in range(cfg.n):
        for w in cfg.succ(u):
            pred[int(w)].append(u)
    return pred


def check_invariants(cfg, res):
    arcs = _arcs(cfg)
    pred = _pred_lists(cfg)
    pps = res.pp_list()
    assert pps == sorted(pps), "canonical order"
    assert len(set(pps)) == len(pps), "no duplicates"
    covered = set()
    for p in pps:
        assert literal.is_simple(p)
        assert all((a, b) in arcs for a, b in zip(p, p[1:]))
        covered |= set(zip(p, p[1:]))
        # no simple one-vertex extension (maximality, Def. 1)
        for w in cfg.succ(p[-1]):
            assert not literal.is_simple(p + (int(w),))
        for u in pred[p[0]]:
            assert not literal.is_simple((u,) + p)
        # every prefix is simple (completeness argument, Sec. 5.4)
        for i in range(1, len(p)):
            assert literal.is_simple(p[:i])
    assert covered == arcs, "every arc lies on some PP"
    if res.tp_offsets is not None:
        tps = res.tp_list()
        assert tps == sorted(set(tps)), "TPs sorted and unique"
        assert len(tps) <= len(pps)
        for t in tps:
            assert t[0] == cfg.entry and t[-1] == cfg.exit
            assert all((a, b) in arcs for a, b in zip(t, t[1:]))
        tp_str = [",".join(map(str, t)) for t in tps]
        for p in pps:
            ps = ",".join(map(str, p))
            assert any(("," + ps + ",") in ("," + s + ",") for s in tp_str), p


def test_invariants_config1():
    cfg = G.config1_cfg()
    check_invariants(cfg, oracle.run_cfg(cfg))


def test_invariants_fig1():
    cfg, _ = fig1_cfg()
    check_invariants(cfg, oracle.run_cfg(cfg))


@pytest.mark.parametrize("seed", [G.BATCH_SEED0 + i for i in range(6)])
def test_invariants_batch_graphs(seed):
    cfg = G.random_cfg(seed)
    check_invariants(cfg, oracle.run_cfg(cfg))


# ---------------------------------------------------------------------------
# BFS tables and the test-path construction
# ---------------------------------------------------------------------------
def _check_bfs(cfg):
    dist, pred = oracle.bfs_tables(cfg.n, cfg.row_ptr, cfg.col)
    adj = sp.csr_matrix((np.ones(cfg.m), cfg.col, cfg.row_ptr), shape=(cfg.n, cfg.n))
    ref = shortest_path(adj, method="D", unweighted=True)
    ref = np.where(np.isinf(ref), -1, ref).astype(np.int32)
    np.testing.assert_array_equal(dist, ref)
    preds = _pred_lists(cfg)
    for a in range(cfg.n):
        for x in range(cfg.n):
            if x == a or dist[a, x] < 0:
                assert pred[a, x] == -1
            else:
                cands = [u for u in preds[x] if dist[a, u] == dist[a, x] - 1]
                assert pred[a, x] == min(cands)
    return dist, pred


def test_bfs_tables_against_scipy():
    for cfg in (G.config1_cfg(), fig1_cfg()[0], G.diamond_chain(4), G.config3_cfg()):
        _check_bfs(cfg)


def test_test_paths_construction_fig1():
    cfg, _ = fig1_cfg()
    res = oracle.run_cfg(cfg)
    dist, pred = _check_bfs(cfg)
    tps = set(res.tp_list())
    for p in res.pp_list():
        # prefix: a shortest entry -> p[0] path; suffix: shortest p[-1] -> exit
        f, l = p[0], p[-1]
        assert dist[cfg.entry, f] >= 0 and dist[l, cfg.exit] >= 0
        lens = dist[cfg.entry, f] + len(p) + dist[l, cfg.exit]
        match = [t for t in tps if len(t) == lens and
                 t[dist[cfg.entry, f]:dist[cfg.entry, f] + len(p)] == p]
        assert match, p
    # the TP set itself, derived by hand from the 13 arcs (golden file)
    golden_map, golden_tps = load_fig1_tps()
    assert res.tp_list() == golden_tps
    assert [p for p, _ in golden_map] == res.pp_list()
    for p, t in golden_map:
        # each PP sits in its TP right after the shortest entry prefix
        d = int(dist[cfg.entry, p[0]])
        assert t[d:d + len(p)] == p and t in tps


def load_fig1_tps():
    pps, tps = [], []
    with open(os.path.join(GOLDEN, "fig1_test_paths.txt")) as f:
        for line in f:
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            if parts[0] == "pp":
                i = parts.index(":")
                pps.append((tuple(int(x) for x in parts[1:i]), tuple(int(x) for x in parts[i + 1:])))
            elif parts[0] == "tp":
                tps.append(tuple(int(x) for x in parts[1:]))
    return pps, tps


def test_unreachable_pp_reports_error():
    # 0 -> 1 -> 3 (exit), 2 -> 2 self-loop unreachable from entry
    rp, col = G.csr_from_arcs(4, [(0, 1), (1, 3), (2, 2)])
    with pytest.raises(oracle.OracleError) as e:
        oracle.run(4, rp, col, 0, 3, test_paths=True)
    assert e.value.code == oracle.ORC_EUNREACH


# ---------------------------------------------------------------------------
# the seeded generator (input side)
# ---------------------------------------------------------------------------
def test_generator_deterministic_and_well_formed():
    for mk in (G.config1_cfg, G.config3_cfg, lambda: G.random_cfg(G.BATCH_SEED0 + 5)):
        a, b = mk(), mk()
        np.testing.assert_array_equal(a.row_ptr, b.row_ptr)
        np.testing.assert_array_equal(a.col, b.col)
        indeg = np.bincount(a.col, minlength=a.n)
        assert indeg[a.entry] == 0
        assert a.row_ptr[a.exit + 1] - a.row_ptr[a.exit] == 0
        for u in range(a.n):
            s = a.succ(u)
            assert np.all(np.diff(s) > 0)
    c1 = G.config1_cfg()
    assert c1.n == 24 and int(np.diff(c1.row_ptr).max()) <= 2
    c3 = G.config3_cfg()
    assert c3.n == 120 and int(np.diff(c3.row_ptr).max()) == 6


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: first outputs of the published generator
    r = G.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    assert r.next_u64() == 0x06C45D188009454F


# ---------------------------------------------------------------------------
# the root-parallel driver (all-core CPU baseline) gives the serial result
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("make", [G.config1_cfg, G.config3_cfg, lambda: G.diamond_chain(9),
                                  lambda: fig1_cfg()[0], lambda: G.random_cfg(G.BATCH_SEED0 + 7)],
                         ids=["config1", "config3", "chain9", "fig1", "random"])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_driver_equals_serial(make, threads):
    cfg = make()
    a = oracle.run_cfg(cfg, test_paths=True)
    b = oracle.run_cfg_parallel(cfg, test_paths=True, threads=threads)
    for f in ("len_counts", "pp_len_counts", "root_paths", "root_pp_ints", "root_pps",
              "pp_offsets", "pp_vertices", "tp_offsets", "tp_vertices"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    assert a.n_simple == b.n_simple


def test_parallel_driver_counts_only_and_digraphs():
    for seed in range(5):
        cfg = G.random_digraph(7, 0.35, 300 + seed, self_loops=True)
        a = oracle.run(cfg.n, cfg.row_ptr, cfg.col)
        b = oracle.run_parallel(cfg.n, cfg.row_ptr, cfg.col, threads=4)
        assert a.pp_list() == b.pp_list()
        c = oracle.run_parallel(cfg.n, cfg.row_ptr, cfg.col, want_paths=False, threads=4)
        np.testing.assert_array_equal(a.root_pps, c.root_pps)
