"""Pins of the oracle's longest-first touring (the Ammann-Offutt TP
construction as Sec. 7.3 describes it: the longest uncovered PP first,
extended to the entry and the exit, until every PP is covered).

The oracle looks the simple windows of each chosen TP up in a hash set of the
PPs.  These tests check it against (1) a brute-force simulation of the rule
that tests every PP against every chosen TP by plain substring search, on
small graphs; (2) closed forms; (3) invariants that any correct result
satisfies; (4) a brute-force minimum set cover of the PPs by one-per-PP TPs,
which the greedy result can never beat.  No test uses the CUDA library.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2210_16998_gb300 import cfggen as G

from .helpers import ring_with_tail, wrap_digraph
from .test_oracle import fig1_cfg


def bfs_path(pred, dist, a, b):
    """path(a -> b) read backwards from b through the lowest-id predecessor
    table (pinned against scipy in test_oracle.py)."""
    if dist[a, b] < 0:
        return None
    out = [b]
    while out[-1] != a:
        out.append(int(pred[a, out[-1]]))
    return out[::-1]


def tp_of(p, pred, dist, entry, exit):
    pre = bfs_path(pred, dist, entry, p[0])
    suf = bfs_path(pred, dist, p[-1], exit)
    return tuple(pre[:-1]) + tuple(p) + tuple(suf[1:])


def is_window(q, t):
    """q is a contiguous subsequence of t"""
    k = len(q)
    return any(t[i:i + k] == q for i in range(len(t) - k + 1))


def greedy_bruteforce(cfg, pps):
    dist, pred = oracle.bfs_tables(cfg.n, cfg.row_ptr, cfg.col)
    order = sorted(range(len(pps)), key=lambda i: (-len(pps[i]), i))
    covered = [False] * len(pps)
    chosen = []
    for i in order:
        if covered[i]:
            continue
        t = tp_of(pps[i], pred, dist, cfg.entry, cfg.exit)
        chosen.append(t)
        for j, q in enumerate(pps):
            if not covered[j] and is_window(q, t):
                covered[j] = True
    return sorted(chosen)


def while_chain(m):
    """entry -> h, h -> b1 -> ... -> bm -> h, h -> exit (ids: entry 0, h 1,
    b_i = i + 1, exit m + 2)"""
    arcs = [(0, 1), (1, 2)] + [(i + 1, i + 2) for i in range(1, m)] + [(m + 1, 1), (1, m + 2)]
    rp, col = G.csr_from_arcs(m + 3, arcs)
    return G.CFG(m + 3, rp, col, 0, m + 2, f"while{m}")


SMALL = [
    ("fig1", lambda: fig1_cfg()[0]),
    ("config1", G.config1_cfg),
    ("diamond-5", lambda: G.diamond_chain(5)),
    ("while-4", lambda: while_chain(4)),
    ("ring-tail-6", lambda: ring_with_tail(6)),
] + [(f"cfg-{s}", (lambda s=s: G.random_cfg(G.BATCH_SEED0 + s))) for s in range(20, 40)] + [
    (f"digraph-{s}", (lambda s=s: wrap_digraph(G.random_digraph(6, 0.4, s, self_loops=True)))) for s in range(6)]


@pytest.mark.parametrize("name,make", SMALL, ids=[c[0] for c in SMALL])
def test_greedy_equals_bruteforce_simulation(name, make):
    cfg = make()
    res = oracle.run_cfg(cfg, test_paths=True, greedy=True)
    pps = res.pp_list()
    if len(pps) > 3000:
        pytest.skip("brute force too slow")
    assert res.gtp_list() == greedy_bruteforce(cfg, pps)


@pytest.mark.parametrize("k", [1, 2, 3, 6, 10])
def test_greedy_diamond_chain_keeps_every_pp(k):
    # every PP runs entry -> exit with 2k + 1 vertices, so TP(p) = p and no
    # TP holds another PP: 2^k TPs, equal to the PPs
    cfg = G.diamond_chain(k)
    res = oracle.run_cfg(cfg, test_paths=False, greedy=True)
    assert len(res.gtp_list()) == 2 ** k
    assert res.gtp_list() == res.pp_list()


@pytest.mark.parametrize("m", [1, 2, 3, 7])
def test_greedy_while_chain_three_tps(m):
    # PPs: the m + 1 rotations of the loop, entry.h.b1..bm, b1..bm.h.exit,
    # entry.h.exit.  One lap (entry h b1..bm h exit) holds the two acyclic
    # long PPs and the rotation at h; two laps hold every rotation; entry h
    # exit is in neither
    cfg = while_chain(m)
    res = oracle.run_cfg(cfg, test_paths=True, greedy=True)
    lap = (1,) + tuple(range(2, m + 2))
    assert res.num_pp == m + 4
    assert res.gtp_list() == sorted([(0,) + lap + (1, m + 2), (0,) + lap + lap + (1, m + 2), (0, 1, m + 2)])


def _check_invariants(res):
    pps, tps, gtps = res.pp_list(), res.tp_list(), res.gtp_list()
    assert gtps == sorted(set(gtps))
    assert set(gtps) <= set(tps)  # each chosen TP is some TP(p)
    assert len(gtps) <= len(tps)
    # every PP is a window of a chosen TP (all windows up to the longest PP)
    kmax = max(len(q) for q in pps)
    windows = {t[i:j] for t in gtps for i in range(len(t)) for j in range(i + 1, min(len(t), i + kmax) + 1)}
    missing = [q for q in pps if q not in windows]
    assert not missing, missing[:3]


@pytest.mark.parametrize("seed", range(40, 60))
def test_greedy_invariants_on_generated_cfgs(seed):
    res = oracle.run_cfg(G.random_cfg(G.BATCH_SEED0 + seed), test_paths=True, greedy=True)
    if res.num_pp > 5000:
        pytest.skip("window sets too large for a quick check")
    _check_invariants(res)


@pytest.mark.parametrize("name,make", SMALL[:12], ids=[c[0] for c in SMALL[:12]])
def test_greedy_never_beats_minimum_cover(name, make):
    cfg = make()
    res = oracle.run_cfg(cfg, test_paths=True, greedy=True)
    pps, tps = res.pp_list(), res.tp_list()
    if len(tps) > 14:
        pytest.skip("set cover by brute force too slow")
    cover = [{j for j, q in enumerate(pps) if is_window(q, t)} for t in tps]
    everything = set(range(len(pps)))
    best = next(r for r in range(1, len(tps) + 1)
                if any(set().union(*(cover[i] for i in c)) == everything
                       for c in itertools.combinations(range(len(tps)), r)))
    assert best <= len(res.gtp_list()) <= len(tps)


def test_greedy_smaller_than_one_tp_per_pp_on_config1():
    # the 24-vertex config: 76 PPs, 45 distinct TP(p), fewer by touring
    res = oracle.run_cfg(G.config1_cfg(), test_paths=True, greedy=True)
    assert len(res.gtp_list()) < len(res.tp_list())
    _check_invariants(res)
