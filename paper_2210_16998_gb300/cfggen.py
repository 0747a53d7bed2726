"""Seeded synthetic control-flow graphs (inputs only).

This module builds the inputs that both the CUDA path and the CPU oracle are
run on.  It holds none of the prime-path arithmetic: it only draws program
shapes, lowers them to a control-flow graph and returns int32 CSR arrays.

The paper's benchmark is a set of Apache Commons CFGs "synthetically augmented
with loops and conditionals" (Sec. 6, Table 1); those graphs are not
available, so these seeded graphs stand in for them.  A program is a statement
tree over the grammar

    Stmt := Block | If(S1, S2) | While(S) | Switch(S1 .. Sk)

and is lowered with one node per Block and per decision (If condition, While
header, Switch head); a Program gets a dedicated entry Block (in-degree 0) and
a dedicated exit node (out-degree 0), the start/end vertices of Problem 1.
Vertex ids are assigned in pre-order; adjacency lists are sorted ascending
and free of duplicate arcs.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition: the state advances by the golden gamma
0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 64-bit finaliser.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood 2014)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive) by rejection sampling."""
        span = hi - lo + 1
        if span <= 0:
            raise ValueError("empty range")
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            x = self.next_u64()
            if x < limit:
                return lo + x % span


# ----------------------------------------------------------------------------
# statement trees
# ----------------------------------------------------------------------------
@dataclass
class Stmt:
    kind: str                      # "block" | "if" | "while" | "switch"
    bodies: list = field(default_factory=list)   # list of Seq (list[Stmt])
    vid: int = -1

    def size(self) -> int:
        return 1 + sum(seq_size(b) for b in self.bodies)


def seq_size(seq) -> int:
    return sum(s.size() for s in seq)


def _make(kind: str, fanout: int = 2) -> Stmt:
    if kind == "block":
        return Stmt("block")
    if kind == "if":
        return Stmt("if", [[Stmt("block")], [Stmt("block")]])
    if kind == "while":
        return Stmt("while", [[Stmt("block")]])
    if kind == "switch":
        return Stmt("switch", [[Stmt("block")] for _ in range(fanout)])
    raise ValueError(kind)


def _min_size(kind: str, fanout: int = 2) -> int:
    return {"block": 1, "if": 3, "while": 2, "switch": 1 + fanout}[kind]


def _slots(body, max_depth: int):
    """All (seq, depth) pairs where a construct may be inserted.

    depth = number of constructs enclosing the seq; a construct inserted into
    a seq at depth d is itself nested d+1 deep.  Only seqs with
    d < max_depth are returned.
    """
    out = []

    def walk(seq, d):
        if d < max_depth:
            out.append((seq, d))
        for s in seq:
            for b in s.bodies:
                walk(b, d + 1)

    walk(body, 0)
    return out


def _all_seqs(body):
    out = []

    def walk(seq):
        out.append(seq)
        for s in seq:
            for b in s.bodies:
                walk(b)

    walk(body)
    return out


def _insert(rng: SplitMix64, seq, stmt: Stmt):
    pos = rng.randint(0, len(seq))
    seq.insert(pos, stmt)


def _pad_blocks(rng: SplitMix64, body, count: int):
    for _ in range(count):
        seqs = _all_seqs(body)
        _insert(rng, seqs[rng.randint(0, len(seqs) - 1)], Stmt("block"))


@dataclass
class CFG:
    """A control-flow graph as int32 CSR plus entry/exit ids."""

    n: int
    row_ptr: np.ndarray   # int32[n+1]
    col: np.ndarray       # int32[m]
    entry: int
    exit: int
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def succ(self, v: int):
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]


def csr_from_arcs(n: int, arcs) -> tuple[np.ndarray, np.ndarray]:
    """Sorted, duplicate-free int32 CSR from an iterable of (u, v) arcs."""
    adj = [set() for _ in range(n)]
    for u, v in arcs:
        adj[u].add(v)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for u in range(n):
        s = sorted(adj[u])
        row_ptr[u + 1] = row_ptr[u] + len(s)
        cols.extend(s)
    return row_ptr, np.asarray(cols, dtype=np.int32)


def lower_program(body, name: str = "") -> CFG:
    """Lower a statement tree to a CFG (entry = 0, exit = n-1, pre-order ids)."""
    counter = [1]                  # 0 is the entry block

    def number(seq):
        for s in seq:
            s.vid = counter[0]
            counter[0] += 1
            for b in s.bodies:
                number(b)

    number(body)
    exit_id = counter[0]
    n = exit_id + 1
    arcs = []

    def lower_seq(seq, nxt):
        for s in reversed(seq):
            nxt = lower_stmt(s, nxt)
        return nxt

    def lower_stmt(s, nxt):
        if s.kind == "block":
            arcs.append((s.vid, nxt))
        elif s.kind == "if" or s.kind == "switch":
            for b in s.bodies:
                arcs.append((s.vid, lower_seq(b, nxt)))
        elif s.kind == "while":
            arcs.append((s.vid, lower_seq(s.bodies[0], s.vid)))
            arcs.append((s.vid, nxt))
        else:
            raise ValueError(s.kind)
        return s.vid

    first = lower_seq(body, exit_id)
    arcs.append((0, first))
    row_ptr, col = csr_from_arcs(n, arcs)
    assert int(row_ptr[-1]) == len(arcs), "duplicate arc in lowering"
    return CFG(n, row_ptr, col, 0, exit_id, name)


def program_size(body) -> int:
    return 2 + seq_size(body)


# ----------------------------------------------------------------------------
# the workload recipes
# ----------------------------------------------------------------------------
def structured_cfg(seed: int, n: int, n_if: int = 0, n_while: int = 0,
                   switch_fanouts=(), max_depth: int = 3,
                   while_chain: int = 0, name: str = "") -> CFG:
    """A structured CFG with exactly n vertices and the given constructs.

    Constructs are inserted one by one at uniformly drawn insertion points
    (any position of any statement sequence whose nesting depth lets the
    construct stay within ``max_depth``); each starts with one-Block bodies.
    ``while_chain`` first places that many Whiles nested inside each other,
    so the requested loop depth is actually reached.  The remaining node
    budget is filled with Blocks at uniformly drawn positions.
    """
    rng = SplitMix64(seed)
    body = []
    kinds = []
    chain_seq = body
    for _ in range(while_chain):
        w = _make("while")
        _insert(rng, chain_seq, w)
        chain_seq = w.bodies[0]
    kinds += ["while"] * (n_while - while_chain)
    kinds += [("switch", k) for k in switch_fanouts]
    kinds += ["if"] * n_if
    # deterministic shuffle (Fisher-Yates)
    for i in range(len(kinds) - 1, 0, -1):
        j = rng.randint(0, i)
        kinds[i], kinds[j] = kinds[j], kinds[i]
    for k in kinds:
        if isinstance(k, tuple):
            st = _make("switch", k[1])
        else:
            st = _make(k)
        slots = _slots(body, max_depth)
        seq, _ = slots[rng.randint(0, len(slots) - 1)]
        _insert(rng, seq, st)
    need = n - program_size(body)
    if need < 0:
        raise ValueError(f"constructs need {program_size(body)} nodes > n={n}")
    _pad_blocks(rng, body, need)
    cfg = lower_program(body, name)
    assert cfg.n == n
    return cfg


def config1_cfg() -> CFG:
    """Plain method, 24 nodes: 4 If, 2 While, nesting <= 3, seed 1."""
    return structured_cfg(seed=1, n=24, n_if=4, n_while=2, max_depth=3,
                          name="structured-24")


# Fixed by the reading of the cyclic high-Npath workload: 10 Whiles with a
# 4-deep chain, 3 Switches of fan-out 6, and CONFIG3_N_IF If-else decisions;
# the rest is Block padding.
CONFIG3_N = 120
CONFIG3_N_IF = 20
CONFIG3_SEED = 3


def config3_cfg(seed: int = CONFIG3_SEED) -> CFG:
    return structured_cfg(seed=seed, n=CONFIG3_N, n_if=CONFIG3_N_IF,
                          n_while=10, switch_fanouts=(6, 6, 6), max_depth=4,
                          while_chain=4, name="structured-120")


def diamond_chain(k: int) -> CFG:
    """Sequential chain of k if-else diamonds.

    d_i = 3i, a_i = 3i+1, b_i = 3i+2, d_k = 3k; arcs d_i->a_i, d_i->b_i,
    a_i->d_{i+1}, b_i->d_{i+1}.  Entry 0, exit 3k, n = 3k+1, m = 4k.
    """
    n = 3 * k + 1
    arcs = []
    for i in range(k):
        d, a, b, d2 = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        arcs += [(d, a), (d, b), (a, d2), (b, d2)]
    row_ptr, col = csr_from_arcs(n, arcs)
    return CFG(n, row_ptr, col, 0, n - 1, f"diamond-chain-{k}")


def binarise_switches(cfg: CFG) -> CFG:
    """The input restriction of Sec. 3: every vertex of out-degree k > 2
    (a switch) gets k - 2 new intermediate vertices, so that no vertex has
    more than two successors.  For v with successors w1 < ... < wk:
    v -> w1, v -> x1; x1 -> w2, x1 -> x2; ...; x(k-2) -> w(k-1), x(k-2) -> wk.
    Every original arc v -> wi becomes the path v, x1, ..., x(i-1), wi.  New
    ids follow the original ones (n, n+1, ...) in order of v, then of the
    chain; entry and exit are kept."""
    arcs = []
    nxt = cfg.n
    for v in range(cfg.n):
        ws = [int(w) for w in cfg.succ(v)]
        if len(ws) <= 2:
            arcs += [(v, w) for w in ws]
            continue
        cur = v
        for i, w in enumerate(ws[:-2]):
            arcs += [(cur, w), (cur, nxt)]
            cur = nxt
            nxt += 1
        arcs += [(cur, ws[-2]), (cur, ws[-1])]
    rp, col = csr_from_arcs(nxt, arcs)
    return CFG(nxt, rp, col, cfg.entry, cfg.exit, f"{cfg.name}-binarised")


def ring(n: int) -> CFG:
    """Directed cycle 0 -> 1 -> ... -> n-1 -> 0 (no valid entry/exit)."""
    row_ptr, col = csr_from_arcs(n, [(i, (i + 1) % n) for i in range(n)])
    return CFG(n, row_ptr, col, -1, -1, f"ring-{n}")


def complete_digraph(n: int) -> CFG:
    """K_n without self-loops (no valid entry/exit)."""
    arcs = [(u, v) for u in range(n) for v in range(n) if u != v]
    row_ptr, col = csr_from_arcs(n, arcs)
    return CFG(n, row_ptr, col, -1, -1, f"complete-{n}")


def random_digraph(n: int, p: float, seed: int, self_loops: bool = False) -> CFG:
    """Erdos-Renyi style digraph: each ordered pair is an arc with prob. p."""
    rng = SplitMix64(seed)
    arcs = []
    for u in range(n):
        for v in range(n):
            if u == v and not self_loops:
                continue
            if rng.uniform() < p:
                arcs.append((u, v))
    row_ptr, col = csr_from_arcs(n, arcs)
    return CFG(n, row_ptr, col, -1, -1, f"random-{n}-{seed}")


NPATH_CAP = 100_000


def random_cfg(seed: int, n_min: int = 10, n_max: int = 150,
               depth_max: int = 4, fan_min: int = 2, fan_max: int = 6,
               mix=(0.4, 0.3, 0.15, 0.15), npath_cap: int = NPATH_CAP) -> CFG:
    """One graph of the batched workload.

    n = round(exp(U(ln n_min, ln n_max))); nesting cap ~ U{0..depth_max};
    constructs drawn Block/If/While/Switch with probabilities ``mix`` while
    the node budget lasts (a draw that no longer fits becomes a Block);
    Switch fan-out ~ U{fan_min..fan_max}.  A draw whose NPATH exceeds
    ``npath_cap`` is redrawn from the next sub-seed (seed + j * 2**32), so
    the batch stays within a bounded path volume without consulting any
    path enumerator.
    """
    for attempt in range(1 << 16):
        body, n = _random_body(SplitMix64(seed + attempt * (1 << 32)), n_min, n_max,
                               depth_max, fan_min, fan_max, mix)
        if npath(body) <= npath_cap:
            cfg = lower_program(body, f"random-cfg-{seed}")
            assert cfg.n == n
            return cfg
    raise RuntimeError("no draw under the NPATH cap")


def _random_body(rng, n_min, n_max, depth_max, fan_min, fan_max, mix):
    u = rng.uniform()
    n = int(round(math.exp(math.log(n_min) + u * (math.log(n_max) - math.log(n_min)))))
    cap = rng.randint(0, depth_max)
    body = []
    while True:
        remaining = n - program_size(body)
        if remaining <= 0:
            break
        r = rng.uniform()
        if r < mix[0]:
            kind = "block"
        elif r < mix[0] + mix[1]:
            kind = "if"
        elif r < mix[0] + mix[1] + mix[2]:
            kind = "while"
        else:
            kind = "switch"
        fan = rng.randint(fan_min, fan_max) if kind == "switch" else 2
        if _min_size(kind, fan) > remaining:
            kind = "block"
        if kind == "block":
            seqs = _all_seqs(body)
            _insert(rng, seqs[rng.randint(0, len(seqs) - 1)], Stmt("block"))
            continue
        slots = _slots(body, cap + 1)
        seq, _ = slots[rng.randint(0, len(slots) - 1)]
        _insert(rng, seq, _make(kind, fan))
    return body, n


def npath(body) -> int:
    """Nejmeh's NPATH of a statement tree (the structural metric of Table 1).

    Sequence multiplies, If/Switch add their branches, While adds one for
    the skipped body; Block contributes 1.
    """
    def seq_np(seq):
        r = 1
        for s in seq:
            r *= stmt_np(s)
        return r

    def stmt_np(s):
        if s.kind == "block":
            return 1
        if s.kind in ("if", "switch"):
            return sum(seq_np(b) for b in s.bodies)
        if s.kind == "while":
            return seq_np(s.bodies[0]) + 1
        raise ValueError(s.kind)

    return seq_np(body)


# batched workload: graph i of the 4096-graph batch uses seed BATCH_SEED0 + i
BATCH_SEED0 = 1_000_000
TRAIN_SEED0 = 2_000_000
HELDOUT_SEED0 = 3_000_000
TUNER_SEED0 = 4_000_000


def batch_cfgs(count: int, seed0: int = BATCH_SEED0):
    return [random_cfg(seed0 + i) for i in range(count)]


def concat_batch(cfgs):
    """Concatenate per-graph CSRs into the batched input layout.

    Returns (n_per_graph int32[G], row_ptr_cat int32[sum(n)+G], col_cat
    int32[sum(m)], entries int32[G], exits int32[G]); each graph keeps its
    own local ids and its own row_ptr starting at 0.
    """
    ns = np.asarray([c.n for c in cfgs], dtype=np.int32)
    rp = np.concatenate([c.row_ptr for c in cfgs]).astype(np.int32)
    col = np.concatenate([c.col for c in cfgs]).astype(np.int32) if cfgs else np.zeros(0, np.int32)
    ent = np.asarray([c.entry for c in cfgs], dtype=np.int32)
    ext = np.asarray([c.exit for c in cfgs], dtype=np.int32)
    return ns, rp, col, ent, ext
