"""Shared helpers for the tests (inputs and comparisons only)."""
import numpy as np

from paper_2210_16998_gb300 import cfggen as G


def ring_with_tail(r: int) -> G.CFG:
    """entry 0 -> ring 1..r (1->2->...->r->1), r -> exit r+1; n = r + 2."""
    n = r + 2
    arcs = [(0, 1), (r, r + 1)] + [(i, i + 1) for i in range(1, r)] + [(r, 1)]
    rp, col = G.csr_from_arcs(n, arcs)
    return G.CFG(n, rp, col, 0, n - 1, f"ring-tail-{r}")


def wrap_digraph(inner: G.CFG) -> G.CFG:
    """Embed an arbitrary digraph between a fresh entry (-> every vertex) and a
    fresh exit (every vertex ->), so every vertex is reachable and co-reachable."""
    k = inner.n
    n = k + 2
    arcs = [(0, v + 1) for v in range(k)] + [(v + 1, n - 1) for v in range(k)]
    for u in range(k):
        for w in inner.succ(u):
            arcs.append((u + 1, int(w) + 1))
    rp, col = G.csr_from_arcs(n, arcs)
    return G.CFG(n, rp, col, 0, n - 1, f"wrapped-{inner.name}")


def assert_paths_equal(gpu_off, gpu_vert, ref_off, ref_vert, what=""):
    gpu_off = np.asarray(gpu_off, dtype=np.int64)
    ref_off = np.asarray(ref_off, dtype=np.int64)
    assert gpu_off.shape == ref_off.shape, f"{what}: {len(gpu_off) - 1} paths vs {len(ref_off) - 1} expected"
    if not np.array_equal(gpu_off, ref_off):
        i = int(np.nonzero(gpu_off != ref_off)[0][0])
        raise AssertionError(f"{what}: offsets differ first at path {i - 1}")
    gv = np.asarray(gpu_vert, dtype=np.int32)
    rv = np.asarray(ref_vert, dtype=np.int32)
    assert gv.shape == rv.shape, f"{what}: {gv.shape} vertices vs {rv.shape}"
    if not np.array_equal(gv, rv):
        j = int(np.nonzero(gv != rv)[0][0])
        p = int(np.searchsorted(ref_off, j, side="right")) - 1
        raise AssertionError(f"{what}: vertex {j} differs (path {p}): {gv[j]} vs {rv[j]}")


def touring_digest_update(h, off, vert):
    """Feed one graph's TP list to a hashlib digest: its count, then every TP
    as (length, vertices), int64 / int32 little-endian."""
    off = np.asarray(off, np.int64)
    vert = np.asarray(vert, np.int32)
    h.update(np.int64(len(off) - 1).tobytes())
    h.update((off[1:] - off[:-1]).astype("<i8").tobytes())
    h.update(vert.astype("<i4").tobytes())
