"""CPU reference of the learned sizer (TEST INFRASTRUCTURE).

Written from the definitions, in float64 numpy:

* features of a vertex v of a CFG with n vertices: log1p(in-degree),
  log1p(out-degree), [v is the entry], [v is the exit], log1p(size of v's
  strongly connected component: the vertices reachable from v that also
  reach v), BFS depth from the entry divided by n (2 if unreachable), BFS
  depth to the exit divided by n (2 if it cannot reach it), log(n) / 5;
* the network: h0 = ReLU(W0 x + b0); for three layers
  h = ReLU(W [h; sum over predecessors of h; sum over successors of h] + b);
  y = Wo h + bo; loss = mean over vertices and the 3 targets of (y - t)^2;
* its gradient by the chain rule (pinned against central finite
  differences in the tests).

`bf16=True` rounds to bfloat16 (round to nearest even) at the same places as
the GPU kernels: layer weights, activations, neighbour sums, and the output
gradient fed to the input-gradient product; it is used to compare the GPU
gradient at matched precision.  The parameter vector uses the GPU layout.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.sparse as sp

H, F, T, L = 64, 8, 3, 3
K = 3 * H
OFF_W0 = 0
OFF_B0 = OFF_W0 + H * F
OFF_WL = OFF_B0 + H
LAYER = H * K + H
OFF_WO = OFF_WL + L * LAYER
OFF_BO = OFF_WO + T * H
NPARAM = OFF_BO + T


def bf16(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32)
    r = ((a >> 16) & 1) + np.uint32(0x7FFF)
    return ((a + r) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    W0 = p[OFF_W0:OFF_W0 + H * F].reshape(H, F)
    b0 = p[OFF_B0:OFF_B0 + H]
    Ws, bs = [], []
    for l in range(L):
        base = OFF_WL + l * LAYER
        Ws.append(p[base:base + H * K].reshape(H, K))
        bs.append(p[base + H * K:base + LAYER])
    Wo = p[OFF_WO:OFF_WO + T * H].reshape(T, H)
    bo = p[OFF_BO:OFF_BO + T]
    return W0, b0, Ws, bs, Wo, bo


def _bfs(n, adj, s):
    d = [-1] * n
    d[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if d[w] < 0:
                d[w] = d[u] + 1
                q.append(w)
    return d


def features(cfg):
    n = cfg.n
    succ = [[int(w) for w in cfg.succ(v)] for v in range(n)]
    pred = [[] for _ in range(n)]
    for u in range(n):
        for w in succ[u]:
            pred[w].append(u)
    reach = [_bfs(n, succ, v) for v in range(n)]
    x = np.zeros((n, F))
    for v in range(n):
        scc = sum(1 for u in range(n) if reach[v][u] >= 0 and reach[u][v] >= 0)
        de, dx = reach[cfg.entry][v], reach[v][cfg.exit]
        x[v] = [np.log1p(len(pred[v])), np.log1p(len(succ[v])), float(v == cfg.entry), float(v == cfg.exit),
                np.log1p(scc), de / n if de >= 0 else 2.0, dx / n if dx >= 0 else 2.0, np.log(n) / 5.0]
    return x


def batch_inputs(cfgs):
    """Features and the (block-diagonal) adjacency of a batch of CFGs."""
    xs, rows, cols, base = [], [], [], 0
    for c in cfgs:
        xs.append(features(c))
        for u in range(c.n):
            for w in c.succ(u):
                rows.append(base + u)
                cols.append(base + int(w))
        base += c.n
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(base, base))
    return np.concatenate(xs), A


def forward(p, X, A, bf=False):
    W0, b0, Ws, bs, Wo, bo = unpack(p)
    r = bf16 if bf else (lambda a: a)
    z0 = X @ W0.T + b0
    h = r(np.maximum(z0, 0.0))
    cache = {"h": [h], "xc": [], "W": []}
    for l in range(L):
        xc = np.concatenate([h, r(A.T @ h), r(A @ h)], axis=1)
        W = r(Ws[l])
        h = r(np.maximum(xc @ W.T + bs[l], 0.0))
        cache["xc"].append(xc)
        cache["W"].append(W)
        cache["h"].append(h)
    y = h @ Wo.T + bo
    return y, cache


def loss_grad(p, X, A, Tt, bf=False):
    W0, b0, Ws, bs, Wo, bo = unpack(p)
    r = bf16 if bf else (lambda a: a)
    y, c = forward(p, X, A, bf)
    N = X.shape[0]
    d = y - Tt
    loss = float(np.mean(d * d))
    g = np.zeros(NPARAM)
    dy = 2.0 * d / (T * N)
    h3 = c["h"][L]
    g[OFF_WO:OFF_WO + T * H] = (dy.T @ h3).ravel()
    g[OFF_BO:OFF_BO + T] = dy.sum(0)
    dz = (dy @ Wo) * (h3 > 0)
    for l in range(L - 1, -1, -1):
        base = OFF_WL + l * LAYER
        xc = c["xc"][l]
        g[base:base + H * K] = (dz.T @ xc).ravel()
        g[base + H * K:base + LAYER] = dz.sum(0)
        dxc = r(dz) @ c["W"][l]
        dh = dxc[:, :H] + A @ dxc[:, H:2 * H] + A.T @ dxc[:, 2 * H:]
        dz = dh * (c["h"][l] > 0)
    g[OFF_W0:OFF_W0 + H * F] = (dz.T @ X).ravel()
    g[OFF_B0:OFF_B0 + H] = dz.sum(0)
    return loss, g
