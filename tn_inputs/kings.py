"""Independent-set networks on King's subgraphs (the combinatorial family of Sec. III-C:
tropical and counting semiring contractions of local-constraint tensors).

Graph: an L x L grid, each site kept with probability rho (seeded), edges between kept
sites at Chebyshev distance 1 (the eight King's-move neighbours).

Network (one tensor per vertex, one label per edge, no hyper-edges): for edge e = (u, v)
with u < v the constraint matrix is folded into u's tensor and v's tensor copies its
occupation s in {0, 1} onto the bond, as in the Ising construction:
  counting  (+, x):    T_u[b..] = sum_s x^s prod_{e=(u,v),u<v} B[s, b_e] prod_{e=(w,u),w<u} delta[s, b_e],
                       B[s, t] = 0 if s = t = 1 else 1; with x = 1 the network sums to the
                       number of independent sets;
  tropical (max, +):   T_u[b..] = max_s ( s + sum_{u<v} B[s, b_e] + sum_{w<u} delta[s, b_e] ),
                       B[s, t] = -inf if s = t = 1 else 0, delta = 0 if equal else -inf; the
                       network's max-plus value is the size of a maximum independent set.
"""
from __future__ import annotations

import numpy as np

from .network import Network


def kings_subgraph(L: int, rho: float, seed: int):
    """(n, edges) of a seeded King's subgraph; vertices numbered in row-major site order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keep = rng.random((L, L)) < rho
    index = -np.ones((L, L), dtype=np.int64)
    n = 0
    for r in range(L):
        for c in range(L):
            if keep[r, c]:
                index[r, c] = n
                n += 1
    edges = []
    for r in range(L):
        for c in range(L):
            if index[r, c] < 0:
                continue
            for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < L and 0 <= cc < L and index[rr, cc] >= 0:
                    u, v = int(index[r, c]), int(index[rr, cc])
                    edges.append((min(u, v), max(u, v)))
    return n, sorted(edges)


def independent_set_network(n: int, edges, semiring: str = "tropical", name: str = "") -> Network:
    """The network of the header for an arbitrary simple graph (n vertices, edges u < v)."""
    assert semiring in ("tropical", "counting")
    trop = semiring == "tropical"
    inc = [[] for _ in range(n)]
    for e, (u, v) in enumerate(edges):
        inc[u].append(e)
        inc[v].append(e)
    tensors, modes = [], []
    for u in range(n):
        es = inc[u]
        shape = (2,) * len(es)
        t = np.full(shape, -np.inf if trop else 0.0, dtype=np.float64)
        for idx in np.ndindex(*shape):
            for s in (0, 1):
                ok = True
                for e, b in zip(es, idx):
                    a, v = edges[e]
                    if a == u:       # u < v: the constraint B[s, b]
                        if s == 1 and b == 1:
                            ok = False
                    elif b != s:     # u is the larger end: copy s onto the bond
                        ok = False
                if ok:
                    t[idx] = max(t[idx], float(s)) if trop else t[idx] + 1.0
        if not es:                   # an isolated vertex: a scalar factor
            t = np.array(1.0 if trop else 2.0)
        tensors.append(t)
        modes.append(tuple(es))
    ext = {e: 2 for e in range(len(edges))}
    net = Network(tensors, modes, ext, (), name=name or f"mis_{semiring}_{n}",
                  meta=dict(n=n, edges=list(edges), semiring=semiring))
    net.check()
    return net


def kings_network(L: int, rho: float, seed: int, semiring: str = "tropical") -> Network:
    n, edges = kings_subgraph(L, rho, seed)
    net = independent_set_network(n, edges, semiring, name=f"kings_{L}x{L}_r{rho}_s{seed}_{semiring}")
    net.meta.update(L=L, rho=rho, seed=seed)
    return net


def kings_ensemble(count: int, seed: int, sizes=(6, 10), rho: float = 0.8, semiring: str = "tropical"):
    """`count` King's subgraph networks, L uniform in [sizes[0], sizes[1]], one seed each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ls = rng.integers(sizes[0], sizes[1] + 1, size=count)
    return [kings_network(int(L), rho, seed * 100003 + i, semiring) for i, L in enumerate(Ls)]
