"""Seeded Ising partition-function networks on random 3-regular graphs (the
counting/combinatorial family of Sec. III-C, real arithmetic).

Z = sum_{s in {+1,-1}^N} exp(beta * sum_{(u,v) in E} J_uv s_u s_v), label value 0 <-> s=+1.

Network: one rank-3 tensor per vertex and one label per edge (no hyper-edges). For
edge e = (u, v) with u < v the weight W_e[s, t] = exp(beta J_e s t) is folded into u's
tensor and v's tensor copies its spin onto the bond:
    T_u[b_e ...] = sum_s prod_{e=(u,v), u<v} W_e[s, b_e] * prod_{e=(w,u), w<u} delta[s, b_e].
Also: a ring of N spins (uniform J, h = 0) for the transfer-matrix closed form.
"""
from __future__ import annotations

import numpy as np

from .network import Network


def random_3regular(n: int, rng: np.random.Generator, max_tries: int = 10000):
    """Configuration model with rejection of self-loops and multi-edges."""
    assert n % 2 == 0 and n >= 4
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = True
        seen = set()
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in seen:
                ok = False
                break
            seen.add(e)
        if ok:
            return sorted(seen)
    raise RuntimeError("no simple 3-regular graph found")


def spin(idx):
    return 1.0 - 2.0 * np.asarray(idx, dtype=np.float64)


def graph_network(n: int, edges, J, beta: float, name: str = "") -> Network:
    """Partition-function network of an arbitrary simple graph with per-edge couplings J."""
    inc = [[] for _ in range(n)]
    for e, (u, v) in enumerate(edges):
        inc[u].append(e)
        inc[v].append(e)
    s = spin([0, 1])
    tensors, modes = [], []
    for u in range(n):
        es = inc[u]
        shape = (2,) * len(es)
        t = np.zeros(shape, dtype=np.float64)
        for idx in np.ndindex(*shape):
            acc = 0.0
            for si in (0, 1):
                w = 1.0
                for ax, e in enumerate(es):
                    a, b = edges[e]
                    if a == u:   # u is the lower endpoint: weight
                        w *= np.exp(beta * J[e] * s[si] * s[idx[ax]])
                    else:        # copy of u's spin
                        w *= 1.0 if idx[ax] == si else 0.0
                acc += w
            t[idx] = acc
        tensors.append(t)
        modes.append(tuple(es))
    net = Network(tensors, modes, {e: 2 for e in range(len(edges))}, (), name=name,
                  meta=dict(n=n, edges=list(edges), J=list(J), beta=beta))
    net.check()
    return net


def random_3regular_network(n: int, seed: int, beta: float = 0.5) -> Network:
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = random_3regular(n, rng)
    J = rng.choice(np.array([-1.0, 1.0]), size=len(edges))
    return graph_network(n, edges, J, beta, name=f"ising3r_n{n}_s{seed}")


def ensemble(count: int, seed: int, n_min: int = 20, n_max: int = 60, beta: float = 0.5):
    """`count` networks with N even, uniform in [n_min, n_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(n_min // 2, n_max // 2 + 1, size=count) * 2
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [random_3regular_network(int(n), int(s), beta) for n, s in zip(sizes, seeds)]


def lattice_network(rows: int, cols: int, beta: float, seed=None, J: float = 1.0) -> Network:
    """Square lattice of rows x cols spins with open boundaries (nearest-neighbour bonds).
    seed None: uniform coupling J (the ferromagnet); otherwise J_ij uniform in {-1, +1}
    from a seeded generator (a +-J spin glass)."""
    idx = lambda r, c: r * cols + c
    edges = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols:
                edges.append((idx(r, c), idx(r, c + 1)))
            if r + 1 < rows:
                edges.append((idx(r, c), idx(r + 1, c)))
    if seed is None:
        Js = [J] * len(edges)
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        Js = list(rng.choice(np.array([-1.0, 1.0]), size=len(edges)))
    return graph_network(rows * cols, edges, Js, beta,
                         name=f"ising_lattice_{rows}x{cols}" + ("" if seed is None else f"_s{seed}"))


def ring_network(n: int, J: float, beta: float) -> Network:
    edges = [(i, (i + 1) % n) for i in range(n)]
    edges = [(min(a, b), max(a, b)) for a, b in edges]
    return graph_network(n, edges, [J] * n, beta, name=f"ring_n{n}")
