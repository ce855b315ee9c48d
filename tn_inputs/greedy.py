"""Seeded greedy contraction paths and a greedy slicer.

These produce the *inputs* the method consumes (a fixed path and slicing metadata,
Sec. IV opening); they are not part of the method. The cost the greedy uses is the
log2 size of a pairwise output (number of modes when every extent is 2), which is
counting, not contraction arithmetic.

greedy_path: among pairs of live tensors that share a label, contract the pair whose
output is smallest, with `alpha` weighting the sizes it frees (opt-einsum style
size(out) - alpha*(size(a)+size(b))); ties broken by a seeded random key. A
disconnected remainder is joined by outer products, smallest first.
"""
from __future__ import annotations

import heapq
import math

import numpy as np

from .network import Network, Path


def _out_modes(ma: frozenset, mb: frozenset, keep: frozenset, count: dict):
    # a label shared by both operands is summed unless something else still needs it
    shared = ma & mb
    out = (ma | mb) - frozenset(x for x in shared if x not in keep and count[x] == 2)
    return frozenset(out)


def _log2size(ms, ext) -> float:
    return sum(math.log2(ext[x]) for x in ms)


def greedy_path(net: Network, seed: int = 0, alpha: float = 0.0, temperature: float = 0.0,
                sliced=()) -> Path:
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = dict(net.extent)
    sl = frozenset(sliced)
    keep = frozenset(net.open_modes)
    live = {}
    count = {}
    for i, ms in enumerate(net.modes):
        s = frozenset(x for x in ms if x not in sl)
        live[i] = s
        for x in s:
            count[x] = count.get(x, 0) + 1
    where = {}
    for i, s in live.items():
        for x in s:
            where.setdefault(x, set()).add(i)
    next_id = len(net.modes)
    pairs = []

    def cost(i, j):
        out = _out_modes(live[i], live[j], keep, count)
        c = 2.0 ** _log2size(out, ext) - alpha * (2.0 ** _log2size(live[i], ext) + 2.0 ** _log2size(live[j], ext))
        if temperature > 0:
            c += temperature * rng.gumbel()
        return c

    heap = []

    def push(i, j):
        if i > j:
            i, j = j, i
        heapq.heappush(heap, (cost(i, j), float(rng.random()), i, j))

    for x, ts in where.items():
        ts = sorted(ts)
        for a in range(len(ts)):
            for b in range(a + 1, len(ts)):
                push(ts[a], ts[b])
    while heap:
        c, _, i, j = heapq.heappop(heap)
        if i not in live or j not in live:
            continue
        out = _out_modes(live[i], live[j], keep, count)
        for x in live[i] & live[j]:
            if x not in out:
                count[x] -= 2
        del_i, del_j = live.pop(i), live.pop(j)
        for x in del_i:
            where[x].discard(i)
        for x in del_j:
            where[x].discard(j)
        k = next_id
        next_id += 1
        live[k] = out
        pairs.append((i, j))
        nbrs = set()
        for x in out:
            nbrs |= where[x]
            where[x].add(k)
        for t in nbrs:
            push(t, k)
    # join disconnected components by outer products, smallest first
    while len(live) > 1:
        ids = sorted(live, key=lambda t: (_log2size(live[t], ext), t))
        i, j = ids[0], ids[1]
        out = live.pop(i) | live.pop(j)
        live[next_id] = frozenset(out)
        pairs.append((min(i, j), max(i, j)))
        next_id += 1
    return Path(pairs)


def path_log2_sizes(net: Network, path: Path, sliced=()):
    """log2 size of every intermediate along the path (slices removed)."""
    ext = net.extent
    sl = set(sliced)
    keep = frozenset(net.open_modes)
    tens = [frozenset(x for x in ms if x not in sl) for ms in net.modes]
    count = {}
    for s in tens:
        for x in s:
            count[x] = count.get(x, 0) + 1
    out_sizes = []
    for (i, j) in path.pairs:
        out = _out_modes(tens[i], tens[j], keep, count)
        for x in tens[i] & tens[j]:
            if x not in out:
                count[x] -= 2
        tens.append(out)
        out_sizes.append(_log2size(out, ext))
    return out_sizes


def path_peak(net: Network, path: Path, sliced=()) -> float:
    s = path_log2_sizes(net, path, sliced)
    leaf = max(_log2size([x for x in ms if x not in set(sliced)], net.extent) for ms in net.modes)
    return max(max(s) if s else 0.0, leaf)


def path_log2_flops(net: Network, path: Path, sliced=()) -> float:
    """log2 of sum over steps of the step's dense index-space size (|A u B| modes)."""
    ext = net.extent
    sl = set(sliced)
    keep = frozenset(net.open_modes)
    tens = [frozenset(x for x in ms if x not in sl) for ms in net.modes]
    count = {}
    for s in tens:
        for x in s:
            count[x] = count.get(x, 0) + 1
    tot = 0.0
    for (i, j) in path.pairs:
        out = _out_modes(tens[i], tens[j], keep, count)
        for x in tens[i] & tens[j]:
            if x not in out:
                count[x] -= 2
        tens.append(out)
        tot += 2.0 ** _log2size(tens[i] | tens[j], ext)
    return math.log2(tot)


def best_greedy(net: Network, seeds, alphas=(0.0, 1.0), temperatures=(0.0,), sliced=(),
                key="peak"):
    """Best of several seeded greedy runs by (peak, flops) or (flops, peak)."""
    best = None
    for s in seeds:
        for a in alphas:
            for t in temperatures:
                p = greedy_path(net, seed=s, alpha=a, temperature=t, sliced=sliced)
                pk, fl = path_peak(net, p, sliced), path_log2_flops(net, p, sliced)
                score = (pk, fl) if key == "peak" else (fl, pk)
                if best is None or score < best[0]:
                    best = (score, p, dict(seed=s, alpha=a, temperature=t, peak=pk, log2flops=fl))
    return best[1], best[2]


def greedy_slicer(net: Network, path: Path, target_log2: float, max_slices: int = 64):
    """Slice labels one at a time, each time the one that lowers the peak most
    (ties: the one with the smallest resulting flop count), until peak <= target."""
    sliced = []
    labels = [x for x in net.labels() if x not in net.open_modes]
    while path_peak(net, path, sliced) > target_log2 and len(sliced) < max_slices:
        best = None
        for x in labels:
            if x in sliced:
                continue
            s2 = sliced + [x]
            sc = (path_peak(net, path, s2), path_log2_flops(net, path, s2) + len(s2))
            if best is None or sc < best[0]:
                best = (sc, x)
        sliced.append(best[1])
    return sliced
