"""Search for the 14-cycle 40-qubit circuit's contraction path and slicing.

Runs seeded greedy path finding (greedy.greedy_path) over a grid of seeds and
size-weighting exponents, keeps the path of least total flops (the sum over steps of
the step's index-space size, log2), and slices it greedily (greedy.greedy_slicer) until
every slice's largest intermediate holds at most 2^30 elements, then two labels further
for the CPU oracle's pieces. Prints what workloads.RC40C14_PATH, RC40C14_SLICED and
RC40C14_SUBSLICED record. Takes a few minutes on one core:
    python -m tn_inputs.search_paths
"""
from __future__ import annotations

import time

from . import circuits, greedy

SEEDS = range(1200)
ALPHAS = (0.75, 0.875, 1.0)
PEAK_LOG2 = 30.0


def search(rows=5, cols=8, cycles=14, seed=40, seeds=SEEDS, alphas=ALPHAS):
    net = circuits.amplitude_network(rows, cols, cycles, seed)
    best = None
    for s in seeds:
        for a in alphas:
            p = greedy.greedy_path(net, seed=s, alpha=a, temperature=0.0)
            fl = greedy.path_log2_flops(net, p)
            if best is None or (fl, s, a) < best[0]:
                best = ((fl, s, a), p)
    (fl, s, a), path = best
    sliced = greedy.greedy_slicer(net, path, PEAK_LOG2, max_slices=40)
    sub = greedy.greedy_slicer(net, path, -1.0, max_slices=len(sliced) + 2)
    return dict(seed=s, alpha=a, temperature=0.0, log2flops=fl), tuple(sliced), tuple(sub)


if __name__ == "__main__":
    t = time.time()
    choice, sliced, sub = search()
    print("path", choice)
    print("sliced", sliced)
    print("subsliced", sub)
    print(f"{time.time() - t:.0f} s")
