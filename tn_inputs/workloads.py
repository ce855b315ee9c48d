"""Named workloads: network + fixed path + sliced labels, all seeded.

  rc12      : 12-qubit 3x4 grid random circuit, 8 brick-wall cycles, one amplitude,
              greedy path, no slicing (the tiny circuit case).
  kising6   : 6x6 kicked Ising, 10 Trotter steps, J=1, dt=0.25, h=0.9, <Z_centre>
              (the dynamics expectation case; the headline workload).
  rc40      : 40-qubit 5x8 grid random circuit, 14 cycles, one amplitude, greedy path,
              8 sliced labels (256 slices).
  ising3r   : an ensemble of Ising partition functions on random 3-regular graphs.
Smaller variants with the same structure serve as parity cases.
"""
from __future__ import annotations

import functools

from . import circuits, kicked_ising, ising_pf, greedy
from .network import Path


class Workload:
    def __init__(self, name, net, path, sliced=(), info=None):
        self.name, self.net, self.path, self.sliced = name, net, path, list(sliced)
        self.info = dict(info or {})

    @property
    def n_slices(self) -> int:
        out = 1
        for x in self.sliced:
            out *= self.net.extent[x]
        return out


def _pathed(name, net, seeds=range(4), alphas=(0.0, 1.0), sliced_target=None, n_sliced=None):
    path, info = greedy.best_greedy(net, seeds, alphas)
    sliced = []
    if sliced_target is not None:
        sliced = greedy.greedy_slicer(net, path, sliced_target)
    if n_sliced is not None:
        # exactly n_sliced labels: extend or trim the greedy choice
        sliced = greedy.greedy_slicer(net, path, -1.0, max_slices=n_sliced)
    info["peak_sliced"] = greedy.path_peak(net, path, sliced)
    info["log2flops_sliced"] = greedy.path_log2_flops(net, path, sliced)
    return Workload(name, net, path, sliced, info)


@functools.lru_cache(maxsize=None)
def random_circuit(rows, cols, cycles, seed, n_sliced=0):
    net = circuits.amplitude_network(rows, cols, cycles, seed)
    return _pathed(net.name, net, n_sliced=n_sliced or None)


@functools.lru_cache(maxsize=None)
def kicked(L, T, J=1.0, h=0.9, dt=0.25, seeds=4):
    net = kicked_ising.expectation_network(L, T, J, h, dt)
    return _pathed(net.name, net, seeds=range(seeds))


def rc12():
    return random_circuit(3, 4, 8, 12)


def kising6():
    return kicked(6, 10)


def rc40():
    return random_circuit(5, 8, 14, 40, n_sliced=8)


def ising_workload(net, seed=0):
    path, info = greedy.best_greedy(net, range(2), (0.0, 1.0))
    return Workload(net.name, net, path, (), info)


def ising3r(count, seed=3):
    return [ising_workload(n) for n in ising_pf.ensemble(count, seed)]
