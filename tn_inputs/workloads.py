"""Named workloads: network + fixed path + sliced labels, all seeded.

  rc12      : 12-qubit 3x4 grid random circuit, 8 brick-wall cycles, one amplitude,
              greedy path, no slicing (the tiny circuit case).
  rc40c14   : 40-qubit 5x8 grid random circuit, 14 cycles, one amplitude, the greedy path
              of least total flops found by search_paths.py, sliced greedily until each
              slice's largest intermediate is <= 2^30 elements (7 labels, 128 slices).
              The headline workload.
  rc40c14sub: the same network and path with two more greedily sliced labels (512 slices,
              every 4 consecutive ones make up one rc40c14 slice): the pieces the CPU
              oracle contracts for parity at this depth.
  rc40      : 40-qubit 5x8 grid random circuit, 13 cycles, one amplitude, greedy path
              with 8 sliced labels (256 slices).
  rc40u     : rc40 with no slicing (the same network and path; largest intermediate 2^32
              complex64 = 32 GiB, which one GPU's HBM holds).
  rc40open  : rc40 with the 2x2 corner block of qubits left open, so one contraction
              yields 16 correlated amplitudes (a [2,2,2,2] output tensor); 256 slices.
  kising44  : 4x4 kicked Ising, 10 Trotter steps, J=1, dt=0.25, h=0.9, <Z_centre>
              (the dynamics expectation case at a size one GPU and the oracle can
              contract unsliced).
  khex45    : kicked Ising, same couplings, on a 4x5 honeycomb lattice (brick-wall form),
              6 Trotter steps;
  ktri44    : kicked Ising on a 4x4 triangular lattice, 8 Trotter steps;
  tcgemm    : one dense step of the 14-cycle circuit's shape (2^14 x 2^14 outputs, k = 2^13), the
              small case the tensor-core kernel is profiled on;
  sv26      : a 2^26-element state leaf in a shuffled declared order absorbing 4 gates (the
              large-leaf permutation case);
  kings16   : maximum independent set of a 16x16 King's subgraph (site density 0.8, seed 1;
              209 vertices), contracted in the max-plus semiring (FP32, exact integers);
  kings_batch: maximum independent sets of many King's subgraphs (L in [4, 7], density 0.8),
              max-plus, for the one-launch batch engine;
  ising3r   : an ensemble of Ising partition functions on random 3-regular graphs.
Smaller variants with the same structure serve as parity cases.

Paths: the best (by total flops, then peak) of seeded greedy runs over a small grid of
(seed, alpha, temperature); slicing: the greedy slicer picks n labels one at a time.
"""
from __future__ import annotations

import functools

import numpy as np

from . import circuits, kicked_ising, ising_pf, greedy, kings, network

PATH_SEEDS = range(6)
PATH_ALPHAS = (0.0, 0.5, 1.0)
PATH_TEMPS = (0.0, 0.05)


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


def _pathed(name, net, n_sliced=0, seeds=PATH_SEEDS):
    path, info = greedy.best_greedy(net, seeds, PATH_ALPHAS, PATH_TEMPS, key="flops")
    sliced = greedy.greedy_slicer(net, path, -1.0, max_slices=n_sliced) if n_sliced else []
    info["peak_sliced"] = greedy.path_peak(net, path, sliced)
    info["log2flops_sliced"] = greedy.path_log2_flops(net, path, sliced)
    return Workload(name, net, path, sliced, info)


@functools.lru_cache(maxsize=None)
def random_circuit(rows, cols, cycles, seed, n_sliced=0, open_qubits=()):
    net = circuits.amplitude_network(rows, cols, cycles, seed, open_qubits=open_qubits)
    name = net.name + (f"_sl{n_sliced}" if n_sliced else "")
    return _pathed(name, net, n_sliced=n_sliced)


@functools.lru_cache(maxsize=None)
def kicked(L, T, J=1.0, h=0.9, dt=0.25, cols=None, lattice="square"):
    net = kicked_ising.expectation_network(L, T, J, h, dt, cols=cols, lattice=lattice)
    return _pathed(net.name, net)


def rc12():
    return random_circuit(3, 4, 8, 12)


def rc40():
    return random_circuit(5, 8, 13, 40, n_sliced=8)


# The 14-cycle circuit: the greedy run of least total flops over the grid that
# tn_inputs/search_paths.py scans (seeds 0-1199, alpha in {0.75, 0.875, 1.0}, temperature 0;
# unsliced 2^50.81 complex MACs), and the labels the greedy slicer picks for it: the first
# seven bring every slice's largest intermediate to 2^30 elements, the last two are the
# oracle's finer pieces. Both are reproduced by tests/test_workloads.py.
RC40C14_PATH = dict(seed=364, alpha=1.0, temperature=0.0)
RC40C14_SLICED = (320, 328, 446, 350, 210, 461, 453)
RC40C14_SUBSLICED = RC40C14_SLICED + (357, 344)


@functools.lru_cache(maxsize=None)
def _rc40c14_net_path():
    net = circuits.amplitude_network(5, 8, 14, 40)
    return net, greedy.greedy_path(net, **RC40C14_PATH)


def _rc40c14(sliced, name):
    net, path = _rc40c14_net_path()
    info = dict(RC40C14_PATH)
    info["peak_sliced"] = greedy.path_peak(net, path, sliced)
    info["log2flops_sliced"] = greedy.path_log2_flops(net, path, sliced)
    return Workload(name, net, path, sliced, info)


def rc40c14():
    """40 qubits on 5x8, 14 cycles, one amplitude; 7 sliced labels (128 slices), each
    slice's largest intermediate 2^30 complex64 elements (8 GiB)."""
    return _rc40c14(RC40C14_SLICED, "rc_5x8_m14_s40_sl7")


def rc40c14sub():
    """rc40c14 sliced two labels further (512 slices): slice 4s + j of this workload is
    piece j of rc40c14's slice s (the added labels are the least significant)."""
    return _rc40c14(RC40C14_SUBSLICED, "rc_5x8_m14_s40_sl9")


def rc40u():
    """rc40 without slicing: the same network and path, every intermediate whole (largest
    2^32 elements, a 51 GiB workspace in complex64)."""
    return random_circuit(5, 8, 13, 40)


# the 2x2 block of qubits in the grid's last corner (rows 3-4, columns 6-7) stays open
RC40_OPEN = (30, 31, 38, 39)


def rc40open():
    """rc40 with four output qubits left open: the 16 correlated amplitudes that share
    the other 36 bits, from one sliced contraction (output tensor [2,2,2,2])."""
    return random_circuit(5, 8, 13, 40, n_sliced=8, open_qubits=RC40_OPEN)


@functools.lru_cache(maxsize=None)
def sv26():
    """A 26-qubit state (one 2^26-element leaf, 512 MiB in complex64) declared in a shuffled
    qubit order, absorbing four Haar-random two-qubit gates; the open output is the new
    state in qubit order. Its leaf is the permutation the staging kernel exists for."""
    net = circuits.state_network(26, 4, 26)
    return Workload(net.name, net, circuits.state_path(net), (), {})


@functools.lru_cache(maxsize=None)
def tcgemm(m_bits=14, n_bits=14, k_bits=13, seed=5):
    """One dense pairwise step of the 14-cycle circuit's shape at a size that fits a small
    profiling case: A[M, K] . B[N, K] with 2^14 x 2^14 outputs over k = 2^13 (complex64: 1 GiB
    per operand), closed by two vectors (the steps after it are tiny)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = list(range(m_bits))
    N = list(range(m_bits, m_bits + n_bits))
    K = list(range(m_bits + n_bits, m_bits + n_bits + k_bits))
    ext = {x: 2 for x in M + N + K}
    gauss = lambda shape: (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    A = gauss((2,) * (m_bits + k_bits))
    B = gauss((2,) * (n_bits + k_bits))
    u = gauss((2,) * m_bits)
    v = gauss((2,) * n_bits)
    net = network.Network([A, B, u, v], [tuple(M + K), tuple(N + K), tuple(M), tuple(N)], ext, (),
                          name=f"gemm_m{m_bits}_n{n_bits}_k{k_bits}")
    net.check()
    return Workload(net.name, net, network.Path([(0, 1), (4, 2), (5, 3)]), (), {})


def kising44():
    return kicked(4, 10)


def kising55():
    """Kicked Ising on a 5 x 5 lattice, 2 Trotter steps (greedy peak 2^26): the serving
    mix's large request."""
    return kicked(5, 2)


def khex45():
    """Kicked Ising on a 4 x 5 honeycomb (brick-wall) lattice, 6 Trotter steps."""
    return kicked(4, 6, cols=5, lattice="hexagonal")


def ktri44():
    """Kicked Ising on a 4 x 4 triangular lattice, 8 Trotter steps."""
    return kicked(4, 8, lattice="triangular")


@functools.lru_cache(maxsize=None)
def kings_mis(L, rho, seed, n_sliced=0):
    """Maximum independent set of a King's subgraph: the max-plus (tropical) network."""
    net = kings.kings_network(L, rho, seed, "tropical")
    name = net.name + (f"_sl{n_sliced}" if n_sliced else "")
    w = _pathed(name, net, n_sliced=n_sliced)
    w.info["semiring"] = "maxplus"
    return w


def kings16():
    """MIS of a 16 x 16 King's subgraph (site density 0.8, seed 1: 209 vertices)."""
    return kings_mis(16, 0.8, 1)


def ising_workload(net):
    path, info = greedy.best_greedy(net, range(2), (0.0, 1.0))
    return Workload(net.name, net, path, (), info)


def isingsq20():
    """Partition function of a +-J Ising spin glass on an open 20 x 20 square lattice
    (400 spins, beta = 0.44, couplings from seed 1), real FP32 with per-intermediate
    exponent scaling (ln Z ~ 350: Z is far beyond FP32), no slicing. Path: the greedy
    search's seed 1, alpha 0 (2^40.1 flops, largest intermediate 2^29 elements, the least
    flops of seeds 0-2 x alpha 0, 1 under a 2^30 cap)."""
    net = ising_pf.lattice_network(20, 20, 0.44, seed=1)
    w = Workload("isingsq20", net, greedy.greedy_path(net, seed=1, alpha=0.0))
    w.info["exp_scaling"] = True
    return w


def ising3r(count, seed=3):
    return [ising_workload(n) for n in ising_pf.ensemble(count, seed)]


def kings_batch(count, seed=5):
    """Maximum independent sets of `count` King's subgraphs, L in [4, 7], density 0.8."""
    out = []
    for n in kings.kings_ensemble(count, seed, sizes=(4, 7)):
        wl = ising_workload(n)
        wl.info["semiring"] = "maxplus"
        out.append(wl)
    return out


BY_NAME = {"rc12": rc12, "rc40": rc40, "rc40c14": rc40c14, "rc40c14sub": rc40c14sub, "rc40u": rc40u, "kising44": kising44, "kising55": kising55,
           "rc40open": rc40open,
           "khex45": khex45, "ktri44": ktri44, "kings16": kings16, "sv26": sv26, "tcgemm": tcgemm,
           "isingsq20": isingsq20}
