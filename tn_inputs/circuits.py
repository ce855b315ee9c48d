"""Seeded random-circuit amplitude networks on a 2D grid (the random-circuit-sampling
workload family of Sec. III-A, shaped like the 2D-grid circuits the paper contracts).

Each gate is a Haar-random 4x4 unitary: QR of a complex Gaussian matrix with the
column phases fixed by diag(R)/|diag(R)| (Mezzadri's recipe). Gates are laid out in a
brick-wall pattern that cycles through four layers: horizontal pairs starting at even
columns, horizontal pairs starting at odd columns, vertical pairs starting at even rows,
vertical pairs starting at odd rows. The network is the closed amplitude <x|C|0...0>.
"""
from __future__ import annotations

import numpy as np

from .network import Network


def haar_unitary(rng: np.random.Generator, d: int = 4) -> np.ndarray:
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def brickwall_layers(rows: int, cols: int):
    """The four gate layers of one period, as lists of (q0, q1) qubit pairs (q = r*cols + c)."""
    q = lambda r, c: r * cols + c
    layers = []
    for start in (0, 1):  # horizontal
        layers.append([(q(r, c), q(r, c + 1)) for r in range(rows) for c in range(start, cols - 1, 2)])
    for start in (0, 1):  # vertical
        layers.append([(q(r, c), q(r + 1, c)) for r in range(start, rows - 1, 2) for c in range(cols)])
    return layers


def circuit_gates(rows: int, cols: int, cycles: int, seed: int):
    """Gate list [(q0, q1, U)] for `cycles` brick-wall layers; U acts on |q0 q1> with q0 the high bit."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = brickwall_layers(rows, cols)
    gates = []
    for cyc in range(cycles):
        for (a, b) in layers[cyc % 4]:
            gates.append((a, b, haar_unitary(rng, 4)))
    return gates


class _Builder:
    def __init__(self):
        self.tensors, self.modes, self.extent = [], [], {}
        self.next_label = 0

    def new_label(self) -> int:
        x = self.next_label
        self.next_label += 1
        self.extent[x] = 2
        return x

    def add(self, data: np.ndarray, modes) -> None:
        self.tensors.append(np.ascontiguousarray(data))
        self.modes.append(tuple(modes))


def amplitude_network(rows: int, cols: int, cycles: int, seed: int, bitstring=None, open_qubits=()) -> Network:
    """Closed network for <x|C|0>; x is drawn from the same seed unless given. Qubits in
    `open_qubits` get no projection: their output wires stay open (in that order), so the
    network is the tensor of the 2^len(open_qubits) amplitudes that share the other bits
    (a batch of correlated amplitudes from one contraction)."""
    n = rows * cols
    gates = circuit_gates(rows, cols, cycles, seed)
    if bitstring is None:
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        bitstring = tuple(int(b) for b in rng.integers(0, 2, size=n))
    b = _Builder()
    wire = []
    for _ in range(n):
        x = b.new_label()
        b.add(np.array([1.0, 0.0], dtype=np.complex128), (x,))
        wire.append(x)
    for (q0, q1, u) in gates:
        o0, o1 = b.new_label(), b.new_label()
        g = u.reshape(2, 2, 2, 2)  # [o0, o1, i0, i1]
        b.add(g, (o0, o1, wire[q0], wire[q1]))
        wire[q0], wire[q1] = o0, o1
    for q in range(n):
        if q in open_qubits:
            continue
        e = np.zeros(2, dtype=np.complex128)
        e[bitstring[q]] = 1.0
        b.add(e, (wire[q],))
    suffix = f"_open{len(open_qubits)}" if open_qubits else ""
    net = Network(b.tensors, b.modes, b.extent, tuple(wire[q] for q in open_qubits),
                  name=f"rc_{rows}x{cols}_m{cycles}_s{seed}{suffix}",
                  meta=dict(rows=rows, cols=cols, cycles=cycles, seed=seed, bitstring=bitstring,
                            gates=gates, open_qubits=tuple(open_qubits)))
    net.check()
    return net


def state_network(n_qubits: int, n_gates: int, seed: int, shuffle: bool = True, extents=None,
                  gate_pairs=None) -> Network:
    """An n-qubit input state (a seeded complex Gaussian tensor, one large leaf) whose
    declared mode order is a seeded permutation of its qubits when `shuffle`, followed by
    `n_gates` Haar-random two-qubit gates on seeded qubit pairs (or `gate_pairs`); the
    output is the final state with its qubits open in order. `extents` (per qubit) replaces
    the qubit dimension 2 by other sizes (gates then act on dimension d0*d1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = list(extents) if extents is not None else [2] * n_qubits
    b = _Builder()
    wire = []
    for q in range(n_qubits):
        x = b.new_label()
        b.extent[x] = ext[q]
        wire.append(x)
    order = list(rng.permutation(n_qubits)) if shuffle else list(range(n_qubits))
    shape = tuple(ext[q] for q in order)
    psi = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    b.add(psi, tuple(wire[q] for q in order))
    pairs = gate_pairs if gate_pairs is not None else [
        tuple(int(v) for v in rng.choice(n_qubits, size=2, replace=False)) for _ in range(n_gates)]
    for (q0, q1) in pairs:
        d = ext[q0] * ext[q1]
        u = haar_unitary(rng, d).reshape(ext[q0], ext[q1], ext[q0], ext[q1])
        o0, o1 = b.new_label(), b.new_label()
        b.extent[o0], b.extent[o1] = ext[q0], ext[q1]
        b.add(u, (o0, o1, wire[q0], wire[q1]))
        wire[q0], wire[q1] = o0, o1
    net = Network(b.tensors, b.modes, b.extent, tuple(wire),
                  name=f"state_{n_qubits}q_g{len(pairs)}_s{seed}" + ("_shuf" if shuffle else ""),
                  meta=dict(n_qubits=n_qubits, seed=seed, order=order, pairs=pairs))
    net.check()
    return net


def state_path(net: Network):
    """The state-vector order for state_network: the state absorbs the gates one by one."""
    from .network import Path
    pairs, cur = [], 0
    n = len(net.modes)
    for g in range(1, n):
        pairs.append((cur, g))
        cur = n + g - 1
    return Path(pairs)
