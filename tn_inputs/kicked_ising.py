"""Seeded 2D kicked-Ising dynamics networks (the many-body dynamics family of Sec. III-D,
on the rectangular, hexagonal and triangular lattices the paper's dynamics workloads use).

One Trotter step applies exp(-i J dt Z_a Z_b) on every nearest-neighbour bond of an
open lattice, then the kick exp(-i h dt X) on every site. The network is the closed
expectation value <0| U^dagger Z_c U |0> with U the product of T steps and Z_c the
Pauli Z at the centre site ((rows-1)//2, (cols-1)//2), 0-based.

Lattices, with sites on a rows x cols grid (q = r * cols + c):
  square     : bonds (r,c)-(r,c+1) and (r,c)-(r+1,c); interior degree 4;
  hexagonal  : the honeycomb lattice in its brick-wall form: every horizontal bond, and the
               vertical bond (r,c)-(r+1,c) only where r + c is even; degree <= 3;
  triangular : the square bonds plus the diagonal (r,c)-(r+1,c+1); interior degree 6.

Gates enter the network as dense tensors (rank 4 for a bond gate, rank 2 for a kick):
the diagonal structure of the bond gate is data, not a hyper-edge.
"""
from __future__ import annotations

import numpy as np

from .network import Network
from .circuits import _Builder


def zz_gate(J: float, dt: float) -> np.ndarray:
    th = J * dt
    return np.diag(np.exp(-1j * th * np.array([1.0, -1.0, -1.0, 1.0]))).astype(np.complex128)


def x_kick(h: float, dt: float) -> np.ndarray:
    a = h * dt
    return np.array([[np.cos(a), -1j * np.sin(a)], [-1j * np.sin(a), np.cos(a)]], dtype=np.complex128)


LATTICES = ("square", "hexagonal", "triangular")


def lattice_bonds(L: int, cols: int | None = None, lattice: str = "square"):
    """Nearest-neighbour bonds (a, b), a < b, of an L x cols open lattice."""
    rows, cols = L, (L if cols is None else cols)
    if lattice not in LATTICES:
        raise ValueError(f"unknown lattice {lattice!r}")
    q = lambda r, c: r * cols + c
    bonds = [(q(r, c), q(r, c + 1)) for r in range(rows) for c in range(cols - 1)]
    bonds += [(q(r, c), q(r + 1, c)) for r in range(rows - 1) for c in range(cols)
              if lattice != "hexagonal" or (r + c) % 2 == 0]
    if lattice == "triangular":
        bonds += [(q(r, c), q(r + 1, c + 1)) for r in range(rows - 1) for c in range(cols - 1)]
    return bonds


def trotter_ops(L: int, T: int, J: float, h: float, dt: float, cols: int | None = None,
                lattice: str = "square"):
    """The forward operator sequence of U: [('zz', a, b, U4) | ('x', q, U2)]."""
    ops = []
    g2, k1 = zz_gate(J, dt), x_kick(h, dt)
    n = L * (L if cols is None else cols)
    for _ in range(T):
        for (a, b) in lattice_bonds(L, cols, lattice):
            ops.append(("zz", a, b, g2))
        for qb in range(n):
            ops.append(("x", qb, k1))
    return ops


def center_site(L: int, cols: int | None = None) -> int:
    cols = L if cols is None else cols
    return ((L - 1) // 2) * cols + (cols - 1) // 2


def expectation_network(L: int, T: int, J: float = 1.0, h: float = 0.9, dt: float = 0.25,
                        cols: int | None = None, lattice: str = "square") -> Network:
    """<Z_centre> after T kicked-Ising steps on an L x cols lattice (cols defaults to L)."""
    cols_ = L if cols is None else cols
    n = L * cols_
    ops = trotter_ops(L, T, J, h, dt, cols, lattice)
    b = _Builder()
    wire = []
    for _ in range(n):
        x = b.new_label()
        b.add(np.array([1.0, 0.0], dtype=np.complex128), (x,))
        wire.append(x)

    def apply(op, dagger: bool):
        if op[0] == "zz":
            _, qa, qb, u = op
            if dagger:
                u = u.conj().T
            o0, o1 = b.new_label(), b.new_label()
            b.add(u.reshape(2, 2, 2, 2), (o0, o1, wire[qa], wire[qb]))
            wire[qa], wire[qb] = o0, o1
        else:
            _, q, u = op
            if dagger:
                u = u.conj().T
            o = b.new_label()
            b.add(u, (o, wire[q]))
            wire[q] = o

    for op in ops:
        apply(op, False)
    c = center_site(L, cols)
    o = b.new_label()
    b.add(np.diag([1.0, -1.0]).astype(np.complex128), (o, wire[c]))
    wire[c] = o
    for op in reversed(ops):
        apply(op, True)
    for q in range(n):
        b.add(np.array([1.0, 0.0], dtype=np.complex128), (wire[q],))
    tag = "" if lattice == "square" else f"_{lattice[:3]}"
    net = Network(b.tensors, b.modes, b.extent, (), name=f"kising{tag}_{L}x{cols_}_T{T}",
                  meta=dict(L=L, cols=cols_, T=T, J=J, h=h, dt=dt, ops=ops, center=c, lattice=lattice,
                            n_sites=n))
    net.check()
    return net
