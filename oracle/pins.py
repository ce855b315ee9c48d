"""Independent references that pin the oracle (TEST INFRASTRUCTURE ONLY).

None of these evaluates a network pairwise; each reaches the same number another way:
  * brute_force: the definition of Sec. II-A written out -- the sum, over every
    assignment of every label, of the product of all tensor entries;
  * statevector_*: a direct simulation of the circuit on a 2^n state vector, applying
    each gate to the two (or one) qubit axes it acts on;
  * ising_*: the Ising partition function by enumerating spin configurations, and the
    1D ring's transfer-matrix closed form Z = l1^N + l2^N with l = e^{bJ} +- e^{-bJ};
  * kicked-Ising special cases with closed forms;
  * independent sets: count and maximum size by checking every vertex subset, and the
    closed forms for paths (Fibonacci), cycles (Lucas) and the full King's graph.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def brute_force(net, max_labels: int = 22):
    """sum_{all label values} prod_t T_t[...]; open labels are kept as result axes."""
    labels = net.labels()
    closed = [x for x in labels if x not in net.open_modes]
    assert len(closed) + len(net.open_modes) <= max_labels, "network too large for brute force"
    dtype = np.complex128 if net.is_complex else np.float64
    out_shape = tuple(net.extent[x] for x in net.open_modes)
    result = np.zeros(out_shape, dtype=dtype)
    # enumerate every closed assignment at once (vectorised over the assignment index)
    sizes = [net.extent[x] for x in closed]
    total = int(np.prod(sizes, dtype=np.int64)) if closed else 1
    digits = {}
    r = np.arange(total, dtype=np.int64)
    for x, d in zip(reversed(closed), reversed(sizes)):
        digits[x] = r % d
        r = r // d
    for opn in itertools.product(*[range(net.extent[x]) for x in net.open_modes]):
        val = dict(zip(net.open_modes, opn))
        prod = np.ones(total, dtype=dtype)
        for t, ms in zip(net.tensors, net.modes):
            idx = tuple(digits[x] if x in digits else np.full(total, val[x]) for x in ms)
            prod = prod * np.asarray(t, dtype=dtype)[idx]
        result[opn] = prod.sum()
    return result if out_shape else result.reshape(())[()]


# ---- state-vector simulation ------------------------------------------------------------

def _apply_1q(psi, n, q, u):
    psi = np.moveaxis(psi.reshape((2,) * n), q, 0)
    shp = psi.shape
    psi = (u @ psi.reshape(2, -1)).reshape(shp)
    return np.moveaxis(psi, 0, q).reshape(-1)


def _apply_2q(psi, n, q0, q1, u):
    psi = np.moveaxis(psi.reshape((2,) * n), (q0, q1), (0, 1))
    shp = psi.shape
    psi = (u @ psi.reshape(4, -1)).reshape(shp)
    return np.moveaxis(psi, (0, 1), (q0, q1)).reshape(-1)


def statevector_circuit(n, gates):
    """psi = C|0...0>, qubit 0 the most significant bit of the basis index."""
    psi = np.zeros(2**n, dtype=np.complex128)
    psi[0] = 1.0
    for (q0, q1, u) in gates:
        psi = _apply_2q(psi, n, q0, q1, u)
    return psi


def amplitude_statevector(rows, cols, gates, bitstring):
    psi = statevector_circuit(rows * cols, gates)
    idx = 0
    for b in bitstring:
        idx = idx * 2 + int(b)
    return psi[idx]


def kicked_ising_statevector(L, ops, center, n_sites=None):
    """<Z_center> after applying the operator list `ops` to |0...0> of n_sites qubits
    (default L * L)."""
    n = L * L if n_sites is None else n_sites
    psi = np.zeros(2**n, dtype=np.complex128)
    psi[0] = 1.0
    for op in ops:
        if op[0] == "zz":
            psi = _apply_2q(psi, n, op[1], op[2], op[3])
        else:
            psi = _apply_1q(psi, n, op[1], op[2])
    z = np.ones(2**n)
    bit = (np.arange(2**n) >> (n - 1 - center)) & 1
    z[bit == 1] = -1.0
    return float(np.real(np.vdot(psi, z * psi)))


def kicked_ising_closed_form(L, T, J, h, dt):
    """Special cases: h = 0 or dt = 0 gives 1; J = 0 gives cos(2 h dt T)."""
    if h == 0.0 or dt == 0.0:
        return 1.0
    if J == 0.0:
        return math.cos(2.0 * h * dt * T)
    raise ValueError("no closed form for J, h, dt all nonzero")


# ---- Ising partition functions ------------------------------------------------------------

def ising_enumerate(n, edges, J, beta):
    """Z by summing exp(beta sum J s_u s_v) over all 2^n spin configurations."""
    assert n <= 24
    idx = np.arange(2**n, dtype=np.int64)
    s = 1.0 - 2.0 * ((idx[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1)
    energy = np.zeros(2**n)
    for (u, v), j in zip(edges, J):
        energy += j * s[:, u] * s[:, v]
    return float(np.exp(beta * energy).sum())


def ising_ring_closed_form(n, J, beta):
    l1 = math.exp(beta * J) + math.exp(-beta * J)
    l2 = math.exp(beta * J) - math.exp(-beta * J)
    return l1**n + l2**n


# ---- independent sets (the semiring family of Sec. III-C) --------------------------------

def independent_sets_enumerate(n, edges):
    """(number of independent sets, size of a maximum one) by checking every vertex subset."""
    adj = [0] * n
    for u, v in edges:
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    count, best = 0, 0
    for mask in range(1 << n):
        ok = True
        m = mask
        while m:
            u = (m & -m).bit_length() - 1
            if adj[u] & mask:
                ok = False
                break
            m &= m - 1
        if ok:
            count += 1
            best = max(best, bin(mask).count("1"))
    return count, best


def _fib(k):
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def path_graph_closed_form(n):
    """Path on n >= 1 vertices: F(n + 2) independent sets (Fibonacci, F(1) = F(2) = 1), and
    a maximum one has ceil(n / 2) vertices."""
    return _fib(n + 2), (n + 1) // 2


def cycle_graph_closed_form(n):
    """Cycle on n >= 3 vertices: the Lucas number L(n) = F(n - 1) + F(n + 1) independent
    sets, and a maximum one has floor(n / 2) vertices."""
    return _fib(n - 1) + _fib(n + 1), n // 2


def kings_full_mis(L):
    """The full L x L King's graph: every 2 x 2 block holds at most one vertex of an
    independent set and the sites with even row and column reach that, ceil(L/2)^2."""
    return ((L + 1) // 2) ** 2
