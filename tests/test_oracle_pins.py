"""The CPU oracle against references that do not evaluate a network pairwise:
brute-force summation (the definition of Sec. II-A), state-vector simulation, closed
forms, and the identities of Sec. II-B/C (path independence, sliced sum = unsliced)."""
import math

import numpy as np
import pytest

import oracle
from oracle import pins
from oracle import core as oc
from tn_inputs import circuits, kicked_ising, ising_pf, greedy, kings
from tn_inputs.network import Network, Path


def random_network(seed, n_tensors=7, n_labels=14, n_open=0, complex_=True):
    """Random connected network: every closed label joins two distinct tensors."""
    rng = np.random.default_rng(seed)
    modes = [[] for _ in range(n_tensors)]
    lab = 0
    for t in range(1, n_tensors):  # spanning tree keeps it connected
        u = int(rng.integers(0, t))
        modes[u].append(lab)
        modes[t].append(lab)
        lab += 1
    while lab < n_labels - n_open:
        u, v = rng.choice(n_tensors, size=2, replace=False)
        modes[int(u)].append(lab)
        modes[int(v)].append(lab)
        lab += 1
    open_ = []
    for _ in range(n_open):
        u = int(rng.integers(0, n_tensors))
        modes[u].append(lab)
        open_.append(lab)
        lab += 1
    for ms in modes:
        rng.shuffle(ms)
    extent = {x: int(rng.integers(2, 4)) for x in range(lab)}
    tensors = []
    for ms in modes:
        shp = tuple(extent[x] for x in ms)
        t = rng.standard_normal(shp)
        if complex_:
            t = t + 1j * rng.standard_normal(shp)
        tensors.append(t)
    rng.shuffle(open_)
    net = Network(tensors, [tuple(m) for m in modes], extent, tuple(open_))
    net.check()
    return net


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n_open", [0, 2])
def test_brute_force_random(seed, n_open):
    net = random_network(seed, n_open=n_open, complex_=(seed % 2 == 0))
    path = greedy.greedy_path(net, seed=seed)
    got = oracle.contract(net, path)
    want = pins.brute_force(net)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11 * np.max(np.abs(want)))


def test_brute_force_catches_transposed_operand(monkeypatch):
    """A planted mistake in the oracle (B used transposed) must fail the brute-force pin."""
    net = random_network(11, n_open=2)
    path = greedy.greedy_path(net, seed=1)
    want = pins.brute_force(net)
    real_pairwise = oc.pairwise

    def wrong(a, ma, b, mb, keep, semiring="standard"):
        # operand B's data transposed against its labels (first two axes of equal extent)
        for i in range(b.ndim):
            for j in range(i + 1, b.ndim):
                if b.shape[i] == b.shape[j]:
                    return real_pairwise(a, ma, np.swapaxes(b, i, j), mb, keep, semiring)
        return real_pairwise(a, ma, b, mb, keep, semiring)

    monkeypatch.setattr(oc, "pairwise", wrong)
    got = oc.contract(net, path)
    assert not np.allclose(got, want, rtol=1e-8)


def test_brute_force_catches_conjugation(monkeypatch):
    net = random_network(12)
    path = greedy.greedy_path(net, seed=2)
    want = pins.brute_force(net)
    real_pairwise = oc.pairwise
    monkeypatch.setattr(oc, "pairwise", lambda a, ma, b, mb, keep, semiring="standard":
                        real_pairwise(a, ma, np.conj(b), mb, keep, semiring))
    assert not np.allclose(oc.contract(net, path), want, rtol=1e-8)


def test_circuit_amplitude_vs_statevector():
    for (r, c, m, seed) in [(2, 3, 6, 1), (3, 3, 8, 2), (3, 4, 8, 12)]:
        net = circuits.amplitude_network(r, c, m, seed)
        path = greedy.greedy_path(net, seed=0, alpha=1.0)
        got = oracle.contract(net, path)
        want = pins.amplitude_statevector(r, c, net.meta["gates"], net.meta["bitstring"])
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (got, want)


def test_open_qubit_amplitudes_vs_statevector():
    """Leaving qubits unprojected gives the tensor of the amplitudes that share the other
    bits: entry [b_0, b_1, ...] (open qubits in the given order) is <x'|C|0> where x' is
    the bitstring with those qubits set to b_i. Sliced over two labels, the sum agrees."""
    for (r, c, m, seed, open_q) in [(2, 3, 6, 1, (4, 0)), (3, 3, 8, 2, (7, 8, 5))]:
        net = circuits.amplitude_network(r, c, m, seed, open_qubits=open_q)
        assert net.open_modes and len(net.open_modes) == len(open_q)
        path = greedy.greedy_path(net, seed=0, alpha=1.0)
        got = np.asarray(oracle.contract(net, path))
        assert got.shape == (2,) * len(open_q)
        psi = pins.statevector_circuit(r * c, net.meta["gates"])
        base = list(net.meta["bitstring"])
        for bits in np.ndindex(*got.shape):
            x = list(base)
            for q, b in zip(open_q, bits):
                x[q] = b
            idx = int("".join(map(str, x)), 2)
            assert abs(got[bits] - psi[idx]) <= 1e-12, (bits, got[bits], psi[idx])
        closed = [x for x in net.extent if x not in net.open_modes
                  and sum(x in m_ for m_ in net.modes) == 2][:2]
        sliced = np.asarray(oracle.contract_slices(net, path, closed))
        assert np.allclose(sliced, got, rtol=0, atol=1e-12)


def test_circuit_normalisation():
    r, c, m, seed = 3, 3, 8, 5
    gates = circuits.circuit_gates(r, c, m, seed)
    tot = 0.0
    for x in range(2 ** (r * c)):
        bits = tuple((x >> (r * c - 1 - q)) & 1 for q in range(r * c))
        net = circuits.amplitude_network(r, c, m, seed, bitstring=bits)
        if x == 0:
            path = greedy.greedy_path(net, seed=0, alpha=1.0)
        tot += abs(oracle.contract(net, path)) ** 2
    assert abs(tot - 1.0) < 1e-11


def test_kicked_ising_vs_statevector_and_real():
    L, T = 3, 3
    net = kicked_ising.expectation_network(L, T, 1.0, 0.9, 0.25)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    got = oracle.contract(net, path)
    want = pins.kicked_ising_statevector(L, net.meta["ops"], net.meta["center"])
    assert abs(got.imag) < 1e-12
    assert -1.0 <= got.real <= 1.0
    assert abs(got.real - want) < 1e-12


@pytest.mark.parametrize("J,h,dt", [(1.0, 0.0, 0.25), (0.0, 0.9, 0.25), (1.0, 0.9, 0.0), (0.0, 0.7, 0.3)])
def test_kicked_ising_closed_forms(J, h, dt):
    L, T = 3, 4
    net = kicked_ising.expectation_network(L, T, J, h, dt)
    path = greedy.greedy_path(net, seed=1, alpha=1.0)
    got = oracle.contract(net, path)
    assert abs(got - pins.kicked_ising_closed_form(L, T, J, h, dt)) < 1e-12


@pytest.mark.parametrize("rows,cols", [(3, 4), (4, 5), (5, 5)])
def test_lattice_bond_structure(rows, cols):
    """Bond sets of the three lattices: counts in closed form and the coordination numbers
    (square 4, honeycomb 3, triangular 6 for interior sites)."""
    import collections
    sq = kicked_ising.lattice_bonds(rows, cols, "square")
    hx = kicked_ising.lattice_bonds(rows, cols, "hexagonal")
    tr = kicked_ising.lattice_bonds(rows, cols, "triangular")
    assert len(sq) == rows * (cols - 1) + (rows - 1) * cols
    assert len(tr) == len(sq) + (rows - 1) * (cols - 1)
    n_vert = sum(1 for r in range(rows - 1) for c in range(cols) if (r + c) % 2 == 0)
    assert len(hx) == rows * (cols - 1) + n_vert
    for bonds in (sq, hx, tr):
        assert len(set(bonds)) == len(bonds) and all(a < b for a, b in bonds)
    deg = {name: collections.Counter(x for e in b for x in e) for name, b in (("sq", sq), ("hx", hx), ("tr", tr))}
    interior = [r * cols + c for r in range(1, rows - 1) for c in range(1, cols - 1)]
    assert all(deg["sq"][q] == 4 and deg["hx"][q] == 3 and deg["tr"][q] == 6 for q in interior)
    assert max(deg["hx"].values()) == 3


@pytest.mark.parametrize("lattice,rows,cols,T", [("hexagonal", 3, 4, 2), ("triangular", 3, 3, 2),
                                                  ("hexagonal", 2, 5, 3)])
def test_kicked_ising_lattices_vs_statevector(lattice, rows, cols, T):
    net = kicked_ising.expectation_network(rows, T, 1.0, 0.9, 0.25, cols=cols, lattice=lattice)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    got = oracle.contract(net, path)
    want = pins.kicked_ising_statevector(rows, net.meta["ops"], net.meta["center"], n_sites=rows * cols)
    assert abs(got.imag) < 1e-12 and abs(got.real - want) < 1e-12, (got, want)


@pytest.mark.parametrize("lattice", ["hexagonal", "triangular"])
@pytest.mark.parametrize("J,h,dt", [(1.0, 0.0, 0.25), (0.0, 0.7, 0.3)])
def test_kicked_ising_lattices_closed_forms(lattice, J, h, dt):
    rows, cols, T = 3, 3, 3
    net = kicked_ising.expectation_network(rows, T, J, h, dt, cols=cols, lattice=lattice)
    path = greedy.greedy_path(net, seed=1, alpha=1.0)
    got = oracle.contract(net, path)
    assert abs(got - pins.kicked_ising_closed_form(rows, T, J, h, dt)) < 1e-12


@pytest.mark.parametrize("n,seed", [(10, 1), (16, 2), (20, 3)])
def test_ising_3regular_vs_enumeration(n, seed):
    net = ising_pf.random_3regular_network(n, seed, beta=0.5)
    path = greedy.greedy_path(net, seed=seed, alpha=1.0)
    got = oracle.contract(net, path)
    m = net.meta
    want = pins.ising_enumerate(n, m["edges"], m["J"], m["beta"])
    assert abs(got / want - 1.0) < 1e-12


@pytest.mark.parametrize("n,J,beta", [(8, 1.0, 0.5), (30, -1.0, 0.3), (60, 1.0, 0.5)])
def test_ising_ring_transfer_matrix(n, J, beta):
    net = ising_pf.ring_network(n, J, beta)
    path = greedy.greedy_path(net, seed=0)
    got = oracle.contract(net, path)
    assert abs(got / pins.ising_ring_closed_form(n, J, beta) - 1.0) < 1e-12


def test_ising_beta_zero():
    net = ising_pf.random_3regular_network(12, 4, beta=0.0)
    got = oracle.contract(net, greedy.greedy_path(net, seed=0))
    assert abs(got - 2.0**12) < 1e-9


def test_sliced_sum_equals_unsliced():
    net = circuits.amplitude_network(3, 4, 8, 3)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    full = oracle.contract(net, path)
    sl = greedy.greedy_slicer(net, path, -1.0, max_slices=4)
    assert len(sl) == 4
    sliced = oracle.contract(net, path, sl)
    assert abs(sliced - full) < 1e-13
    # the partials are a genuine partition: no single slice carries the sum
    _, parts = oracle.contract_slices(net, path, sl, return_partials=True)
    assert len(parts) == 16 and max(abs(p - full) for p in parts) > 1e-6


def test_path_independence():
    net = random_network(21, n_tensors=9, n_labels=16, n_open=1)
    a = oracle.contract(net, greedy.greedy_path(net, seed=0))
    b = oracle.contract(net, greedy.greedy_path(net, seed=5, alpha=1.0, temperature=0.5))
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_neumaier():
    acc = oracle.Neumaier(np.float64(0.0))
    for v in [1e16, 1.0, -1e16, 3.0]:
        acc.add(v)
    assert acc.value() == 4.0


def test_step_costs_hand_counted():
    # A[a,b,c,d] x B[e,f,c,d] -> C[a,b,e,f] with extents a=2,b=3,c=4,d=5,e=6,f=7
    ext = dict(zip(range(6), [2, 3, 4, 5, 6, 7]))
    A = np.zeros((2, 3, 4, 5))
    B = np.zeros((6, 7, 4, 5))
    net = Network([A, B], [(0, 1, 2, 3), (4, 5, 2, 3)], ext, (0, 1, 4, 5))
    (s,) = oracle.step_costs(net, Path([(0, 1)]))
    m, n, k = 6, 42, 20
    assert (s["m"], s["n"], s["k"]) == (m, n, k)
    assert s["Ct"] == 5040 and s["Cs"] == max(120, 840, 252) and s["Cm"] == 120 + 840 + 252


# ---- semirings: independent sets (Sec. III-C) -------------------------------------------

def _mis_and_count(n, edges, sliced_k=0, seed=0):
    t = kings.independent_set_network(n, edges, "tropical")
    c = kings.independent_set_network(n, edges, "counting")
    path = greedy.greedy_path(t, seed=seed, alpha=1.0)
    sl = list(range(min(sliced_k, len(edges))))
    mis = oracle.contract(t, path, sl, semiring="maxplus")
    cnt = oracle.contract(c, path, sl)
    return float(mis), float(cnt)


@pytest.mark.parametrize("seed", range(6))
def test_independent_sets_vs_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(8, 15))
    edges = sorted({(int(min(u, v)), int(max(u, v))) for u, v in rng.integers(0, n, size=(2 * n, 2)) if u != v})
    want_count, want_mis = pins.independent_sets_enumerate(n, edges)
    for k in (0, 3):  # unsliced, and 3 sliced labels (max / sum over the 8 slices)
        mis, cnt = _mis_and_count(n, edges, sliced_k=k, seed=seed)
        assert mis == want_mis and cnt == want_count, (k, mis, want_mis, cnt, want_count)


@pytest.mark.parametrize("n", [5, 8, 13])
def test_independent_sets_path_and_cycle_closed_forms(n):
    path_edges = [(i, i + 1) for i in range(n - 1)]
    cycle_edges = path_edges + [(0, n - 1)]
    assert _mis_and_count(n, path_edges)[::-1] == tuple(float(x) for x in pins.path_graph_closed_form(n))
    assert _mis_and_count(n, cycle_edges)[::-1] == tuple(float(x) for x in pins.cycle_graph_closed_form(n))


@pytest.mark.parametrize("L", [3, 4, 5])
def test_full_kings_graph_mis(L):
    net = kings.kings_network(L, 1.0, 0)
    assert net.meta["n"] == L * L and len(net.meta["edges"]) == 2 * (L - 1) * (2 * L - 1)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    assert float(oracle.contract(net, path, semiring="maxplus")) == pins.kings_full_mis(L)


def test_kings_subgraph_vs_enumeration():
    net = kings.kings_network(5, 0.8, 11)
    n, edges = net.meta["n"], net.meta["edges"]
    want_count, want_mis = pins.independent_sets_enumerate(n, edges)
    mis, cnt = _mis_and_count(n, edges)
    assert (mis, cnt) == (want_mis, want_count)
