"""GPU parity: the CUDA path through the C ABI against the CPU complex128 oracle, on
the same seeded inputs.

Tolerance (complex64/FP32 arithmetic): each step rounds every product and every
partial sum to FP32 (unit roundoff u = 2^-24 ~ 6e-8). Along a path of depth d the
relative error of a result without heavy cancellation grows roughly like
sqrt(sum of k over the path) * u; for the networks here that is below 1e-6, so
scalar results must match to a relative 1e-5 (the bar the method is held to), and
tensor results to a relative Frobenius norm of 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from tests._lib import ensure_built
from tests.test_oracle_pins import random_network
from tn_inputs import circuits, greedy, ising_pf, kicked_ising, workloads
from tn_inputs.network import Network, Path

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def dev_inputs(net, cplx=True):
    dt = torch.complex64 if cplx else torch.float32
    return [torch.tensor(np.asarray(t), dtype=dt, device="cuda").contiguous() for t in net.tensors]


def run(tn, plan, net, cplx=True, begin=None, count=None):
    ins = dev_inputs(net, cplx)
    shape = tuple(net.extent[x] for x in net.open_modes)
    out = torch.zeros(shape, dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    if begin is None:
        plan.contract(ins, out, ls)
    else:
        plan.contract_slices(ins, begin, count, out, ls)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(ls.cpu()[0])


def rel_err(got, want):
    got, want = np.asarray(got), np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / max(np.linalg.norm(want.ravel()), 1e-300))


def test_rc12_amplitude(tn):
    w = workloads.rc12()
    plan = tn.Plan(w.net, w.path)
    got, _ = run(tn, plan, w.net)
    want = oracle.contract(w.net, w.path)
    assert rel_err(got, want) < REL


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n_open", [0, 3])
def test_random_networks(tn, seed, n_open):
    cplx = seed % 3 != 2
    net = random_network(100 + seed, n_tensors=8, n_labels=15, n_open=n_open, complex_=cplx)
    path = greedy.greedy_path(net, seed=seed, temperature=0.5)
    plan = tn.Plan(net, path, prec=0 if cplx else 4)
    got, _ = run(tn, plan, net, cplx)
    want = oracle.contract(net, path)
    assert rel_err(got, want) < REL


def test_single_tensor_network(tn):
    rng = np.random.default_rng(1)
    t = rng.standard_normal((2, 3, 4)) + 1j * rng.standard_normal((2, 3, 4))
    from tn_inputs.network import Network, Path
    net = Network([t], [(0, 1, 2)], {0: 2, 1: 3, 2: 4}, (2, 0, 1))
    plan = tn.Plan(net, Path([]))
    got, _ = run(tn, plan, net)
    assert rel_err(got, np.transpose(t, (2, 0, 1))) < 1e-6


def test_disconnected_outer_product(tn):
    from tn_inputs.network import Network, Path
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    b = rng.standard_normal((2, 5)) + 1j * rng.standard_normal((2, 5))
    c = rng.standard_normal((4,)) + 1j * rng.standard_normal((4,))
    net = Network([a, b, c], [(0, 1), (1, 2), (3,)], {0: 3, 1: 2, 2: 5, 3: 4}, (3, 2, 0))
    path = Path([(0, 1), (3, 2)])  # the second step has k = 1
    plan = tn.Plan(net, path)
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path)) < REL


@pytest.mark.parametrize("arity,real", [(1, False), (2, True), (2, False), (3, False), (4, False), (4, True)])
def test_stream_gate_widths(tn, arity, real):
    """The streaming kernel's forms on a 2^18 state: k = 2 (registers, one float at a
    time) and k = 4, 8, 16 (rows staged in shared memory by bulk copies; n = 4, 8, 16),
    complex and real; element by element against the oracle (largest error relative to the
    largest amplitude)."""
    net, path = gate_chain_network(n_qubits=18, n_gates=6, seed=10 + arity, arity=arity, real=real)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT if real else 0)
    classes = [plan.step(s)["cls"] for s in range(len(path.pairs))]
    assert classes.count(tn.TN_CLASS_STREAM) == len(classes)
    got, _ = run(tn, plan, net, cplx=not real)
    want = oracle.contract(net, path)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-5


@pytest.mark.parametrize("batch", [1, 2, 4])
def test_stream_sliced_big_operand(tn, batch):
    """A gate chain with the original label of a gated qubit sliced (4 slices over two
    labels): the state and the first gates are batched, so the streaming steps read a
    batched big operand (batch stride between slices) at 1, 2 and 4 slices per pass."""
    net, path = gate_chain_network(n_qubits=18, n_gates=6, seed=21, arity=2)
    sliced = [net.modes[1][2], net.modes[1][3]]
    plan = tn.Plan(net, path, sliced, max_slice_batch=batch)
    assert plan.step(0)["cls"] == tn.TN_CLASS_STREAM and plan.step(0)["batched"] == 1
    got, _ = run(tn, plan, net)
    want = oracle.contract(net, path, sliced)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-5


@pytest.mark.parametrize("batch", [1, 3, 16, 0])
def test_sliced_sum_and_partials(tn, batch):
    w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=batch)
    got, _ = run(tn, plan, w.net)
    want, parts = oracle.contract_slices(w.net, w.path, w.sliced, return_partials=True)
    assert rel_err(got, want) < REL
    for sid in (0, 5, 15):
        g, _ = run(tn, plan, w.net, begin=sid, count=1)
        assert rel_err(g, parts[sid]) < REL
    g, _ = run(tn, plan, w.net, begin=2, count=7)
    assert rel_err(g, sum(parts[2:9])) < REL


def test_kicked_ising_small(tn):
    net = kicked_ising.expectation_network(3, 3)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    plan = tn.Plan(net, path)
    got, _ = run(tn, plan, net)
    want = oracle.contract(net, path)
    assert abs(got - want) < REL * max(1.0, abs(want))


def gate_chain_network(n_qubits=12, n_gates=10, seed=4, arity=2, real=False):
    """A 2^n state tensor absorbing a chain of `arity`-qubit gates (state-vector style
    path): every step is big x small, with the gate's new modes landing at arbitrary
    positions of the open result. real: a real state and orthogonal gates."""
    from tn_inputs.network import Network, Path
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((2,) * n_qubits)
    if not real:
        psi = psi + 1j * rng.standard_normal((2,) * n_qubits)
    wire = list(range(n_qubits))
    tensors, modes, nxt = [psi], [tuple(wire)], n_qubits
    d = 2 ** arity
    for _ in range(n_gates):
        qs = [int(x) for x in rng.choice(n_qubits, size=arity, replace=False)]
        u = np.linalg.qr(rng.standard_normal((d, d)))[0] if real else circuits.haar_unitary(rng, d)
        tensors.append(u.reshape((2,) * (2 * arity)))
        modes.append(tuple(range(nxt, nxt + arity)) + tuple(wire[q] for q in qs))
        for i, q in enumerate(qs):
            wire[q] = nxt + i
        nxt += arity
    net = Network(tensors, modes, {x: 2 for x in range(nxt)}, tuple(wire))
    net.check()
    pairs, cur = [], 0
    for g in range(1, n_gates + 1):
        pairs.append((cur, g))
        cur = n_gates + g
    return net, Path(pairs)


def test_stream_class_steps(tn):
    """Big x small steps run on the streaming kernel and match the oracle."""
    net, path = gate_chain_network()
    plan = tn.Plan(net, path)
    classes = [plan.step(s)["cls"] for s in range(len(path.pairs))]
    assert classes.count(tn.TN_CLASS_STREAM) == len(classes)
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path)) < REL


@pytest.mark.parametrize("n,seed", [(20, 1), (40, 2), (60, 3)])
def test_ising_partition_function_scaled(tn, n, seed):
    net = ising_pf.random_3regular_network(n, seed, beta=0.5)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    got, ls = run(tn, plan, net, cplx=False)
    want = oracle.contract(net, path)
    lnz = np.log(got) + ls
    assert abs(lnz - np.log(want)) < 1e-5


def test_ising_ring_overflow_needs_scaling(tn):
    """Z = (2 cosh 1)^300 + (2 sinh 1)^300 ~ 1e146 overflows FP32 intermediates; the
    exponent-scaled path recovers ln Z (transfer-matrix closed form)."""
    from oracle import pins
    n, J, beta = 300, 1.0, 1.0
    net = ising_pf.ring_network(n, J, beta)
    path = greedy.greedy_path(net, seed=0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    got, ls = run(tn, plan, net, cplx=False)
    want_ln = np.log(pins.ising_ring_closed_form(n, J, beta)) if n < 300 else \
        n * np.log(2 * np.cosh(1.0)) + np.log1p(np.tanh(1.0) ** n)
    assert abs(np.log(got) + ls - want_ln) < 1e-5 * abs(want_ln)


def test_contract_host_roundtrip(tn):
    w = workloads.rc12()
    plan = tn.Plan(w.net, w.path)
    host = [np.ascontiguousarray(np.asarray(t, dtype=np.complex64)) for t in w.net.tensors]
    out = np.zeros((), dtype=np.complex128)
    ls = np.zeros(1)
    plan.contract_host(host, out, ls)
    want = oracle.contract(w.net, w.path)
    assert rel_err(out, want) < REL and ls[0] == 0.0


def dot_network(out_a, out_b, k_dims, seed=9, sliced_dim=None):
    """A[a..., k...] . B[b..., k...] with few open labels and a long reduction."""
    from tn_inputs.network import Network
    rng = np.random.default_rng(seed)
    ext, lab = {}, 0
    A_open, B_open, K = [], [], []
    for grp, dims in ((A_open, out_a), (B_open, out_b), (K, k_dims)):
        for d in dims:
            ext[lab] = d
            grp.append(lab)
            lab += 1
    am, bm = tuple(A_open + K), tuple(B_open + K)
    if sliced_dim:
        ext[lab] = sliced_dim
        am, bm = am + (lab,), (lab,) + bm
        lab += 1
    shp = lambda ms: tuple(ext[x] for x in ms)
    A = rng.standard_normal(shp(am)) + 1j * rng.standard_normal(shp(am))
    B = rng.standard_normal(shp(bm)) + 1j * rng.standard_normal(shp(bm))
    net = Network([A, B], [am, bm], ext, tuple(B_open + A_open))
    net.check()
    from tn_inputs.network import Path
    return net, Path([(0, 1)]), ([lab - 1] if sliced_dim else [])


@pytest.mark.parametrize("out_a,out_b,k_dims", [((), (), (2,) * 16), ((2,), (2,), (5, 7, 500)),
                                                ((4,), (2, 2), (2,) * 14)])
def test_splitk_long_reduction(tn, out_a, out_b, k_dims):
    """Few outputs and a long k (a dot product of two big tensors): split-K partials in
    FP64, summed in a fixed order; includes a ragged last chunk (k = 17500)."""
    net, path, _ = dot_network(out_a, out_b, k_dims)
    plan = tn.Plan(net, path)
    assert plan.step(0)["cls"] == tn.TN_CLASS_SPLITK
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path)) < REL


def test_splitk_sliced_batch(tn):
    net, path, sliced = dot_network((2,), (), (2,) * 13, sliced_dim=4)
    plan = tn.Plan(net, path, sliced, max_slice_batch=3)
    assert plan.step(0)["cls"] == tn.TN_CLASS_SPLITK and plan.step(0)["batched"] == 1
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path, sliced)) < REL


@pytest.mark.parametrize("k_bits", [11, 13])
def test_simt_ksplit_underfilled_grid(tn, k_bits):
    """A 64 x 96 output over k = 2^11 or 2^13: too few 64 x 64 tiles to fill the GPU, so the
    CUDA-core kernel cuts k into parts and a second kernel combines them in part order."""
    rng = np.random.default_rng(k_bits)
    kd = (2,) * k_bits
    A = rng.standard_normal((64,) + kd) + 1j * rng.standard_normal((64,) + kd)
    B = rng.standard_normal((96,) + kd) + 1j * rng.standard_normal((96,) + kd)
    K = tuple(range(2, 2 + k_bits))
    ext = {0: 64, 1: 96, **{x: 2 for x in K}}
    net = Network([A, B], [(0,) + K, (1,) + K], ext, (1, 0))
    path = Path([(0, 1)])
    plan = tn.Plan(net, path, prec="fp32")
    assert plan.step(0)["cls"] == tn.TN_CLASS_SIMT
    got, _ = run(tn, plan, net)
    want = oracle.contract(net, path)
    assert rel_err(got, want) < 1e-5
    plan.destroy()
