"""GPU parity of the step chains (runs of tiny CUDA-core steps executed by one CTA in one
launch) in the cases their kernel treats specially: passes after the first (the chain skips
its slice-invariant steps, computed once and kept), exponent scaling (a step's scale record
written and read inside the one launch), the max-plus semiring, complex outputs in the split
storage form (a chain step feeding a BF16x3 tensor-core step), and one pass. Every case
asserts that the plan has chains and compares with the CPU oracle: FP32 arithmetic to 1e-5
(complex), ln Z to 1e-5 (scaled), maximum independent sets exactly."""
import numpy as np
import pytest

import oracle
from oracle import pins
from tests._lib import ensure_built
from tn_inputs import greedy, ising_pf, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def chains(plan, n_steps):
    steps = [plan.step(s) for s in range(n_steps)]
    ids = {st["chain"] for st in steps if st["chain"] >= 0}
    mixed = any({st["batched"] for st in steps if st["chain"] == c} == {0, 1} for c in ids)
    return len(ids), mixed


def contract_host(plan, net, cplx):
    dt = np.complex64 if cplx else np.float32
    host = [np.ascontiguousarray(np.asarray(t, dtype=dt)) for t in net.tensors]
    out = np.zeros(tuple(plan.out_shape), dtype=np.complex128 if cplx else np.float64)
    ls = np.zeros(1)
    plan.contract_host(host, out, ls)
    return out, float(ls[0])


@pytest.mark.parametrize("batch", [3, 16])
def test_chains_over_passes(tn, batch):
    """A sliced circuit (16 slices) in passes of 3 (six passes: later ones skip the chains'
    slice-invariant steps) and in one pass of 16."""
    w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=batch)
    try:
        n, mixed = chains(plan, len(w.path.pairs))
        assert n >= 1
        if batch == 3:
            assert mixed, "a chain holding slice-invariant and batched steps"
        got, _ = contract_host(plan, w.net, True)
    finally:
        plan.destroy()
    want = complex(oracle.contract(w.net, w.path, w.sliced))
    assert abs(complex(got) - want) < 1e-5 * abs(want)


def test_chains_with_exponent_scaling(tn):
    """An Ising ring of 300 spins (Z ~ 1e146, beyond FP32): every step is tiny, so the whole
    path is chains; ln Z against the transfer-matrix closed form."""
    n, J, beta = 300, 1.0, 1.0
    net = ising_pf.ring_network(n, J, beta)
    path = greedy.greedy_path(net, seed=0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    try:
        assert chains(plan, len(path.pairs))[0] >= 1
        got, ls = contract_host(plan, net, False)
    finally:
        plan.destroy()
    want_ln = n * np.log(2 * np.cosh(beta * J)) + np.log1p(np.tanh(beta * J) ** n)
    assert abs(np.log(float(got)) + ls - want_ln) < 1e-5 * abs(want_ln)
    small = ising_pf.ring_network(40, J, beta)
    spath = greedy.greedy_path(small, seed=0)
    plan = tn.Plan(small, spath, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    try:
        got, ls = contract_host(plan, small, False)
    finally:
        plan.destroy()
    assert abs(np.log(float(got)) + ls - np.log(pins.ising_ring_closed_form(40, J, beta))) < 1e-5


def test_chains_in_the_maxplus_semiring(tn):
    """Maximum independent set of a King's subgraph, sliced, in passes of 4: exact."""
    w = workloads.kings_mis(10, 0.8, 5, 3)
    plan = tn.Plan(w.net, w.path, w.sliced, prec=tn.TN_R32_FP32_SIMT, semiring="maxplus", max_slice_batch=4)
    try:
        assert chains(plan, len(w.path.pairs))[0] >= 1
        got, _ = contract_host(plan, w.net, False)
    finally:
        plan.destroy()
    assert float(got) == float(oracle.contract(w.net, w.path, w.sliced, semiring="maxplus"))


def test_chains_feeding_bf16x3_steps(tn):
    """The 20-qubit circuit in the BF16x3 form: chain steps whose outputs feed tensor-core
    steps store the split form; the amplitude within BF16x3's bound."""
    w = workloads.random_circuit(4, 5, 12, 40)
    plan = tn.Plan(w.net, w.path, prec="bf16x3")
    try:
        n_steps = len(w.path.pairs)
        assert chains(plan, n_steps)[0] >= 1
        split_out = [plan.tensor(plan.n_leaves + s)["format"] for s in range(n_steps)
                     if plan.step(s)["chain"] >= 0]
        assert any(x != 0 for x in split_out), "a chain step writes the split form"
        got, _ = contract_host(plan, w.net, True)
    finally:
        plan.destroy()
    want = complex(oracle.contract(w.net, w.path))
    assert abs(complex(got) - want) < 3 * 2.0 ** -16 * abs(want)
