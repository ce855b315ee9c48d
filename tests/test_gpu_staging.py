"""Tiled leaf staging on the GPU against the CPU oracle, element by element: a 2^26-element
state in a shuffled declared order absorbing gates (the staged copy is planar FP32), two
large leaves meeting in a tensor-core step (staged in the split-BF16 form), extents other
than 2, and a sliced large leaf. Staging itself is exact (a copy, plus the exact hi/lo
split), so the bounds are those of the steps after it."""
import numpy as np
import pytest
import torch

import oracle
from tests._lib import BF16X3_BOUND, FP32_BAR, ensure_built
from tn_inputs import circuits
from tn_inputs.network import Network, Path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def run(tn, net, path, sliced=(), prec="fp32", batch=0):
    plan = tn.Plan(net, path, sliced, prec=prec, max_slice_batch=batch)
    plan.check_staging()
    assert plan.tensor(0)["tiled"] >= 1
    ins = [torch.tensor(np.asarray(t), dtype=torch.complex64, device="cuda") for t in net.tensors]
    out = torch.zeros(tuple(net.extent[x] for x in net.open_modes), dtype=torch.complex128, device="cuda")
    plan.contract(ins, out)
    torch.cuda.synchronize()
    plan.destroy()
    return out.cpu().numpy()


def elementwise(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


def test_state_2_to_26_shuffled(tn):
    """The largest leaf of the staging tests: 2^26 complex64 (512 MiB), declared in a
    shuffled qubit order, then three gates (streaming steps, k = 4)."""
    net = circuits.state_network(26, 3, 26)
    path = circuits.state_path(net)
    got = run(tn, net, path)
    want = oracle.contract(net, path)
    assert elementwise(got, want) < FP32_BAR


def test_other_extents_and_identity_order(tn):
    ext = [3, 5, 2, 7, 4, 3, 2, 6]
    for shuffle in (True, False):
        net = circuits.state_network(8, 0, 5, shuffle=shuffle, extents=ext,
                                     gate_pairs=[(0, 1), (2, 3), (4, 5), (6, 7)])
        path = circuits.state_path(net)
        assert elementwise(run(tn, net, path), oracle.contract(net, path)) < FP32_BAR


def test_sliced_large_leaf(tn):
    net = circuits.state_network(18, 0, 7, gate_pairs=[(q, q + 1) for q in range(0, 18, 2)])
    path = circuits.state_path(net)
    for sliced in (list(net.modes[0][:2]), list(net.modes[0][-2:])):
        got = run(tn, net, path, sliced, batch=3)
        assert elementwise(got, oracle.contract(net, path, sliced)) < FP32_BAR


def two_big_leaves(seed=3, n_a=10, n_b=10, n_k=10):
    """A[shuffled M + K] . B[shuffled N + K] over 2^10 x 2^10 x 2^10: a tensor-core step
    in the BF16x3 form, so both leaves are staged in the split form."""
    rng = np.random.default_rng(seed)
    M = list(range(n_a))
    N = list(range(n_a, n_a + n_b))
    K = list(range(n_a + n_b, n_a + n_b + n_k))
    am = [M[i] for i in rng.permutation(n_a)] + [K[i] for i in rng.permutation(n_k)]
    am = [am[i] for i in rng.permutation(len(am))]
    bm = [N[i] for i in rng.permutation(n_b)] + [K[i] for i in rng.permutation(n_k)]
    bm = [bm[i] for i in rng.permutation(len(bm))]
    shp = lambda ms: (2,) * len(ms)
    A = rng.standard_normal(shp(am)) + 1j * rng.standard_normal(shp(am))
    B = rng.standard_normal(shp(bm)) + 1j * rng.standard_normal(shp(bm))
    net = Network([A, B], [tuple(am), tuple(bm)], {x: 2 for x in M + N + K}, tuple(M + N))
    net.check()
    return net, Path([(0, 1)])


def test_two_large_leaves_split_form(tn):
    net, path = two_big_leaves()
    plan = tn.Plan(net, path, prec="bf16x3", host_only=True)
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC and plan.tensor(0)["format"] == 1 and plan.tensor(1)["format"] == 1
    plan.destroy()
    want = oracle.contract(net, path)
    got = run(tn, net, path, prec="bf16x3")
    assert elementwise(got, want) < BF16X3_BOUND
    got32 = run(tn, net, path, prec="fp32")
    assert elementwise(got32, want) < FP32_BAR
