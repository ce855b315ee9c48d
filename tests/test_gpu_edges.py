"""Degenerate and edge inputs through the C ABI against the oracle: an all-zero leaf (with
and without exponent scaling), labels of extent 1, the smallest tensor-core step (128 x 16
outputs over k = 8), the last slice alone, and slice ranges the plan refuses."""
import numpy as np
import pytest
import torch

import oracle
from tests._lib import FP32_BAR, ensure_built
from tests.test_gpu_parity import rel_err, run
from tests.test_oracle_pins import random_network
from tn_inputs import greedy, ising_pf, workloads
from tn_inputs.network import Network, Path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def test_zero_leaf_complex(tn):
    """A zero gate makes the amplitude exactly zero in every form."""
    w = workloads.rc12()
    tensors = list(w.net.tensors)
    tensors[20] = np.zeros_like(np.asarray(tensors[20]))
    net = Network(tensors, w.net.modes, w.net.extent, w.net.open_modes)
    for prec in ("fp32", "3xtf32", "bf16x3"):
        plan = tn.Plan(net, w.path, prec=prec)
        got, ls = run(tn, plan, net)
        assert complex(got) == 0 and ls == 0.0, prec
        plan.destroy()


def test_zero_leaf_scaled_partition_function(tn):
    """An all-zero vertex tensor under exponent scaling: the zero tensor is not rescaled
    (its exponent is taken as 0), the value is exactly zero and the log scale finite."""
    net = ising_pf.random_3regular_network(20, 4, beta=0.5)
    tensors = list(net.tensors)
    tensors[3] = np.zeros_like(np.asarray(tensors[3]))
    net = Network(tensors, net.modes, net.extent, net.open_modes)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    got, ls = run(tn, plan, net, cplx=False)
    assert float(got) == 0.0 and np.isfinite(ls)


@pytest.mark.parametrize("seed", range(3))
def test_extent_one_labels(tn, seed):
    """Labels of extent 1 (a bond dimension that collapsed): the same as the oracle."""
    net = random_network(300 + seed, n_tensors=7, n_labels=12, n_open=2, complex_=True)
    rng = np.random.default_rng(seed)
    ones = set(int(x) for x in rng.choice(sorted(net.extent), size=4, replace=False))
    ext = {x: (1 if x in ones else e) for x, e in net.extent.items()}
    tensors = [np.asarray(t)[tuple(slice(0, ext[x]) for x in ms)] for t, ms in zip(net.tensors, net.modes)]
    net = Network(tensors, net.modes, ext, net.open_modes)
    path = greedy.greedy_path(net, seed=seed, temperature=0.5)
    plan = tn.Plan(net, path)
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path)) < FP32_BAR


@pytest.mark.parametrize("prec,tol", [("3xtf32", FP32_BAR), ("bf16x3", 5e-5)])
def test_smallest_tensor_core_step(tn, prec, tol):
    """m = 128 rows, n = 16 columns, k = 8: the smallest step the tensor-core kernels take
    (a single partial k-block and an eighth of the column tile)."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((128, 8)) + 1j * rng.standard_normal((128, 8))
    B = rng.standard_normal((16, 8)) + 1j * rng.standard_normal((16, 8))
    net = Network([A, B], [(0, 2), (1, 2)], {0: 128, 1: 16, 2: 8}, (0, 1))
    old = tn.binding.cost_model()
    tn.binding.set_cost_model(old["hbm_bytes_per_s"], old["simt_flops"], [10 * f for f in old["tc_flops"]])
    try:
        plan = tn.Plan(net, Path([(0, 1)]), prec=prec)
        assert plan.step(0)["cls"] == tn.TN_CLASS_TC
        got, _ = run(tn, plan, net)
    finally:
        tn.binding.set_cost_model(old["hbm_bytes_per_s"], old["simt_flops"], old["tc_flops"])
    assert rel_err(got, A @ B.T) < tol


def test_last_slice_and_refused_ranges(tn):
    w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=5)
    _, parts = oracle.contract_slices(w.net, w.path, w.sliced, return_partials=True)
    got, _ = run(tn, plan, w.net, begin=15, count=1)
    assert rel_err(got, parts[15]) < FP32_BAR
    got, _ = run(tn, plan, w.net, begin=11, count=5)  # a ragged last pass of one slice
    assert rel_err(got, sum(parts[11:16])) < FP32_BAR
    ins = [torch.tensor(np.asarray(t), dtype=torch.complex64, device="cuda") for t in w.net.tensors]
    out = torch.zeros((), dtype=torch.complex128, device="cuda")
    for begin, count in ((15, 2), (-1, 1), (0, 0), (16, 1)):
        with pytest.raises(tn.TnError) as e:
            plan.contract_slices(ins, begin, count, out)
        assert e.value.status == tn.TN_ERR_INVALID


@pytest.mark.parametrize("batch", [1, 3, 4])
def test_scaled_ring_sliced_passes(tn, batch):
    """Exponent scaling across passes: the 300-spin Ising ring (Z ~ 1e146, beyond FP32)
    sliced on two edges (4 slices) at 1, 3 (ragged: 3 + 1) and 4 slices per pass. The
    reference exponent of the first slice carries over the passes and the last pass writes
    the value and its log scale: ln Z within 1e-5 relative of the transfer-matrix closed
    form."""
    n = 300
    net = ising_pf.ring_network(n, 1.0, 1.0)
    path = greedy.greedy_path(net, seed=0)
    plan = tn.Plan(net, path, [0, n // 2], prec=tn.TN_R32_FP32_SIMT, exp_scaling=True, max_slice_batch=batch)
    assert plan.info()["n_passes"] == -(-4 // batch)
    got, ls = run(tn, plan, net, cplx=False)
    want_ln = n * np.log(2 * np.cosh(1.0)) + np.log1p(np.tanh(1.0) ** n)
    assert abs(np.log(got) + ls - want_ln) < 1e-5 * abs(want_ln)
    plan.destroy()


@pytest.mark.parametrize("batch", [1, 5, 16])
def test_open_output_sliced_passes(tn, batch):
    """An open 2^5-amplitude output over 16 slices in 16, 4 (ragged: 5+5+5+1) and 1 passes:
    the earlier passes keep the FP64 compensated sums, the last one writes the tensor.
    Element by element against the oracle's sum of slices."""
    w = workloads.random_circuit(3, 4, 8, 5, n_sliced=4, open_qubits=(0, 3, 5, 8, 11))
    plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=batch)
    assert plan.info()["n_passes"] == -(-16 // batch)
    got, _ = run(tn, plan, w.net)
    want = oracle.contract(w.net, w.path, w.sliced)
    assert got.shape == want.shape
    assert np.abs(got - want).max() / np.abs(want).max() < FP32_BAR
    plan.destroy()


@pytest.mark.parametrize("cplx", [False, True])
def test_one_slice_output_exact_fp64(tn, cplx):
    """A one-tensor network (no steps, one slice, one pass): the output is the staged leaf
    widened to FP64, and every FP32 class (normal, subnormal, signed zeros, infinities,
    NaN, the extremes) comes out as the same value, bit for bit."""
    vals = np.array([1.0, -2.5, 3.4028235e38, 1.1754944e-38, 1e-45, -3e-42, 7.0e-40, 0.0, -0.0,
                     np.inf, -np.inf, np.nan, 1 / 3, -1e-30, 65504.0, -2.0 ** -126], dtype=np.float32)
    want = vals.astype(np.float64).reshape(4, 4)
    t = want.copy()
    if cplx:  # set the parts directly: 1j * inf would put a NaN in the real part
        t = np.empty((4, 4), dtype=np.complex128)
        t.real, t.imag = want, want[::-1, ::-1]
    net = Network([t], [(0, 1)], {0: 4, 1: 4}, (1, 0))
    plan = tn.Plan(net, Path([]), prec=0 if cplx else tn.TN_R32_FP32_SIMT)
    got, ls = run(tn, plan, net, cplx=cplx)
    assert ls == 0.0
    if cplx:
        parts = [(got.real, want.T), (got.imag, want[::-1, ::-1].T)]
    else:
        parts = [(got, want.T)]
    for g, w in parts:
        assert np.array_equal(np.ascontiguousarray(g).view(np.uint64), np.ascontiguousarray(w).view(np.uint64))
    plan.destroy()


def test_fma_rate_probes(tn):
    """The FP32 and FP64 FMA probes return positive rates below what the SMs could issue at
    the maximum clock (152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s), and FP64
    well below FP32 on this part (the cross-slice sum's arithmetic)."""
    f32, ms32 = tn.binding.measure_ffma(1 << 16)
    f64, ms64 = tn.binding.measure_dfma(1 << 10)
    assert ms32 > 0 and ms64 > 0
    assert 1e12 < f32 < 81e12
    assert 0 < f64 < f32
