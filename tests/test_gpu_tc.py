"""GPU parity of the tensor-core (tcgen05) GEMM path against the CPU oracle.

Tolerances, derived from the arithmetic of each form:
  * TF32: operands keep 10 explicit mantissa bits (truncated), u_tf32 = 2^-10 ~ 1e-3
    relative per product; FP32 accumulation adds little. A single GEMM step is then
    within ~1e-3 relative (Frobenius), and a path of several TF32 steps within a few
    1e-3: tested at 5e-3 per step and 3e-2 along a path.
  * 3xTF32: hi + lo carry 21 bits; the dropped lo*lo term and lo's own truncation are
    ~2^-20 relative per product, below FP32 accumulation error: held to the FP32 bar,
    1e-5 (relative), the bar the method is held to.
  * BF16x3: hi = RN_bf16(v), lo = RN_bf16(v - hi) leave |v - hi - lo| <= 2^-16 |v|;
    with the dropped lo*lo term (<= 2^-16) each product is within 3 * 2^-16 ~ 4.6e-5
    relative, so a single GEMM step is held to 5e-5 and a path of several such steps
    (errors adding roughly in quadrature, plus cancellation in the amplitude) to 2e-4.
  * BF16x3 with the 3M product: the imaginary part is P3 - P1 - P2, where P3's operands
    (the sums re + im) are up to twice as large: twice the BF16x3 bounds, 1e-4 per step
    and 4e-4 along a path.
"""
import numpy as np
import pytest
import torch

import oracle
from tests._lib import ensure_built
from tests.test_gpu_parity import rel_err, run
from tn_inputs import workloads
from tn_inputs.network import Network, Path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


@pytest.fixture(autouse=True)
def tensor_core_rates(tn):
    """These tests exercise the tensor-core kernels on narrow and ragged tiles (down to a
    quarter of the 128-column tile), which the Eq. 6 choice at the peak rates can hand to
    the CUDA cores instead: the tensor-core rates are raised for the duration of a test."""
    old = tn.binding.cost_model()
    tn.binding.set_cost_model(old["hbm_bytes_per_s"], old["simt_flops"], [10 * f for f in old["tc_flops"]])
    yield
    tn.binding.set_cost_model(old["hbm_bytes_per_s"], old["simt_flops"], old["tc_flops"])


def gemm_network(dims_m, dims_n, dims_k, out_order, seed=0, sliced_dim=None, vec_slice=None):
    """A[m..., k...] x B[n..., k...] with the open result in `out_order` (labels)."""
    rng = np.random.default_rng(seed)
    ext = {}
    lab = 0
    M, N, K = [], [], []
    for grp, dims in ((M, dims_m), (N, dims_n), (K, dims_k)):
        for d in dims:
            ext[lab] = d
            grp.append(lab)
            lab += 1
    tensors, modes = [], []
    am = tuple(M + K)
    bm = tuple(N + K)
    if sliced_dim is not None:      # a closed label on both operands, sliced
        ext[lab] = sliced_dim
        am = (lab,) + am
        bm = (lab,) + bm
        lab += 1
    if vec_slice is not None:       # a label joining A to a vector only (A batched, B not)
        ext[lab] = vec_slice
        am = am + (lab,)
        v = rng.standard_normal(vec_slice) + 1j * rng.standard_normal(vec_slice)
        vlab = lab
        lab += 1
    shp = lambda ms: tuple(ext[x] for x in ms)
    A = rng.standard_normal(shp(am)) + 1j * rng.standard_normal(shp(am))
    B = rng.standard_normal(shp(bm)) + 1j * rng.standard_normal(shp(bm))
    tensors = [A, B]
    modes = [am, bm]
    open_ = tuple(M[i] if kind == "m" else N[i] for kind, i in out_order)
    if vec_slice is not None:
        tensors.append(v)
        modes.append((vlab,))
        path = Path([(0, 2), (3, 1)])
    else:
        path = Path([(0, 1)])
    net = Network(tensors, modes, ext, open_)
    net.check()
    sliced = [lab - 1] if (sliced_dim is not None or vec_slice is not None) else []
    return net, path, sliced


CASES = [
    # (m dims, n dims, k dims, output interleaving)
    ((2, 64), (2, 64), (64,), [("m", 0), ("m", 1), ("n", 0), ("n", 1)]),         # full tiles
    ((5, 40), (3, 50), (72,), [("m", 0), ("n", 0), ("m", 1), ("n", 1)]),         # ragged m, n, k tails
    ((128,), (2, 2, 32), (8, 4), [("n", 0), ("m", 0), ("n", 1), ("n", 2)]),      # interleaved columns
    ((256,), (96,), (16,), [("n", 0), ("m", 0)]),                                 # rows land strided
    ((2, 128), (128,), (8,), [("m", 0), ("n", 0), ("m", 1)]),                     # k = 8: half a k-block
    ((4, 512), (32,), (2, 32), [("m", 0), ("n", 0), ("m", 1)]),                   # n = 32: a quarter tile
]


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("3xtf32", 1e-5), ("bf16x3", 5e-5), ("bf16x3m", 1e-4)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_single_gemm_step(tn, prec, tol, case):
    dm, dn, dk, order = CASES[case]
    net, path, sliced = gemm_network(dm, dn, dk, order, seed=case)
    plan = tn.Plan(net, path, prec=prec)
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path)) < tol


PAIR_CASES = [
    # (m dims, n dims, k dims, output order, sliced extent): m >= 256 and k > 256
    ((2, 256), (128,), (512,), [("m", 0), ("m", 1), ("n", 0)], None),            # two fold chunks
    ((384,), (136,), (776,), [("m", 0), ("n", 0)], None),                        # 1.5 pair tiles, n and k tails
    ((3, 100), (2, 64), (24, 16), [("m", 0), ("n", 0), ("m", 1), ("n", 1)], None),  # m = 300, interleaved
    ((512,), (256,), (264,), [("m", 0), ("n", 0)], 3),                           # batched, k just above 256
    ((4096,), (2048,), (512,), [("m", 0), ("n", 0)], None),                      # 256 tiles: several per cluster
    ((1000,), (1000,), (320,), [("n", 0), ("m", 0)], 4),                         # ragged, 4 entries, 128 tiles
    ((2, 256), (136,), (4104,), [("m", 0), ("m", 1), ("n", 0)], None),          # k > 2048: a cluster per tile
]


@pytest.mark.parametrize("case", range(len(PAIR_CASES)))
def test_paired_sm_tiles_same_bits(tn, case):
    """BF16x3 4M steps with m >= 256 and k > 256 run 256 x 128 output tiles on pairs of SMs
    (tcgen05 cta_group::2; up to k = 2048 persistent clusters, each walking several tiles in
    the larger cases, beyond it one cluster per tile). Every output has the same bits as from the single-SM kernel
    (TN_PLAN_SINGLE_SM_TILES: the same products accumulated in the same order), and matches
    the oracle within the BF16x3 bound."""
    dm, dn, dk, order, sl = PAIR_CASES[case]
    net, path, sliced = gemm_network(dm, dn, dk, order, seed=30 + case, sliced_dim=sl)
    pair = tn.Plan(net, path, sliced, prec="bf16x3")
    one = tn.Plan(net, path, sliced, prec="bf16x3", single_sm_tiles=True)
    st = pair.step(0)
    assert st["cls"] == tn.TN_CLASS_TC and st["m"] >= 256 and st["k"] > 256
    got, _ = run(tn, pair, net)
    ref, _ = run(tn, one, net)
    g, r = np.ascontiguousarray(got), np.ascontiguousarray(ref)
    assert np.array_equal(g.view(np.uint64), r.view(np.uint64))
    want = oracle.contract(net, path, sliced) if sliced else oracle.contract(net, path)
    assert rel_err(got, want) < 5e-5
    pair.destroy()
    one.destroy()


def test_paired_sm_tiles_row_operand_batched(tn):
    """Paired-SM tiles when only the row operand depends on the slice (the column operand
    shared by every batch entry), 3 slices per pass: the same bits as on one SM."""
    net, path, sliced = gemm_network((512,), (384,), (512,), [("m", 0), ("n", 0)], seed=41, vec_slice=4)
    pair = tn.Plan(net, path, sliced, prec="bf16x3", max_slice_batch=3)
    one = tn.Plan(net, path, sliced, prec="bf16x3", max_slice_batch=3, single_sm_tiles=True)
    st = pair.step(1)
    assert st["cls"] == tn.TN_CLASS_TC and st["batched"] == 1 and st["m"] >= 256 and st["k"] > 256
    got, _ = run(tn, pair, net)
    ref, _ = run(tn, one, net)
    g, r = np.ascontiguousarray(got), np.ascontiguousarray(ref)
    assert np.array_equal(g.view(np.uint64), r.view(np.uint64))
    assert rel_err(got, oracle.contract(net, path, sliced)) < 5e-5
    pair.destroy()
    one.destroy()


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("3xtf32", 1e-5), ("bf16x3", 5e-5), ("bf16x3m", 1e-4)])
def test_batched_both_operands(tn, prec, tol):
    """A sliced label on both operands: the batch runs as TMA planes of both maps."""
    net, path, sliced = gemm_network((2, 64), (160,), (32,), [("m", 1), ("n", 0), ("m", 0)], seed=7,
                                     sliced_dim=3)
    plan = tn.Plan(net, path, sliced, prec=prec)
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC and plan.step(0)["batched"] == 1
    got, _ = run(tn, plan, net)
    want, parts = oracle.contract_slices(net, path, sliced, return_partials=True)
    assert rel_err(got, want) < tol
    g1, _ = run(tn, plan, net, begin=1, count=1)
    assert rel_err(g1, parts[1]) < tol


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("3xtf32", 1e-5), ("bf16x3", 5e-5), ("bf16x3m", 1e-4)])
def test_batched_row_operand_only(tn, prec, tol):
    """Only the row operand depends on the slice (the column operand is shared)."""
    net, path, sliced = gemm_network((192,), (128,), (64,), [("m", 0), ("n", 0)], seed=8, vec_slice=4)
    plan = tn.Plan(net, path, sliced, prec=prec, max_slice_batch=3)
    st = plan.step(1)
    assert st["cls"] == tn.TN_CLASS_TC and st["batched"] == 1
    got, _ = run(tn, plan, net)
    assert rel_err(got, oracle.contract(net, path, sliced)) < tol


@pytest.mark.parametrize("prec,tol", [("tf32", 3e-2), ("3xtf32", 1e-5), ("bf16x3", 2e-4), ("bf16x3m", 4e-4)])
def test_circuit_path_with_tc_steps(tn, prec, tol):
    w = workloads.random_circuit(4, 5, 12, 40)
    plan = tn.Plan(w.net, w.path, prec=prec)
    n_tc = sum(1 for s in range(len(w.path.pairs)) if plan.step(s)["cls"] == tn.TN_CLASS_TC)
    assert n_tc >= 1
    got, _ = run(tn, plan, w.net)
    assert rel_err(got, oracle.contract(w.net, w.path)) < tol


def test_tf32_operand_rounding(tn):
    """How tcgen05 kind::tf32 reads an FP32 operand: with A = 1 + 3*2^-12 and B = 1,
    truncation to 10 mantissa bits gives 1, round-to-nearest 1 + 2^-10. The 3xTF32
    kernel writes hi = RN_tf32(value) itself (read exactly) and lo = value - hi, which
    the hardware truncates without a bias; the 3xTF32 product is exact here."""
    from tn_inputs.network import Network, Path
    ext = {0: 128, 1: 64, 2: 16}
    A = np.full((128, 16), 1.0 + 3.0 * 2.0**-12, dtype=np.complex128)
    B = np.ones((64, 16), dtype=np.complex128)
    net = Network([A, B], [(0, 2), (1, 2)], ext, (0, 1))
    plan = tn.Plan(net, Path([(0, 1)]), prec="tf32")
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC
    got, _ = run(tn, plan, net)
    vals = np.unique(got.real)
    assert vals.size == 1 and vals[0] == 16.0, vals  # truncation
    exact = tn.Plan(net, Path([(0, 1)]), prec="3xtf32")
    g3, _ = run(tn, exact, net)
    assert np.allclose(g3.real, 16.0 * (1.0 + 3.0 * 2.0**-12), rtol=0, atol=1e-6)


@pytest.mark.parametrize("k", [4096, 32768])
def test_3xtf32_long_k_accumulation(tn, k):
    """The tensor core truncates each FP32 accumulation, which over a long k drifts a
    positive sum toward zero by ~k * 2^-25 relative. The 3xTF32 kernel accumulates
    64-term chunks in tensor memory and adds the chunks with round-to-nearest FP32, so
    the error must not grow with k: on positive data (no cancellation) the mean relative
    error of the imaginary part stays below 5e-6 and every element below 1e-5."""
    from tn_inputs.network import Network, Path
    rng = np.random.default_rng(k)
    m = n = 128
    A = (rng.random((m, k)) + 1j * rng.random((m, k))).astype(np.complex64).astype(np.complex128)
    B = (rng.random((n, k)) + 1j * rng.random((n, k))).astype(np.complex64).astype(np.complex128)
    net = Network([A, B], [(0, 2), (1, 2)], {0: m, 1: n, 2: k}, (0, 1))
    plan = tn.Plan(net, Path([(0, 1)]), prec="3xtf32")
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC
    got, _ = run(tn, plan, net)
    want = A @ B.T
    rel = (got.imag - want.imag) / want.imag
    assert abs(rel.mean()) < 5e-6 and np.abs(rel).max() < 1e-5, (rel.mean(), np.abs(rel).max())


@pytest.mark.parametrize("prec,tol", [("tf32", 3e-2), ("3xtf32", 1e-5), ("bf16x3", 2e-4), ("bf16x3m", 4e-4)])
def test_sliced_circuit_with_tc_steps(tn, prec, tol):
    w = workloads.random_circuit(4, 5, 12, 40, n_sliced=3)
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=4)
    got, _ = run(tn, plan, w.net)
    assert rel_err(got, oracle.contract(w.net, w.path, w.sliced)) < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("3xtf32", 1e-5), ("tf32", 3e-2), ("bf16x3", 2e-4),
                                      ("bf16x3m", 4e-4)])
def test_sliced_circuit_open_qubits(tn, prec, tol):
    """Several amplitudes from one contraction: four qubits of a 20-qubit circuit left
    open (a [2,2,2,2] output), three labels sliced, TC steps on the path."""
    w = workloads.random_circuit(4, 5, 12, 40, n_sliced=3, open_qubits=(13, 14, 18, 19))
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=4)
    assert plan.out_shape == (2, 2, 2, 2)
    got, _ = run(tn, plan, w.net)
    assert rel_err(got, oracle.contract(w.net, w.path, w.sliced)) < tol


@pytest.mark.parametrize("prec,bound", [("bf16x3", 5e-5), ("bf16x3m", 1e-4), ("3xtf32", 1e-5)])
def test_stream_step_feeding_tensor_core_step(tn, prec, bound):
    """A 2^22-element state absorbs a two-qubit gate (a streaming big x small step) and the
    result is contracted with a 2^21-element tensor over 14 labels (a tensor-core step,
    256 x 128 outputs, k = 2^14). The streaming kernel writes its output in the form the
    tensor-core step reads (split BF16 planes for BF16x3, the six planes of the 3M form);
    the open result against the oracle in the Frobenius norm and element by element."""
    rng = np.random.default_rng(7)
    psi = rng.standard_normal((2,) * 22) + 1j * rng.standard_normal((2,) * 22)
    g = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))).reshape(2, 2, 2, 2)
    x = rng.standard_normal((2,) * 21) + 1j * rng.standard_normal((2,) * 21)
    # psi(0..21); gate(22, 23, 0, 1) -> new labels 22, 23 for qubits 0, 1; x(22, 23, 2..13, 24..30)
    modes = [tuple(range(22)), (22, 23, 0, 1), (22, 23) + tuple(range(2, 14)) + tuple(range(24, 31))]
    out = tuple(range(14, 22)) + tuple(range(24, 31))
    net = Network([psi, g, x], modes, {q: 2 for q in range(31)}, out)
    net.check()
    path = Path([(0, 1), (2, 3)])
    plan = tn.Plan(net, path, prec=prec, complex_mult=3 if prec == "bf16x3m" else 4)
    assert plan.step(0)["cls"] == tn.TN_CLASS_STREAM and plan.step(1)["cls"] == tn.TN_CLASS_TC
    got, _ = run(tn, plan, net)
    want = oracle.contract(net, path)
    assert rel_err(got, want) < bound
    assert np.abs(got - want).max() / np.abs(want).max() < 4 * bound
    plan.destroy()


@pytest.mark.parametrize("seed", range(10))
def test_paired_sm_tiles_random_shapes(tn, seed):
    """Seeded random shapes through the paired-SM kernels (rows 256-1500, columns 16-700,
    depth 264-5000 in steps of 8, with and without a sliced label on both operands): the
    same bits as the single-SM kernel every time."""
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(256, 1501))
    n = int(rng.integers(16, 701))
    k = 8 * int(rng.integers(33, 626))
    sl = int(rng.integers(2, 4)) if seed % 2 else None
    net, path, sliced = gemm_network((m,), (n,), (k,), [("m", 0), ("n", 0)], seed=seed, sliced_dim=sl)
    pair = tn.Plan(net, path, sliced, prec="bf16x3", max_slice_batch=2 if sl else 0)
    one = tn.Plan(net, path, sliced, prec="bf16x3", max_slice_batch=2 if sl else 0, single_sm_tiles=True)
    st = pair.step(0)
    assert st["cls"] == tn.TN_CLASS_TC and st["m"] >= 256
    got, _ = run(tn, pair, net)
    ref, _ = run(tn, one, net)
    g, r = np.ascontiguousarray(got), np.ascontiguousarray(ref)
    assert np.array_equal(g.view(np.uint64), r.view(np.uint64)), (m, n, k, sl)
    if seed < 3:
        assert rel_err(got, oracle.contract(net, path, sliced)) < 5e-5
    pair.destroy()
    one.destroy()


def test_autotune_keeps_the_bits(tn):
    """tn_plan_autotune times paired SMs against one SM per tile for each paired-SM step and
    keeps the faster; the result of the plan is the same bits before and after, and the launch
    count follows the choice."""
    net, path, sliced = gemm_network((4096,), (2048,), (4104,), [("m", 0), ("n", 0)], seed=51, sliced_dim=2)
    plan = tn.Plan(net, path, sliced, prec="bf16x3")
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC and plan.step(0)["single_sm"] == 0
    before, _ = run(tn, plan, net)
    ins = [torch.tensor(np.asarray(t), dtype=torch.complex64, device="cuda") for t in net.tensors]
    scratch = torch.zeros(plan.out_shape, dtype=torch.complex128, device="cuda")
    plan.autotune(ins, scratch)
    assert plan.step(0)["single_sm"] in (0, 1)
    after, _ = run(tn, plan, net)
    assert np.array_equal(np.ascontiguousarray(before).view(np.uint64), np.ascontiguousarray(after).view(np.uint64))
    assert plan.launches_per_call() >= 4
    plan.destroy()
