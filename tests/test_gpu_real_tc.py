"""GPU parity of the real tensor-core forms (TN_R32_TF32, TN_R32_3XTF32) and of exponent
scaling on tensor-core steps, against the CPU float64 / complex128 oracle.

Real partition functions (Sec. III-C counting family): Ising spin glasses on open
square lattices, Z = sum over spin configurations of exp(beta sum J_ij s_i s_j), whose
greedy paths have tensor-core-sized steps (m up to 2^14 here) and whose Z overflows FP32
(ln Z ~ 150-200), so the tensor-core epilogues must carry the per-intermediate
power-of-two scales (ln Z = ln(value) + log_scale).

Tolerances. 3xTF32 is FP32-accurate: Z's relative error (|ln Z_got - ln Z|) within
max(1e-5, 2 x the plain FP32 form's error on the same network), the bar the complex forms
are held to. TF32 reads every operand with 10 fraction bits
(truncated), so each tensor-core step lowers its result by ~2^-11 relative on average and
a path of a few dozen such steps moves Z by a few percent: the TF32 error is measured and
held only to a loose bound (|ln Z_got - ln Z| < 0.2; a lost power-of-two scale would be
off by ln 2 or more), as the method reports TF32 rather than bounding it.

Scaling is exact: a power-of-two scale commutes with every rounding, so a scaled
contraction's value times 2^(log scale) equals the unscaled contraction's value wherever
the unscaled one does not overflow (checked to 1e-12 relative, i.e. up to the final FP64
conversion), when both runs take the same kernels. (An unscaled CUDA-core step may split
its k across CTAs, a scaled one never does: the two then differ by FP32 rounding, 1e-6.)
"""
import numpy as np
import pytest

import oracle
from tests._lib import ensure_built
from tn_inputs import greedy, ising_pf, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def contract_host(tn, net, path, prec, exp_scaling, cplx=False):
    """One contraction through the host-buffer C-ABI call (which also reads the plan's
    device error word); returns (value, log scale, plan step (class, k split) pairs)."""
    plan = tn.Plan(net, path, prec=prec, exp_scaling=exp_scaling)
    try:
        dt = np.complex64 if cplx else np.float32
        host = [np.ascontiguousarray(np.asarray(t, dtype=dt)) for t in net.tensors]
        shape = tuple(net.extent[x] for x in net.open_modes)
        out = np.zeros(shape, dtype=np.complex128 if cplx else np.float64)
        ls = np.zeros(1)
        plan.contract_host(host, out, ls)
        n_steps = len(path.pairs) if hasattr(path, "pairs") else len(path)
        steps = [(plan.step(s)["cls"], plan.step(s)["ksplit"]) for s in range(n_steps)]
        return out, float(ls[0]), steps
    finally:
        plan.destroy()


def lattice(rows, cols, seed=1, beta=0.44):
    net = ising_pf.lattice_network(rows, cols, beta, seed=seed)
    return net, greedy.greedy_path(net, seed=0, alpha=1.0)


@pytest.mark.parametrize("rows,cols", [(14, 14), (16, 16)])
def test_real_partition_function_on_tensor_cores(tn, rows, cols):
    net, path = lattice(rows, cols)
    want = oracle.contract(net, path)  # float64; Z ~ 1e68 .. 1e89, beyond FP32
    ln_want = float(np.log(want))
    z32, ls32, _ = contract_host(tn, net, path, tn.TN_R32_FP32_SIMT, True)
    err32 = abs(np.log(float(z32)) + ls32 - ln_want)  # |ln Z_got - ln Z| ~ relative error of Z
    bar = max(1e-5, 2 * err32)
    for prec, tol in ((tn.TN_R32_3XTF32, bar), (tn.TN_R32_TF32, 0.2)):
        z, ls, steps = contract_host(tn, net, path, prec, True)
        assert [c for c, _ in steps].count(tn.TN_CLASS_TC) >= 10, "the large steps run on tensor cores"
        err = abs(np.log(float(z)) + ls - ln_want)
        assert err < tol, (prec, err, tol, err32)


def test_real_scaled_equals_unscaled_times_its_scale(tn):
    """A real network whose value stays inside FP32 (the lattice's tensors halved:
    Z' = Z 2^-196): with and without exponent scaling the tensor-core forms give the same
    value up to the reported power of two, and both match the oracle."""
    net, path = lattice(14, 14)
    net.tensors = [0.5 * np.asarray(t) for t in net.tensors]
    want = float(oracle.contract(net, path))
    for prec in (tn.TN_R32_TF32, tn.TN_R32_3XTF32):
        z0, ls0, st0 = contract_host(tn, net, path, prec, False)
        z1, ls1, st1 = contract_host(tn, net, path, prec, True)
        assert ls0 == 0.0 and [c for c, _ in st0].count(tn.TN_CLASS_TC) >= 10
        e2 = ls1 / np.log(2.0)
        assert abs(e2 - round(e2)) < 1e-9, "the log scale is a whole power of two"
        same = 1e-12 if st0 == st1 else 1e-6
        assert abs(np.ldexp(float(z1), int(round(e2))) - float(z0)) <= same * abs(float(z0))
        tol = 1e-5 if prec == tn.TN_R32_3XTF32 else 0.2
        assert abs(float(z0) - want) < tol * abs(want), (prec, float(z0), want)


def test_real_tensor_core_tiles_ragged_and_batched(tn):
    """Real tensor-core steps whose n is not a multiple of the 256-column tile (second B
    tile partly or wholly past n) on a sliced lattice (batched steps, one plane per batch
    entry in the TMA maps): the sum over slices equals the unsliced oracle value."""
    net, path = lattice(12, 20, seed=3, beta=0.3)
    want = float(np.log(oracle.contract(net, path)))
    sliced = greedy.greedy_slicer(net, path, greedy.path_peak(net, path) - 2, max_slices=4)
    assert len(sliced) == 3
    errs = {}
    for prec in (tn.TN_R32_FP32_SIMT, tn.TN_R32_3XTF32):
        plan = tn.Plan(net, path, sliced=sliced, prec=prec, exp_scaling=True)
        try:
            n_tc = sum(plan.step(s)["cls"] == tn.TN_CLASS_TC and plan.step(s)["batched"] != 0
                       for s in range(len(path.pairs)))
            host = [np.ascontiguousarray(np.asarray(t, dtype=np.float32)) for t in net.tensors]
            out = np.zeros((), dtype=np.float64)
            ls = np.zeros(1)
            plan.contract_host(host, out, ls)
        finally:
            plan.destroy()
        errs[prec] = abs(np.log(float(out)) + ls[0] - want)
    assert n_tc >= 3, "batched tensor-core steps"
    assert errs[tn.TN_R32_3XTF32] < max(1e-5, 2 * errs[tn.TN_R32_FP32_SIMT]), errs


def test_complex_tensor_cores_with_exponent_scaling(tn):
    """Complex TF32, 3xTF32 and BF16x3 steps with exponent scaling: the 20-qubit circuit's
    amplitude equals the unscaled run's up to the reported power of two (scaled BF16x3
    steps keep one SM per tile, which gives the paired-SM kernels' bits), and the oracle."""
    w = workloads.random_circuit(4, 5, 12, 40)
    want = complex(oracle.contract(w.net, w.path))
    for prec in (tn.TN_C64_TF32, tn.TN_C64_3XTF32, tn.TN_C64_BF16X3):
        a0, ls0, st0 = contract_host(tn, w.net, w.path, prec, False, cplx=True)
        a1, ls1, st1 = contract_host(tn, w.net, w.path, prec, True, cplx=True)
        assert tn.TN_CLASS_TC in [c for c, _ in st0]
        e2 = int(round(ls1 / np.log(2.0)))
        a1 = complex(a1) * 2.0 ** e2
        same = 1e-12 if st0 == st1 else 1e-6
        assert abs(a1 - complex(a0)) <= same * abs(complex(a0))
        # BF16x3: its one-product bound 3 x 2^-16 (R20); TF32 measured, loosely bounded
        tol = {tn.TN_C64_3XTF32: 1e-5, tn.TN_C64_BF16X3: 3 * 2.0 ** -16}.get(prec, 5e-2)
        assert abs(complex(a0) - want) < tol * abs(want)
