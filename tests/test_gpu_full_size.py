"""Parity at the benchmark's full sizes and launch configuration, against oracle values
stored by tests/golden/make_oracle_values.py, make_rc40_total.py and
make_rc40c14_values.py (CPU complex128 oracle; sampled slices of the sliced circuits,
which the oracle can compute one by one).

Bounds (tests/_lib.py): the FP32-accurate forms (FP32, 3xTF32) within max(1e-5, 2x the
plain FP32 error on the same workload, measured in the same run); BF16x3 within its
one-product bound 3 * 2^-16; TF32 within per-test bounds (biased truncation). A slice
partial of a random-circuit amplitude is itself a sum with heavy cancellation (partials
of different slices differ by orders of magnitude and have random phases), so its error
is measured relative to the typical partial size (the RMS of the sampled partials).
Tensor outputs are checked both in the Frobenius norm and element by element (the
largest elementwise error over the samples relative to their largest element).
"""
import functools
import json
import os

import numpy as np
import pytest
import torch

from tests._lib import BF16X3_BOUND, BF16X3M_BOUND, FP32_BAR, ROOT, ensure_built, fp32_accurate_bound

FAST_BOUND = {"bf16x3": BF16X3_BOUND, "bf16x3m": BF16X3M_BOUND}
from tn_inputs import workloads

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_values.json")))
C14 = os.path.join(ROOT, "tests", "golden", "rc40c14_values.json")


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def dev(net):
    return [torch.tensor(np.asarray(t), dtype=torch.complex64, device="cuda") for t in net.tensors]


def slice_partials(tn, w, prec, ids, batch):
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=batch)
    try:
        assert plan.info()["slice_batch"] == batch
        ins = dev(w.net)
        out = torch.zeros(plan.out_shape, dtype=torch.complex128, device="cuda")
        got = []
        for sid in ids:
            plan.contract_slices(ins, sid, 1, out)
            torch.cuda.synchronize()
            got.append(out.cpu().numpy().copy())
    finally:
        plan.destroy()
    return np.array(got)


def full_value(tn, w, prec, expect_tc=True):
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec)
    if prec != "fp32" and expect_tc:
        assert plan.info()["steps_per_class"][tn.TN_CLASS_TC] > 0
    out = torch.zeros((), dtype=torch.complex128, device="cuda")
    plan.contract(dev(w.net), out)
    torch.cuda.synchronize()
    plan.destroy()
    return complex(out.cpu())


# ---- the 14-cycle circuit (the benchmark's workload) ---------------------------------

@functools.lru_cache(maxsize=None)
def _c14_pieces_err(prec):
    """Error of the four pieces of the stored slice (the finer 512-slice plan, 4 slices per
    pass) relative to the RMS piece, elementwise maximum over the pieces."""
    tn = ensure_built()
    gold = json.load(open(C14))
    w = workloads.rc40c14sub()
    assert list(w.sliced) == gold["subsliced"]
    want = np.array([complex(*p) for p in gold["pieces"]])
    got = slice_partials(tn, w, prec, gold["piece_ids"], 4)
    typical = np.sqrt(np.mean(np.abs(want) ** 2))
    return float(np.max(np.abs(got - want)) / typical)


def test_rc40c14_pieces_fp32(tn):
    assert _c14_pieces_err("fp32") < FP32_BAR


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3", "bf16x3m"])
def test_rc40c14_pieces_fast_forms(tn, prec):
    err, fp32 = _c14_pieces_err(prec), _c14_pieces_err("fp32")
    bound = fp32_accurate_bound(fp32) if prec == "3xtf32" else FAST_BOUND[prec]
    assert err < bound, (prec, err, fp32)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x3m", "3xtf32"])
def test_rc40c14_slice_bench_config(tn, prec):
    """The benchmark's plan (7 sliced labels, 8 slices per pass): the stored slice against
    the oracle's sum of its four pieces (Sec. II-C: slicing partitions the sum exactly), and
    an 8-slice range equal to the sum of its slices contracted one by one."""
    gold = json.load(open(C14))
    w = workloads.rc40c14()
    assert list(w.sliced) == gold["sliced"] and w.n_slices == 128
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=8)
    assert plan.info()["peak_elems"] == 2 ** 30
    ins = dev(w.net)
    out = torch.zeros((), dtype=torch.complex128, device="cuda")
    sid = gold["slice"]
    plan.contract_slices(ins, sid, 1, out)
    torch.cuda.synchronize()
    want = complex(*gold["slice_partial"])
    typical = np.sqrt(np.mean(np.abs([complex(*p) for p in gold["pieces"]]) ** 2))
    bound = FAST_BOUND[prec] if prec in FAST_BOUND else fp32_accurate_bound(_c14_pieces_err("fp32"))
    assert abs(complex(out.cpu()) - want) / typical < bound
    b0 = (sid // 8) * 8
    plan.contract_slices(ins, b0, 8, out)
    torch.cuda.synchronize()
    batch_sum = complex(out.cpu())
    singles = []
    for s in range(b0, b0 + 8):
        plan.contract_slices(ins, s, 1, out)
        torch.cuda.synchronize()
        singles.append(complex(out.cpu()))
    scale = np.sqrt(np.mean(np.abs(singles) ** 2))
    # the same kernels on the same data: only the FP64 cross-slice order differs
    assert abs(batch_sum - sum(singles)) / scale < 1e-9
    plan.destroy()


# ---- the 13-cycle circuit --------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def _rc40_slices_err(prec, name):
    tn = ensure_built()
    gold = GOLD[name]
    w = workloads.BY_NAME[name]()
    got = slice_partials(tn, w, prec, gold["slices"], 128)
    if name == "rc40":
        want = np.array([complex(*p) for p in gold["partials"]])
        typical = np.sqrt(np.mean(np.abs(want) ** 2))
        err = np.abs(got - want) / typical
        return float(err.max()), float(err.max())
    want = np.array([[complex(*v) for v in p] for p in gold["partials"]])
    got = got.reshape(want.shape)
    typical = np.sqrt(np.mean(np.sum(np.abs(want) ** 2, axis=1)))
    frob = np.linalg.norm(got - want, axis=1) / typical
    elem = np.abs(got - want).max() / np.abs(want).max()
    return float(frob.max()), float(elem.max())


@pytest.mark.parametrize("name", ["rc40", "rc40open"])
@pytest.mark.parametrize("prec", ["fp32", "3xtf32", "bf16x3", "bf16x3m"])
def test_rc40_sampled_slices_bench_config(tn, name, prec):
    """Four sampled slices at the benchmark launch configuration (128 slices per pass);
    rc40open's slices are [2,2,2,2] tensors of partial amplitudes: Frobenius and
    elementwise errors both held to the bound."""
    frob, elem = _rc40_slices_err(prec, name)
    if prec == "fp32":
        bound = FP32_BAR
    elif prec == "3xtf32":
        bound = fp32_accurate_bound(max(_rc40_slices_err("fp32", name)))
    else:
        bound = FAST_BOUND[prec]
    assert frob < bound and elem < bound, (name, prec, frob, elem)


# ---- dynamics expectation values -------------------------------------------------------

@functools.lru_cache(maxsize=None)
def _dyn_err(name, prec):
    w = workloads.BY_NAME[name]()
    want = complex(*GOLD[name]["value"])
    return abs(full_value(ensure_built(), w, prec) - want) / abs(want)


# Plain FP32 misses 1e-5 on the 4x4 kicked Ising (830 steps; measured 1.3e-5): held to 2e-5
# there and the fast forms to twice the FP32 error (the reading of the bar).
FP32_DYN = {"kising44": 2e-5}
# Measured misses of that bar, reported rather than claimed (none at present: 3xTF32 on the
# triangular lattice missed it with 64-term tensor-memory accumulation chunks, 2.0e-5 against
# a plain FP32 error of 9.0e-6, and meets it with 32-term chunks, 1.5e-5).
KNOWN_MISSES = {}


@pytest.mark.parametrize("name", ["kising44", "khex45", "ktri44", "kising55"])
def test_dynamics_fp32(tn, name):
    assert _dyn_err(name, "fp32") < FP32_DYN.get(name, FP32_BAR)


@pytest.mark.parametrize("name", ["kising44", "khex45", "ktri44", "kising55"])
@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3", "bf16x3m", "tf32"])
def test_dynamics_fast_forms(tn, name, prec):
    """Kicked Ising on the square (4x4, and the serving mix's 5x5), honeycomb and
    triangular lattices. TF32 (biased truncation over hundreds of steps) is held to 1e-1."""
    err = _dyn_err(name, prec)
    bound = {"3xtf32": fp32_accurate_bound(_dyn_err(name, "fp32")), "tf32": 1e-1, **FAST_BOUND}[prec]
    bound = KNOWN_MISSES.get((name, prec), bound)
    assert err < bound, (name, prec, err, _dyn_err(name, "fp32"))


def _rc40_total():
    return complex(*json.load(open(os.path.join(ROOT, "tests", "golden", "rc40_total.json")))["total"])


@pytest.mark.parametrize("prec,batch,bound", [("bf16x3", 128, FP32_BAR), ("3xtf32", 128, FP32_BAR),
                                               ("bf16x3m", 64, BF16X3M_BOUND)])
def test_rc40_full_sum_bench_config(tn, prec, batch, bound):
    """All 256 slices at 128 slices per launch (two passes; the 3M form's 12-byte operands
    at 64 per launch), FP64 Neumaier sum across slices, against the oracle's full sum:
    within 1e-5 for BF16x3 and 3xTF32 (measured 3.3e-6 and 3.6e-6), the 3M form within its
    one-product bound."""
    w = workloads.rc40()
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=batch)
    try:
        assert plan.info()["n_passes"] == 256 // batch
        out = torch.zeros((), dtype=torch.complex128, device="cuda")
        plan.contract(dev(w.net), out)
        torch.cuda.synchronize()
        want = _rc40_total()
        assert abs(complex(out.cpu()) - want) / abs(want) < bound, (complex(out.cpu()), want)
    finally:
        plan.destroy()


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
def test_rc40_unsliced_equals_sliced_sum(tn, prec):
    """The same amplitude with no slicing (intermediates up to 2^32 elements, one
    contraction): equal to the oracle's sum over the 256 slices (Sec. II-C: slicing is an
    exact partition of the sum), within 1e-5 (measured 2.7e-6 for BF16x3)."""
    w = workloads.rc40u()
    plan = tn.Plan(w.net, w.path, prec=prec)
    assert plan.info()["peak_elems"] == 2**32
    out = torch.zeros((), dtype=torch.complex128, device="cuda")
    plan.contract(dev(w.net), out)
    torch.cuda.synchronize()
    want = _rc40_total()
    assert abs(complex(out.cpu()) - want) / abs(want) < FP32_BAR, (complex(out.cpu()), want)
    plan.destroy()


def test_rc12_full(tn):
    w = workloads.rc12()
    want = complex(*GOLD["rc12"]["value"])
    assert abs(full_value(tn, w, "3xtf32", expect_tc=False) - want) / abs(want) < FP32_BAR
