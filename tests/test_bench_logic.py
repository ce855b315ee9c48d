"""Host-side logic of bench.py that the GPU run relies on, checked on CPU with host-only
plans: the path roofline (Sec. IV-C Eq. 6 summed over a contraction's steps)."""
import os
import sys

import numpy as np
import pytest

from tests._lib import ROOT, ensure_built
from tn_inputs import workloads
from tn_inputs.network import Network, Path

sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6684.8, "bf16_tflops_sustained": 1730.2, "sm_max_mhz": 2070.0, "_source": "measured"}


def test_path_roofline_single_gemm_by_hand():
    """One complex 128 x 128 x 128 GEMM: 8 * 128^3 flops, 8 * 3 * 128^2 bytes. FP32 form:
    bound by the ALU (152 * 128 * 2 * 2.07 GHz); BF16x3: by HBM (the form's peak is a third
    of the sustained bf16 rate, far above what these bytes allow)."""
    tn = ensure_built()
    ext = {0: 128, 1: 128, 2: 128}
    net = Network([np.zeros((128, 128), np.complex128), np.zeros((128, 128), np.complex128)],
                  [(0, 2), (1, 2)], ext, (0, 1))
    flops, nbytes = 8.0 * 128 ** 3, 8.0 * 3 * 128 ** 2
    alu = 152 * 128 * 2 * 2.07e9
    plan = tn.Plan(net, Path([(0, 1)]), prec="fp32", host_only=True)
    r = bench.path_roofline(plan, 0, "standard", PEAKS, 1.0)
    assert r["sum_t_roof_ms"] == pytest.approx(max(flops / alu, nbytes / 6684.8e9) * 1e3, rel=1e-12)
    plan = tn.Plan(net, Path([(0, 1)]), prec="bf16x3", host_only=True)
    assert plan.step(0)["cls"] == tn.TN_CLASS_TC
    r = bench.path_roofline(plan, 3, "standard", PEAKS, 2.0)
    want = max(flops / (1730.2e12 / 3), nbytes / 6684.8e9) * 1e3
    assert r["sum_t_roof_ms"] == pytest.approx(want, rel=1e-12) and r["frac"] == pytest.approx(want / 2.0)


def test_path_roofline_sliced_plan():
    """The 40-qubit plan: every step counted over its 256 slices (or once if slice-invariant);
    its roofline time is below the measured contraction time of ~1.3 s."""
    tn = ensure_built()
    w = workloads.rc40()
    plan = tn.Plan(w.net, w.path, w.sliced, prec="bf16x3", max_slice_batch=128, host_only=True)
    r = bench.path_roofline(plan, 3, "standard", PEAKS, 1317.0)
    assert 900.0 < r["sum_t_roof_ms"] < 1317.0
    assert r["frac"] == pytest.approx(r["sum_t_roof_ms"] / 1317.0)


def test_path_roofline_slice_batch_and_flops_per_call():
    """A step of the 14-cycle benchmark contracts 16 of its 128 slices: the flops of one
    call count the sliced steps 16 times and the slice-invariant ones once, and the path
    roofline of such a step is that of the 16 slices."""
    tn = ensure_built()
    w = workloads.rc40c14()
    plan = tn.Plan(w.net, w.path, w.sliced, prec="bf16x3", max_slice_batch=16, host_only=True)
    info = plan.info()
    fixed = batched = 0.0
    for s in range(info["n_steps"]):
        st = plan.step(s)
        f = 8.0 * st["m"] * st["n"] * st["k"]
        if st["batched"]:
            batched += f
        else:
            fixed += f
    assert plan.flops_per_call() == pytest.approx(info["flops"], rel=1e-12)
    assert plan.flops_per_call(16) == pytest.approx(fixed + 16 * batched, rel=1e-12)
    full = bench.path_roofline(plan, 3, "standard", PEAKS, 1000.0)["sum_t_roof_ms"]
    part = bench.path_roofline(plan, 3, "standard", PEAKS, 1000.0, count=16)["sum_t_roof_ms"]
    assert part == pytest.approx(full * 16 / 128, rel=0.02)
    # tensor-bound: the 16 slices' flops at the form's peak, plus a little for HBM-bound steps
    assert part >= plan.flops_per_call(16) * info["flops_per_class"][tn.TN_CLASS_TC] / info["flops"] / (
        1730.2e12 / 3) * 1e3 * 0.999
