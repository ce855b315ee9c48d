"""Shared helpers for the tests: build the library on demand and marshal inputs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def ensure_built():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_tn_build", os.path.join(ROOT, "paper_2606_01852_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2606_01852_gb300 as tn
    return tn


# Tolerances of the forms against the complex128 oracle (the reading of the 1e-5 bar for
# complex64-equivalent paths):
#  * FP32-accurate forms (plain FP32 on the CUDA cores, 3xTF32): relative error <= 1e-5, or
#    <= 2x the plain FP32 form's own error on the same workload where that is larger (a
#    result the plain FP32 form itself cannot reach to 1e-5);
#  * BF16x3 (measured and reported, not held to 1e-5): hi + lo BF16 halves represent each
#    operand to 2^-16 relative and the dropped lo.lo term is below 2^-16, so each product
#    is within 3 * 2^-16 = 4.6e-5 relative; the roundings are unbiased (round to nearest),
#    so results are held to that one-product bound;
#  * TF32 (measured and reported): operands truncated to 10 mantissa bits, a bias of up to
#    2^-10 per product that adds up along a path; bounds per test.
#  * BF16x3 with the 3M product: Im = P3 - P1 - P2 with P3 = (a_re + a_im)(b_re + b_im), whose
#    terms are up to twice |a||b|: each of the three products within 3 * 2^-16 of its own
#    magnitude, 4 |a||b| in all, so 12 * 2^-16 = 1.8e-4 relative to |a||b|.
FP32_BAR = 1e-5
BF16X3_BOUND = 3 * 2.0 ** -16
BF16X3M_BOUND = 12 * 2.0 ** -16


def fp32_accurate_bound(fp32_err):
    return max(FP32_BAR, 2.0 * fp32_err)
