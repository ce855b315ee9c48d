"""Write tests/golden/rc40_total.json: the CPU-oracle (complex128) value of the full
40-qubit amplitude (5x8 grid, 13 cycles, all 256 slices, Neumaier-summed), for
tests/test_gpu_full_size.py. Calls only the oracle and the seeded input generators.
Takes about 50 minutes on 8 cores. Run from the repository root:
    python tests/golden/make_rc40_total.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from tn_inputs import workloads  # noqa: E402


def main():
    t = time.time()
    w = workloads.rc40()
    total = complex(oracle.contract(w.net, w.path, w.sliced))
    out = {"total": [total.real, total.imag], "slices": w.n_slices, "seconds": time.time() - t}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rc40_total.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, out)


if __name__ == "__main__":
    main()
