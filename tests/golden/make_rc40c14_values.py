"""Write tests/golden/rc40c14_values.json: CPU-oracle (complex128) partial results for the
14-cycle 40-qubit circuit (tests/test_gpu_full_size.py).

Calls only the oracle and the seeded input generators. One slice of the benchmark's
slicing (rc40c14: 7 sliced labels, largest intermediate 2^30) is drawn with a fixed
seed; the oracle contracts it as its four pieces of the finer slicing (rc40c14sub: the
same path with two more sliced labels, largest intermediate 2^29, ~3.4e13 flops each),
which keeps the host's memory within bounds. Stores the four piece partials and their
Neumaier sum (= the slice's partial, Sec. II-C: slicing partitions the sum exactly).
Takes roughly 10-20 minutes on 8 cores. Run from the repository root:
    python tests/golden/make_rc40c14_values.py
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

SAMPLE_SEED = 20261203


def main():
    t = time.time()
    w = workloads.rc40c14()
    sub = workloads.rc40c14sub()
    pieces = sub.n_slices // w.n_slices
    s = int(np.random.default_rng(SAMPLE_SEED).integers(0, w.n_slices))
    ids = [s * pieces + j for j in range(pieces)]
    total, parts = oracle.contract_slices(sub.net, sub.path, sub.sliced, slice_ids=ids, return_partials=True)
    total = complex(total)
    out = {"slice": s, "sliced": list(w.sliced), "subsliced": list(sub.sliced), "piece_ids": ids,
           "pieces": [[float(np.real(p)), float(np.imag(p))] for p in parts],
           "slice_partial": [total.real, total.imag], "seconds": time.time() - t}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rc40c14_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, out)


if __name__ == "__main__":
    main()
