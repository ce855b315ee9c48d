"""Write tests/golden/oracle_values.json: CPU-oracle (complex128) values for the
full-size workloads, used by tests/test_gpu_full_size.py.

Calls only the oracle and the seeded input generators:
  * rc40 (40-qubit 5x8 circuit, 13 cycles, 256 slices): the partial results of 4 slices
    drawn with a fixed seed (one slice takes ~10 s here; all 256 would take ~1 h);
  * kising44 (4x4 kicked Ising, 10 Trotter steps): the full value;
  * rc12 (12-qubit circuit): the full value;
  * khex45, ktri44 (kicked Ising on a honeycomb and a triangular lattice): the full values;
  * kings16 (King's subgraph, max-plus semiring): the maximum independent set size;
  * kising55 (5x5 kicked Ising, 2 steps; the serving mix's large request): the full value;
  * rc40open (rc40 with four qubits left open): the [2,2,2,2] partial tensors of 4 slices
    drawn with a second fixed seed.
Run from the repository root: python tests/golden/make_oracle_values.py
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

RC40_SAMPLE_SEED = 20261202
RC40_SAMPLES = 4
RC40OPEN_SAMPLE_SEED = 20261203


def main():
    out = {}
    t = time.time()
    w = workloads.rc40()
    rng = np.random.default_rng(RC40_SAMPLE_SEED)
    ids = sorted(int(x) for x in rng.choice(w.n_slices, size=RC40_SAMPLES, replace=False))
    _, parts = oracle.contract_slices(w.net, w.path, w.sliced, slice_ids=ids, return_partials=True)
    out["rc40"] = {"slices": ids, "partials": [[float(np.real(p)), float(np.imag(p))] for p in parts]}
    w = workloads.rc40open()
    rng = np.random.default_rng(RC40OPEN_SAMPLE_SEED)
    ids = sorted(int(x) for x in rng.choice(w.n_slices, size=RC40_SAMPLES, replace=False))
    _, parts = oracle.contract_slices(w.net, w.path, w.sliced, slice_ids=ids, return_partials=True)
    out["rc40open"] = {"slices": ids, "shape": list(np.shape(parts[0])),
                       "partials": [[[float(v.real), float(v.imag)] for v in np.ravel(p)] for p in parts]}
    for name in ("kising44", "rc12", "khex45", "ktri44", "kings16", "kising55"):
        wl = workloads.BY_NAME[name]()
        v = complex(oracle.contract(wl.net, wl.path, wl.sliced, semiring=wl.info.get("semiring", "standard")))
        out[name] = {"value": [v.real, v.imag]}
    out["seconds"] = time.time() - t
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, out["seconds"])


if __name__ == "__main__":
    main()
