"""Writes tests/golden/raider_like_k10.json from the FP64 oracle only.

Workload: the raider-like planted case (4 subjects x 2000 voxels, 300 TRs,
k = 10, seed 0), 10 EM iterations of Algorithm 1 plus the final
log-likelihood.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    spec = synth.config_spec(0)
    d = synth.planted_dataset(spec, dtype=np.float32)
    r = oracle.fit([x.astype(np.float64) for x in d["X"]], d["W0"], spec.n_iter, final_ll=True)
    out = {
        "workload": spec.name,
        "n_iter": spec.n_iter,
        "input_dtype": "float32",
        "ll": [float(x) for x in r["ll"]],
        "rho2": [float(x) for x in r["rho2"]],
        "sigma_s_trace": float(np.trace(r["Sigma_s"])),
        "sigma_s_eigs": [float(x) for x in np.linalg.eigvalsh(r["Sigma_s"])],
        "es_fro": float(np.linalg.norm(r["ES"])),
        "W0_first_col_head": [float(x) for x in d["W0"][0][:4, 0]],
    }
    with open(os.path.join(HERE, "raider_like_k10.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
