"""Writes tests/golden/tiny_search.json from the CPU oracle alone.

The tiny workload (1,000 references, 100 queries, D=2048, Q=16, +-500 window,
top-1, seed 0) is preprocessed, encoded and searched by ``oracle`` only; the
file pins the oracle against later drift.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2211_16422_gb300 import synth  # noqa: E402


def main():
    refs, qs, spec = synth.make_workload("tiny")
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH,
              n_bins=synth.N_BINS, max_peaks=synth.MAX_PEAKS, n_levels=spec["n_levels"])
    F, L, _, _ = oracle.item_memory(spec["dim"], spec["n_levels"], synth.N_BINS, spec["dim"] // 2, 0)
    r_csr = oracle.preprocess(refs.offsets, refs.mz, refs.intensity, **pp)
    q_csr = oracle.preprocess(qs.offsets, qs.mz, qs.intensity, **pp)
    r_hv = oracle.encode(spec["dim"], F, L, *r_csr)
    q_hv = oracle.encode(spec["dim"], F, L, *q_csr)
    idx, dist = oracle.search(spec["dim"], r_hv, refs.precursor_mz, refs.charge, q_hv,
                              qs.precursor_mz, qs.charge, spec["tol"], spec["unit"], spec["k"])
    out = {
        "_what": "oracle-only regression values for the tiny workload (seed 0, item-memory seed 0)",
        "dim": spec["dim"], "n_levels": spec["n_levels"], "tol": spec["tol"], "k": spec["k"],
        "ref_hv_sha256": hashlib.sha256(r_hv.tobytes()).hexdigest(),
        "query_hv_sha256": hashlib.sha256(q_hv.tobytes()).hexdigest(),
        "ref_csr_nnz": int(r_csr[0][-1]), "query_csr_nnz": int(q_csr[0][-1]),
        "top1_idx": idx[:, 0].tolist(), "top1_dist": dist[:, 0].tolist(),
        "recovered_source": int(np.count_nonzero(idx[:, 0] == qs.source)),
    }
    with open(os.path.join(ROOT, "tests", "golden", "tiny_search.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
