"""The oracle against its stored regression values and Table 1's settings."""
import hashlib
import json
import os

import numpy as np

import oracle
from paper_2211_16422_gb300 import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_table1_settings_used_by_workloads():
    t = json.load(open(os.path.join(HERE, "table1.json")))
    assert synth.MAX_PEAKS == t["max_peaks"]
    assert (synth.MZ_MIN, synth.MZ_MAX) == (t["mz_min"], t["mz_max"])
    assert synth.BIN_WIDTH == t["bin_size"]["small_scale"]
    # f = floor((1500 - 101) / 0.05) + 1 bins
    assert synth.N_BINS == int(round((t["mz_max"] - t["mz_min"]) / t["bin_size"]["small_scale"])) + 1
    for name in ("tiny", "full", "serving"):
        assert synth.WORKLOADS[name]["tol"] == t["precursor_tolerance_wide_da"]["small_scale"]


def test_oracle_tiny_regression():
    g = json.load(open(os.path.join(HERE, "tiny_search.json")))
    refs, qs, spec = synth.make_workload("tiny")
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH,
              n_bins=synth.N_BINS, max_peaks=synth.MAX_PEAKS, n_levels=spec["n_levels"])
    F, L, _, _ = oracle.item_memory(spec["dim"], spec["n_levels"], synth.N_BINS, spec["dim"] // 2, 0)
    r_csr = oracle.preprocess(refs.offsets, refs.mz, refs.intensity, **pp)
    q_csr = oracle.preprocess(qs.offsets, qs.mz, qs.intensity, **pp)
    r_hv = oracle.encode(spec["dim"], F, L, *r_csr)
    q_hv = oracle.encode(spec["dim"], F, L, *q_csr)
    assert hashlib.sha256(r_hv.tobytes()).hexdigest() == g["ref_hv_sha256"]
    assert hashlib.sha256(q_hv.tobytes()).hexdigest() == g["query_hv_sha256"]
    idx, dist = oracle.search(spec["dim"], r_hv, refs.precursor_mz, refs.charge, q_hv,
                              qs.precursor_mz, qs.charge, spec["tol"], spec["unit"], spec["k"])
    assert idx[:, 0].tolist() == g["top1_idx"]
    assert dist[:, 0].tolist() == g["top1_dist"]
