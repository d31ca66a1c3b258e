#!/usr/bin/env python3
"""Benchmark of the HD open-modification search hot path on GB300.

One step = one pass of the hot path over one query batch with the reference
library resident on the device (reference HVs are encoded once and reused,
Section 3.3): encode the 50,000 query spectra (Eq. 1), sort them by charge
and precursor m/z, find their +-500 windows, score every in-window reference
by Hamming distance and keep the top-5.  The library (1,000,000 references,
half decoys, D=8192, Q=32) is built before timing; its one-off costs are
reported beside the step.

The JSON line's `value` is Hamming comparisons per second (algorithmic
in-window candidates only) over the whole job; queries/s and the
end-to-end figure through hd_search_host (host buffers, copies included)
are reported next to it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_16422_gb300 import synth  # noqa: E402

METRIC = "Hamming comparisons/s & queries/s, D=8192, ±500 Da open window; p50/p99 latency"
UNIT = "comparisons/s"
L2_BYTES = 129 * 2**20

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel on the full workload, from one single-pass ncu capture of
# this script.  A figure is used only while the kernel's sources hash to the
# captured value and the launch uses the captured form and schedule;
# otherwise `traffic` is null.
KERNEL_SOURCES = ("paper_2211_16422_gb300/csrc/search_mma.cu", "paper_2211_16422_gb300/csrc/search_common.cuh")
POPC_SOURCES = ("paper_2211_16422_gb300/csrc/search_popc.cu", "paper_2211_16422_gb300/csrc/search_common.cuh")
TRAFFIC = {
    # key: (kernel, form, tile_group, super_group, cluster, cta_group, tiles_per_stage)
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
    #     -k regex:k_search_mma -s 0 -c 1 python bench.py --steps 2 --warmup 3 --no-e2e --no-cpu-baseline
    #     --popc-steps 0 --no-peaks --form <form> --schedule <tile_group,super_group,cluster,cta_group,tiles>
    ("k_search_mma2", "tc_mxf4", 4, 2, 2, 2, 2): {"bytes": 162.048e9 + 0.18906e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 4, 2, 2, 2, 1): {"bytes": 142.911e9 + 0.27436e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 4, 4, 2, 2, 2): {"bytes": 176.168e9 + 0.15872e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 4, 4, 2, 2, 1): {"bytes": 154.274e9 + 0.20655e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 4, 16, 2, 2, 2): {"bytes": 195.379e9 + 0.06076e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 4, 16, 2, 2, 1): {"bytes": 193.309e9 + 0.06281e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 8, 2, 2, 2, 2): {"bytes": 177.418e9 + 0.16138e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 8, 2, 2, 2, 1): {"bytes": 159.751e9 + 0.18949e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 8, 4, 2, 2, 2): {"bytes": 184.797e9 + 0.12673e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 8, 4, 2, 2, 1): {"bytes": 176.310e9 + 0.16065e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 8, 16, 2, 2, 2): {"bytes": 210.660e9 + 0.03568e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 8, 16, 2, 2, 1): {"bytes": 210.051e9 + 0.03628e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 16, 2, 2, 2, 2): {"bytes": 186.900e9 + 0.09986e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 16, 2, 2, 2, 1): {"bytes": 176.523e9 + 0.11182e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 16, 4, 2, 2, 2): {"bytes": 194.750e9 + 0.08237e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 16, 4, 2, 2, 1): {"bytes": 187.700e9 + 0.08059e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 16, 16, 2, 2, 2): {"bytes": 218.315e9 + 0.02146e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 16, 16, 2, 2, 1): {"bytes": 221.438e9 + 0.02168e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 32, 2, 2, 2, 2): {"bytes": 183.868e9 + 0.06897e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 32, 2, 2, 2, 1): {"bytes": 181.403e9 + 0.07096e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 32, 4, 2, 2, 2): {"bytes": 197.430e9 + 0.05047e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 32, 4, 2, 2, 1): {"bytes": 198.752e9 + 0.04694e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 32, 16, 2, 2, 2): {"bytes": 224.915e9 + 0.01352e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
    ("k_search_mma2", "tc_mxf4", 32, 16, 2, 2, 1): {"bytes": 227.719e9 + 0.01352e9,
                                                  "sha256": "6fc3e0e0bf68e41f"},
}

# The arithmetic type the search computes in: the tensor-core operand format
# (products accumulated in fp32, exact), or 32-bit words for XOR + popcount.
DTYPE_OF_FORM = {"tc_mxf4": "e2m1", "tc_fp4": "e2m1", "tc_fp8": "e4m3", "tc_bf16": "bf16", "popc": "u32"}


# Schedule of the tensor-core forms: work-item shape, SM pairing, and the
# kind::mxf4 form's reference tiles per query stage; the library's default.
SCHEDULE_KEYS = ("tile_group", "super_group", "cluster", "cta_group", "tiles_per_stage")
DEFAULT_SCHEDULE = {"tile_group": 16, "super_group": 16, "cluster": 2, "cta_group": 2, "tiles_per_stage": 1}


def parse_schedule(text):
    """'tile_group,super_group,cluster,cta_group[,tiles_per_stage]' -> dict (tiles_per_stage 1 if absent)."""
    v = [int(x) for x in text.split(",")]
    if len(v) not in (4, 5):
        raise SystemExit("--schedule takes 4 or 5 comma-separated integers")
    return dict(zip(SCHEDULE_KEYS, v + [1] * (5 - len(v))))


def apply_schedule(hd, lib, sched):
    hd.hd_library_set_schedule(lib, sched["tile_group"], sched["super_group"], sched["cluster"], sched["cta_group"])
    hd.hd_library_set_stage_tiles(lib, sched.get("tiles_per_stage", 1))
    return sched


def kernel_source_hash(sources=KERNEL_SOURCES):
    """sha256 of the kernel's code: its sources with C/C++ comments and blank
    lines removed, so that editing a comment keeps the captured figures."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            t = fh.read()
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        h.update("\n".join(line.rstrip() for line in t.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--form", default="auto")
    ap.add_argument("--schedule", default=None,
                    help="tile_group,super_group,cluster,cta_group[,tiles_per_stage] of the tensor-core "
                         "form (with --form; default: the library's 16,16,2,2,1)")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (testing only)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--popc-steps", type=int, default=3,
                    help="timed steps of the popcount form beside the headline form (0: skip)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the instruction-rate microbenchmarks")
    ap.add_argument("--workload", choices=("full", "batched", "serving", "cascade", "multibit", "peaks"),
                    default="full",
                    help="full: the headline line; batched / serving / cascade / multibit: the extra workloads; "
                         "peaks: the instruction-rate microbenchmarks alone")
    ap.add_argument("--bits", type=int, default=None,
                    help="component bits (2..5) of --workload multibit (default 3), or of --workload cascade "
                         "(default: binary HVs)")
    return ap.parse_args()


# ------------------------------------------------------------------ workload
def workload(scale: float, rank: int):
    """References are identical on every rank (a replica of the library);
    each rank draws its own queries (weak scaling over query batches)."""
    spec = dict(synth.WORKLOADS["full"])
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    n_r = max(2, int(round(spec["n_refs"] * scale)))
    n_q = max(1, int(round(spec["n_queries"] * scale)))
    refs = synth.make_references(n_r, spec["charges"], spec["weights"], rng,
                                 decoy_fraction=spec["decoy_fraction"])
    qrng = np.random.Generator(np.random.PCG64([spec["seed"], 1000 + rank]))
    queries = synth.make_queries(refs, n_q, qrng)
    spec.update(n_refs=n_r, n_queries=n_q)
    return refs, queries, spec


def tuning_queries(refs, n_q, rank):
    """A second query batch of the same recipe and size, drawn from its own seed:
    the autotuner picks form and schedule on it, not on the batch it is timed on."""
    spec = synth.WORKLOADS["full"]
    return synth.make_queries(refs, n_q, np.random.Generator(np.random.PCG64([spec["seed"], 2000 + rank])))


def pp_args(spec):
    return dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH,
                n_bins=synth.N_BINS, max_peaks=synth.MAX_PEAKS, n_levels=spec["n_levels"])


def config_of(spec, n_gpus):
    return {"workload": "1M-reference library (50% decoys) x 50k queries, synthetic, D=8192, Q=32, "
                        "bins 0.05 m/z, +-500 open window, top-5",
            "n_refs": spec["n_refs"], "n_queries_per_gpu": spec["n_queries"], "dim": spec["dim"],
            "n_levels": spec["n_levels"], "tol": spec["tol"], "tol_unit": spec["unit"], "k": spec["k"],
            "global_batch": spec["n_queries"] * n_gpus,
            "parallelism": f"replicated library, queries sharded, {n_gpus} GPU(s)",
            "l2": "library (1 GiB) and per-step query set exceed L2 (129 MB): no flush needed"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.rows = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[4:8]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": reasons}


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(refs, queries, spec, target_s, lib_fraction=0.05, seed=5, bits=1):
    """The oracle's brute-force windowed top-k search on the host cores, on a
    uniform library sample; returns (comparisons/s, threads, sample text, step fn).
    bits > 1: multi-bit components and the dot-product search."""
    import oracle
    rng = np.random.default_rng(seed)
    n_lib = max(1000, int(refs.n * lib_fraction))
    rsel = np.sort(rng.choice(refs.n, n_lib, replace=False))
    rsub = refs.subset(rsel)
    D, Q = spec["dim"], spec["n_levels"]
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    enc = ((lambda *csr: oracle.encode(D, F, L, *csr)) if bits == 1
           else (lambda *csr: oracle.encode_multibit(D, F, L, *csr, bits)))
    r_hv = enc(*oracle.preprocess(rsub.offsets, rsub.mz, rsub.intensity, **pp_args(spec)))
    threads = os.cpu_count() or 1
    q_all = queries.subset(np.arange(min(queries.n, 20000)))
    q_hv = enc(*oracle.preprocess(q_all.offsets, q_all.mz, q_all.intensity, **pp_args(spec)))
    wc = oracle.window_count(rsub.precursor_mz, rsub.charge, q_all.precursor_mz, q_all.charge, spec["tol"],
                             spec["unit"]).astype(np.int64)

    def step(m, offset=0):
        which = (np.arange(m) + offset) % q_all.n
        t = time.perf_counter()
        if bits == 1:
            oracle.search(D, r_hv, rsub.precursor_mz, rsub.charge, q_hv, q_all.precursor_mz, q_all.charge,
                          spec["tol"], spec["unit"], spec["k"], which=which.astype(np.uint32), n_threads=threads)
        else:
            oracle.search_dot(r_hv, rsub.precursor_mz, rsub.charge, q_hv, q_all.precursor_mz, q_all.charge,
                              spec["tol"], spec["unit"], spec["k"], which=which.astype(np.uint32),
                              n_threads=threads)
        return int(wc[which].sum()), time.perf_counter() - t

    m = 256
    comps, dt = step(m)
    while dt < 1.0 and m < q_all.n:
        m = min(q_all.n, m * 4)
        comps, dt = step(m)
    per_step = max(1, min(q_all.n, int(m * max(1.0, target_s / 4) / max(dt, 1e-3))))
    kind = "search" if bits == 1 else f"dot-product search ({bits}-bit components)"
    sample = (f"oracle brute-force top-{spec['k']} {kind} of {per_step} queries against a uniform "
              f"{n_lib}-reference sample ({lib_fraction:.0%}) of the library, D={D}, +-{spec['tol']:g}; "
              f"oracle encoding of the sample is setup, not timed")
    return per_step, threads, sample, step


# ------------------------------------------------------- multi-rank reduce
def reduce_over_ranks(seconds, units, device=None):
    """Whole-job figures of a weak-scaling step: the slowest rank's time and the
    units (comparisons, queries) of all ranks summed.  With no process group
    the rank's own figures are returned.  `device` holds the reduction tensors
    (cuda for NCCL; None = CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), int(units)
    tt = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cc = torch.tensor([int(units)], dtype=torch.int64, device=device)
    dist.all_reduce(cc)
    return float(tt.item()), int(cc.item())


# ---------------------------------------------------------------- our arm
def measure_peaks(hd, kinds, launches=10, clock_index=0):
    """The instruction-rate microbenchmarks (hd_measure_peak), with the SM clock
    sampled while they run."""
    with ClockSampler(clock_index) as clocks:
        res = {k: hd.hd_measure_peak(k, launches) for k in kinds}
    return res, clocks.summary()


def tensor_roofline(form, comparisons, D, avg_search_ms, peaks, peak_clocks, sched):
    """Roofline of a tensor-core search launch: 2*D flops per in-window comparison
    (masked tile padding not counted) against the measured rate of the kernel's
    own instruction and shape (hd_measure_peak), with the bf16-derived figure
    beside it."""
    achieved = comparisons * 2.0 * D / (avg_search_ms / 1e3) / 1e12
    bf16 = measured_peaks().get("bf16_tflops", 1900.0)
    eight_bit_kind = form in ("tc_fp8", "tc_fp4")   # kind::f8f6f4
    # the recipe's nominal dense ratios to bf16: fp8 4.5 / 2.25, fp4 13.5 / 2.25
    ratio = 2.0 if eight_bit_kind else (6.0 if form == "tc_mxf4" else 1.0)
    derived = bf16 * ratio
    pair = sched.get("cta_group") == 2
    kname = "k_search_mma2" if pair else "k_search_mma"
    r = {"kernel": kname, "bound": "tensor", "unit": "TFLOP/s", "achieved": achieved,
         "schedule": {k_: sched.get(k_) for k_ in SCHEDULE_KEYS},
         "derived_peak": {"peak": derived, "frac": achieved / derived,
                          "basis": "MEASURED_PEAKS burst cuBLAS bf16" + (
                              " x 2 (nominal fp8/bf16 ratio 4.5/2.25)" if eight_bit_kind else
                              " x 6 (nominal fp4/bf16 ratio 13.5/2.25)" if form == "tc_mxf4" else "")}}
    p = (peaks or {}).get(form)
    if p:
        peak = p["best_per_s"] / 1e12
        instr = ("tcgen05.mma.cta_group::2.kind::f8f6f4 (" + ("e2m1" if form == "tc_fp4" else "e4m3") + "), M=256 N=256"
                 if eight_bit_kind else
                 "tcgen05.mma.cta_group::2.kind::mxf4.block_scale (packed e2m1, unit ue8m0 scales), M=256 N=240"
                 if form == "tc_mxf4" else "tcgen05.mma.cta_group::2.kind::f16 (bf16), M=256 N=256")
        r.update({"peak": peak, "frac": achieved / peak,
                  "peak_basis": f"measured (own microbenchmark hd_measure_peak: {instr}, operands "
                                f"resident in shared memory, {p['sms']} SMs, best of {p['launches']} launches, "
                                f"SM clock median {(peak_clocks or {}).get('sm_mhz')} MHz)",
                  "peak_median": p["median_per_s"] / 1e12})
        if not pair:
            r["peak_basis"] += "; the 1-SM kernel issues M=128 cta_group::1 at the same per-SM rate"
    else:
        r.update({"peak": derived, "frac": achieved / derived, "peak_basis": r["derived_peak"]["basis"]
                  + " (of measured)"})
    return r


OPS_PER_WORD = 2.5   # integer-pipe operations per 32-bit word of the carry-save popcount kernel


def popc_roofline(comparisons, D, avg_search_ms, n_sm, sm_mhz, peaks):
    """Roofline of the popcount form: 32-bit words of XOR + popcount work.  The
    paper's form counts one word per popcount (bound: the popcount unit's
    measured rate); the carry-save kernel counts two words per popcount and
    spends 2.5 integer-pipe operations per word: the XOR, and per two words a
    majority, a three-input XOR and a shift-add of one carry count (bound: the
    measured LOP3 rate / 2.5).  Counting two carries per three-input add (2.25
    operations per word) left the kernel's time unchanged (942 ms with the
    two-stage ring), so the integer issue rate is a bound it does not reach."""
    words = comparisons * (D // 32)
    achieved = words / (avg_search_ms / 1e3) / 1e12
    pp, pl = (peaks or {}).get("popc"), (peaks or {}).get("lop3")
    if pp and pl:
        popc_bound = pp["best_per_s"] / 1e12
        issue_bound = pl["best_per_s"] / OPS_PER_WORD / 1e12
        basis = f"measured (own microbenchmarks hd_measure_peak 'lop3' / {OPS_PER_WORD} and 'popc')"
    else:
        popc_bound = n_sm * 16 * sm_mhz * 1e6 / 1e12
        issue_bound = n_sm * 64 / OPS_PER_WORD * sm_mhz * 1e6 / 1e12
        basis = f"{n_sm} SMs x (64 LOP3 / {OPS_PER_WORD}, 16 popc) per clk x {sm_mhz:.0f} MHz (nominal unit counts)"
    return {"kernel": "k_search_popc", "bound": "alu", "unit": "Tword32/s", "achieved": achieved,
            "peak": issue_bound, "frac": achieved / issue_bound,
            "peak_basis": "integer-issue bound of the carry-save kernel: " + basis,
            "popcount_unit_bound": {"peak": popc_bound, "frac": achieved / popc_bound,
                                    "basis": "one popc32 per word (the paper's form): " + basis}}


def popc_mb_roofline(comparisons, D, bits, avg_search_ms, peaks):
    """Roofline of the popcount form of the multi-bit dot product: per pair of
    32-bit words, bits^2 plane-pair terms, each counted by the carry-save adder
    of the binary kernel: 2.5 integer-pipe operations per word and term (the
    AND, and per two words a majority, a three-input XOR and a shift-add;
    bound: the measured LOP3 rate / (2.5 bits^2)) and half a popcount (bound:
    the popcount unit's measured rate / (0.5 bits^2))."""
    words = comparisons * (D // 32)
    achieved = words / (avg_search_ms / 1e3) / 1e12
    pp, pl = (peaks or {}).get("popc"), (peaks or {}).get("lop3")
    issue_bound = pl["best_per_s"] / (OPS_PER_WORD * bits ** 2) / 1e12
    popc_bound = pp["best_per_s"] / (0.5 * bits ** 2) / 1e12
    basis = "measured (own microbenchmarks hd_measure_peak 'lop3' and 'popc')"
    return {"kernel": "k_search_popc_mb", "bound": "alu", "unit": "Tword32/s (pairs of 32-bit words)",
            "achieved": achieved, "peak": issue_bound, "frac": achieved / issue_bound,
            "peak_basis": f"integer-issue bound: LOP3 rate / ({OPS_PER_WORD} x {bits ** 2}) per word pair: " + basis,
            "popcount_unit_bound": {"peak": popc_bound, "frac": achieved / popc_bound,
                                    "basis": f"popcount unit / (0.5 x {bits ** 2}) per word pair: " + basis}}


def pctl(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2211_16422_gb300 import build, hd
    build.build()
    torch.cuda.set_device(local_rank)
    dist_on = world > 1
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist_on:
            import torch.distributed as dist
            dist.barrier()

    refs, queries, spec = workload(args.scale, rank)
    D, Q, k, tol, unit = spec["dim"], spec["n_levels"], spec["k"], spec["tol"], spec["unit"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32
                                     else np.ascontiguousarray(a)).cuda()
    setup = {}
    t = time.perf_counter()
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=0)
    setup["item_memory_s"] = time.perf_counter() - t
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp_args(spec))
    q_csr = hd.hd_preprocess(ctx, dev(queries.offsets), dev(queries.mz), dev(queries.intensity), **pp_args(spec))
    torch.cuda.synchronize()
    t = time.perf_counter()
    r_hv = hd.hd_encode(ctx, *r_csr)
    torch.cuda.synchronize()
    setup["encode_refs_s"] = time.perf_counter() - t
    t = time.perf_counter()
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    setup["build_library_s"] = time.perf_counter() - t
    del r_hv
    form = args.form
    # the autotuner chooses among the prepared tensor-core forms (and popc)
    for f in (("tc_fp4", "tc_fp8") if form == "auto" else ((form,) if form.startswith("tc_") else ())):
        t = time.perf_counter()
        hd.hd_library_prepare(lib, f)
        setup["prepare_" + f + "_s"] = time.perf_counter() - t
    if args.schedule:
        setup["schedule"] = apply_schedule(hd, lib, parse_schedule(args.schedule))
    q_mz, q_z = dev(queries.precursor_mz), dev(queries.charge)
    if args.form == "auto":
        # the library's autotuner picks form and schedule on a second, separately seeded batch
        # of the same size and recipe (setup, not timed)
        t = time.perf_counter()
        tq = tuning_queries(refs, queries.n, rank)
        tq_hv = hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(tq.offsets), dev(tq.mz), dev(tq.intensity),
                                                      **pp_args(spec)))
        tuned, _ = hd.hd_library_autotune(lib, tq_hv, dev(tq.precursor_mz), dev(tq.charge), None, [(tol, unit)], k)
        del tq_hv
        form = tuned["form"]
        setup["autotune_s"] = time.perf_counter() - t
        setup["autotune_choice"] = tuned
        setup["autotune_batch"] = "separate seeded batch of the same recipe and size"
    lo, hi = hd.hd_query_windows(lib, q_mz, q_z, tol, unit)
    comparisons = int((hd.as_u32(hi).astype(np.int64) - hd.as_u32(lo).astype(np.int64)).sum())
    nq = queries.n
    q_hv = torch.empty((nq, D // 64), dtype=torch.int64, device="cuda")
    out_idx = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    out_dist = torch.empty((nq, k), dtype=torch.int16, device="cuda")
    stream = torch.cuda.current_stream()

    def step(f=None):
        hd.hd_encode(ctx, *q_csr, out=q_hv)
        hd.hd_search_open(lib, q_hv, q_mz, q_z, tol, unit, k, form=f or form, out_idx=out_idx, out_dist=out_dist)

    # instruction-rate microbenchmarks (the rooflines' denominators), outside the timed region
    peaks, peak_clocks = None, None
    if not args.no_peaks:
        kinds = ((form,) if form.startswith("tc_") else ()) + (("popc", "lop3") if args.popc_steps > 0
                                                                  or form == "popc" else ())
        peaks, peak_clocks = measure_peaks(hd, kinds, clock_index=local_rank)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.status()
    lib.status()
    barrier()
    torch.cuda.synchronize()
    hd.hd_profile_enable(True)
    launches0 = hd.hd_launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local_rank) as clocks:
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = hd.hd_launch_count() - launches0
    hd.hd_profile_enable(False)
    search_ms, search_n = hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
    encode_ms, encode_n = hd.hd_profile_collect(hd.HD_KERNEL_ENCODE)
    ctx.status()
    lib.status()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    ms = evs[0].elapsed_time(evs[-1]) / args.steps
    ms, total_comparisons = reduce_over_ranks(ms, comparisons, device="cuda")
    p50, _ = reduce_over_ranks(pctl(step_ms, 50), 0, device="cuda")
    p99, _ = reduce_over_ranks(pctl(step_ms, 99), 0, device="cuda")
    value = total_comparisons / (ms / 1e3)
    qps = nq * world / (ms / 1e3)
    ref_idx, ref_dist = out_idx.cpu().numpy(), out_dist.cpu().numpy()

    # the paper's form (XOR + popcount) on the same batch: its own timed steps and
    # its own roofline, and the same top-k as the headline form
    forms = None
    if args.popc_steps > 0 and form != "popc":
        step("popc")
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(out_idx.cpu().numpy(), ref_idx) and np.array_equal(out_dist.cpu().numpy(), ref_dist), \
            "popcount and tensor-core forms differ"
        hd.hd_profile_enable(True)
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as pclocks:
            pe0.record(stream)
            for _ in range(args.popc_steps):
                step("popc")
            pe1.record(stream)
            torch.cuda.synchronize()
        hd.hd_profile_enable(False)
        psearch_ms, psearch_n = hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
        hd.hd_profile_collect(hd.HD_KERNEL_ENCODE)
        lib.status()
        pms = pe0.elapsed_time(pe1) / args.popc_steps
        pms, _ = reduce_over_ranks(pms, 0, device="cuda")
        popc_equal = bool(np.array_equal(out_idx.cpu().numpy(), ref_idx)
                          and np.array_equal(out_dist.cpu().numpy(), ref_dist))
        assert popc_equal, "popcount and tensor-core forms differ"
        forms = {"popc": {"ms_per_step": pms, "search_ms": psearch_ms / max(1, psearch_n),
                          "comparisons_per_s": total_comparisons / (pms / 1e3), "steps": args.popc_steps,
                          "clocks": pclocks.summary()},
                 form: {"ms_per_step": ms, "search_ms": search_ms / max(1, search_n),
                        "comparisons_per_s": value, "steps": args.steps},
                 "speedup": pms / ms, "speedup_of": f"{form} over popc, ms per step",
                 "identical_topk": popc_equal}

    # end to end through hd_search_host: pinned host inputs, copies in the timed region
    e2e = None
    if not args.no_e2e:
        h_off, h_bins, h_lv = (t_.cpu().pin_memory() for t_ in
                               (q_csr[0], q_csr[1][:int(hd.as_u32(q_csr[0])[-1])], q_csr[2][:int(hd.as_u32(q_csr[0])[-1])]))
        h_mz = torch.from_numpy(queries.precursor_mz).pin_memory()
        h_z = torch.from_numpy(queries.charge).pin_memory()
        h_idx = torch.empty((nq, k), dtype=torch.int32).pin_memory()
        h_dist = torch.empty((nq, k), dtype=torch.int16).pin_memory()
        e2e_step = lambda: hd.hd_search_host(ctx, lib, h_off, h_bins, h_lv, h_mz, h_z, tol, unit, k, h_idx, h_dist)
        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        barrier()
        walls = []
        t = time.perf_counter()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            e2e_step()
            walls.append((time.perf_counter() - t1) * 1e3)
        e2e_s = (time.perf_counter() - t) / args.steps
        e2e_s, _ = reduce_over_ranks(e2e_s, 0, device="cuda")
        e50, _ = reduce_over_ranks(pctl(walls, 50), 0, device="cuda")
        e99, _ = reduce_over_ranks(pctl(walls, 99), 0, device="cuda")
        h2d = sum(t_.numel() * t_.element_size() for t_ in (h_off, h_bins, h_lv, h_mz, h_z))
        d2h = nq * k * (4 + 2)
        e2e = {"value": total_comparisons / e2e_s, "unit": UNIT, "queries_per_s": nq * world / e2e_s,
               "ms_per_step": e2e_s * 1e3, "p50_ms": e50, "p99_ms": e99,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        assert np.array_equal(h_idx.numpy(), ref_idx), "end-to-end results differ"

    if rank != 0:
        return
    cs = clocks.summary()
    props = torch.cuda.get_device_properties(local_rank)
    n_sm = props.multi_processor_count
    sm_mhz = (cs or {}).get("sm_mhz") or 1455.0
    avg_search_ms = search_ms / max(1, search_n)
    if form.startswith("tc_"):
        sched = setup.get("autotune_choice") or setup.get("schedule") or dict(DEFAULT_SCHEDULE)
        roofline = tensor_roofline(form, comparisons, D, avg_search_ms, peaks, peak_clocks, sched)
    else:
        roofline = popc_roofline(comparisons, D, avg_search_ms, n_sm, sm_mhz, peaks)
    if forms:
        pr = popc_roofline(comparisons, D, forms["popc"]["search_ms"], n_sm,
                           (forms["popc"]["clocks"] or {}).get("sm_mhz") or sm_mhz, peaks)
        forms["popc"].update({"frac_issue_bound": pr["frac"], "frac_popc_bound": pr["popcount_unit_bound"]["frac"],
                              "roofline": pr})
        forms[form].update({"frac": roofline["frac"], "peak_basis": roofline["peak_basis"]})
    traffic = None
    if form.startswith("tc_") and args.scale == 1.0:
        s_ = roofline["schedule"]
        t_ = TRAFFIC.get((roofline["kernel"], form) + tuple(s_.get(k_) or 1 for k_ in SCHEDULE_KEYS))
        if t_ and t_["sha256"] == kernel_source_hash():
            traffic = t_["bytes"]
    roofline.update({"traffic": traffic, "traffic_unit": "bytes per launch", "avg_launch_ms": avg_search_ms,
                     "launches": search_n, "step_share": search_ms / (ms * args.steps),
                     "kernel_source_sha256": kernel_source_hash(POPC_SOURCES if roofline["kernel"] == "k_search_popc"
                                                                 else KERNEL_SOURCES)})
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        per_step, threads, sample, cstep = cpu_oracle_rate(refs, queries, spec, args.cpu_seconds)
        tot_c, tot_t, off = 0, 0.0, 0
        while tot_t < args.cpu_seconds:
            c_, t_ = cstep(per_step, off)
            tot_c, tot_t, off = tot_c + c_, tot_t + t_, off + per_step
        cpu = {"value": tot_c / tot_t, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": tot_t}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_OF_FORM.get(form, "u32"),
            "data": "synthetic (seeded generator; stands in for the "
            "paper's MassIVE-KB/HEK293 and yeast/iPRG2012 sets)",
            "config": config_of(spec, world), "queries_per_s": qps,
            "latency_ms": {"p50": p50, "p99": p99, "of": "one step (encode + search of the query batch), "
                                                         "CUDA events on the launching stream"},
            "comparisons_per_step": total_comparisons,
            "kernel_ms_per_step": {"search": search_ms / args.steps, "encode": encode_ms / args.steps},
            "setup_s": setup, "roofline": roofline, "forms": forms, "peaks": peaks, "peak_clocks": peak_clocks,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": cs, "form": form, "device": props.name}
    print(json.dumps(line))


def run_peaks(args):
    """The instruction-rate microbenchmarks alone: one JSON line."""
    import torch
    from paper_2211_16422_gb300 import build, hd
    build.build()
    torch.cuda.set_device(0)
    res, clocks = measure_peaks(hd, ("tc_mxf4", "tc_fp4", "tc_fp8", "tc_bf16", "popc", "lop3"),
                                launches=max(3, args.steps))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    per_clk = {k: v["best_per_s"] / (n_sm * mhz * 1e6) for k, v in res.items()}
    line = {"metric": "instruction-rate microbenchmarks (the search rooflines' denominators)",
            "value": res["tc_mxf4"]["best_per_s"] / 1e12, "unit": "TFLOP/s (tc_mxf4)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "peaks": res,
            "per_clock_per_sm": per_clk, "clocks": clocks, "device": torch.cuda.get_device_properties(0).name}
    print(json.dumps(line), flush=True)


# ------------------------------------------------ batched uneven workload
def run_batched(args):
    """200 log-uniform query batches (10..20,000 spectra), charge 1-5, windows
    round-robin over 20 ppm / 150 Da / 500 Da, against a 2,000,000-reference
    library, at D=4096 and D=8192: autotune on the whole query set, capture
    encode + search of every batch as one CUDA graph, time its replays, then
    each batch alone for its latency, with the graph's schedule and with one
    tuned on a median-size batch of the widest window.  One JSON line per D."""
    import torch
    from paper_2211_16422_gb300 import build, hd
    build.build()
    spec = synth.WORKLOADS["batched"]
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    n_r = max(1000, int(spec["n_refs"] * args.scale))
    refs = synth.make_references(n_r, spec["charges"], spec["weights"], rng, decoy_fraction=spec["decoy_fraction"])
    hi = max(20, int(spec["batch_hi"] * args.scale))
    sizes = synth.batch_sizes(spec["n_batches"], spec["batch_lo"], hi, rng)
    qs = synth.make_queries(refs, int(sizes.sum()), rng)
    windows = [(t, u) for t, u in spec["windows"]]
    cls = np.repeat(np.arange(len(sizes)) % len(windows), sizes).astype(np.uint8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32
                                     else np.ascontiguousarray(a)).cuda()
    for D in spec["dims"]:
        Q = spec["n_levels"]
        pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
                  max_peaks=synth.MAX_PEAKS, n_levels=Q)
        ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=0)
        r_hv = hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp))
        lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
        del r_hv
        hd.hd_library_prepare(lib, "tc_fp4")
        hd.hd_library_prepare(lib, "tc_fp8")
        off, bins, lv = hd.hd_preprocess(ctx, dev(qs.offsets), dev(qs.mz), dev(qs.intensity), **pp)
        nnz = int(hd.as_u32(off)[-1])
        q_mz, q_z, q_cls = dev(qs.precursor_mz), dev(qs.charge), dev(cls)
        # comparisons: in-window candidates of every query under its own window
        comparisons = 0
        for c, (tol, unit) in enumerate(windows):
            sel = torch.from_numpy(np.nonzero(cls == c)[0]).cuda()
            lo, hi_ = hd.hd_query_windows(lib, q_mz[sel].contiguous(), q_z[sel].contiguous(), tol, unit)
            comparisons += int((hd.as_u32(hi_).astype(np.int64) - hd.as_u32(lo).astype(np.int64)).sum())
        # autotune on the whole query set (setup, not timed): a subset of the queries has a
        # lower query density per window class, so its sorted blocks span wider m/z ranges
        # than the real set's and can favour another schedule
        q_hv = hd.hd_encode(ctx, off, bins, lv)
        best, table = hd.hd_library_autotune(lib, q_hv, q_mz, q_z, q_cls, windows, spec["k"])
        del q_hv
        plan = hd.Plan(ctx, lib, off, bins[:nnz], lv[:nnz], q_mz, q_z, q_cls, windows, k=spec["k"], form="auto")
        stream = torch.cuda.current_stream()
        for _ in range(args.warmup):
            plan.launch()
        torch.cuda.synchronize()
        lib.status()
        hd.hd_profile_enable(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clocks:
            ev0.record(stream)
            for _ in range(args.steps):
                plan.launch()
            ev1.record(stream)
            torch.cuda.synchronize()
        hd.hd_profile_enable(False)
        hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
        hd.hd_profile_collect(hd.HD_KERNEL_ENCODE)
        ms = ev0.elapsed_time(ev1) / args.steps
        # the dominant kernel's time, from one eager run of the same search (graph
        # replays carry no per-kernel events)
        hd.hd_profile_enable(True)
        hd.hd_search_open_multi(lib, plan.q_hv, q_mz, q_z, q_cls, windows, spec["k"], form=best["form"])
        torch.cuda.synchronize()
        hd.hd_profile_enable(False)
        search_ms, search_n = hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
        # per-batch latency: each batch alone (encode + search with its window), CUDA events around it
        starts = np.r_[0, np.cumsum(sizes)]
        off_np = hd.as_u32(off)
        batches = []
        for b_ in range(len(sizes)):
            a_, e_ = int(starts[b_]), int(starts[b_ + 1])
            p0, p1 = int(off_np[a_]), int(off_np[e_])
            batches.append((dev((off_np[a_:e_ + 1] - p0).astype(np.uint32)), bins[p0:p1].contiguous(),
                            lv[p0:p1].contiguous(), q_mz[a_:e_].contiguous(), q_z[a_:e_].contiguous(),
                            windows[b_ % len(windows)]))
        def alone(form_):
            lat_ = []
            for off_b, bins_b, lv_b, mz_b, z_b, (tol_b, unit_b) in batches:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hv_b = hd.hd_encode(ctx, off_b, bins_b, lv_b)
                hd.hd_search_open(lib, hv_b, mz_b, z_b, tol_b, unit_b, spec["k"], form=form_)
                e1.record(stream)
                torch.cuda.synchronize()
                lat_.append(e0.elapsed_time(e1))
            lib.status()
            return np.asarray(lat_)

        lat_tp = alone(best["form"])   # with the schedule tuned for the whole set's throughput
        # a batch searched alone is a latency question: tune on one batch of the median size
        # with the widest window (setup, not timed) and time every batch alone again
        widest = max((w for w in windows if w[1] == "da"), key=lambda w: w[0], default=windows[-1])
        wide = [b_ for b_ in range(len(sizes)) if batches[b_][5] == widest]
        pick = min(wide, key=lambda b_: (abs(int(sizes[b_]) - float(np.median(sizes))), b_))
        off_b, bins_b, lv_b, mz_b, z_b, win_b = batches[pick]
        best_lat, _ = hd.hd_library_autotune(lib, hd.hd_encode(ctx, off_b, bins_b, lv_b), mz_b, z_b, None,
                                             [win_b], spec["k"])
        lat = alone(best_lat["form"])
        # the roofline comes from one eager launch timed alone, against the measured rate of its instruction
        if best["form"].startswith("tc_"):
            pk, pclk = measure_peaks(hd, (best["form"],))
            roof = tensor_roofline(best["form"], comparisons, D, search_ms / max(1, search_n), pk, pclk, best)
        else:
            pk, _ = measure_peaks(hd, ("popc", "lop3"))
            roof = popc_roofline(comparisons, D, search_ms / max(1, search_n),
                                 torch.cuda.get_device_properties(0).multi_processor_count,
                                 (clocks.summary() or {}).get("sm_mhz") or 2070.0, pk)
        roof.update({"avg_launch_ms": search_ms / max(1, search_n), "traffic": None})
        line = {"metric": "Hamming comparisons/s, batched uneven windows (200 batches, 20 ppm / 150 Da / 500 Da)",
                "value": comparisons / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE_OF_FORM.get(best["form"], "u32"), "data": "synthetic",
                "config": {"workload": f"{n_r}-reference library x {len(sizes)} batches "
                                       f"({int(sizes.sum())} queries, sizes {int(sizes.min())}..{int(sizes.max())}), "
                                       f"D={D}, charge 1-5, windows round-robin", "dim": D,
                           "n_queries": int(qs.n), "n_batches": int(len(sizes))},
                "queries_per_s": qs.n / (ms / 1e3), "comparisons_per_step": comparisons,
                "batch_latency_ms": {"all_batches_one_graph": ms, "one_batch_alone_p50": float(np.percentile(lat, 50)),
                                     "one_batch_alone_p99": float(np.percentile(lat, 99)),
                                     "one_batch_alone_max": float(lat.max()),
                                     "one_batch_alone_schedule": best_lat,
                                     "one_batch_alone_tuned_on": f"batch {pick} ({int(sizes[pick])} queries, "
                                                                 f"{win_b[0]} {win_b[1]})",
                                     "one_batch_alone_with_graph_schedule_p50": float(np.percentile(lat_tp, 50)),
                                     "one_batch_alone_with_graph_schedule_p99": float(np.percentile(lat_tp, 99))},
                "graph_kernel_nodes": plan.kernel_nodes, "gpu_launches": plan.kernel_nodes * args.steps,
                "autotune": {"best": best, "candidates": len(table)},
                "roofline": roof,
                "clocks": clocks.summary()}
        print(json.dumps(line), flush=True)
        plan.close()
        lib.close()
        ctx.close()
        torch.cuda.empty_cache()


# ----------------------------------------------------------------- serving
def run_serving(args):
    """Continuous-batching server on the resident 1,000,000-reference D=8192
    library: Poisson-arriving requests of 1..5000 spectra (log-uniform), +-500,
    top-5, offered at 50..2000 requests/s.  Per load: p50/p99 latency (submit
    to results in host memory) and sustained queries/s.  One JSON line."""
    import torch
    from paper_2211_16422_gb300 import build, hd
    build.build()
    spec = synth.WORKLOADS["serving"]
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    n_r = max(1000, int(spec["n_refs"] * args.scale))
    refs = synth.make_references(n_r, spec["charges"], spec["weights"], rng, decoy_fraction=spec["decoy_fraction"])
    pool = synth.make_queries(refs, max(6000, int(60000 * args.scale)), rng)
    D, Q, k = spec["dim"], spec["n_levels"], spec["k"]
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32
                                     else np.ascontiguousarray(a)).cuda()
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=0)
    r_hv = hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp))
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    del r_hv
    hd.hd_library_prepare(lib, "tc_fp4")
    off_t, bins_t, lv_t = hd.hd_preprocess(ctx, dev(pool.offsets), dev(pool.mz), dev(pool.intensity), **pp)
    off = hd.as_u32(off_t)
    nnz = int(off[-1])
    bins, lv = hd.as_u32(bins_t[:nnz]), lv_t[:nnz].cpu().numpy()
    hi_req = max(2, int(spec["req_hi"] * min(1.0, args.scale * 10)))

    def make_request(size, r):
        a = int(r.integers(0, pool.n - size))
        b = a + size
        return (off[a:b + 1] - off[a], bins[off[a]:off[b]], lv[off[a]:off[b]], pool.precursor_mz[a:b],
                pool.charge[a:b])

    # setup: the autotuner picks the form and schedule the server's AUTO searches use, on one
    # request of the mean request size (latency, not the throughput of a large set, is the aim)
    t_off, t_bins, t_lv, t_mz, t_z = make_request(min(600, hi_req, pool.n - 1), np.random.default_rng(7))
    tuned, _ = hd.hd_library_autotune(lib, hd.hd_encode(ctx, dev(t_off), dev(t_bins), dev(t_lv)), dev(t_mz),
                                      dev(t_z), None, [(spec["tol"], spec["unit"])], k)
    srv = hd.Server(ctx, lib, k=k, slots=3, max_batch_queries=16384)

    # warm-up: a few requests of each size class
    wr = np.random.default_rng(1)
    for s in (1, 100, 1000, 5000):
        s = min(s, hi_req, pool.n - 1)
        srv.wait(srv.submit(*make_request(s, wr), spec["tol"], spec["unit"]))
    loads = []
    launches0 = hd.hd_launch_count()
    clocks = ClockSampler(0)
    clocks.__enter__()
    for lam in (50, 100, 200, 500, 1000, 2000):
        r = np.random.default_rng(100 + lam)
        n_req = int(min(2000, max(100, lam * 6 * min(1.0, args.scale * 10))))
        sizes = synth.batch_sizes(n_req, spec["req_lo"], hi_req, r)
        reqs = [make_request(int(s), r) for s in sizes]
        gaps = r.exponential(1.0 / lam, n_req)
        arrivals = np.cumsum(gaps) - gaps[0]
        ids = [None] * n_req
        t0 = time.perf_counter()

        def submitter():
            for j in range(n_req):
                delay = t0 + arrivals[j] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                ids[j] = srv.submit(*reqs[j], spec["tol"], spec["unit"])

        st0 = srv.stats()
        th = threading.Thread(target=submitter)
        th.start()
        lat, qn = [], 0
        for j in range(n_req):
            while ids[j] is None:
                time.sleep(0.0002)
            _, _, info = srv.wait(ids[j])
            lat.append(info["latency_s"])
            qn += info["n_queries"]
        t_end = time.perf_counter()
        th.join()
        st1 = srv.stats()
        lat_ms = np.asarray(lat) * 1e3
        loads.append({"offered_req_per_s": lam, "requests": n_req, "queries": qn,
                      "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                      "mean_ms": float(lat_ms.mean()), "completed_req_per_s": n_req / (t_end - t0),
                      "queries_per_s": qn / (t_end - t0), "batches": st1["batches"] - st0["batches"],
                      "max_inflight_batches": st1["max_inflight"]})
        print(json.dumps({"load": loads[-1]}), file=sys.stderr, flush=True)
    clocks.__exit__(None, None, None)
    launches = hd.hd_launch_count() - launches0
    srv.close()
    best = max(l["queries_per_s"] for l in loads)
    line = {"metric": "serving: sustained queries/s and p50/p99 request latency under Poisson load, D=8192, +-500",
            "value": best, "unit": "queries/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e2m1", "data": "synthetic",
            "config": {"workload": f"{n_r}-reference resident library, requests of {spec['req_lo']}..{hi_req} "
                                   "spectra (log-uniform), Poisson arrivals", "dim": D, "k": k,
                       "server": {"slots": 3, "max_batch_queries": 16384, "form": "auto",
                                  "autotune_choice": tuned, "autotuned_on": "one request of 600 spectra"}},
            "loads": loads, "gpu_launches": launches, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- cascade
def run_cascade(args):
    """Cascade search with target-decoy FDR on the 1,000,000-reference library
    (half decoys) and 50,000 queries, D=8192: 20 ppm first, then +-500 Da for
    the queries not identified at 1% FDR.  A step = encode the queries + the
    whole cascade (both searches, q-values, compaction, one read-back of the
    survivor count).  One JSON line: queries/s, identifications per level."""
    import torch
    from paper_2211_16422_gb300 import build, hd
    build.build()
    refs, queries, spec = workload(args.scale, 0)
    D, Q = spec["dim"], spec["n_levels"]
    levels, fdr = [(20.0, "ppm"), (500.0, "da")], 0.01
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32
                                     else np.ascontiguousarray(a)).cuda()
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=0)
    bits = args.bits
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp_args(spec))
    if bits:   # multi-bit components (Section 4.3), SSMs ranked by the dot product
        r_comp = hd.hd_encode_multibit(ctx, *r_csr, bits)
        lib = hd.hd_build_library_multibit(ctx, r_comp, dev(refs.precursor_mz), dev(refs.charge), bits)
        del r_comp
        cform = ("tc_mxf4" if D % 256 == 0 else "tc_fp4") if bits <= 3 else "tc_fp8"
    else:
        r_hv = hd.hd_encode(ctx, *r_csr)
        lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
        del r_hv
        hd.hd_library_prepare(lib, "tc_fp4")
        cform = "tc_mxf4" if D % 256 == 0 else "tc_fp4"   # kind::mxf4 on the e2m1 rows
    del r_csr
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    q_csr = hd.hd_preprocess(ctx, dev(queries.offsets), dev(queries.mz), dev(queries.intensity), **pp_args(spec))
    q_mz, q_z = dev(queries.precursor_mz), dev(queries.charge)
    nq = queries.n
    if bits:
        q_comp = torch.empty((nq, D), dtype=torch.int8, device="cuda")

        def step():
            hd.hd_encode_multibit(ctx, *q_csr, bits, out=q_comp)
            return hd.hd_cascade_search_dot(lib, q_comp, q_mz, q_z, levels, fdr, form=cform)
    else:
        q_hv = torch.empty((nq, D // 64), dtype=torch.int64, device="cuda")

        def step():
            hd.hd_encode(ctx, *q_csr, out=q_hv)
            return hd.hd_cascade_search(lib, q_hv, q_mz, q_z, levels, fdr, form=cform)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    lib.status()
    hd.hd_profile_enable(True)
    launches0 = hd.hd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        ev0.record()
        for _ in range(args.steps):
            out = step()
        ev1.record()
        torch.cuda.synchronize()
    launches = hd.hd_launch_count() - launches0
    hd.hd_profile_enable(False)
    search_ms, search_n = hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
    lib.status()
    ms = ev0.elapsed_time(ev1) / args.steps
    level = out[3].cpu().numpy()
    ident = [int((level == i).sum()) for i in range(len(levels))]
    kind = f", {bits}-bit components scored by the dot product" if bits else ""
    line = {"metric": "cascade search queries/s (20 ppm, then +-500 Da for the unidentified; 1% FDR per level), "
                      "D=8192" + kind,
            "value": nq / (ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_OF_FORM.get(cform, "e2m1"),
            "data": "synthetic (seeded generator; decoys are targets with repositioned fragments)",
            "config": {"workload": f"{refs.n}-reference library (50% decoys) x {nq} queries, D={D}, Q={Q}, "
                                   "levels 20 ppm / +-500 Da, top-1, FDR 1%" + kind, "form": cform,
                       "l2": "library and query set exceed L2: no flush needed"},
            "identified_per_level": ident, "identified_fraction": sum(ident) / nq,
            "search_ms_per_step": search_ms / args.steps, "search_launches_per_step": search_n / args.steps,
            "gpu_launches": launches, "clocks": clocks.summary(), "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_multibit(args):
    """Multi-bit HV components (Section 4.3) on the headline workload: the
    1,000,000 references encoded once with `--bits` bits per component and
    kept as e2m1 (bits <= 3) or e4m3; a step encodes the 50,000 queries and
    runs the windowed dot-product top-5 search.  One JSON line: in-window
    comparisons/s, with the search kernel's roofline and the oracle's
    dot-product search as the CPU baseline."""
    import torch
    from paper_2211_16422_gb300 import build, hd
    build.build()
    bits = args.bits or 3
    refs, queries, spec = workload(args.scale, 0)
    D, Q, k, tol, unit = spec["dim"], spec["n_levels"], spec["k"], spec["tol"], spec["unit"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32
                                     else np.ascontiguousarray(a)).cuda()
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=0)
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp_args(spec))
    r_comp = hd.hd_encode_multibit(ctx, *r_csr, bits)
    lib = hd.hd_build_library_multibit(ctx, r_comp, dev(refs.precursor_mz), dev(refs.charge), bits)
    del r_comp
    q_csr = hd.hd_preprocess(ctx, dev(queries.offsets), dev(queries.mz), dev(queries.intensity), **pp_args(spec))
    tuned = None
    if args.form == "auto" and not args.schedule:
        # the autotuner picks form and schedule on a second batch of the same recipe
        tq = tuning_queries(refs, queries.n, 0)
        tq_comp = hd.hd_encode_multibit(ctx, *hd.hd_preprocess(ctx, dev(tq.offsets), dev(tq.mz), dev(tq.intensity),
                                                               **pp_args(spec)), bits)
        tuned, _ = hd.hd_library_autotune(lib, tq_comp, dev(tq.precursor_mz), dev(tq.charge), None, [(tol, unit)], k)
        del tq_comp
        form = tuned["form"]
        sched = {key: tuned[key] for key in SCHEDULE_KEYS}
    else:
        form = args.form if args.form != "auto" else ("tc_mxf4" if bits <= 3 else "tc_fp8")
        hd.hd_library_prepare(lib, form)
        sched = parse_schedule(args.schedule) if args.schedule else dict(DEFAULT_SCHEDULE)
    apply_schedule(hd, lib, sched)
    q_mz, q_z = dev(queries.precursor_mz), dev(queries.charge)
    lo, hi = hd.hd_query_windows(lib, q_mz, q_z, tol, unit)
    comparisons = int((hd.as_u32(hi).astype(np.int64) - hd.as_u32(lo).astype(np.int64)).sum())
    nq = queries.n
    q_comp = torch.empty((nq, D), dtype=torch.int8, device="cuda")
    out_idx = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    out_score = torch.empty((nq, k), dtype=torch.int32, device="cuda")

    def step():
        hd.hd_encode_multibit(ctx, *q_csr, bits, out=q_comp)
        hd.hd_search_dot(lib, q_comp, q_mz, q_z, tol, unit, k, form, out_idx=out_idx, out_score=out_score)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.status()
    lib.status()
    hd.hd_profile_enable(True)
    launches0 = hd.hd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    launches = hd.hd_launch_count() - launches0
    hd.hd_profile_enable(False)
    search_ms, search_n = hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
    encode_ms, _ = hd.hd_profile_collect(hd.HD_KERNEL_ENCODE)
    ctx.status()
    lib.status()
    ms = ev0.elapsed_time(ev1) / args.steps
    avg_search_ms = search_ms / max(1, search_n)
    if form == "popc":
        pk, pclk = measure_peaks(hd, ("popc", "lop3"))
        roofline = popc_mb_roofline(comparisons, D, bits, avg_search_ms, pk)
    else:
        pk, pclk = measure_peaks(hd, (form,))
        roofline = tensor_roofline(form, comparisons, D, avg_search_ms, pk, pclk, sched)
    roofline.update({"traffic": None, "avg_launch_ms": avg_search_ms, "launches": search_n,
                     "step_share": search_ms / (ms * args.steps)})
    cpu = None
    if not args.no_cpu_baseline:
        per_step, threads, sample, cstep = cpu_oracle_rate(refs, queries, spec, args.cpu_seconds, bits=bits)
        tot_c, tot_t, off = 0, 0.0, 0
        while tot_t < args.cpu_seconds:
            c_, t_ = cstep(per_step, off)
            tot_c, tot_t, off = tot_c + c_, tot_t + t_, off + per_step
        cpu = {"value": tot_c / tot_t, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": tot_t}
    line = {"metric": f"in-window comparisons/s, dot-product search over {bits}-bit HV components (Section 4.3)",
            "value": comparisons / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_OF_FORM.get(form, "e4m3"), "data": "synthetic (seeded generator)",
            "config": {"workload": f"{refs.n}-reference library x {nq} queries, D={D}, {bits}-bit components "
                                   f"(|h| <= {2 ** (bits - 1) - 1}), +-500 open window, top-5", "form": form,
                       "schedule": sched, "autotuned_on": "a second seeded query batch" if tuned else None,
                       "l2": "library and query set exceed L2: no flush needed"},
            "queries_per_s": nq / (ms / 1e3), "comparisons_per_step": comparisons,
            "kernel_ms_per_step": {"search": search_ms / args.steps, "encode": encode_ms / args.steps},
            "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores (the paper publishes no
    code; its method's plain CPU restatement is the reference)."""
    if rank != 0:
        return
    refs, queries, spec = workload(args.scale, 0)
    per_step, threads, sample, cstep = cpu_oracle_rate(refs, queries, spec, target_s=8.0)
    off = 0
    for _ in range(args.warmup):
        cstep(per_step, off)
        off += per_step
    tot_c, tot_t = 0, 0.0
    for _ in range(args.steps):
        c_, t_ = cstep(per_step, off)
        tot_c, tot_t, off = tot_c + c_, tot_t + t_, off + per_step
    v = tot_c / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config_of(spec, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "cascade":
        run_cascade(args)
    elif args.workload == "multibit":
        run_multibit(args)
    elif args.workload == "peaks":
        run_peaks(args)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
