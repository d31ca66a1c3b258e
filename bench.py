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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--form", default="auto")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (testing only)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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
def cpu_oracle_rate(refs, queries, spec, target_s, lib_fraction=0.05, seed=5):
    """The oracle's brute-force windowed top-k search on the host cores, on a
    uniform library sample; returns (comparisons/s, threads, sample text, step fn)."""
    import oracle
    rng = np.random.default_rng(seed)
    n_lib = max(1000, int(refs.n * lib_fraction))
    rsel = np.sort(rng.choice(refs.n, n_lib, replace=False))
    rsub = refs.subset(rsel)
    D, Q = spec["dim"], spec["n_levels"]
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    r_hv = oracle.encode(D, F, L, *oracle.preprocess(rsub.offsets, rsub.mz, rsub.intensity, **pp_args(spec)))
    threads = os.cpu_count() or 1
    q_all = queries.subset(np.arange(min(queries.n, 20000)))
    q_hv = oracle.encode(D, F, L, *oracle.preprocess(q_all.offsets, q_all.mz, q_all.intensity, **pp_args(spec)))
    wc = oracle.window_count(rsub.precursor_mz, rsub.charge, q_all.precursor_mz, q_all.charge, spec["tol"],
                             spec["unit"]).astype(np.int64)

    def step(m, offset=0):
        which = (np.arange(m) + offset) % q_all.n
        t = time.perf_counter()
        oracle.search(D, r_hv, rsub.precursor_mz, rsub.charge, q_hv, q_all.precursor_mz, q_all.charge,
                      spec["tol"], spec["unit"], spec["k"], which=which.astype(np.uint32), n_threads=threads)
        return int(wc[which].sum()), time.perf_counter() - t

    m = 256
    comps, dt = step(m)
    while dt < 1.0 and m < q_all.n:
        m = min(q_all.n, m * 4)
        comps, dt = step(m)
    per_step = max(1, min(q_all.n, int(m * max(1.0, target_s / 4) / max(dt, 1e-3))))
    sample = (f"oracle brute-force top-{spec['k']} search of {per_step} queries against a uniform "
              f"{n_lib}-reference sample ({lib_fraction:.0%}) of the library, D={D}, +-{spec['tol']:g}; "
              f"oracle encoding of the sample is setup, not timed")
    return per_step, threads, sample, step


# ---------------------------------------------------------------- our arm
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
    form = args.form if args.form != "auto" else "tc_fp8"
    if form.startswith("tc_"):
        t = time.perf_counter()
        hd.hd_library_prepare(lib, form)
        setup["prepare_" + form + "_s"] = time.perf_counter() - t
    q_mz, q_z = dev(queries.precursor_mz), dev(queries.charge)
    lo, hi = hd.hd_query_windows(lib, q_mz, q_z, tol, unit)
    comparisons = int((hd.as_u32(hi).astype(np.int64) - hd.as_u32(lo).astype(np.int64)).sum())
    nq = queries.n
    q_hv = torch.empty((nq, D // 64), dtype=torch.int64, device="cuda")
    out_idx = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    out_dist = torch.empty((nq, k), dtype=torch.int16, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        hd.hd_encode(ctx, *q_csr, out=q_hv)
        hd.hd_search_open(lib, q_hv, q_mz, q_z, tol, unit, k, form=form, out_idx=out_idx, out_dist=out_dist)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.status()
    lib.status()
    barrier()
    torch.cuda.synchronize()
    hd.hd_profile_enable(True)
    launches0 = hd.hd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = hd.hd_launch_count() - launches0
    hd.hd_profile_enable(False)
    search_ms, search_n = hd.hd_profile_collect(hd.HD_KERNEL_SEARCH)
    encode_ms, encode_n = hd.hd_profile_collect(hd.HD_KERNEL_ENCODE)
    ctx.status()
    lib.status()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist_on:
        import torch.distributed as dist
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        cc = torch.tensor([comparisons], device="cuda", dtype=torch.int64)
        dist.all_reduce(cc)
        total_comparisons = int(cc.item())
    else:
        total_comparisons = comparisons
    value = total_comparisons / (ms / 1e3)
    qps = nq * world / (ms / 1e3)

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
        t = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = (time.perf_counter() - t) / args.steps
        if dist_on:
            import torch.distributed as dist
            tt = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt.item())
        h2d = sum(t_.numel() * t_.element_size() for t_ in (h_off, h_bins, h_lv, h_mz, h_z))
        d2h = nq * k * (4 + 2)
        e2e = {"value": total_comparisons / e2e_s, "unit": UNIT, "queries_per_s": nq * world / e2e_s,
               "ms_per_step": e2e_s * 1e3, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        assert np.array_equal(h_idx.numpy(), out_idx.cpu().numpy()), "end-to-end results differ"

    if rank != 0:
        return
    cs = clocks.summary()
    props = torch.cuda.get_device_properties(local_rank)
    n_sm = props.multi_processor_count
    sm_mhz = (cs or {}).get("sm_mhz") or 1455.0
    avg_search_ms = search_ms / max(1, search_n)
    if form.startswith("tc_"):
        # dense +-1 contraction: 2*D flops per in-window comparison (masked tile
        # padding is not counted)
        peaks = measured_peaks()
        bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
        peak = bf16 * (2.0 if form == "tc_fp8" else 1.0)
        achieved = comparisons * 2.0 * D / (avg_search_ms / 1e3) / 1e12
        basis = ("measured sustained cuBLAS bf16 x 2 (nominal fp8/bf16 ratio 4.5/2.25)" if form == "tc_fp8"
                 else "measured sustained cuBLAS bf16")
        roofline = {"kernel": "k_search_mma", "bound": "tensor", "unit": "TFLOP/s", "achieved": achieved,
                    "peak": peak, "frac": achieved / peak, "peak_basis": basis + " (of measured)"}
    else:
        popc_per_launch = comparisons * (D // 32)
        achieved = popc_per_launch / (avg_search_ms / 1e3) / 1e12
        peak = n_sm * 16 * sm_mhz * 1e6 / 1e12
        roofline = {"kernel": "k_search_popc", "bound": "alu", "unit": "Tpopc32/s",
                    "achieved": achieved, "peak": peak, "frac": achieved / peak,
                    "peak_basis": f"{n_sm} SMs x 16 popc32/clk/SM x {sm_mhz:.0f} MHz median SM clock sampled"}
    roofline.update({"traffic": None, "avg_launch_ms": avg_search_ms, "launches": search_n,
                     "step_share": search_ms / (ms * args.steps)})
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
            "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded generator; stands in for the "
            "paper's MassIVE-KB/HEK293 and yeast/iPRG2012 sets)",
            "config": config_of(spec, world), "queries_per_s": qps,
            "comparisons_per_step": total_comparisons,
            "kernel_ms_per_step": {"search": search_ms / args.steps, "encode": encode_ms / args.steps},
            "setup_s": setup, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": cs, "form": form, "device": props.name}
    print(json.dumps(line))


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
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
