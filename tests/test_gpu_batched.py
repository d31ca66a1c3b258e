"""Batched uneven workload (many query batches, each with its own window:
Table 1's 20 ppm narrow search next to 150 and 500 Da open searches) through
the multi-window search, the CUDA-graph plan and the autotuner, against the
oracle answering each window class separately."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_16422_gb300 import synth
from tests import oracle_side

pytestmark = pytest.mark.gpu
WINDOWS = [(20.0, "ppm"), (150.0, "da"), (500.0, "da")]


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_16422_gb300 import build, hd as _hd
    build.build()
    return _hd


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def _batched_workload(seed, n_refs, n_batches, lo, hi):
    """Library + concatenated query batches (log-uniform sizes), class per
    query = its batch's window, round-robin over WINDOWS."""
    rng = np.random.Generator(np.random.PCG64(seed))
    spec = synth.WORKLOADS["batched"]
    refs = synth.make_references(n_refs, spec["charges"], spec["weights"], rng, decoy_fraction=0.5)
    sizes = synth.batch_sizes(n_batches, lo, hi, rng)
    qs = synth.make_queries(refs, int(sizes.sum()), rng)
    cls = np.repeat(np.arange(n_batches) % len(WINDOWS), sizes).astype(np.uint8)
    return refs, qs, cls, sizes


def _oracle_by_class(D, r_hv, refs, q_hv, qs, cls, k, which=None):
    n = qs.n
    oi = np.full((n, k), 0xFFFFFFFF, np.uint32)
    od = np.full((n, k), 0xFFFF, np.uint16)
    for c, (tol, unit) in enumerate(WINDOWS):
        idx = np.nonzero(cls == c)[0]
        if which is not None:
            idx = np.intersect1d(idx, which)
        if idx.size == 0:
            continue
        i, d = oracle.search(D, r_hv, refs.precursor_mz, refs.charge, q_hv, qs.precursor_mz, qs.charge, tol, unit,
                             k, which=idx.astype(np.uint32))
        oi[idx], od[idx] = i, d
    return oi, od


def _setup(hd, refs, qs, D, Q, seed=0):
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp)
    q_csr = hd.hd_preprocess(ctx, dev(qs.offsets), dev(qs.mz), dev(qs.intensity), **pp)
    r_hv = hd.hd_encode(ctx, *r_csr)
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    return ctx, lib, r_hv, q_csr


@pytest.mark.parametrize("D", [4096, 8192])
def test_multi_window_all_forms_exact(hd, D):
    refs, qs, cls, _ = _batched_workload(D, 8000, 12, 10, 200)
    ctx, lib, r_hv, q_csr = _setup(hd, refs, qs, D, 32)
    q_hv = hd.hd_encode(ctx, *q_csr)
    for f in ("tc_fp8", "tc_bf16", "tc_fp4"):
        hd.hd_library_prepare(lib, f)
    oi, od = _oracle_by_class(D, oracle_side.hvs(refs, D, 32, 0), refs, oracle_side.hvs(qs, D, 32, 0), qs, cls, 5)
    for form in ("popc", "tc_fp8", "tc_bf16", "tc_fp4", "tc_mxf4"):
        i, d = hd.hd_search_open_multi(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, 5,
                                       form=form)
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(i), oi), form
        assert np.array_equal(hd.as_u16(d), od), form
    # one class for everybody equals hd_search_open
    i1, d1 = hd.hd_search_open_multi(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), None, [(150.0, "da")], 3)
    i2, d2 = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), 150.0, "da", 3)
    torch.cuda.synchronize()
    assert torch.equal(i1, i2) and torch.equal(d1, d2)


def test_plan_graph_matches_eager_and_refills(hd):
    D = 4096
    refs, qs, cls, _ = _batched_workload(7, 6000, 20, 10, 300)
    ctx, lib, r_hv, q_csr = _setup(hd, refs, qs, D, 32)
    hd.hd_library_prepare(lib, "tc_fp8")
    off, bins, lv = q_csr
    nnz = int(hd.as_u32(off)[-1])
    plan = hd.Plan(ctx, lib, off, bins[:nnz], lv[:nnz], dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS,
                   k=5, form="tc_fp8")
    assert plan.kernel_nodes > 5
    for _ in range(2):
        i, d = plan.launch()
        torch.cuda.synchronize()
        lib.status()
        oi, od = _oracle_by_class(D, oracle_side.hvs(refs, D, 32, 0), refs, oracle_side.hvs(qs, D, 32, 0), qs,
                                  cls, 5)
        assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)
    # refill the bound buffers with another query set of the same shape
    rng = np.random.Generator(np.random.PCG64(99))
    qs2 = synth.make_queries(refs, qs.n, rng)
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=32)
    off2, bins2, lv2 = oracle.preprocess(qs2.offsets, qs2.mz, qs2.intensity, **pp)
    nnz2 = int(off2[-1])
    # the plan reads the CSR through its offsets: a refill may use fewer peaks
    if nnz2 <= nnz:
        plan.offsets.copy_(dev(off2))
        plan.bins[:nnz2].copy_(dev(bins2))
        plan.levels[:nnz2].copy_(dev(lv2))
        plan.q_mz.copy_(dev(qs2.precursor_mz))
        plan.q_charge.copy_(dev(qs2.charge))
        i, d = plan.launch()
        torch.cuda.synchronize()
        oi, od = _oracle_by_class(D, oracle_side.hvs(refs, D, 32, 0), refs, oracle_side.hvs(qs2, D, 32, 0), qs2,
                                  cls, 5)
        assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)


def test_autotune_keeps_results(hd):
    D = 4096
    refs, qs, cls, _ = _batched_workload(11, 12000, 9, 50, 400)
    ctx, lib, r_hv, q_csr = _setup(hd, refs, qs, D, 32)
    q_hv = hd.hd_encode(ctx, *q_csr)
    hd.hd_library_prepare(lib, "tc_fp8")
    args = (lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS)
    i0, d0 = hd.hd_search_open_multi(*args, 5, form="popc")
    best, allr = hd.hd_library_autotune(*args, 5)
    # popc, then 4 tile groups x 3 super groups x {(1, 1), (2, 2)} for the prepared e4m3 copy
    assert best["ms"] > 0 and len(allr) == 1 + 24
    assert {(r["cluster"], r["cta_group"]) for r in allr[1:]} == {(1, 1), (2, 2)}
    assert best["ms"] == min(r["ms"] for r in allr)
    i1, d1 = hd.hd_search_open_multi(*args, 5, form="auto")
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)


def test_multi_window_mixed_units_exact(hd):
    """Window classes mixing m/z (Da, ppm) and neutral-mass tolerances in one
    launch give, per class, the oracle's top-k for that window."""
    windows = [(20.0, "ppm"), (300.0, "mass"), (150.0, "da"), (1000.0, "mass")]
    D = 2048
    rng = np.random.Generator(np.random.PCG64(77))
    spec = synth.WORKLOADS["batched"]
    refs = synth.make_references(6000, spec["charges"], spec["weights"], rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, 900, rng)
    cls = (np.arange(qs.n) % len(windows)).astype(np.uint8)
    ctx, lib, r_hv, q_csr = _setup(hd, refs, qs, D, 16)
    q_hv = hd.hd_encode(ctx, *q_csr)
    hd.hd_library_prepare(lib, "tc_fp8")
    o_r, o_q = oracle_side.hvs(refs, D, 16, 0), oracle_side.hvs(qs, D, 16, 0)
    oi = np.full((qs.n, 4), 0xFFFFFFFF, np.uint32)
    od = np.full((qs.n, 4), 0xFFFF, np.uint16)
    for c, (tol, unit) in enumerate(windows):
        idx = np.nonzero(cls == c)[0].astype(np.uint32)
        oi[idx], od[idx] = oracle.search(D, o_r, refs.precursor_mz, refs.charge, o_q, qs.precursor_mz, qs.charge,
                                         tol, unit, 4, which=idx)
    for form in ("popc", "tc_fp8"):
        i, d = hd.hd_search_open_multi(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), windows, 4,
                                       form=form)
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(i), oi), form
        assert np.array_equal(hd.as_u16(d), od), form


def test_batched_full_size_sampled(hd):
    """The benchmark's batched workload at full size (2,000,000 references, 200
    batches, 445,653 queries, D=4096) through the CUDA-graph plan with e2m1 SM
    pairs: every query equals the popcount form (an independent GPU path),
    and a seeded sample of 20 ppm queries equals the oracle, which encodes
    only those queries' candidate references."""
    spec = synth.WORKLOADS["batched"]
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    refs = synth.make_references(spec["n_refs"], spec["charges"], spec["weights"], rng,
                                 decoy_fraction=spec["decoy_fraction"])
    sizes = synth.batch_sizes(spec["n_batches"], spec["batch_lo"], spec["batch_hi"], rng)
    qs = synth.make_queries(refs, int(sizes.sum()), rng)
    windows = [(t, u) for t, u in spec["windows"]]
    assert windows == WINDOWS
    cls = np.repeat(np.arange(len(sizes)) % len(windows), sizes).astype(np.uint8)
    D, Q, k = 4096, spec["n_levels"], spec["k"]
    ctx, lib, r_hv, q_csr = _setup(hd, refs, qs, D, Q)
    del r_hv
    hd.hd_library_prepare(lib, "tc_fp4")
    nnz = int(hd.as_u32(q_csr[0])[-1])
    q_mz, q_z, q_cls = dev(qs.precursor_mz), dev(qs.charge), dev(cls)
    plan = hd.Plan(ctx, lib, q_csr[0], q_csr[1][:nnz], q_csr[2][:nnz], q_mz, q_z, q_cls, windows, k=k,
                   form="tc_fp4")
    pi, pd = plan.launch()
    torch.cuda.synchronize()
    lib.status()
    pi, pd = hd.as_u32(pi).copy(), hd.as_u16(pd).copy()
    ci, cd = hd.hd_search_open_multi(lib, plan.q_hv, q_mz, q_z, q_cls, windows, k, form="popc")
    torch.cuda.synchronize()
    lib.status()
    assert np.array_equal(pi, hd.as_u32(ci)) and np.array_equal(pd, hd.as_u16(cd))
    mi, md = hd.hd_search_open_multi(lib, plan.q_hv, q_mz, q_z, q_cls, windows, k, form="tc_mxf4")
    torch.cuda.synchronize()
    lib.status()
    assert np.array_equal(pi, hd.as_u32(mi)) and np.array_equal(pd, hd.as_u16(md))
    # oracle on sampled 20 ppm queries: their candidates are few, so only those references are encoded
    s_rng = np.random.default_rng(31)
    which = np.sort(s_rng.choice(np.nonzero(cls == 0)[0], 300, replace=False))
    tol_q = qs.precursor_mz[which] * (20.0 * 1e-6)
    cand = set()
    order = np.argsort(refs.precursor_mz, kind="stable")
    mz_sorted = refs.precursor_mz[order]
    for j, q in enumerate(which):
        a = np.searchsorted(mz_sorted, qs.precursor_mz[q] - tol_q[j] - 1e-6, "left")
        b = np.searchsorted(mz_sorted, qs.precursor_mz[q] + tol_q[j] + 1e-6, "right")
        cand.update(order[a:b].tolist())
    sub_idx = np.array(sorted(cand), dtype=np.int64)
    sub = refs.subset(sub_idx)
    r_np = oracle_side.hvs(sub, D, Q, 0)
    q_sub = qs.subset(which)
    q_np = oracle_side.hvs(q_sub, D, Q, 0)
    oi, od = oracle.search(D, r_np, sub.precursor_mz, sub.charge, q_np, q_sub.precursor_mz, q_sub.charge,
                           20.0, "ppm", k)
    oi_g = np.where(oi == 0xFFFFFFFF, 0xFFFFFFFF, sub_idx[np.minimum(oi, sub_idx.size - 1)]).astype(np.uint32)
    assert np.array_equal(pi[which], oi_g) and np.array_equal(pd[which], od)
    assert np.mean(oi[:, 0] != 0xFFFFFFFF) > 0.5


# ------------------------------------------------ multi-bit components (Section 4.3)
def _oracle_dot_by_class(r_comp, refs, q_comp, qs, cls, k):
    n = qs.n
    oi = np.full((n, k), 0xFFFFFFFF, np.uint32)
    osc = np.full((n, k), np.iinfo(np.int32).min, np.int32)
    for c, (tol, unit) in enumerate(WINDOWS):
        idx = np.nonzero(cls == c)[0]
        if idx.size == 0:
            continue
        i, s = oracle.search_dot(r_comp, refs.precursor_mz, refs.charge, q_comp, qs.precursor_mz, qs.charge, tol,
                                 unit, k, which=idx.astype(np.uint32))
        oi[idx], osc[idx] = i, s
    return oi, osc


def _setup_mb(hd, refs, qs, D, Q, bits, seed=0):
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp)
    q_csr = hd.hd_preprocess(ctx, dev(qs.offsets), dev(qs.mz), dev(qs.intensity), **pp)
    lib = hd.hd_build_library_multibit(ctx, hd.hd_encode_multibit(ctx, *r_csr, bits), dev(refs.precursor_mz),
                                       dev(refs.charge), bits)
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, seed)
    o_r = oracle.encode_multibit(D, F, L, *oracle.preprocess(refs.offsets, refs.mz, refs.intensity, **pp), bits)
    o_q = oracle.encode_multibit(D, F, L, *oracle.preprocess(qs.offsets, qs.mz, qs.intensity, **pp), bits)
    return ctx, lib, q_csr, o_r, o_q, pp


@pytest.mark.parametrize("bits,forms", [(3, ("tc_mxf4", "tc_fp4", "tc_bf16", "popc")), (4, ("tc_fp8", "popc"))])
def test_multi_window_dot_exact(hd, bits, forms):
    D, Q = 2048, 32
    refs, qs, cls, _ = _batched_workload(11 + bits, 5000, 24, 10, 300)
    ctx, lib, q_csr, o_r, o_q, _ = _setup_mb(hd, refs, qs, D, Q, bits)
    q_comp = hd.hd_encode_multibit(ctx, *q_csr, bits)
    want = _oracle_dot_by_class(o_r, refs, o_q, qs, cls, 5)
    for form in forms:
        if form in ("tc_bf16", "popc"):
            hd.hd_library_prepare(lib, form)
        i, s = hd.hd_search_dot_multi(lib, q_comp, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, k=5,
                                      form=form)
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(i), want[0]), form
        assert np.array_equal(s.cpu().numpy(), want[1]), form
    # without classes every query takes windows[0]
    i, s = hd.hd_search_dot_multi(lib, q_comp, dev(qs.precursor_mz), dev(qs.charge), None, [(150.0, "da")], k=2)
    torch.cuda.synchronize()
    oi, osc = oracle.search_dot(o_r, refs.precursor_mz, refs.charge, o_q, qs.precursor_mz, qs.charge, 150.0, "da", 2)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(s.cpu().numpy(), osc)


def test_plan_dot_matches_oracle_and_refills(hd):
    D, Q, bits = 4096, 32, 3
    refs, qs, cls, _ = _batched_workload(17, 6000, 20, 10, 300)
    ctx, lib, q_csr, o_r, o_q, pp = _setup_mb(hd, refs, qs, D, Q, bits)
    off, b, lv = q_csr       # bins / levels hold n * max_peaks entries: room for any refill
    plan = hd.Plan(ctx, lib, off, b, lv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, k=5)
    assert plan.multibit and plan.kernel_nodes > 5
    want = _oracle_dot_by_class(o_r, refs, o_q, qs, cls, 5)
    for _ in range(2):
        i, s = plan.launch()
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(i), want[0]) and np.array_equal(s.cpu().numpy(), want[1])
    assert np.array_equal(plan.q_comp.cpu().numpy(), o_q)     # the plan's own multi-bit encode
    hd.hd_library_prepare(lib, "popc")                           # the popcount form in a plan of its own
    pplan = hd.Plan(ctx, lib, off, b, lv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, k=5, form="popc")
    i, s = pplan.launch()
    torch.cuda.synchronize()
    lib.status()
    assert np.array_equal(hd.as_u32(i), want[0]) and np.array_equal(s.cpu().numpy(), want[1])
    pplan.close()
    rng = np.random.Generator(np.random.PCG64(98))
    qs2 = synth.make_queries(refs, qs.n, rng)
    off2, bins2, lv2 = oracle.preprocess(qs2.offsets, qs2.mz, qs2.intensity, **pp)
    nnz2 = int(off2[-1])
    plan.offsets.copy_(dev(off2))
    plan.bins[:nnz2].copy_(dev(bins2))
    plan.levels[:nnz2].copy_(dev(lv2))
    plan.q_mz.copy_(dev(qs2.precursor_mz))
    plan.q_charge.copy_(dev(qs2.charge))
    i, s = plan.launch()
    torch.cuda.synchronize()
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    o_q2 = oracle.encode_multibit(D, F, L, off2, bins2, lv2, bits)
    want2 = _oracle_dot_by_class(o_r, refs, o_q2, qs2, cls, 5)
    assert np.array_equal(hd.as_u32(i), want2[0]) and np.array_equal(s.cpu().numpy(), want2[1])


def test_multibit_batched_argument_errors(hd):
    D, Q = 1024, 8
    refs, qs, cls, _ = _batched_workload(23, 600, 4, 5, 20)
    ctx, lib, q_csr, o_r, o_q, _ = _setup_mb(hd, refs, qs, D, Q, 3)
    off, b, lv = q_csr
    q_hv = dev(np.zeros((qs.n, D // 64), np.uint64))
    with pytest.raises(hd.HDError) as e:       # the binary multi-window search refuses a multi-bit library
        hd.hd_search_open_multi(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    q_comp = hd.hd_encode_multibit(ctx, *q_csr, 3)
    for kw in (dict(form="popc"), dict(form="tc_bf16"), dict(k=0), dict(k=17)):
        with pytest.raises(hd.HDError) as e:
            hd.hd_search_dot_multi(lib, q_comp, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, **kw)
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    blib = hd.hd_build_library(ctx, dev(np.zeros((refs.n, D // 64), np.uint64)), dev(refs.precursor_mz),
                               dev(refs.charge))
    with pytest.raises(hd.HDError) as e:       # the dot search refuses a binary library
        hd.hd_search_dot_multi(blib, q_comp, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS)
    assert e.value.status == hd.HD_ERR_INVALID_ARG


def test_autotune_dot_keeps_results(hd):
    """The multi-bit autotuner: mxf4 pairs (12 schedules, each with one and
    with two reference tiles per query stage) and e2m1 (24) for a 3-bit
    library; the chosen form and schedule serve AUTO in the dot search and in
    a multi-bit plan, with the oracle's results."""
    D, Q, bits = 2048, 32, 3
    refs, qs, cls, _ = _batched_workload(29, 8000, 9, 50, 400)
    ctx, lib, q_csr, o_r, o_q, _ = _setup_mb(hd, refs, qs, D, Q, bits)
    q_comp = hd.hd_encode_multibit(ctx, *q_csr, bits)
    args = (lib, q_comp, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS)
    best, allr = hd.hd_library_autotune(*args, 5)
    forms = [r["form"] for r in allr]
    assert forms.count("tc_mxf4") == 24 and forms.count("tc_fp4") == 24 and len(allr) == 48
    assert all((r["cluster"], r["cta_group"]) == (2, 2) for r in allr if r["form"] == "tc_mxf4")
    assert sorted(r["tiles_per_stage"] for r in allr if r["form"] == "tc_mxf4") == [1] * 12 + [2] * 12
    assert all(r["tiles_per_stage"] == 1 for r in allr if r["form"] == "tc_fp4")
    assert best["ms"] == min(r["ms"] for r in allr) and best["form"] in ("tc_mxf4", "tc_fp4")
    want = _oracle_dot_by_class(o_r, refs, o_q, qs, cls, 5)
    i, s = hd.hd_search_dot_multi(*args, 5, form="auto")
    torch.cuda.synchronize()
    assert np.array_equal(hd.as_u32(i), want[0]) and np.array_equal(s.cpu().numpy(), want[1])
    off, b, lv = q_csr
    plan = hd.Plan(ctx, lib, off, b, lv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, k=5)
    i, s = plan.launch()
    torch.cuda.synchronize()
    lib.status()
    assert np.array_equal(hd.as_u32(i), want[0]) and np.array_equal(s.cpu().numpy(), want[1])
    blib = hd.hd_build_library(ctx, dev(np.zeros((refs.n, D // 64), np.uint64)), dev(refs.precursor_mz),
                               dev(refs.charge))
    q_hv = dev(np.zeros((qs.n, D // 64), np.uint64))
    with pytest.raises(hd.HDError) as e:       # a binary library without a tensor-core copy is tuned as binary
        hd.hd_search_dot_multi(blib, q_comp, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    best_b, allr_b = hd.hd_library_autotune(blib, q_hv, dev(qs.precursor_mz), dev(qs.charge), dev(cls), WINDOWS, 5)
    assert [r["form"] for r in allr_b] == ["popc"]
