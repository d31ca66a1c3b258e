"""Tensor-core search forms (tcgen05, +-1 operands, fp32 accumulation) against
the oracle and the popcount form: identical distances and indices.

Exactness argument: products are +-1 and every partial sum is an integer of
magnitude <= D < 2^24.  The adversarial cases below put the accumulator near
+-D (near-duplicates and complements) where a narrower internal accumulator
would lose low bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_16422_gb300 import synth
from tests import oracle_side

pytestmark = pytest.mark.gpu
FORMS = ("tc_fp8", "tc_bf16", "tc_fp4", "tc_mxf4")


def forms_for(D):
    """The tensor-core forms that serve dimension D (kind::mxf4 needs D % 256 == 0)."""
    return tuple(f for f in FORMS if f != "tc_mxf4" or D % 256 == 0)


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


def _rand_hv(rng, n, W):
    return rng.integers(-2**63, 2**63, (n, W), dtype=np.int64).view(np.uint64)


def _search_all(hd, lib, q, qmz, qz, tol, unit, k):
    out = {}
    for form in ("popc",) + forms_for(lib.dim):
        i, d = hd.hd_search_open(lib, dev(q), dev(qmz), dev(qz), tol, unit, k, form=form)
        torch.cuda.synchronize()
        lib.status()
        out[form] = (hd.as_u32(i), hd.as_u16(d))
    return out


@pytest.mark.parametrize("D", [128, 256, 384, 768, 2048, 8192, 16384, 32768])
def test_tc_forms_small_exact(hd, D):
    rng = np.random.default_rng(D)
    W = D // 64
    n = 700
    refs = _rand_hv(rng, n, W)
    mz = rng.uniform(400, 700, n)
    z = rng.integers(1, 4, n).astype(np.uint8)
    q = refs[rng.choice(n, 150)].copy()
    # flip a few bits: near-duplicates put S close to D
    for i in range(len(q)):
        for b in rng.choice(D, int(rng.integers(0, 6)), replace=False):
            q[i, b // 64] ^= np.uint64(1) << np.uint64(b % 64)
    q[:10] = ~refs[:10]                      # complements: S = -D
    qmz = rng.uniform(400, 700, len(q))
    qz = rng.integers(1, 4, len(q)).astype(np.uint8)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(refs), dev(mz), dev(z))
    for f in forms_for(D):
        hd.hd_library_prepare(lib, f)
    if D % 256:   # kind::mxf4 reads K in 256-component stages: refused before anything runs
        with pytest.raises(hd.HDError) as e:
            hd.hd_search_open(lib, dev(q), dev(qmz), dev(qz), 500.0, "da", 5, form="tc_mxf4")
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    for k, tol, unit in ((5, 500.0, "da"), (1, 60.0, "da"), (16, 2e5, "ppm")):
        res = _search_all(hd, lib, q, qmz, qz, tol, unit, k)
        oi, od = oracle.search(D, refs, mz, z, q, qmz, qz, tol, unit, k)
        for form, (i, d) in res.items():
            assert np.array_equal(i, oi), form
            assert np.array_equal(d, od), form


def test_tc_forms_all_distances_exact(hd):
    """k = n: every candidate distance of every query compared, including the
    extremes dist = 0 and dist = D."""
    rng = np.random.default_rng(5)
    D, W, n = 8192, 128, 256
    refs = _rand_hv(rng, n, W)
    refs[1] = ~refs[0]
    refs[2] = refs[0]
    q = refs[:16].copy()
    mz, z = np.full(n, 500.0), np.full(n, 2, np.uint8)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(refs), dev(mz), dev(z))
    for f in forms_for(D):
        hd.hd_library_prepare(lib, f)
    # k is at most 16; sweep windows that each hold 16 references at a time
    for start in range(0, n, 16):
        sub_mz = mz.copy()
        sub_mz[:] = 1000.0
        sub_mz[start:start + 16] = 500.0
        lib2 = hd.hd_build_library(ctx, dev(refs), dev(sub_mz), dev(z))
        for f in forms_for(D):
            hd.hd_library_prepare(lib2, f)
        res = _search_all(hd, lib2, q, np.full(16, 500.0), np.full(16, 2, np.uint8), 0.5, "da", 16)
        oi, od = oracle.search(D, refs, sub_mz, z, q, np.full(16, 500.0), np.full(16, 2, np.uint8), 0.5, "da", 16)
        for form, (i, d) in res.items():
            assert np.array_equal(i, oi) and np.array_equal(d, od), form
    assert od.max() <= D


@pytest.mark.parametrize("D,k", [(8192, 5), (4096, 2), (12288, 8)])
def test_tc_forms_workload_exact(hd, D, k):
    rng = np.random.Generator(np.random.PCG64(D + k))
    refs = synth.make_references(6000, (1, 2, 3, 4), (0.1, 0.5, 0.3, 0.1), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, 900, rng)
    Q = 32
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 1)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    r_hv, q_hv = enc(refs), enc(qs)
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    for f in forms_for(D):
        hd.hd_library_prepare(lib, f)
    for tol, unit in ((500.0, "da"), (20.0, "ppm")):
        res = {}
        for form in ("popc",) + forms_for(D):
            i, d = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), tol, unit, k, form=form)
            torch.cuda.synchronize()
            res[form] = (hd.as_u32(i), hd.as_u16(d))
        o_r, o_q = oracle_side.hvs(refs, D, Q, 1), oracle_side.hvs(qs, D, Q, 1)
        oi, od = oracle.search(D, o_r, refs.precursor_mz, refs.charge, o_q,
                               qs.precursor_mz, qs.charge, tol, unit, k)
        for form, (i, d) in res.items():
            assert np.array_equal(i, oi), form
            assert np.array_equal(d, od), form
    lib.status()


def test_auto_prefers_prepared_tc_form(hd):
    rng = np.random.default_rng(2)
    D, W = 1024, 16
    refs = _rand_hv(rng, 100, W)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(refs), dev(rng.uniform(400, 500, 100)), dev(np.full(100, 2, np.uint8)))
    q, qm, qz = dev(refs[:5]), dev(np.full(5, 450.0)), dev(np.full(5, 2, np.uint8))
    with pytest.raises(hd.HDError):
        hd.hd_search_open(lib, q, qm, qz, 100.0, "da", 1, form="tc_fp8")   # not prepared
    i0, d0 = hd.hd_search_open(lib, q, qm, qz, 100.0, "da", 3, form="auto")
    hd.hd_library_prepare(lib, "tc_fp8")
    i1, d1 = hd.hd_search_open(lib, q, qm, qz, 100.0, "da", 3, form="auto")
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)


@pytest.mark.parametrize("tg,sg,cs,cg", [(1, 1, 1, 1), (2, 3, 1, 1), (64, 64, 1, 1), (8, 4, 1, 1), (16, 8, 1, 1),
                                         (3, 5, 1, 1), (1, 1, 2, 2), (3, 5, 2, 2), (16, 8, 2, 2), (64, 64, 2, 2),
                                         (16, 16, 2, 2), (32, 2, 2, 2)])
def test_tc_schedule_does_not_change_results(hd, tg, sg, cs, cg):
    """Work-item shape (tiles per item, groups per L2 slice) and SM pairing
    are pure performance knobs: the top-k must not move."""
    rng = np.random.Generator(np.random.PCG64(17))
    refs = synth.make_references(9000, (2, 3), (0.7, 0.3), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, 700, rng)
    D, Q, k = 2048, 16, 4
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 2)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    r_hv, q_hv = enc(refs), enc(qs)
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    hd.hd_library_prepare(lib, "tc_fp8")
    hd.hd_library_set_schedule(lib, tg, sg, cs, cg)
    i, d = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), 500.0, "da", k, form="tc_fp8")
    torch.cuda.synchronize()
    lib.status()
    o_r, o_q = oracle_side.hvs(refs, D, Q, 2), oracle_side.hvs(qs, D, Q, 2)
    oi, od = oracle.search(D, o_r, refs.precursor_mz, refs.charge, o_q,
                           qs.precursor_mz, qs.charge, 500.0, "da", k)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)


@pytest.mark.parametrize("D,k,n_q,tol,unit", [(2048, 1, 300, 500.0, "da"), (4096, 16, 257, 150.0, "da"),
                                              (8192, 5, 1, 500.0, "da"), (2048, 2, 700, 20.0, "ppm")])
def test_tc_pair_form_exact(hd, D, k, n_q, tol, unit):
    """The 2-SM form (one M = 256 tensor-core operation per SM pair) gives the
    oracle's top-k for both operand types, with ragged query blocks (257, 1)
    and narrow windows."""
    rng = np.random.Generator(np.random.PCG64(40 + k))
    refs = synth.make_references(6000, (2, 3, 4), (0.6, 0.3, 0.1), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, n_q, rng)
    Q = 16
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 5)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    lib = hd.hd_build_library(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge))
    q_hv = enc(qs)
    o_r, o_q = oracle_side.hvs(refs, D, Q, 5), oracle_side.hvs(qs, D, Q, 5)
    oi, od = oracle.search(D, o_r, refs.precursor_mz, refs.charge, o_q, qs.precursor_mz, qs.charge, tol, unit, k)
    for form in FORMS:
        hd.hd_library_prepare(lib, form)
        hd.hd_library_set_schedule(lib, 4, 2, 2, 2)
        i, d = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), tol, unit, k, form=form)
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od), form


def test_schedule_arguments_checked(hd):
    rng = np.random.default_rng(3)
    D, W, n = 2048, 32, 100
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(rng.integers(-2**63, 2**63, (n, W), dtype=np.int64)),
                              dev(rng.uniform(400, 600, n)), dev(np.full(n, 2, np.uint8)))
    # clusters of 1-SM CTAs (2, 1) and (4, 1) shared tiles by TMA multicast and are gone
    for args in [(0, 0, 3, 1), (0, 0, 0, 3), (0, 0, 4, 2), (0, 0, 1, 2), (0, 0, 2, 1), (0, 0, 4, 1), (0, 0, 4, 0),
                 (5000, 0, 0, 0)]:
        with pytest.raises(hd.HDError) as e:
            hd.hd_library_set_schedule(lib, *args)
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    hd.hd_library_set_schedule(lib, 0, 0, 0, 2)
    hd.hd_library_set_schedule(lib, 0, 0, 2, 2)
    hd.hd_library_set_schedule(lib, 0, 0, 1, 0)
    hd.hd_library_set_schedule(lib, 0, 0, 0, 1)
    hd.hd_library_set_schedule(lib, 0, 0, 1, 1)
    hd.hd_library_set_schedule(lib, 0, 0, 0, 0)


@pytest.mark.parametrize("form,tg,sg,cs,cg", [("tc_fp4", 1, 1, 1, 1), ("tc_fp4", 8, 4, 1, 1), ("tc_fp4", 3, 5, 2, 2),
                                              ("tc_fp4", 16, 16, 2, 2), ("tc_mxf4", 1, 1, 2, 2),
                                              ("tc_mxf4", 3, 5, 2, 2), ("tc_mxf4", 16, 2, 2, 2),
                                              ("tc_mxf4", 64, 64, 2, 2), ("tc_mxf4", 8, 4, 1, 1)])
def test_e2m1_schedules_exact(hd, form, tg, sg, cs, cg):
    """The e2m1 rows (4-bit operands in HBM) under kind::f8f6f4 (unpacked by
    the TMA) with the 1-SM and the SM-pair schedules, and under the
    block-scaled kind::mxf4 (kept packed; 240-row tiles, SM pairs whatever
    the schedule asks)."""
    rng = np.random.default_rng(90 + tg)
    D, n, m = 2048, 5000, 333
    refs = _rand_hv(rng, n, D // 64)
    mz = rng.uniform(400, 700, n)
    z = rng.integers(2, 4, n).astype(np.uint8)
    q = refs[:m] ^ (_rand_hv(rng, m, D // 64) & np.uint64(0x0000FFFF0000FFFF))
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(refs), dev(mz), dev(z))
    hd.hd_library_prepare(lib, form)
    hd.hd_library_set_schedule(lib, tg, sg, cs, cg)
    i, d = hd.hd_search_open(lib, dev(q), dev(mz[:m]), dev(z[:m]), 100.0, "da", 4, form=form)
    torch.cuda.synchronize()
    lib.status()
    oi, od = oracle.search(D, refs, mz, z, q, mz[:m], z[:m], 100.0, "da", 4)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)


@pytest.mark.parametrize("D,tg,sg,k,n_q,tol,unit", [(256, 1, 1, 4, 333, 100.0, "da"), (2048, 3, 5, 4, 333, 100.0, "da"),
                                                    (2048, 16, 2, 1, 257, 500.0, "da"),
                                                    (2048, 5, 16, 16, 700, 20.0, "ppm"),
                                                    (8192, 16, 2, 5, 1, 500.0, "da"),
                                                    (8192, 7, 3, 8, 513, 150.0, "da")])
def test_mxf4_two_tiles_per_stage_exact(hd, D, tg, sg, k, n_q, tol, unit):
    """kind::mxf4 with each staged query chunk scored against two reference
    tiles (both accumulators filled and drained together): odd tile groups
    leave one-tile stage runs at the end of items, blocks are ragged (257,
    513, 1 queries) and windows narrow or wide; the top-k is the oracle's and
    that of one tile per stage."""
    rng = np.random.default_rng(300 + D + tg)
    n = 7000 if D <= 2048 else 3000
    refs = _rand_hv(rng, n, D // 64)
    mz = rng.uniform(400, 700, n)
    z = rng.integers(2, 4, n).astype(np.uint8)
    src = rng.integers(0, n, n_q)
    q = refs[src] ^ (_rand_hv(rng, n_q, D // 64) & np.uint64(0x0000FFFF0000FFFF))
    qm, qz = mz[src] + rng.uniform(-1, 1, n_q), z[src]
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(refs), dev(mz), dev(z))
    hd.hd_library_prepare(lib, "tc_mxf4")
    hd.hd_library_set_schedule(lib, tg, sg, 2, 2)
    got = []
    for tps in (2, 1):
        hd.hd_library_set_stage_tiles(lib, tps)
        i, d = hd.hd_search_open(lib, dev(q), dev(qm), dev(qz), tol, unit, k, form="tc_mxf4")
        torch.cuda.synchronize()
        lib.status()
        got.append((hd.as_u32(i), hd.as_u16(d)))
    oi, od = oracle.search(D, refs, mz, z, q, qm, qz, tol, unit, k)
    assert np.array_equal(got[0][0], oi) and np.array_equal(got[0][1], od)
    assert np.array_equal(got[1][0], oi) and np.array_equal(got[1][1], od)


def test_stage_tiles_argument_checked(hd):
    rng = np.random.default_rng(4)
    D, W, n = 2048, 32, 100
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(rng.integers(-2**63, 2**63, (n, W), dtype=np.int64)),
                              dev(rng.uniform(400, 600, n)), dev(np.full(n, 2, np.uint8)))
    with pytest.raises(hd.HDError) as e:
        hd.hd_library_set_stage_tiles(lib, 3)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    for tps in (0, 1, 2):
        hd.hd_library_set_stage_tiles(lib, tps)
