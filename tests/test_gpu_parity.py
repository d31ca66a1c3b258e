"""GPU path (through the C ABI) against the CPU oracle, element by element.

Integer and bit results must be identical: item memory, CSR spectrum
vectors, hypervectors, library order, windows, distances and top-k indices.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2211_16422_gb300 import synth
from tests import oracle_side

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def pp_args(n_levels, bin_width=synth.BIN_WIDTH, max_peaks=synth.MAX_PEAKS, n_bins=synth.N_BINS):
    return dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=bin_width, n_bins=n_bins,
                max_peaks=max_peaks, n_levels=n_levels)


def gpu_csr(hd, ctx, sp, **pp):
    off, b, lv = hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp)
    torch.cuda.synchronize()
    return off, b, lv


def host_csr(hd, csr):
    off, b, lv = csr
    o = hd.as_u32(off)
    n = int(o[-1])
    return o, hd.as_u32(b[:n]) if n else np.zeros(0, np.uint32), lv[:n].cpu().numpy()


# ------------------------------------------------------------ item memory
@pytest.mark.parametrize("D,Q,f,alpha,seed", [(2048, 16, synth.N_BINS, 1024, 0), (8192, 32, synth.N_BINS, 4096, 7),
                                              (384, 3, 5, 384, 123), (128, 2, 1, 0, 1)])
def test_item_memory_bit_exact(hd, D, Q, f, alpha, seed):
    ctx = hd.Ctx(D, Q, f, alpha, seed)
    F, L, rF, rL = hd.hd_ctx_item_memory(ctx)
    torch.cuda.synchronize()
    oF, oL, orF, orL = oracle.item_memory(D, Q, f, alpha, seed)
    assert np.array_equal(hd.as_u32(rF), orF)
    assert np.array_equal(hd.as_u32(rL), orL)
    assert np.array_equal(hd.as_u64(F), oF)
    assert np.array_equal(hd.as_u64(L), oL)


@pytest.mark.parametrize("seed,stream,n", [(0, 0, 4_000_000), (0x0123456789ABCDEF, 3, 4_000_000),
                                           (2**64 - 1, 5, 1_000_003), (7, 1, 1)])
def test_philox_word_stream_bit_exact(hd, seed, stream, n):
    """The GPU's Philox4x32-10 word stream (the item memory's random words)
    equals the oracle's, written independently, on 10^6 counters; the first
    block of stream 0 under seed 0 is the first Random123 known-answer vector."""
    got = hd.as_u32(hd.hd_random_words(seed, stream, n))
    want = oracle.random_words(seed, stream, n)
    assert np.array_equal(got, want)
    if seed == 0 and stream == 0:
        assert [int(x) for x in got[:4]] == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]


# ---------------------------------------------------------- preprocessing
@pytest.mark.parametrize("n_levels,bin_width,max_peaks", [(16, 0.05, 50), (32, 0.04, 50), (256, 0.05, 3),
                                                          (2, 0.05, 1023)])
def test_preprocess_bit_exact(hd, n_levels, bin_width, max_peaks):
    n_bins = int(np.floor((synth.MZ_MAX - synth.MZ_MIN) / bin_width)) + 1
    rng = np.random.Generator(np.random.PCG64(11))
    refs, qs, _ = synth.make_workload("tiny", scale=0.4)
    soup = synth.raw_peak_soup(300, rng, max_len=1200)
    ctx = hd.Ctx(128, n_levels, n_bins, 64, 0)
    pp = pp_args(n_levels, bin_width, max_peaks, n_bins)
    for sp in (refs, qs, soup):
        got = host_csr(hd, gpu_csr(hd, ctx, sp, **pp))
        want = oracle.preprocess(sp.offsets, sp.mz, sp.intensity, **pp)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
    ctx.status()


# ---------------------------------------------------------------- encode
def _random_csr(rng, n, n_bins, n_levels, lens):
    lens = np.asarray(lens)
    off = np.zeros(n + 1, np.uint32)
    off[1:] = np.cumsum(lens[:n])
    nnz = int(off[-1])
    return off, rng.integers(0, n_bins, nnz).astype(np.uint32), rng.integers(0, n_levels, nnz).astype(np.uint8)


@pytest.mark.parametrize("D,f,Q", [(128, 50, 4), (2048, synth.N_BINS, 16), (8192, 3000, 32), (12288, 700, 16),
                                   (32768, 300, 256)])
def test_encode_bit_exact(hd, D, f, Q):
    rng = np.random.default_rng(D)
    special = [0, 1, 2, 3, 4, 5, 11, 12, 49, 50, 51, 150, 1023]
    n = 200 if D <= 8192 else 40
    lens = special + list(rng.integers(0, 160, n - len(special)))
    off, b, lv = _random_csr(rng, n, f, Q, lens)
    ctx = hd.Ctx(D, Q, f, D // 2, 5)
    got = hd.hd_encode(ctx, dev(off), dev(b), dev(lv))
    torch.cuda.synchronize()
    ctx.status()
    F, L, _, _ = oracle.item_memory(D, Q, f, D // 2, 5)
    assert np.array_equal(hd.as_u64(got), oracle.encode(D, F, L, off, b, lv))


def _drop_peaks(off, b, lv, keep):
    """CSR rows without the peaks where keep is False."""
    n = len(off) - 1
    row = np.repeat(np.arange(n), np.diff(off.astype(np.int64)))
    cnt = np.bincount(row[keep], minlength=n)
    o = np.zeros(len(off), np.uint32)
    o[1:] = np.cumsum(cnt)
    return o, b[keep], lv[keep]


@pytest.mark.parametrize("D,f,Q", [(128, 50, 4), (2048, 3000, 16), (8192, 3000, 32), (12288, 700, 16)])
def test_encode_skips_bad_peaks(hd, D, f, Q):
    """A peak whose bin or level is out of range is left out of its row's
    bundle (Eq. 1 over the remaining peaks) and flags the status; a row over
    1023 peaks encodes as an empty row.  Bad peaks sit at chunk starts and
    ends and inside full 16-peak groups."""
    rng = np.random.default_rng(D + 7)
    lens = [1, 2, 16, 17, 31, 32, 33, 48, 50, 64, 65, 100, 1023, 1024] + list(rng.integers(0, 130, 60))
    off, b, lv = _random_csr(rng, len(lens), f, Q, lens)
    nnz = len(b)
    bad_b = np.zeros(nnz, bool)
    bad_l = np.zeros(nnz, bool)
    bad_b[rng.choice(nnz, nnz // 40, replace=False)] = True
    bad_l[rng.choice(nnz, nnz // 40, replace=False)] = True
    starts = off[:-1][np.diff(off) > 0].astype(np.int64)
    bad_b[starts[::3]] = True                      # first peak of some rows
    bad_l[(off[1:][np.diff(off) > 0] - 1)[::4].astype(np.int64)] = True   # last peak of others
    b = np.where(bad_b, f + rng.integers(0, 4, nnz), b).astype(np.uint32)
    lv = np.where(bad_l, Q + rng.integers(0, 2, nnz), lv).astype(np.uint8) if Q < 255 else lv
    keep = ~(bad_b | (lv >= Q))
    row_len = np.diff(off.astype(np.int64))
    too_long = np.repeat(row_len > 1023, row_len)
    keep &= ~too_long                              # an over-long row encodes as empty
    want_off, want_b, want_lv = _drop_peaks(off, b, lv, keep)
    F, L, _, _ = oracle.item_memory(D, Q, f, D // 2, 5)
    ctx = hd.Ctx(D, Q, f, D // 2, 5)
    got = hd.hd_encode(ctx, dev(off), dev(b), dev(lv))
    torch.cuda.synchronize()
    with pytest.raises(hd.HDError) as e:
        ctx.status()
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    assert np.array_equal(hd.as_u64(got), oracle.encode(D, F, L, want_off, want_b, want_lv))
    for bits in (2, 3):
        got = hd.hd_encode_multibit(ctx, dev(off), dev(b), dev(lv), bits)
        torch.cuda.synchronize()
        with pytest.raises(hd.HDError):
            ctx.status()
        want = oracle.encode_multibit(D, F, L, want_off, want_b, want_lv, bits)
        assert np.array_equal(got.cpu().numpy(), want), bits
    ctx.status()   # cleared


# --------------------------------------------------------------- library
def _refs_with_ties(rng, n):
    mz = np.round(rng.uniform(400, 420, n), 1)
    mz[:3] = [0.0, -0.0, 0.0][:min(3, n)]
    z = rng.integers(0, 6, n).astype(np.uint8)
    hv = rng.integers(-2**63, 2**63, (n, 4), dtype=np.int64).view(np.uint64)
    return hv, mz, z


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 4095, 4096, 4097, 20000])
def test_library_order_and_rows(hd, n):
    """Sorted rows against the oracle's order, through the one-CTA sort (up to
    4096 rows) and the radix passes (above), with equal m/z values and +-0.0."""
    rng = np.random.default_rng(3 + n)
    hv, mz, z = _refs_with_ties(rng, n)
    ctx = hd.Ctx(256, 4, 10, 128, 0)
    lib = hd.hd_build_library(ctx, dev(hv), dev(mz), dev(z))
    s_hv, s_mz, s_z, s_orig = hd.hd_library_export(lib)
    torch.cuda.synchronize()
    order = oracle.library_order(mz, z)
    assert np.array_equal(hd.as_u32(s_orig), order)
    assert np.array_equal(hd.as_u64(s_hv), hv[order])
    assert np.array_equal(s_z.cpu().numpy(), z[order])
    assert np.array_equal(s_mz.cpu().numpy().view(np.uint64), mz[order].view(np.uint64))


def test_library_rejects_nan_mz(hd):
    ctx = hd.Ctx(128, 4, 10, 64, 0)
    mz = np.array([500.0, np.nan, 600.0])
    with pytest.raises(hd.HDError) as e:
        hd.hd_build_library(ctx, dev(np.zeros((3, 2), np.uint64)), dev(mz), dev(np.full(3, 2, np.uint8)))
    assert e.value.status == hd.HD_ERR_INVALID_ARG


# --------------------------------------------------------------- windows
@pytest.mark.parametrize("tol,unit", [(500.0, "da"), (150.0, "da"), (20.0, "ppm"), (0.0, "da"), (0.05, "da"),
                                      (500.0, "mass"), (37.5, "mass"), (0.0, "mass")])
def test_windows_match_oracle(hd, tol, unit):
    rng = np.random.default_rng(4)
    n = 5000
    mz = np.round(rng.uniform(400, 1500, n), 2)
    z = rng.integers(1, 5, n).astype(np.uint8)
    qmz = np.concatenate([rng.uniform(350, 1550, 400), mz[:50], mz[50:60] + tol, mz[60:70] - tol,
                          [np.nan, np.inf, -np.inf]])
    qz = np.concatenate([rng.integers(0, 6, 400), z[:70], [2, 2, 2]]).astype(np.uint8)
    ctx = hd.Ctx(128, 4, 10, 64, 0)
    lib = hd.hd_build_library(ctx, dev(np.zeros((n, 2), np.uint64)), dev(mz), dev(z))
    lo, hi = hd.hd_query_windows(lib, dev(qmz), dev(qz), tol, unit)
    _, s_mz, s_z, s_orig = hd.hd_library_export(lib)
    torch.cuda.synchronize()
    lo, hi = hd.as_u32(lo).astype(np.int64), hd.as_u32(hi).astype(np.int64)
    want = oracle.window_count(mz, z, qmz, qz, tol, unit)
    assert np.array_equal(hi - lo, want.astype(np.int64))
    so = hd.as_u32(s_orig)
    cnt = oracle.window_count(mz, z, qmz, qz, tol, unit)
    for q in range(len(qmz)):
        rows = so[lo[q]:hi[q]]
        # every row of the range is a candidate and their number is the oracle's count
        if len(rows):
            sub = oracle.window_count(mz[rows], z[rows], qmz[q:q + 1], qz[q:q + 1], tol, unit)
            assert sub[0] == len(rows)
        assert len(rows) == cnt[q]


# ---------------------------------------------------------------- search
def _pipeline(hd, refs, qs, D, Q, k, tol, unit, seed=0, form="auto"):
    pp = pp_args(Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    r_hv = hd.hd_encode(ctx, *gpu_csr(hd, ctx, refs, **pp))
    q_hv = hd.hd_encode(ctx, *gpu_csr(hd, ctx, qs, **pp))
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    idx, dist = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), tol, unit, k, form=form)
    torch.cuda.synchronize()
    ctx.status()
    lib.status()
    return ctx, lib, r_hv, q_hv, hd.as_u32(idx), hd.as_u16(dist)


def test_search_tiny_golden(hd):
    g = json.load(open(os.path.join(GOLDEN, "tiny_search.json")))
    refs, qs, spec = synth.make_workload("tiny")
    _, _, r_hv, q_hv, idx, dist = _pipeline(hd, refs, qs, spec["dim"], spec["n_levels"], 1, spec["tol"],
                                            spec["unit"])
    import hashlib
    assert hashlib.sha256(hd.as_u64(r_hv).tobytes()).hexdigest() == g["ref_hv_sha256"]
    assert hashlib.sha256(hd.as_u64(q_hv).tobytes()).hexdigest() == g["query_hv_sha256"]
    assert idx[:, 0].tolist() == g["top1_idx"]
    assert dist[:, 0].tolist() == g["top1_dist"]


def _medium(seed, n_refs=3000, n_q=500):
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = synth.make_references(n_refs, (1, 2, 3, 4), (0.1, 0.5, 0.3, 0.1), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, n_q, rng)
    return refs, qs


@pytest.mark.parametrize("D,k,tol,unit", [(2048, 1, 500.0, "da"), (8192, 5, 500.0, "da"), (8192, 16, 150.0, "da"),
                                          (12288, 3, 500.0, "da"), (4096, 5, 20.0, "ppm"), (2048, 2, 0.0, "da"),
                                          (128, 8, 1e6, "da"), (4096, 5, 300.0, "mass"), (2048, 3, 1000.0, "mass")])
def test_search_bit_exact(hd, D, k, tol, unit):
    refs, qs = _medium(D + k)
    Q = 32
    _, lib, r_hv, q_hv, idx, dist = _pipeline(hd, refs, qs, D, Q, k, tol, unit)
    o_r, o_q = oracle_side.hvs(refs, D, Q, 0), oracle_side.hvs(qs, D, Q, 0)
    assert np.array_equal(hd.as_u64(r_hv), o_r) and np.array_equal(hd.as_u64(q_hv), o_q)
    oi, od = oracle.search(D, o_r, refs.precursor_mz, refs.charge, o_q, qs.precursor_mz,
                           qs.charge, tol, unit, k)
    assert np.array_equal(idx, oi)
    assert np.array_equal(dist, od)


def test_search_edge_cases(hd):
    rng = np.random.default_rng(9)
    D, W = 256, 4
    n = 300
    hv = rng.integers(-2**63, 2**63, (n, W), dtype=np.int64).view(np.uint64)
    hv[100:110] = hv[0]                                   # ties broken by lowest index
    mz = rng.uniform(400, 600, n)
    z = np.where(np.arange(n) < 250, 2, 3).astype(np.uint8)
    q = np.concatenate([hv[:5], hv[250:252], hv[:3]])
    qmz = np.array([500, 500, 500, 500, 500, 450, 450, np.nan, 500, 500], float)
    qz = np.array([2, 2, 2, 2, 2, 3, 3, 2, 9, 2], np.uint8)   # charge 9 has no reference
    ctx = hd.Ctx(D, 4, 10, 128, 0)
    lib = hd.hd_build_library(ctx, dev(hv), dev(mz), dev(z))
    for k, tol in ((16, 1000.0), (1, 1000.0), (4, 0.5), (16, 0.0)):
        i, d = hd.hd_search_open(lib, dev(q), dev(qmz), dev(qz), tol, "da", k)
        torch.cuda.synchronize()
        oi, od = oracle.search(D, hv, mz, z, q, qmz, qz, tol, "da", k)
        assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)
    # empty query set is a no-op
    hd.hd_search_open(lib, dev(q[:0]), dev(qmz[:0]), dev(qz[:0]), 10.0, "da", 3)
    # a library of one row
    lib1 = hd.hd_build_library(ctx, dev(hv[:1]), dev(mz[:1]), dev(z[:1]))
    i, d = hd.hd_search_open(lib1, dev(q), dev(qmz), dev(qz), 1000.0, "da", 2)
    torch.cuda.synchronize()
    oi, od = oracle.search(D, hv[:1], mz[:1], z[:1], q, qmz, qz, 1000.0, "da", 2)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)


def test_search_host_matches_device(hd):
    refs, qs = _medium(77, 2000, 300)
    D, Q, k = 4096, 16, 5
    ctx, lib, _, q_hv, idx, dist = _pipeline(hd, refs, qs, D, Q, k, 500.0, "da")
    q_csr = oracle.preprocess(qs.offsets, qs.mz, qs.intensity, **pp_args(Q))
    hi, hd_ = hd.hd_search_host(ctx, lib, *q_csr, qs.precursor_mz, qs.charge, 500.0, "da", k)
    assert np.array_equal(hi, idx) and np.array_equal(hd_, dist)


def test_invalid_arguments(hd):
    with pytest.raises(hd.HDError) as e:
        hd.Ctx(100, 16, 10)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    ctx = hd.Ctx(256, 4, 10, 128, 0)
    rng = np.random.default_rng(1)
    hv = rng.integers(-2**63, 2**63, (50, 4), dtype=np.int64)
    lib = hd.hd_build_library(ctx, dev(hv), dev(rng.uniform(400, 500, 50)), dev(np.full(50, 2, np.uint8)))
    q, qm, qz = dev(hv[:4]), dev(np.full(4, 450.0)), dev(np.full(4, 2, np.uint8))
    for kw in (dict(k=0), dict(k=17), dict(tol=-1.0), dict(tol=float("nan")), dict(tol=float("inf"))):
        args = dict(tol=10.0, k=1)
        args.update(kw)
        with pytest.raises(hd.HDError) as e:
            hd.hd_search_open(lib, q, qm, qz, args["tol"], "da", args["k"])
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    flat = dev(np.zeros(4 * 4 + 1, np.uint64))
    with pytest.raises(hd.HDError) as e:      # rows not 16-byte aligned
        hd.hd_search_open(lib, flat[1:].view(4, 4), qm, qz, 10.0, "da", 1)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    # a bin beyond n_bins is found on the device and reported by the ctx status
    off, b, lv = dev(np.array([0, 2], np.uint32)), dev(np.array([3, 10], np.uint32)), dev(np.array([0, 1], np.uint8))
    hd.hd_encode(ctx, off, b, lv)
    torch.cuda.synchronize()
    with pytest.raises(hd.HDError) as e:
        ctx.status()
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    ctx.status()   # cleared


# ----------------------------------------------- full-size workload, sampled
def test_full_size_sampled(hd):
    """The 1,000,000 x 50,000, D=8192, Q=32, +-500, top-5 workload: the
    popcount form, then the benchmark's launch configurations (e2m1 SM pairs
    at the schedules the autotuner picks, e4m3, the 1-SM form); the oracle
    answers a seeded sample of queries and encodes a sample of spectra, and
    every form must equal the popcount form on all 50,000 queries."""
    refs, qs, spec = synth.make_workload("full")
    D, Q, k = spec["dim"], spec["n_levels"], spec["k"]
    pp = pp_args(Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 0)
    r_csr = gpu_csr(hd, ctx, refs, **pp)
    q_csr = gpu_csr(hd, ctx, qs, **pp)
    r_hv = hd.hd_encode(ctx, *r_csr)
    q_hv = hd.hd_encode(ctx, *q_csr)
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    idx, dist = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), spec["tol"], spec["unit"], k)
    torch.cuda.synchronize()
    ctx.status()
    lib.status()
    rng = np.random.default_rng(2024)
    # encode: a sample of spectra through the oracle's own preprocessing and encoder
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    rs = np.sort(rng.choice(refs.n, 200, replace=False))
    sub = refs.subset(rs)
    o_csr = oracle.preprocess(sub.offsets, sub.mz, sub.intensity, **pp)
    assert np.array_equal(hd.as_u64(r_hv[torch.from_numpy(rs).cuda()]), oracle.encode(D, F, L, *o_csr))
    # search: a sample of queries by brute force over the whole library, on
    # the oracle's own encoding of every reference and of the sampled queries
    which = np.sort(rng.choice(qs.n, 48, replace=False)).astype(np.uint32)
    r_np = oracle_side.workload_ref_hvs("full", D, Q, 0)
    q_sub = qs.subset(which)
    q_np = oracle_side.hvs(q_sub, D, Q, 0)
    assert np.array_equal(hd.as_u64(q_hv[torch.from_numpy(which.astype(np.int64)).cuda()]), q_np)
    oi, od = oracle.search(D, r_np, refs.precursor_mz, refs.charge, q_np, q_sub.precursor_mz, q_sub.charge,
                           spec["tol"], spec["unit"], k)
    gi, gd = hd.as_u32(idx), hd.as_u16(dist)
    assert np.array_equal(gi[which], oi)
    assert np.array_equal(gd[which], od)
    # properties that hold for every query: ascending keys, candidates only
    assert np.all((gd[:, 1:] > gd[:, :-1]) | ((gd[:, 1:] == gd[:, :-1]) & (gi[:, 1:] > gi[:, :-1])))
    ok = gi != 0xFFFFFFFF
    rows = gi[ok]
    qq = np.nonzero(ok)[0]
    assert np.all(refs.charge[rows] == qs.charge[qq])
    assert np.all(np.abs(refs.precursor_mz[rows] - qs.precursor_mz[qq]) <= spec["tol"])
    # the benchmark's form and schedules: e2m1 SM pairs at the autotuner's usual picks (kind::mxf4
    # with one and with two reference tiles per query stage), e4m3, and the 1-SM form; each equal
    # to the oracle on the sample and to the popcount form on every query
    hd.hd_library_prepare(lib, "tc_fp4")
    hd.hd_library_prepare(lib, "tc_fp8")
    for form, sched in (("tc_fp4", (16, 16, 2, 2)), ("tc_fp4", (32, 16, 2, 2)), ("tc_fp4", (32, 2, 2, 2)),
                        ("tc_fp4", (16, 2, 2, 2)), ("tc_fp8", (16, 16, 2, 2)), ("tc_fp4", (16, 16, 1, 1)),
                        ("tc_mxf4", (16, 2, 2, 2)), ("tc_mxf4", (32, 2, 2, 2)), ("tc_mxf4", (16, 16, 2, 2)),
                        ("tc_mxf4", (4, 2, 2, 2)), ("tc_mxf4", (16, 2, 2, 2, 2)), ("tc_mxf4", (32, 2, 2, 2, 2)),
                        ("tc_mxf4", (16, 16, 2, 2, 2))):
        hd.hd_library_set_schedule(lib, *sched[:4])
        hd.hd_library_set_stage_tiles(lib, sched[4] if len(sched) > 4 else 1)
        ti, td = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), spec["tol"], spec["unit"], k,
                                   form=form)
        torch.cuda.synchronize()
        lib.status()
        ti, td = hd.as_u32(ti), hd.as_u16(td)
        assert np.array_equal(ti[which], oi) and np.array_equal(td[which], od), (form, sched)
        assert np.array_equal(ti, gi) and np.array_equal(td, gd), (form, sched)
