"""Seeded randomised parity: many small searches with drawn shapes -- D (a
multiple of 128), library and query sizes that straddle tile and block edges,
charge mixes, window units and widths, k -- through every applicable form,
binary and multi-bit, each compared element by element with the oracle's
brute force on the same inputs."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
UNITS = ("da", "ppm", "mass")


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


def draw(rng):
    """One case: D, sizes, precursors over a narrow m/z range (dense windows),
    a charge mix, a window and k."""
    D = int(rng.choice([128, 256, 384, 640, 1024, 1152, 2048, 2304, 4096]))
    n_ref = int(rng.choice([1, 2, 63, 64, 65, 239, 240, 241, 255, 256, 257, 1000, 2999]))
    n_q = int(rng.choice([1, 2, 31, 63, 64, 65, 127, 128, 129, 255, 256, 257, 700]))
    z_sets = ([2], [2, 3], [1, 2, 3, 4, 5], [0, 2])
    z_set = z_sets[int(rng.integers(len(z_sets)))]
    ref_z = rng.choice(z_set, n_ref).astype(np.uint8)
    q_z = rng.choice(z_set, n_q).astype(np.uint8)
    ref_mz = rng.uniform(400, 430, n_ref)
    q_mz = rng.uniform(398, 432, n_q)
    dup = rng.integers(0, n_ref, min(n_ref, 8))          # equal m/z values among the references
    ref_mz[dup] = ref_mz[dup[0]]
    unit = str(rng.choice(UNITS))
    tol = {"da": float(rng.choice([0.0, 0.5, 3.0, 40.0])), "ppm": float(rng.choice([20.0, 5000.0, 80000.0])),
           "mass": float(rng.choice([1.0, 12.0, 100.0]))}[unit]
    k = int(rng.choice([1, 2, 3, 5, 8, 13, 16]))
    return D, n_ref, n_q, ref_mz, ref_z, q_mz, q_z, unit, tol, k


@pytest.mark.parametrize("seed", range(96))
def test_fuzz_binary(hd, seed):
    rng = np.random.default_rng(1000 + seed)
    D, n_ref, n_q, ref_mz, ref_z, q_mz, q_z, unit, tol, k = draw(rng)
    W = D // 64
    hv = rng.integers(-2**63, 2**63, (n_ref, W), dtype=np.int64).view(np.uint64)
    src = rng.integers(0, n_ref, n_q)
    q = hv[src].copy()                                   # near-duplicates of references: small distances
    flip = rng.random((n_q, W)) < 0.02
    q[flip] ^= rng.integers(-2**63, 2**63, int(flip.sum()), dtype=np.int64).view(np.uint64)
    q[: n_q // 4] = rng.integers(-2**63, 2**63, (n_q // 4, W), dtype=np.int64).view(np.uint64)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(hv), dev(ref_mz), dev(ref_z))
    oi, od = oracle.search(D, hv, ref_mz, ref_z, q, q_mz, q_z, tol, unit, k)
    forms = ["popc", "tc_fp4", "tc_fp8", "tc_bf16"] + (["tc_mxf4"] if D % 256 == 0 else [])
    for form in forms:
        if form != "popc":
            hd.hd_library_prepare(lib, form)
        gi, gd = hd.hd_search_open(lib, dev(q), dev(q_mz), dev(q_z), tol, unit, k, form=form)
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(gi), oi), (form, D, n_ref, n_q, unit, tol, k)
        assert np.array_equal(hd.as_u16(gd), od), (form, D, n_ref, n_q, unit, tol, k)


@pytest.mark.parametrize("seed", range(64))
def test_fuzz_multibit(hd, seed):
    rng = np.random.default_rng(2000 + seed)
    D, n_ref, n_q, ref_mz, ref_z, q_mz, q_z, unit, tol, k = draw(rng)
    bits = int(rng.integers(2, 6))
    m = (1 << (bits - 1)) - 1
    R = rng.integers(-m, m + 1, (n_ref, D)).astype(np.int8)
    Qv = R[rng.integers(0, n_ref, n_q)].copy()
    redraw = rng.random((n_q, D)) < 0.3
    Qv[redraw] = rng.integers(-m, m + 1, int(redraw.sum()))
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(ref_mz), dev(ref_z), bits)
    oi, osc = oracle.search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, tol, unit, k)
    forms = ["popc", "tc_fp8", "tc_bf16"] + (["tc_fp4"] + (["tc_mxf4"] if D % 256 == 0 else []) if bits <= 3 else [])
    for form in forms:
        if form in ("popc", "tc_bf16") or (form == "tc_fp8" and bits <= 3):
            hd.hd_library_prepare(lib, form)
        gi, gs = hd.hd_search_dot(lib, dev(Qv), dev(q_mz), dev(q_z), tol, unit, k, form)
        torch.cuda.synchronize()
        lib.status()
        assert np.array_equal(hd.as_u32(gi), oi), (form, bits, D, n_ref, n_q, unit, tol, k)
        assert np.array_equal(gs.cpu().numpy(), osc), (form, bits, D, n_ref, n_q, unit, tol, k)


def draw_windows(rng, n):
    out = []
    for _ in range(n):
        unit = str(rng.choice(UNITS))
        tol = {"da": float(rng.choice([0.0, 1.0, 10.0, 40.0])), "ppm": float(rng.choice([20.0, 2000.0, 50000.0])),
               "mass": float(rng.choice([2.0, 25.0]))}[unit]
        out.append((tol, unit))
    return out


@pytest.mark.parametrize("seed", range(32))
def test_fuzz_window_classes(hd, seed):
    """Per-query window classes (1..16 windows) in one launch, binary forms and
    a multi-bit form, against the oracle answering each class on its own."""
    rng = np.random.default_rng(3000 + seed)
    D, n_ref, n_q, ref_mz, ref_z, q_mz, q_z, _, _, k = draw(rng)
    windows = draw_windows(rng, int(rng.integers(1, 17)))
    cls = rng.integers(0, len(windows), n_q).astype(np.uint8)
    W = D // 64
    hv = rng.integers(-2**63, 2**63, (n_ref, W), dtype=np.int64).view(np.uint64)
    q = hv[rng.integers(0, n_ref, n_q)].copy()
    q[::3] = rng.integers(-2**63, 2**63, (len(q[::3]), W), dtype=np.int64).view(np.uint64)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(hv), dev(ref_mz), dev(ref_z))
    oi = np.full((n_q, k), 0xFFFFFFFF, np.uint32)
    od = np.full((n_q, k), 0xFFFF, np.uint16)
    for c, (tol, unit) in enumerate(windows):
        w = np.nonzero(cls == c)[0].astype(np.uint32)
        if w.size:
            oi[w], od[w] = oracle.search(D, hv, ref_mz, ref_z, q, q_mz, q_z, tol, unit, k, which=w)
    form = str(rng.choice(["popc", "tc_fp4", "tc_fp8"] + (["tc_mxf4"] if D % 256 == 0 else [])))
    if form != "popc":
        hd.hd_library_prepare(lib, form)
    gi, gd = hd.hd_search_open_multi(lib, dev(q), dev(q_mz), dev(q_z), dev(cls), windows, k, form=form)
    torch.cuda.synchronize()
    lib.status()
    assert np.array_equal(hd.as_u32(gi), oi) and np.array_equal(hd.as_u16(gd), od), (form, windows, k)
    bits = int(rng.integers(2, 6))
    m = (1 << (bits - 1)) - 1
    R = rng.integers(-m, m + 1, (n_ref, D)).astype(np.int8)
    Qv = R[rng.integers(0, n_ref, n_q)].copy()
    Qv[::2] = rng.integers(-m, m + 1, (len(Qv[::2]), D))
    mlib = hd.hd_build_library_multibit(ctx, dev(R), dev(ref_mz), dev(ref_z), bits)
    oi2 = np.full((n_q, k), 0xFFFFFFFF, np.uint32)
    os2 = np.full((n_q, k), np.iinfo(np.int32).min, np.int32)
    for c, (tol, unit) in enumerate(windows):
        w = np.nonzero(cls == c)[0].astype(np.uint32)
        if w.size:
            oi2[w], os2[w] = oracle.search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, tol, unit, k, which=w)
    gi, gs = hd.hd_search_dot_multi(mlib, dev(Qv), dev(q_mz), dev(q_z), dev(cls), windows, k)
    torch.cuda.synchronize()
    mlib.status()
    assert np.array_equal(hd.as_u32(gi), oi2) and np.array_equal(gs.cpu().numpy(), os2), (bits, windows, k)


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_cascade(hd, seed):
    """Cascades of 1..4 drawn levels and FDR thresholds over seeded targets,
    decoys and noisy queries, binary and multi-bit, against the oracle's
    cascades (index, distance or score, level and q-value bit for bit)."""
    rng = np.random.default_rng(4000 + seed)
    D = int(rng.choice([256, 512, 1024]))
    n_t, n_q = int(rng.integers(50, 800)), int(rng.integers(1, 400))
    mz_t = rng.uniform(400, 460, n_t)
    z_t = rng.integers(2, 4, n_t).astype(np.uint8)
    mz, z = np.r_[mz_t, mz_t], np.r_[z_t, z_t]
    dec = np.r_[np.zeros(n_t, np.uint8), np.ones(n_t, np.uint8)]
    src = rng.integers(0, n_t, n_q)
    q_mz = mz[src] + np.where(rng.random(n_q) < 0.5, 0.0, rng.uniform(-60, 60, n_q)) / z[src]
    q_z = z[src]
    levels = draw_windows(rng, int(rng.integers(1, 5)))
    fdr = float(rng.choice([-1.0, 0.0, 0.01, 0.05, 0.5, 1e9]))
    W = D // 64
    hv = rng.integers(-2**63, 2**63, (2 * n_t, W), dtype=np.int64).view(np.uint64)
    bits_ = np.unpackbits(hv[src].view(np.uint8), bitorder="little").reshape(n_q, D)
    flip = rng.random((n_q, D)) < rng.uniform(0.02, 0.45, (n_q, 1))
    q_hv = np.packbits(bits_ ^ flip, axis=1, bitorder="little").view(np.uint64)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(hv), dev(mz), dev(z))
    hd.hd_library_set_decoys(lib, dev(dec))
    form = str(rng.choice(["popc", "tc_fp4", "tc_mxf4"]))
    if form != "popc":
        hd.hd_library_prepare(lib, form)
    gi, gd, gq, gl = hd.hd_cascade_search(lib, dev(q_hv), dev(q_mz), dev(q_z), levels, fdr, form=form)
    torch.cuda.synchronize()
    lib.status()
    oi, od, ol, oq = oracle.cascade(D, hv, mz, z, dec, q_hv, q_mz, q_z, levels, fdr)
    assert np.array_equal(hd.as_u32(gi), oi) and np.array_equal(hd.as_u16(gd), od), (form, levels, fdr)
    assert np.array_equal(gl.cpu().numpy(), ol) and np.array_equal(gq.cpu().numpy(), oq, equal_nan=True)
    bits = int(rng.integers(2, 6))
    m = (1 << (bits - 1)) - 1
    R = rng.integers(-m, m + 1, (2 * n_t, D)).astype(np.int8)
    Qc = R[src].copy()
    redraw = rng.random((n_q, D)) < rng.uniform(0.05, 0.8, (n_q, 1))
    Qc[redraw] = rng.integers(-m, m + 1, int(redraw.sum()))
    mlib = hd.hd_build_library_multibit(ctx, dev(R), dev(mz), dev(z), bits)
    hd.hd_library_set_decoys(mlib, dev(dec))
    gi, gs, gq, gl = hd.hd_cascade_search_dot(mlib, dev(Qc), dev(q_mz), dev(q_z), levels, fdr)
    torch.cuda.synchronize()
    mlib.status()
    oi, osc, ol, oq = oracle.cascade_dot(R, mz, z, dec, Qc, q_mz, q_z, levels, fdr)
    assert np.array_equal(hd.as_u32(gi), oi) and np.array_equal(gs.cpu().numpy(), osc), (bits, levels, fdr)
    assert np.array_equal(gl.cpu().numpy(), ol) and np.array_equal(gq.cpu().numpy(), oq, equal_nan=True)
