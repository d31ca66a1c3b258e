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
