"""hd_search_open_noalloc: the search for callers that cannot allocate device
memory while running (a server that reserved its memory up front, a host
thread that must not block in the allocator).  Its scratch is one fixed
device buffer inside libhd; these checks call it through the C ABI, compare
it with hd_search_open (which allocates its own scratch) and with the
oracle, and check that a call allocates nothing.

This file is collected last on purpose: it passes both alone in a fresh
process and after the rest of the suite (the buffer keeps whatever earlier
calls left in it, which must not matter).
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

import oracle
from paper_2211_16422_gb300 import synth

from tests import oracle_side

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_16422_gb300 import build, hd as _hd
    build.build()
    return _hd


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def test_noalloc_matches_allocating_search_and_oracle_twice(hd):
    rng = np.random.Generator(np.random.PCG64(31))
    refs = synth.make_references(4000, (2, 3, 4), (0.6, 0.3, 0.1), rng, decoy_fraction=0.5)
    qa = synth.make_queries(refs, 700, rng)
    qb = synth.make_queries(refs, 333, rng)
    D, Q, seed = 4096, 32, 3
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=seed)

    def encode(sp):
        csr = hd.hd_preprocess(ctx, _dev(sp.offsets), _dev(sp.mz), _dev(sp.intensity), **pp)
        return hd.hd_encode(ctx, *csr)

    lib = hd.hd_build_library(ctx, encode(refs), _dev(refs.precursor_mz), _dev(refs.charge))
    o_r = oracle_side.hvs(refs, D, Q, seed)
    for qs, k, tol, unit in ((qa, 5, 500.0, "da"), (qb, 16, 150.0, "da")):
        q_hv, q_mz, q_z = encode(qs), _dev(qs.precursor_mz), _dev(qs.charge)
        want_i, want_d = hd.hd_search_open(lib, q_hv, q_mz, q_z, tol, unit, k)
        got_i = torch.full((qs.n, k), 7, dtype=torch.int32, device="cuda")
        got_d = torch.full((qs.n, k), 7, dtype=torch.int16, device="cuda")
        hd.hd_search_open_noalloc(lib, q_hv, q_mz, q_z, tol, unit, k, out_idx=got_i, out_dist=got_d)
        torch.cuda.synchronize()
        lib.status()
        assert torch.equal(got_i, want_i) and torch.equal(got_d, want_d)
        # the oracle encodes the raw spectra itself and searches by brute force
        oi, od = oracle.search(D, o_r, refs.precursor_mz, refs.charge, oracle_side.hvs(qs, D, Q, seed),
                               qs.precursor_mz, qs.charge, tol, unit, k)
        assert np.array_equal(hd.as_u32(got_i), oi) and np.array_equal(hd.as_u16(got_d), od)


def test_noalloc_rejects_requests_beyond_its_buffer(hd):
    rng = np.random.default_rng(8)
    ctx = hd.Ctx(128, 4, 10, 64, 0)
    hv = rng.integers(-2**63, 2**63, (64, 2), dtype=np.int64)
    lib = hd.hd_build_library(ctx, _dev(hv), _dev(rng.uniform(400, 500, 64)), _dev(np.full(64, 2, np.uint8)))
    n = 400_000
    q = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    qm = torch.full((n,), 450.0, dtype=torch.float64, device="cuda")
    qz = torch.full((n,), 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.hd_search_open_noalloc(lib, q, qm, qz, 10.0, "da", 16)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    assert "scratch" in str(e.value)


def test_noalloc_binding_checks_caller_outputs(hd):
    """The kernels write the caller's buffers in place: a too-small, wrongly typed
    or non-contiguous output is refused before anything is launched."""
    rng = np.random.default_rng(9)
    ctx = hd.Ctx(128, 4, 10, 64, 0)
    hv = rng.integers(-2**63, 2**63, (64, 2), dtype=np.int64)
    lib = hd.hd_build_library(ctx, _dev(hv), _dev(rng.uniform(400, 500, 64)), _dev(np.full(64, 2, np.uint8)))
    n, k = 10, 4
    q, qm, qz = _dev(hv[:n]), _dev(np.full(n, 450.0)), _dev(np.full(n, 2, np.uint8))
    ok_i = torch.empty((n, k), dtype=torch.int32, device="cuda")
    ok_d = torch.empty((n, k), dtype=torch.int16, device="cuda")
    bad = [dict(out_idx=torch.empty((n, k - 1), dtype=torch.int32, device="cuda"), out_dist=ok_d),
           dict(out_idx=ok_i, out_dist=torch.empty((n, k), dtype=torch.int32, device="cuda")),
           dict(out_idx=torch.empty((k, n), dtype=torch.int32, device="cuda").t(), out_dist=ok_d),
           dict(out_idx=torch.empty((n, k), dtype=torch.int32), out_dist=ok_d)]
    for kw in bad:
        with pytest.raises((TypeError, ValueError)):
            hd.hd_search_open_noalloc(lib, q, qm, qz, 100.0, "da", k, **kw)
    with pytest.raises(ValueError):
        hd.hd_search_open_noalloc(lib, q[:n - 1], qm, qz, 100.0, "da", k, out_idx=ok_i, out_dist=ok_d)


class _DefaultPool:
    """The device's default stream-ordered memory pool (where cudaMallocAsync
    takes memory), read through the CUDA driver API."""
    RELEASE_THRESHOLD, USED_MEM_CURRENT, USED_MEM_HIGH = 4, 7, 8

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_noalloc_call_allocates_nothing(hd):
    """After a first call (the per-device set-up), a call leaves the pool's
    high-water mark where it was, allocates nothing through torch and takes no
    free device memory.  Objects of earlier tests are collected before the
    measured call and the collector is off during it (a library or tensor
    freed then would otherwise move the figures).  The same check run on
    hd_search_open sees its scratch allocation, so it can tell the two apart."""
    rng = np.random.Generator(np.random.PCG64(47))
    D, n_r, n_q, k = 2048, 20000, 2000, 5
    hv = rng.integers(-2**63, 2**63, (n_r, D // 64), dtype=np.int64)
    mz = rng.uniform(400, 1500, n_r)
    z = rng.integers(2, 4, n_r).astype(np.uint8)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, _dev(hv), _dev(mz), _dev(z))
    q, qm, qz = _dev(hv[:n_q]), _dev(mz[:n_q]), _dev(z[:n_q])
    oi = torch.empty((n_q, k), dtype=torch.int32, device="cuda")
    od = torch.empty((n_q, k), dtype=torch.int16, device="cuda")
    pool = _DefaultPool()

    def watched(call):
        call()                      # loads every kernel the call uses
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.synchronize()
        gc.disable()
        try:
            free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
            pool.reset_high()
            call()
            torch.cuda.synchronize()
            grew = pool.get(pool.USED_MEM_HIGH) - pool.get(pool.USED_MEM_CURRENT)
            return grew, free0 - torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated() - torch0
        finally:
            gc.enable()

    grew, free_drop, torch_grew = watched(
        lambda: hd.hd_search_open_noalloc(lib, q, qm, qz, 500.0, "da", k, out_idx=oi, out_dist=od))
    lib.status()
    assert grew == 0 and free_drop <= 0 and torch_grew <= 0, (grew, free_drop, torch_grew)
    grew_alloc, _, _ = watched(lambda: hd.hd_search_open(lib, q, qm, qz, 500.0, "da", k, out_idx=oi, out_dist=od))
    assert grew_alloc > 0
    # a call with no queries is a valid set-up call and launches nothing
    n0 = hd.hd_launch_count()
    hd.hd_search_open_noalloc(lib, q[:0], qm[:0], qz[:0], 500.0, "da", k)
    assert hd.hd_launch_count() == n0


def test_ctx_keeps_scratch_mapped(hd):
    """A context raises the default pool's release threshold to 4 GiB (stream-
    ordered scratch stays mapped across synchronising calls) and never lowers
    a higher one."""
    pool = _DefaultPool()
    hd.Ctx(128, 4, 10, 64, 0)
    assert pool.get(pool.RELEASE_THRESHOLD) >= 4 << 30
    big = ctypes.c_uint64(8 << 30)
    assert pool.cu.cuMemPoolSetAttribute(pool.pool, pool.RELEASE_THRESHOLD, ctypes.byref(big)) == 0
    hd.Ctx(128, 4, 10, 64, 0)
    assert pool.get(pool.RELEASE_THRESHOLD) == 8 << 30
