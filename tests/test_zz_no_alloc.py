"""hd_search_open_noalloc: the search for callers that cannot allocate device
memory while running (a server that reserved its memory up front, a host
thread that must not block in the allocator).  Its scratch is one fixed
device buffer inside libhd; these checks call it through the C ABI and
compare it with hd_search_open, which allocates its own scratch.

This file is collected last on purpose: it passes both alone in a fresh
process and after the rest of the suite (the buffer keeps whatever earlier
calls left in it, which must not matter).
"""
import numpy as np
import pytest
import torch

from paper_2211_16422_gb300 import synth

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


def test_noalloc_matches_allocating_search_twice(hd):
    rng = np.random.Generator(np.random.PCG64(31))
    refs = synth.make_references(4000, (2, 3, 4), (0.6, 0.3, 0.1), rng, decoy_fraction=0.5)
    qa = synth.make_queries(refs, 700, rng)
    qb = synth.make_queries(refs, 333, rng)
    D, Q = 4096, 32
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed=3)

    def encode(sp):
        csr = hd.hd_preprocess(ctx, _dev(sp.offsets), _dev(sp.mz), _dev(sp.intensity), **pp)
        return hd.hd_encode(ctx, *csr)

    lib = hd.hd_build_library(ctx, encode(refs), _dev(refs.precursor_mz), _dev(refs.charge))
    for qs, k, tol, unit in ((qa, 5, 500.0, "da"), (qb, 16, 150.0, "da")):
        q_hv, q_mz, q_z = encode(qs), _dev(qs.precursor_mz), _dev(qs.charge)
        want_i, want_d = hd.hd_search_open(lib, q_hv, q_mz, q_z, tol, unit, k)
        got_i = torch.full((qs.n, k), 7, dtype=torch.int32, device="cuda")
        got_d = torch.full((qs.n, k), 7, dtype=torch.int16, device="cuda")
        hd.hd_search_open_noalloc(lib, q_hv, q_mz, q_z, tol, unit, k, out_idx=got_i, out_dist=got_d)
        torch.cuda.synchronize()
        lib.status()
        assert torch.equal(got_i, want_i) and torch.equal(got_d, want_d)


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
