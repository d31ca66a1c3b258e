"""Continuous-batching server: every request's top-k is exactly what the
request gets when searched alone, whether it ran coalesced with others, in an
overlapping batch on another stream, or squeezed by a small memory budget."""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2211_16422_gb300 import synth
from tests import oracle_side

pytestmark = pytest.mark.gpu
D, Q, K = 4096, 32, 5


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
    return torch.from_numpy(a).cuda()


@pytest.fixture(scope="module")
def world(hd):
    rng = np.random.Generator(np.random.PCG64(41))
    refs = synth.make_references(15000, (2, 3, 4), (0.6, 0.3, 0.1), rng, decoy_fraction=0.5)
    pool = synth.make_queries(refs, 6000, rng)
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 0)
    r_hv = hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp))
    lib = hd.hd_build_library(ctx, r_hv, dev(refs.precursor_mz), dev(refs.charge))
    hd.hd_library_prepare(lib, "tc_fp8")
    csr = oracle.preprocess(pool.offsets, pool.mz, pool.intensity, **pp)
    return ctx, lib, refs, pool, csr, r_hv


def _requests(pool, csr, n_req, rng, lo=1, hi=400):
    sizes = synth.batch_sizes(n_req, lo, hi, rng)
    off, bins, lv = csr
    out = []
    for i, s in enumerate(sizes):
        a = int(rng.integers(0, pool.n - s))
        b = a + int(s)
        o = off[a:b + 1] - off[a]
        win = (500.0, "da") if i % 3 else (20.0, "ppm")
        out.append((o, bins[off[a]:off[b]], lv[off[a]:off[b]], pool.precursor_mz[a:b], pool.charge[a:b], win))
    return out


def _alone(hd, ctx, lib, req):
    o, b, lv, mz, z, (tol, unit) = req
    q_hv = hd.hd_encode(ctx, dev(o), dev(b), dev(lv))
    i, d = hd.hd_search_open(lib, q_hv, dev(mz), dev(z), tol, unit, K)
    torch.cuda.synchronize()
    return hd.as_u32(i), hd.as_u16(d)


def test_server_results_equal_alone(hd, world):
    ctx, lib, refs, pool, csr, r_hv = world
    reqs = _requests(pool, csr, 60, np.random.default_rng(3))
    srv = hd.Server(ctx, lib, k=K, slots=3, max_batch_queries=3000)
    ids = [None] * len(reqs)

    def submit(part):
        for j in part:
            o, b, lv, mz, z, (tol, unit) = reqs[j]
            ids[j] = srv.submit(o, b, lv, mz, z, tol, unit)

    th = [threading.Thread(target=submit, args=(range(t, len(reqs), 2),)) for t in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = [srv.wait(r) for r in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["batches"] < len(reqs)
    for req, (i, d, info) in zip(reqs, got):
        ai, ad = _alone(hd, ctx, lib, req)
        assert np.array_equal(i, ai) and np.array_equal(d, ad)
        assert info["n_queries"] == len(req[3]) and info["latency_s"] >= info["queue_s"] >= 0


def _overlapping_pairs(log):
    return [(a["batch"], b["batch"]) for i, a in enumerate(log) for b in log[i + 1:]
            if a["slot"] != b["slot"] and a["device_start_ms"] < b["device_end_ms"]
            and b["device_start_ms"] < a["device_end_ms"]]


@pytest.mark.parametrize("slots", [3, 1])
def test_server_batches_overlap_on_the_device(hd, world, slots):
    """Requests that arrive while others run go to free slots, and their batches
    run on the device at the same time: with three slots some pair of batches on
    different streams has intersecting device-time intervals (CUDA events around
    each batch's copies, encode and search), and each result still equals the
    request searched alone.  One slot serialises the batches: no overlap."""
    ctx, lib, refs, pool, csr, r_hv = world
    off, bins, lv = csr
    n_req, size = 6, 5000
    rng = np.random.default_rng(21)
    reqs = []
    for j in range(n_req):
        a = int(rng.integers(0, pool.n - size))
        b = a + size
        reqs.append((off[a:b + 1] - off[a], bins[off[a]:off[b]], lv[off[a]:off[b]], pool.precursor_mz[a:b],
                     pool.charge[a:b], (500.0, "da")))
    # the popcount form keeps each batch on the device for a while
    srv = hd.Server(ctx, lib, k=K, slots=slots, max_batch_queries=size, form="popc")
    ids = [srv.submit(*r[:5], *r[5]) for r in reqs]
    got = [srv.wait(r) for r in ids]
    st, log = srv.stats(), srv.batch_log()
    srv.close()
    assert st["completed"] == n_req and len(log) == st["batches"] == n_req
    assert all(r["device_end_ms"] > r["device_start_ms"] >= 0 for r in log)
    pairs = _overlapping_pairs(log)
    if slots == 1:
        assert st["max_inflight"] == 1 and not pairs
    else:
        assert st["max_inflight"] >= 2 and pairs, log
    for req, (i, d, _) in zip(reqs, got):
        ai, ad = _alone(hd, ctx, lib, req)
        assert np.array_equal(i, ai) and np.array_equal(d, ad)


def test_server_matches_oracle_sample(hd, world):
    ctx, lib, refs, pool, csr, r_hv = world
    req = _requests(pool, csr, 1, np.random.default_rng(5), 200, 200)[0]
    srv = hd.Server(ctx, lib, k=K, slots=2)
    rid = srv.submit(*req[:5], *req[5])
    i, d, _ = srv.wait(rid)
    srv.close()
    o, b, lv, mz, z, (tol, unit) = req
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    q_hv = oracle.encode(D, F, L, o, b, lv)
    oi, od = oracle.search(D, oracle_side.hvs(refs, D, Q, 0), refs.precursor_mz, refs.charge, q_hv, mz, z, tol,
                           unit, K)
    assert np.array_equal(i, oi) and np.array_equal(d, od)


def test_server_small_memory_budget(hd, world):
    """A budget of ~2 requests' worth forces many small batches, never a stall."""
    ctx, lib, refs, pool, csr, r_hv = world
    reqs = _requests(pool, csr, 25, np.random.default_rng(9), 50, 300)
    srv = hd.Server(ctx, lib, k=K, slots=4, mem_budget_bytes=300 * (D // 8 + 2 * D + 1024 + K * 32))
    ids = [srv.submit(*r[:5], *r[5]) for r in reqs]
    got = [srv.wait(r) for r in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    for req, (i, d, info) in zip(reqs, got):
        ai, ad = _alone(hd, ctx, lib, req)
        assert np.array_equal(i, ai) and np.array_equal(d, ad)


def test_server_multibit_library(hd, world):
    """A server on a multi-bit library (Section 4.3 components, 3 bits):
    requests are encoded into components and scored by the dot-product
    search; every result equals hd_search_dot of the request alone, one
    request equals the oracle, and the binary submit call is refused."""
    import ctypes
    ctx, lib, refs, pool, csr, r_hv = world
    bits = 3
    pp = oracle_side.pp_args(Q)
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp)
    mlib = hd.hd_build_library_multibit(ctx, hd.hd_encode_multibit(ctx, *r_csr, bits), dev(refs.precursor_mz),
                                        dev(refs.charge), bits)
    reqs = _requests(pool, csr, 12, np.random.default_rng(33), 1, 300)
    srv = hd.Server(ctx, mlib, k=K, slots=3, max_batch_queries=1000)
    ids = [srv.submit(*r[:5], *r[5]) for r in reqs]
    got = [srv.wait(r) for r in ids]
    # the binary submit call on a multi-bit server is refused before anything is queued
    o, b, lv, mz, z, (tol, unit) = reqs[0]
    oi = np.empty((len(mz), K), np.uint32)
    od = np.empty((len(mz), K), np.uint16)
    rid = ctypes.c_uint64()
    st = hd.load().hd_server_submit(srv._h, hd._ptr(np.ascontiguousarray(o, np.uint32)),
                                    hd._ptr(np.ascontiguousarray(b, np.uint32)), hd._ptr(np.ascontiguousarray(lv)),
                                    hd._ptr(np.ascontiguousarray(mz)), hd._ptr(np.ascontiguousarray(z)), len(mz),
                                    float(tol), hd._unit(unit), hd._ptr(oi), hd._ptr(od), ctypes.byref(rid))
    assert st == hd.HD_ERR_INVALID_ARG
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(reqs)
    for req, (i, sc, info) in zip(reqs, got):
        o, b, lv, mz, z, (tol, unit) = req
        q = hd.hd_encode_multibit(ctx, dev(o), dev(b), dev(lv), bits)
        ai, asc = hd.hd_search_dot(mlib, q, dev(mz), dev(z), tol, unit, K)
        torch.cuda.synchronize()
        assert sc.dtype == np.int32
        assert np.array_equal(i, hd.as_u32(ai)) and np.array_equal(sc, asc.cpu().numpy())
    o, b, lv, mz, z, (tol, unit) = reqs[1]
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    R = oracle.encode_multibit(D, F, L, *oracle.preprocess(refs.offsets, refs.mz, refs.intensity, **pp), bits)
    oi, osc = oracle.search_dot(R, refs.precursor_mz, refs.charge, oracle.encode_multibit(D, F, L, o, b, lv, bits),
                                mz, z, tol, unit, K)
    assert np.array_equal(got[1][0], oi) and np.array_equal(got[1][1], osc)
