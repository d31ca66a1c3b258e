"""Cascade search with target-decoy FDR on the GPU (through the C ABI)
against the oracle's cascade, element by element: identifying level,
top-1 index and distance, and the q-value in IEEE double, bit for bit.
The FDR-path cases take seeded random hypervectors as inputs of both sides
(true matches far above chance, so every level accepts queries); the
spectra cases have each side preprocess and encode the raw synthetic
spectra itself."""
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


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def _setup(hd, n_refs, n_q, D, Q, seed, charges=(2, 3, 4), weights=(0.6, 0.3, 0.1)):
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = synth.make_references(n_refs, charges, weights, rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, n_q, rng)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    pp = oracle_side.pp_args(Q)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    lib = hd.hd_build_library(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge))
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    return refs, qs, ctx, lib, enc(qs)


def _check(hd, got, want):
    gi, gd, gq, gl = got
    oi, od, ol, oq = want
    assert np.array_equal(hd.as_u32(gi), oi)
    assert np.array_equal(hd.as_u16(gd), od)
    assert np.array_equal(gl.cpu().numpy(), ol)
    assert np.array_equal(gq.cpu().numpy(), oq, equal_nan=True)


LEVELS2 = [(20.0, "ppm"), (500.0, "da")]
LEVELS3 = [(5.0, "ppm"), (150.0, "da"), (500.0, "da")]


def _hv_workload(seed, D, n_t, n_q):
    """Seeded random reference HVs (targets, then as many decoys with the same
    precursors) and queries that are noisy copies of targets, 40% at the
    target's precursor and the rest shifted: true
    matches stand far above chance, so every level identifies queries.  Shifts of
    U(-900, 900) Da / charge put some true matches beyond +-150 Th."""
    rng = np.random.default_rng(seed)
    W = D // 64
    hv = rng.integers(-2**63, 2**63, (2 * n_t, W), dtype=np.int64).view(np.uint64)
    mz_t = rng.uniform(400, 1500, n_t)
    z_t = rng.integers(2, 5, n_t).astype(np.uint8)
    mz, z = np.r_[mz_t, mz_t], np.r_[z_t, z_t]
    dec = np.r_[np.zeros(n_t, np.uint8), np.ones(n_t, np.uint8)]
    src = rng.integers(0, n_t, n_q)
    shift = np.where(rng.random(n_q) < 0.4, 0.0, rng.uniform(-900, 900, n_q))
    q_mz, q_z = mz[src] + shift / z[src], z[src]
    bits = np.unpackbits(hv[src].view(np.uint8), bitorder="little").reshape(n_q, D)
    flip = rng.random((n_q, D)) < rng.uniform(0.05, 0.35, (n_q, 1))
    q_hv = np.packbits(bits ^ flip, axis=1, bitorder="little").view(np.uint64)
    return hv, mz, z, dec, q_hv, q_mz, q_z


@pytest.mark.parametrize("form", ["popc", "tc_fp8", "tc_bf16", "tc_fp4", "tc_mxf4"])
@pytest.mark.parametrize("levels,fdr", [(LEVELS2, 0.01), (LEVELS3, 0.05)])
def test_cascade_matches_oracle(hd, form, levels, fdr):
    D = 2048
    hv, mz, z, dec, q_hv, q_mz, q_z = _hv_workload(31, D, 12000, 3000)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(hv), dev(mz), dev(z))
    hd.hd_library_set_decoys(lib, dev(dec))
    if form != "popc":
        hd.hd_library_prepare(lib, form)
    got = hd.hd_cascade_search(lib, dev(q_hv), dev(q_mz), dev(q_z), levels, fdr, form=form)
    torch.cuda.synchronize()
    lib.status()
    want = oracle.cascade(D, hv, mz, z, dec, q_hv, q_mz, q_z, levels, fdr)
    _check(hd, got, want)
    lv = want[2]
    assert (lv == 0).sum() > 0 and (lv == len(levels) - 1).sum() > 0   # first and last level identify


def test_cascade_spectra_pipeline(hd):
    """Preprocess + encode + cascade on synthetic spectra (each side encodes its own)."""
    D, Q, seed = 2048, 16, 21
    refs, qs, ctx, lib, q_hv = _setup(hd, 20000, 1500, D, Q, seed)
    hd.hd_library_prepare(lib, "tc_fp8")
    got = hd.hd_cascade_search(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), LEVELS2, 0.01, form="tc_fp8")
    torch.cuda.synchronize()
    lib.status()
    o_r, o_q = oracle_side.hvs(refs, D, Q, seed), oracle_side.hvs(qs, D, Q, seed)
    want = oracle.cascade(D, o_r, refs.precursor_mz, refs.charge, refs.decoy, o_q, qs.precursor_mz, qs.charge,
                          LEVELS2, 0.01)
    _check(hd, got, want)


def test_cascade_edges(hd):
    D, Q, seed = 1024, 8, 5
    # charge 5 queries have no candidate at any level (the library holds 2 and 3)
    refs, qs, ctx, lib, q_hv = _setup(hd, 3000, 400, D, Q, seed, charges=(2, 3), weights=(0.5, 0.5))
    z = qs.charge.copy()
    z[::7] = 5
    o_r, o_q = oracle_side.hvs(refs, D, Q, seed), oracle_side.hvs(qs, D, Q, seed)
    for fdr in (-1.0, 0.0, 0.02, 1e9):
        got = hd.hd_cascade_search(lib, q_hv, dev(qs.precursor_mz), dev(z), LEVELS2, fdr, form="popc")
        torch.cuda.synchronize()
        lib.status()
        want = oracle.cascade(D, o_r, refs.precursor_mz, refs.charge, refs.decoy, o_q, qs.precursor_mz, z,
                              LEVELS2, fdr)
        _check(hd, got, want)
        assert np.all(got[3].cpu().numpy()[::7] == 255)
        assert np.all(np.isnan(got[2].cpu().numpy()[::7]))
    # one query, one level
    got = hd.hd_cascade_search(lib, q_hv[:1], dev(qs.precursor_mz[:1]), dev(qs.charge[:1]), [(500.0, "da")], 0.01)
    torch.cuda.synchronize()
    want = oracle.cascade(D, o_r, refs.precursor_mz, refs.charge, refs.decoy, o_q[:1], qs.precursor_mz[:1],
                          qs.charge[:1], [(500.0, "da")], 0.01)
    _check(hd, got, want)


def test_cascade_argument_errors(hd):
    D, Q, seed = 1024, 8, 6
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = synth.make_references(500, (2,), (1.0,), rng, decoy_fraction=0.5)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    pp = oracle_side.pp_args(Q)
    hv = hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp))
    lib = hd.hd_build_library(ctx, hv, dev(refs.precursor_mz), dev(refs.charge))
    args = (lib, hv[:4], dev(refs.precursor_mz[:4]), dev(refs.charge[:4]))
    with pytest.raises(hd.HDError) as e:            # no decoy flags yet
        hd.hd_cascade_search(*args, LEVELS2, 0.01)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    for levels, fdr in [([], 0.01), ([(1.0, "da")] * 17, 0.01), ([(-1.0, "da")], 0.01), (LEVELS2, float("nan"))]:
        with pytest.raises(hd.HDError) as e:
            hd.hd_cascade_search(*args, levels, fdr)
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    hd.hd_cascade_search(*args, LEVELS2, 0.01)
    torch.cuda.synchronize()
    lib.status()


def test_cascade_full_size_one_level(hd):
    """1,000,000 references x 50,000 queries, D=8192: one +-500 level, so every
    query's SSM is reported; the q-values are recomputed by the oracle from
    the GPU's own SSM scores and decoy flags (bit for bit), and a seeded sample
    of SSMs is checked against the oracle's brute-force top-1."""
    refs, qs, spec = synth.make_workload("full")
    D, Q = spec["dim"], spec["n_levels"]
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 0)
    pp = oracle_side.pp_args(Q)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    lib = hd.hd_build_library(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge))
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    hd.hd_library_prepare(lib, "tc_fp8")
    q_hv = enc(qs)
    gi, gd, gq, gl = hd.hd_cascade_search(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), [(500.0, "da")], 0.01,
                                          form="tc_fp8")
    torch.cuda.synchronize()
    lib.status()
    gi, gd, gq, gl = hd.as_u32(gi), hd.as_u16(gd), gq.cpu().numpy(), gl.cpu().numpy()
    has = gi != 0xFFFFFFFF
    qv = oracle.fdr_qvalues(D - gd[has].astype(np.int64), refs.decoy[gi[has]])
    assert np.array_equal(gq[has], qv)
    ident = np.zeros(qs.n, bool)
    ident[np.nonzero(has)[0]] = (refs.decoy[gi[has]] == 0) & (qv <= 0.01)
    assert np.array_equal(gl == 0, ident) and np.all(gl[~ident] == 255)
    rng = np.random.default_rng(77)
    which = np.sort(rng.choice(qs.n, 24, replace=False)).astype(np.uint32)
    r_np = oracle_side.workload_ref_hvs("full", D, Q, 0)
    q_np = oracle_side.hvs(qs.subset(which), D, Q, 0)
    sub = qs.subset(which)
    oi, od = oracle.search(D, r_np, refs.precursor_mz, refs.charge, q_np, sub.precursor_mz, sub.charge, 500.0,
                           "da", 1)
    assert np.array_equal(gi[which], oi[:, 0]) and np.array_equal(gd[which], od[:, 0])


# ------------------------------------------------ multi-bit components (Section 4.3)
def _comp_workload(seed, D, n_t, n_q, m):
    """Seeded random component rows in [-m, m] (targets, then as many decoys
    with the same precursors) and queries that are copies of targets with 5-60%
    of their components redrawn, 40% at the target's precursor and the rest
    shifted."""
    rng = np.random.default_rng(seed)
    comp = rng.integers(-m, m + 1, (2 * n_t, D)).astype(np.int8)
    mz_t = rng.uniform(400, 1500, n_t)
    z_t = rng.integers(2, 5, n_t).astype(np.uint8)
    mz, z = np.r_[mz_t, mz_t], np.r_[z_t, z_t]
    dec = np.r_[np.zeros(n_t, np.uint8), np.ones(n_t, np.uint8)]
    src = rng.integers(0, n_t, n_q)
    shift = np.where(rng.random(n_q) < 0.4, 0.0, rng.uniform(-900, 900, n_q))
    q_mz, q_z = mz[src] + shift / z[src], z[src]
    q = comp[src].copy()
    redraw = rng.random((n_q, D)) < rng.uniform(0.05, 0.6, (n_q, 1))
    q[redraw] = rng.integers(-m, m + 1, int(redraw.sum()))
    return comp, mz, z, dec, q, q_mz, q_z


def _check_dot(hd, got, want):
    gi, gs, gq, gl = got
    oi, os_, ol, oq = want
    assert np.array_equal(hd.as_u32(gi), oi)
    assert np.array_equal(gs.cpu().numpy(), os_)
    assert np.array_equal(gl.cpu().numpy(), ol)
    assert np.array_equal(gq.cpu().numpy(), oq, equal_nan=True)


@pytest.mark.parametrize("bits,form", [(2, "tc_mxf4"), (3, "tc_mxf4"), (3, "tc_fp4"), (4, "tc_fp8"),
                                       (5, "tc_bf16"), (3, "auto"), (4, "popc")])
@pytest.mark.parametrize("levels,fdr", [(LEVELS2, 0.01), (LEVELS3, 0.05)])
def test_cascade_dot_matches_oracle(hd, bits, form, levels, fdr):
    D, m = 2048, (1 << (bits - 1)) - 1
    comp, mz, z, dec, q, q_mz, q_z = _comp_workload(40 + bits, D, 6000, 2000, m)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library_multibit(ctx, dev(comp), dev(mz), dev(z), bits)
    hd.hd_library_set_decoys(lib, dev(dec))
    if form in ("tc_bf16", "popc"):   # bits <= 3 come with the e2m1 copy, bits 4..5 with e4m3
        hd.hd_library_prepare(lib, form)
    got = hd.hd_cascade_search_dot(lib, dev(q), dev(q_mz), dev(q_z), levels, fdr, form=form)
    torch.cuda.synchronize()
    lib.status()
    want = oracle.cascade_dot(comp, mz, z, dec, q, q_mz, q_z, levels, fdr)
    _check_dot(hd, got, want)
    lv = want[2]
    assert (lv == 0).sum() > 0 and (lv == len(levels) - 1).sum() > 0


def test_cascade_dot_encoded_spectra_and_edges(hd):
    """Multi-bit encode of synthetic spectra on each side, a charge with no
    candidates, the FDR extremes and one query."""
    D, Q, seed, bits = 1024, 8, 5, 3
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = synth.make_references(3000, (2, 3), (0.5, 0.5), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, 400, rng)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    pp = oracle_side.pp_args(Q)

    def enc(sp):
        return hd.hd_encode_multibit(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity),
                                                            **pp), bits)

    lib = hd.hd_build_library_multibit(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge), bits)
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    q_comp = enc(qs)
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, seed)
    o_r = oracle.encode_multibit(D, F, L, *oracle.preprocess(refs.offsets, refs.mz, refs.intensity, **pp), bits)
    o_q = oracle.encode_multibit(D, F, L, *oracle.preprocess(qs.offsets, qs.mz, qs.intensity, **pp), bits)
    z = qs.charge.copy()
    z[::7] = 5
    for fdr in (-1.0, 0.0, 0.02, 1e9):
        got = hd.hd_cascade_search_dot(lib, q_comp, dev(qs.precursor_mz), dev(z), LEVELS2, fdr)
        torch.cuda.synchronize()
        lib.status()
        want = oracle.cascade_dot(o_r, refs.precursor_mz, refs.charge, refs.decoy, o_q, qs.precursor_mz, z,
                                  LEVELS2, fdr)
        _check_dot(hd, got, want)
        assert np.all(got[3].cpu().numpy()[::7] == 255)
        assert np.all(got[1].cpu().numpy()[::7] == np.iinfo(np.int32).min)
    got = hd.hd_cascade_search_dot(lib, q_comp[:1], dev(qs.precursor_mz[:1]), dev(qs.charge[:1]),
                                   [(500.0, "da")], 0.01)
    torch.cuda.synchronize()
    want = oracle.cascade_dot(o_r, refs.precursor_mz, refs.charge, refs.decoy, o_q[:1], qs.precursor_mz[:1],
                              qs.charge[:1], [(500.0, "da")], 0.01)
    _check_dot(hd, got, want)


def test_cascade_dot_argument_errors(hd):
    D = 1024
    comp, mz, z, dec, q, q_mz, q_z = _comp_workload(9, D, 200, 8, 3)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library_multibit(ctx, dev(comp), dev(mz), dev(z), 3)
    args = (dev(q), dev(q_mz), dev(q_z), LEVELS2, 0.01)
    with pytest.raises(hd.HDError) as e:            # no decoy flags yet
        hd.hd_cascade_search_dot(lib, *args)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    hd.hd_library_set_decoys(lib, dev(dec))
    for form in ("popc", "tc_bf16"):                # not a tensor-core form / not prepared
        with pytest.raises(hd.HDError) as e:
            hd.hd_cascade_search_dot(lib, *args, form=form)
        assert e.value.status == hd.HD_ERR_INVALID_ARG
    hv = dev(np.zeros((8, D // 64), np.uint64))
    with pytest.raises(hd.HDError) as e:            # the binary entry point refuses a multi-bit library
        hd.hd_cascade_search(lib, hv, dev(q_mz), dev(q_z), LEVELS2, 0.01)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    blib = hd.hd_build_library(ctx, dev(np.zeros((400, D // 64), np.uint64)), dev(mz), dev(z))
    hd.hd_library_set_decoys(blib, dev(dec))
    with pytest.raises(hd.HDError) as e:            # and the dot entry point a binary one
        hd.hd_cascade_search_dot(blib, *args)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    lib384 = hd.hd_build_library_multibit(hd.Ctx(384, 4, 10, 192, 0), dev(comp[:, :384]), dev(mz), dev(z), 3)
    hd.hd_library_set_decoys(lib384, dev(dec))
    with pytest.raises(hd.HDError) as e:            # kind::mxf4 needs D % 256 == 0
        hd.hd_cascade_search_dot(lib384, dev(q[:, :384]), dev(q_mz), dev(q_z), LEVELS2, 0.01, form="tc_mxf4")
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    got = hd.hd_cascade_search_dot(lib, *args, form="tc_fp4")
    torch.cuda.synchronize()
    lib.status()
    _check_dot(hd, got, oracle.cascade_dot(comp, mz, z, dec, q, q_mz, q_z, LEVELS2, 0.01))


def test_cascade_dot_full_size_one_level(hd):
    """1,000,000 references x 50,000 queries, D=8192, 3-bit components, one
    +-500 level under kind::mxf4: every query's SSM equals the dot-product
    search's top-1, the q-values are recomputed by the oracle from the GPU's
    own SSM scores and decoy flags (bit for bit), and 16 sampled charge-4
    SSMs are checked against the oracle encoding and searching every charge-4
    reference."""
    refs, qs, spec = synth.make_workload("full")
    D, Q, bits = spec["dim"], spec["n_levels"], 3
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 0)
    pp = oracle_side.pp_args(Q)

    def enc(sp):
        return hd.hd_encode_multibit(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity),
                                                            **pp), bits)

    lib = hd.hd_build_library_multibit(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge), bits)
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    q_comp = enc(qs)
    q_mz, q_z = dev(qs.precursor_mz), dev(qs.charge)
    gi, gs, gq, gl = hd.hd_cascade_search_dot(lib, q_comp, q_mz, q_z, [(500.0, "da")], 0.01, form="tc_mxf4")
    si, ss = hd.hd_search_dot(lib, q_comp, q_mz, q_z, 500.0, "da", 1, "tc_mxf4")
    torch.cuda.synchronize()
    lib.status()
    gi, gs, gq, gl = hd.as_u32(gi), gs.cpu().numpy(), gq.cpu().numpy(), gl.cpu().numpy()
    assert np.array_equal(gi, hd.as_u32(si)[:, 0]) and np.array_equal(gs, ss.cpu().numpy()[:, 0])
    has = gi != 0xFFFFFFFF
    qv = oracle.fdr_qvalues(gs[has].astype(np.int64), refs.decoy[gi[has]])
    assert np.array_equal(gq[has], qv) and np.all(np.isnan(gq[~has]))
    ident = np.zeros(qs.n, bool)
    ident[np.nonzero(has)[0]] = (refs.decoy[gi[has]] == 0) & (qv <= 0.01)
    assert np.array_equal(gl == 0, ident) and np.all(gl[~ident] == 255)
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    z4 = np.nonzero(refs.charge == 4)[0]
    r4 = refs.subset(z4)
    R4 = oracle.encode_multibit(D, F, L, *oracle.preprocess(r4.offsets, r4.mz, r4.intensity, **pp), bits)
    rng = np.random.default_rng(78)
    which = np.sort(rng.choice(np.nonzero(qs.charge == 4)[0], 16, replace=False))
    q4 = qs.subset(which)
    Q4 = oracle.encode_multibit(D, F, L, *oracle.preprocess(q4.offsets, q4.mz, q4.intensity, **pp), bits)
    oi, osc = oracle.search_dot(R4, r4.precursor_mz, r4.charge, Q4, q4.precursor_mz, q4.charge, 500.0, "da", 1)
    oi_g = np.where(oi[:, 0] == 0xFFFFFFFF, 0xFFFFFFFF, z4[np.minimum(oi[:, 0], z4.size - 1)]).astype(np.uint32)
    assert np.array_equal(gi[which], oi_g) and np.array_equal(gs[which], osc[:, 0])


def test_cascade_dot_empty_library_and_queries(hd):
    D = 1024
    comp, mz, z, dec, q, q_mz, q_z = _comp_workload(12, D, 50, 20, 3)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    empty = hd.hd_build_library_multibit(ctx, dev(np.zeros((0, D), np.int8)), dev(np.zeros(0)),
                                         dev(np.zeros(0, np.uint8)), 3)
    # an empty library needs no decoy flags
    gi, gs, gq, gl = hd.hd_cascade_search_dot(empty, dev(q), dev(q_mz), dev(q_z), LEVELS2, 0.01)
    torch.cuda.synchronize()
    empty.status()
    assert np.all(hd.as_u32(gi) == 0xFFFFFFFF) and np.all(gs.cpu().numpy() == np.iinfo(np.int32).min)
    assert np.all(gl.cpu().numpy() == 255) and np.all(np.isnan(gq.cpu().numpy()))
    _check_dot(hd, (gi, gs, gq, gl),
               oracle.cascade_dot(np.zeros((0, D), np.int8), np.zeros(0), np.zeros(0, np.uint8),
                                  np.zeros(0, np.uint8), q, q_mz, q_z, LEVELS2, 0.01))
    lib = hd.hd_build_library_multibit(ctx, dev(comp), dev(mz), dev(z), 3)
    hd.hd_library_set_decoys(lib, dev(dec))
    gi, gs, gq, gl = hd.hd_cascade_search_dot(lib, dev(q[:0]), dev(q_mz[:0]), dev(q_z[:0]), LEVELS2, 0.01)
    torch.cuda.synchronize()
    assert gi.numel() == 0 and gs.numel() == 0 and gq.numel() == 0 and gl.numel() == 0
