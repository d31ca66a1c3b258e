"""Multi-bit HV components (Section 4.3) on the GPU against the oracle:
the encoder bit for bit (both encoders, bits 2..5, empty and long spectra),
and the dot-product search through every tensor-core form and schedule,
with exact indices and scores, on encoded spectra and on random components
with ties and extreme scores; plus the boundary's argument checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_16422_gb300 import synth

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


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def random_csr(rng, n, f, Q, lens):
    off = np.zeros(n + 1, np.uint32)
    off[1:] = np.cumsum(lens)
    b = np.concatenate([np.sort(rng.choice(f, l, replace=False)) for l in lens]).astype(np.uint32) \
        if sum(lens) else np.zeros(0, np.uint32)
    lv = rng.integers(0, Q, int(off[-1])).astype(np.uint8)
    return off, b, lv


@pytest.mark.parametrize("D,Q,f,encoder", [(128, 4, 60, "id_level"), (2048, 16, 3000, "id_level"),
                                           (4096, 16, 3000, "id_level"), (8192, 32, synth.N_BINS, "id_level"),
                                           (32768, 32, 3000, "id_level"), (1024, 64, 2000, "projection"),
                                           (4096, 256, 5000, "projection")])
def test_encode_multibit_bit_exact(hd, D, Q, f, encoder):
    rng = np.random.default_rng(D + Q)
    lens = [0, 1, 2, 3, 50, min(1023, f)] + list(rng.integers(0, 120, 90))
    lens = [min(l, f) for l in lens]
    off, b, lv = random_csr(rng, len(lens), f, Q, lens)
    ctx = hd.Ctx(D, Q, f, D // 2, 3, encoder=encoder)
    F, L, _, _ = oracle.item_memory(D, Q, f, D // 2, 3)
    enc = 1 if encoder == "projection" else 0
    for bits in (2, 3, 4, 5):
        got = hd.hd_encode_multibit(ctx, dev(off), dev(b), dev(lv), bits)
        torch.cuda.synchronize()
        ctx.status()
        want = oracle.encode_multibit(D, F, L, off, b, lv, bits, encoder=enc)
        assert np.array_equal(got.cpu().numpy(), want), bits


def windowed(rng, n_ref, n_q, lo=400.0, hi=460.0):
    ref_mz = rng.uniform(lo, hi, n_ref)
    ref_z = rng.integers(2, 4, n_ref).astype(np.uint8)
    q_mz = rng.uniform(lo, hi, n_q)
    q_z = rng.integers(2, 4, n_q).astype(np.uint8)
    return ref_mz, ref_z, q_mz, q_z


def check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, tol, unit, k, form):
    gi, gs = hd.hd_search_dot(lib, dev(Qv), dev(q_mz), dev(q_z), tol, unit, k, form)
    torch.cuda.synchronize()
    lib.status()
    oi, osc = oracle.search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, tol, unit, k)
    assert np.array_equal(u32(gi), oi), (form, unit, k)
    assert np.array_equal(gs.cpu().numpy(), osc), (form, unit, k)
    return oi


@pytest.mark.parametrize("bits", [2, 3, 4, 5])
def test_search_dot_encoded_spectra(hd, bits):
    """Encoded synthetic-style spectra: 3000 references (12 tiles, ragged), 700
    queries, every applicable form, three window units, k 1 / 5 / 16."""
    D, Q, f = 2048, 16, 4000
    rng = np.random.default_rng(bits)
    n_ref, n_q = 3000, 700
    r_off, r_b, r_lv = random_csr(rng, n_ref, f, Q, list(rng.integers(1, 60, n_ref)))
    q_off, q_b, q_lv = random_csr(rng, n_q, f, Q, list(rng.integers(0, 60, n_q)))
    ctx = hd.Ctx(D, Q, f, D // 2, 9)
    r_gpu = hd.hd_encode_multibit(ctx, dev(r_off), dev(r_b), dev(r_lv), bits)
    q_gpu = hd.hd_encode_multibit(ctx, dev(q_off), dev(q_b), dev(q_lv), bits)
    F, L, _, _ = oracle.item_memory(D, Q, f, D // 2, 9)
    R = oracle.encode_multibit(D, F, L, r_off, r_b, r_lv, bits)
    Qv = oracle.encode_multibit(D, F, L, q_off, q_b, q_lv, bits)
    assert np.array_equal(r_gpu.cpu().numpy(), R) and np.array_equal(q_gpu.cpu().numpy(), Qv)
    ref_mz, ref_z, q_mz, q_z = windowed(rng, n_ref, n_q)
    lib = hd.hd_build_library_multibit(ctx, r_gpu, dev(ref_mz), dev(ref_z), bits)
    assert hd.hd_library_component_bits(lib) == bits
    forms = ["tc_fp8", "tc_bf16", "popc"] + (["tc_fp4", "tc_mxf4"] if bits <= 3 else [])
    for form in forms:
        hd.hd_library_prepare(lib, form)
    for form in forms:
        for unit, tol, k in (("da", 6.0, 5), ("ppm", 9000.0, 1), ("mass", 15.0, 16)):
            check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, tol, unit, k, form)
    # 'auto' takes e2m1 (kind::mxf4) when the library holds it, else e4m3
    oi = check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, 6.0, "da", 5, "auto")
    assert np.mean(oi[:, 0] != 0xFFFFFFFF) > 0.9


@pytest.mark.parametrize("cluster,cta_group", [(2, 2), (1, 1)])
@pytest.mark.parametrize("form,bits", [("tc_fp4", 3), ("tc_fp8", 4), ("tc_mxf4", 3), ("popc", 5)])
def test_search_dot_random_components_schedules(hd, form, bits, cluster, cta_group):
    """Random components in [-m, m], duplicate rows (ties go to the lower input
    index) and rows of all +m / all -m (scores D m^2 and -D m^2, the ends of
    the key range), under the pair and 1-SM schedules."""
    D, m = 1024, 2 ** (bits - 1) - 1
    rng = np.random.default_rng(bits * 10 + cluster + cta_group)
    n_ref, n_q = 2600, 450
    R = rng.integers(-m, m + 1, (n_ref, D)).astype(np.int8)
    Qv = rng.integers(-m, m + 1, (n_q, D)).astype(np.int8)
    ref_mz, ref_z, q_mz, q_z = windowed(rng, n_ref, n_q, 400.0, 410.0)
    for a, b_ in ((100, 5), (2000, 7), (611, 2599)):     # duplicate rows b_ of rows a
        R[b_], ref_mz[b_], ref_z[b_] = R[a], ref_mz[a], ref_z[a]
    R[10], R[11] = m, -m
    ref_z[11], ref_mz[11] = ref_z[10], ref_mz[10]
    Qv[0], q_mz[0], q_z[0] = m, ref_mz[10], ref_z[10]    # S = D m^2 with row 10, -D m^2 with row 11
    Qv[1], q_mz[1], q_z[1] = R[100], ref_mz[100], ref_z[100]
    ctx = hd.Ctx(D, 8, 100, D // 2, 1)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(ref_mz), dev(ref_z), bits)
    hd.hd_library_prepare(lib, form)
    hd.hd_library_set_schedule(lib, 4, 2, cluster, cta_group)
    oi = check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, 1.5, "da", 16, form)
    assert oi[0, 0] == 10 and oi[1, 0] == 5 and oi[1, 1] == 100
    gi, gs = hd.hd_search_dot(lib, dev(Qv[:1]), dev(q_mz[:1]), dev(q_z[:1]), 0.0, "da", 16, form)
    s = gs.cpu().numpy()[0]
    assert s[0] == D * m * m and s[u32(gi)[0] == 11][0] == -D * m * m


def test_search_dot_d8192_tiles_and_tail(hd):
    """D = 8192 (64 K-chunks per tile), 100,003 references: many tiles and a
    ragged last tile; 40 queries over wide windows checked in full."""
    D, bits, m = 8192, 3, 3
    rng = np.random.default_rng(77)
    n_ref, n_q = 100003, 40
    R = rng.integers(-m, m + 1, (n_ref, D), dtype=np.int8)
    Qv = rng.integers(-m, m + 1, (n_q, D), dtype=np.int8)
    ref_mz = rng.uniform(400, 1500, n_ref)
    ref_z = rng.integers(2, 4, n_ref).astype(np.uint8)
    q_mz = rng.uniform(400, 1500, n_q)
    q_z = rng.integers(2, 4, n_q).astype(np.uint8)
    ctx = hd.Ctx(D, 8, 100, D // 2, 1)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(ref_mz), dev(ref_z), bits)
    for form in ("tc_fp4", "tc_fp8"):
        hd.hd_library_prepare(lib, form)
        check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, 500.0, "da", 5, form)


def test_multibit_argument_checks(hd):
    D = 256
    rng = np.random.default_rng(0)
    ctx = hd.Ctx(D, 8, 100, D // 2, 1)
    R = rng.integers(-3, 4, (300, D)).astype(np.int8)
    mz = rng.uniform(400, 401, 300)
    z = np.full(300, 2, np.uint8)
    with pytest.raises(hd.HDError):                    # bits out of range
        hd.hd_build_library_multibit(ctx, dev(R), dev(mz), dev(z), 6)
    bad = R.copy()
    bad[17, 5] = 4                                     # |h| > m for bits 3
    with pytest.raises(hd.HDError) as e:
        hd.hd_build_library_multibit(ctx, dev(bad), dev(mz), dev(z), 3)
    assert e.value.status == 1
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(mz), dev(z), 3)
    lib4 = hd.hd_build_library_multibit(ctx, dev(R), dev(mz), dev(z), 4)
    with pytest.raises(hd.HDError) as e:               # e2m1 cannot hold 4..7
        hd.hd_library_prepare(lib4, "tc_fp4")
    assert e.value.status == 5
    with pytest.raises(hd.HDError):                    # binary entry points refuse it
        hd.hd_search_open(lib, torch.zeros((4, D // 64), dtype=torch.int64, device="cuda"),
                          dev(mz[:4]), dev(z[:4]), 1.0, "da", 1)
    with pytest.raises(hd.HDError):                    # the popcount form needs its bit planes first
        hd.hd_search_dot(lib, dev(R[:4]), dev(mz[:4]), dev(z[:4]), 1.0, "da", 1, "popc")
    hd.hd_library_prepare(lib, "popc")
    check_dot(hd, lib, R, mz, z, R[:4], mz[:4], z[:4], 1.0, "da", 3, "popc")
    binary = hd.hd_build_library(ctx, torch.zeros((300, D // 64), dtype=torch.int64, device="cuda"),
                                 dev(mz), dev(z))
    with pytest.raises(hd.HDError):                    # hd_search_dot refuses a binary library
        hd.hd_search_dot(binary, dev(R[:4]), dev(mz[:4]), dev(z[:4]), 1.0, "da", 1)
    with pytest.raises(hd.HDError):                    # not prepared for this form
        hd.hd_search_dot(lib, dev(R[:4]), dev(mz[:4]), dev(z[:4]), 1.0, "da", 1, "tc_bf16")
    # a query component out of range flags the library's status
    q = R[:4].copy()
    q[2, 9] = -5
    hd.hd_search_dot(lib, dev(q), dev(mz[:4]), dev(z[:4]), 1.0, "da", 1, "tc_fp4")
    torch.cuda.synchronize()
    with pytest.raises(hd.HDError):
        lib.status()
    lib.status()                                       # the flag is consumed
    # no queries, and an empty library: every slot padded
    gi, gs = hd.hd_search_dot(lib, dev(R[:0]), dev(mz[:0]), dev(z[:0]), 1.0, "da", 3)
    assert gi.shape == (0, 3)
    empty = hd.hd_build_library_multibit(ctx, dev(R[:0]), dev(mz[:0]), dev(z[:0]), 3)
    gi, gs = hd.hd_search_dot(empty, dev(R[:5]), dev(mz[:5]), dev(z[:5]), 1.0, "da", 3)
    torch.cuda.synchronize()
    assert np.all(u32(gi) == 0xFFFFFFFF) and np.all(gs.cpu().numpy() == np.iinfo(np.int32).min)


def test_search_dot_full_size_sampled(hd):
    """The multi-bit benchmark's shapes: the 1,000,000-reference "full" library
    and 50,000 queries, D=8192, 3-bit components, +-500 Da, top-5, e2m1 SM
    pairs.  e4m3 gives the same result on every query; the oracle encodes every
    charge-4 reference and answers 16 sampled charge-4 queries by brute force;
    a sample of spectra is encoded by both sides."""
    refs, qs, spec = synth.make_workload("full")
    D, Q, k, bits = spec["dim"], spec["n_levels"], spec["k"], 3
    pp = dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
              max_peaks=synth.MAX_PEAKS, n_levels=Q)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, 0)
    r_csr = hd.hd_preprocess(ctx, dev(refs.offsets), dev(refs.mz), dev(refs.intensity), **pp)
    q_csr = hd.hd_preprocess(ctx, dev(qs.offsets), dev(qs.mz), dev(qs.intensity), **pp)
    r_comp = hd.hd_encode_multibit(ctx, *r_csr, bits)
    q_comp = hd.hd_encode_multibit(ctx, *q_csr, bits)
    lib = hd.hd_build_library_multibit(ctx, r_comp, dev(refs.precursor_mz), dev(refs.charge), bits)
    q_mz, q_z = dev(qs.precursor_mz), dev(qs.charge)
    gi, gs = hd.hd_search_dot(lib, q_comp, q_mz, q_z, spec["tol"], spec["unit"], k, "tc_fp4")
    torch.cuda.synchronize()
    lib.status()
    gi, gs = u32(gi), gs.cpu().numpy()
    hd.hd_library_prepare(lib, "tc_fp8")
    for form in ("tc_fp8", "tc_mxf4"):
        ei, es = hd.hd_search_dot(lib, q_comp, q_mz, q_z, spec["tol"], spec["unit"], k, form)
        torch.cuda.synchronize()
        assert np.array_equal(u32(ei), gi) and np.array_equal(es.cpu().numpy(), gs), form
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, D // 2, 0)
    rng = np.random.default_rng(8)
    rs = np.sort(rng.choice(refs.n, 100, replace=False))
    sub = refs.subset(rs)
    want = oracle.encode_multibit(D, F, L, *oracle.preprocess(sub.offsets, sub.mz, sub.intensity, **pp), bits)
    assert np.array_equal(r_comp[torch.from_numpy(rs).cuda()].cpu().numpy(), want)
    z4 = np.nonzero(refs.charge == 4)[0]
    r4 = refs.subset(z4)
    R4 = oracle.encode_multibit(D, F, L, *oracle.preprocess(r4.offsets, r4.mz, r4.intensity, **pp), bits)
    which = np.sort(rng.choice(np.nonzero(qs.charge == 4)[0], 16, replace=False))
    q4 = qs.subset(which)
    Q4 = oracle.encode_multibit(D, F, L, *oracle.preprocess(q4.offsets, q4.mz, q4.intensity, **pp), bits)
    oi, osc = oracle.search_dot(R4, r4.precursor_mz, r4.charge, Q4, q4.precursor_mz, q4.charge, spec["tol"],
                                spec["unit"], k)
    oi_g = np.where(oi == 0xFFFFFFFF, 0xFFFFFFFF, z4[np.minimum(oi, z4.size - 1)]).astype(np.uint32)
    assert np.array_equal(gi[which], oi_g) and np.array_equal(gs[which], osc)


@pytest.mark.parametrize("bits,D", [(2, 128), (3, 1024), (3, 1152), (4, 2176), (5, 4096)])
def test_search_dot_popc_chunks(hd, bits, D):
    """The popcount form on bit planes: one chunk of 1024 components, a ragged
    last chunk (1152 = 1024 + 128, 2176 = 2 x 1024 + 128), D below one chunk;
    random components with duplicate rows and all +m / all -m rows; k 1 / 5 /
    16 and the three window units against the oracle; equal to a tensor-core
    form on every query."""
    m = 2 ** (bits - 1) - 1
    rng = np.random.default_rng(bits * 100 + D)
    n_ref, n_q = 1500, 300
    R = rng.integers(-m, m + 1, (n_ref, D)).astype(np.int8)
    Qv = rng.integers(-m, m + 1, (n_q, D)).astype(np.int8)
    ref_mz, ref_z, q_mz, q_z = windowed(rng, n_ref, n_q, 400.0, 420.0)
    R[7], ref_mz[7], ref_z[7] = R[3], ref_mz[3], ref_z[3]
    R[10], R[11] = m, -m
    ref_z[11], ref_mz[11] = ref_z[10], ref_mz[10]
    Qv[0], q_mz[0], q_z[0] = m, ref_mz[10], ref_z[10]
    Qv[1], q_mz[1], q_z[1] = R[3], ref_mz[3], ref_z[3]
    ctx = hd.Ctx(D, 8, 100, D // 2, 1)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(ref_mz), dev(ref_z), bits)
    hd.hd_library_prepare(lib, "popc")
    for unit, tol, k in (("da", 3.0, 5), ("ppm", 5000.0, 1), ("mass", 9.0, 16)):
        oi = check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, tol, unit, k, "popc")
    gi, gs = hd.hd_search_dot(lib, dev(Qv[:2]), dev(q_mz[:2]), dev(q_z[:2]), 0.0, "da", 16, "popc")
    s0, i0 = gs.cpu().numpy(), u32(gi)
    assert s0[0, 0] == D * m * m and s0[0][i0[0] == 11][0] == -D * m * m
    assert i0[1, 0] == 3 and i0[1, 1] == 7 and s0[1, 0] == s0[1, 1]
    tc = "tc_fp4" if bits <= 3 else "tc_fp8"
    hd.hd_library_prepare(lib, tc)
    a = hd.hd_search_dot(lib, dev(Qv), dev(q_mz), dev(q_z), 10.0, "da", 5, "popc")
    b = hd.hd_search_dot(lib, dev(Qv), dev(q_mz), dev(q_z), 10.0, "da", 5, tc)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("bits,tg", [(2, 3), (3, 16)])
def test_search_dot_mxf4_two_tiles_per_stage(hd, bits, tg):
    """Multi-bit components through kind::mxf4 with each staged query chunk
    scored against two reference tiles: the oracle's scores and indices."""
    D, m = 1024, 2 ** (bits - 1) - 1
    rng = np.random.default_rng(500 + bits)
    n_ref, n_q = 5200, 300
    R = rng.integers(-m, m + 1, (n_ref, D)).astype(np.int8)
    Qv = rng.integers(-m, m + 1, (n_q, D)).astype(np.int8)
    ref_mz, ref_z, q_mz, q_z = windowed(rng, n_ref, n_q, 400.0, 410.0)
    ctx = hd.Ctx(D, 8, 100, D // 2, 1)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(ref_mz), dev(ref_z), bits)
    hd.hd_library_prepare(lib, "tc_mxf4")
    hd.hd_library_set_schedule(lib, tg, 2, 2, 2)
    hd.hd_library_set_stage_tiles(lib, 2)
    check_dot(hd, lib, R, ref_mz, ref_z, Qv, q_mz, q_z, 3.0, "da", 8, "tc_mxf4")
