"""Encoder variants (Section 4.2, "Encoding strategy"; Section 3.3.1's
random-walk reading) on the GPU against the oracle, bit for bit: the
position tables of the walk and of independent random IDs, the
random-projection encoder, and a search on variant HVs."""
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


MODES = {"nested": 0, "walk": 1, "random": 2}


@pytest.mark.parametrize("mode,D,Q,f,alpha,seed", [("walk", 512, 4, 300, 1, 3), ("walk", 2048, 16, 5000, 37, 4),
                                                   ("walk", 8192, 32, synth.N_BINS, 256, 0),
                                                   ("walk", 384, 3, 7, 0, 9),
                                                   ("random", 2048, 16, 3000, 0, 5),
                                                   ("random", 8192, 32, synth.N_BINS, 0, 0),
                                                   ("random", 128, 2, 1, 0, 1)])
def test_item_memory_variants_bit_exact(hd, mode, D, Q, f, alpha, seed):
    ctx = hd.Ctx(D, Q, f, alpha, seed, position_mode=mode)
    F, L, _, _ = hd.hd_ctx_item_memory(ctx)
    torch.cuda.synchronize()
    oF, oL, _, _ = oracle.item_memory(D, Q, f, alpha, seed, mode=MODES[mode])
    assert np.array_equal(hd.as_u64(F), oF)
    assert np.array_equal(hd.as_u64(L), oL)


def _random_csr(rng, n, f, Q, lens):
    off = np.zeros(n + 1, np.uint32)
    off[1:] = np.cumsum(lens)
    b = np.concatenate([np.sort(rng.choice(f, l, replace=False)) for l in lens]).astype(np.uint32) \
        if sum(lens) else np.zeros(0, np.uint32)
    lv = rng.integers(0, Q, int(off[-1])).astype(np.uint8)
    return off, b, lv


@pytest.mark.parametrize("mode,D,f,Q", [("random", 2048, 3000, 16), ("nested", 8192, synth.N_BINS, 32),
                                        ("walk", 1024, 2000, 256), ("random", 128, 50, 4)])
def test_projection_encoder_bit_exact(hd, mode, D, f, Q):
    rng = np.random.default_rng(D + Q)
    special = [0, 1, 2, 3, 50, 1023]
    n = 160
    lens = special + list(rng.integers(0, 120, n - len(special)))
    lens = [min(l, f) for l in lens]
    off, b, lv = _random_csr(rng, n, f, Q, lens)
    alpha = 7 if mode == "walk" else D // 2
    ctx = hd.Ctx(D, Q, f, alpha, 6, position_mode=mode, encoder="projection")
    got = hd.hd_encode(ctx, dev(off), dev(b), dev(lv))
    torch.cuda.synchronize()
    ctx.status()
    F, L, _, _ = oracle.item_memory(D, Q, f, alpha, 6, mode=MODES[mode])
    assert np.array_equal(hd.as_u64(got), oracle.encode(D, F, L, off, b, lv, encoder=1))


@pytest.mark.parametrize("mode,encoder", [("random", "id_level"), ("walk", "id_level"), ("random", "projection")])
def test_search_on_variant_hvs(hd, mode, encoder):
    """Preprocess + encode (variant) + library + e4m3 search against the
    oracle's own pipeline with the same variant."""
    D, Q, seed = 2048, 16, 12
    alpha = 16 if mode == "walk" else D // 2
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = synth.make_references(6000, (2, 3), (0.5, 0.5), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, 400, rng)
    ctx = hd.Ctx(D, Q, synth.N_BINS, alpha, seed, position_mode=mode, encoder=encoder)
    pp = oracle_side.pp_args(Q)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    lib = hd.hd_build_library(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge))
    hd.hd_library_prepare(lib, "tc_fp8")
    q_hv = enc(qs)
    i, d = hd.hd_search_open(lib, q_hv, dev(qs.precursor_mz), dev(qs.charge), 500.0, "da", 3, form="tc_fp8")
    torch.cuda.synchronize()
    lib.status()
    F, L, _, _ = oracle.item_memory(D, Q, synth.N_BINS, alpha, seed, mode=MODES[mode])
    ecode = 1 if encoder == "projection" else 0

    def o_enc(sp):
        return oracle.encode(D, F, L, *oracle.preprocess(sp.offsets, sp.mz, sp.intensity, **pp), encoder=ecode)

    o_r, o_q = o_enc(refs), o_enc(qs)
    assert np.array_equal(hd.as_u64(q_hv), o_q)
    oi, od = oracle.search(D, o_r, refs.precursor_mz, refs.charge, o_q, qs.precursor_mz, qs.charge, 500.0, "da", 3)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)


def test_variant_arguments_checked(hd):
    for kw in (dict(position_mode="walk", alpha=257), ):
        with pytest.raises(hd.HDError) as e:
            hd.Ctx(512, 4, 10, seed=0, **kw)
        assert e.value.status == hd.HD_ERR_INVALID_ARG
