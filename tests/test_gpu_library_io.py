"""Library save / load (reference HVs encoded once and reused, Section 3.3):
a loaded library is the saved one row for row, and searches on it --
plain, tensor-core and cascade -- return identical results.  Files written
with other item-memory parameters, corrupted or truncated are rejected."""
import os

import numpy as np
import pytest
import torch

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
    return torch.from_numpy(a).cuda()


def _lib(hd, seed=3, D=2048, Q=16, n=6000, n_q=500):
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = synth.make_references(n, (2, 3, 4), (0.6, 0.3, 0.1), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, n_q, rng)
    ctx = hd.Ctx(D, Q, synth.N_BINS, D // 2, seed)
    pp = oracle_side.pp_args(Q)

    def enc(sp):
        return hd.hd_encode(ctx, *hd.hd_preprocess(ctx, dev(sp.offsets), dev(sp.mz), dev(sp.intensity), **pp))

    lib = hd.hd_build_library(ctx, enc(refs), dev(refs.precursor_mz), dev(refs.charge))
    hd.hd_library_set_decoys(lib, dev(refs.decoy))
    return ctx, lib, refs, qs, enc(qs)


def test_round_trip_is_identical(hd, tmp_path):
    ctx, lib, refs, qs, q_hv = _lib(hd)
    path = str(tmp_path / "lib.hdl")
    hd.hd_library_save(lib, ctx, path)
    ctx2 = hd.Ctx(2048, 16, synth.N_BINS, 1024, 3)          # same parameters, a new context
    lib2 = hd.hd_library_load(ctx2, path)
    assert lib2.n == lib.n and lib2.dim == lib.dim
    a, b = hd.hd_library_export(lib), hd.hd_library_export(lib2)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    qm, qz = dev(qs.precursor_mz), dev(qs.charge)
    for form in ("popc", "tc_fp8"):
        for L in (lib, lib2):
            if form != "popc":
                hd.hd_library_prepare(L, form)
        r1 = hd.hd_search_open(lib, q_hv, qm, qz, 500.0, "da", 5, form=form)
        r2 = hd.hd_search_open(lib2, q_hv, qm, qz, 500.0, "da", 5, form=form)
        torch.cuda.synchronize()
        assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1]), form
    c1 = hd.hd_cascade_search(lib, q_hv, qm, qz, [(20.0, "ppm"), (500.0, "da")], 0.01)
    c2 = hd.hd_cascade_search(lib2, q_hv, qm, qz, [(20.0, "ppm"), (500.0, "da")], 0.01)
    torch.cuda.synchronize()
    for x, y in zip(c1, c2):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy(), equal_nan=True)
    lib2.status()


def test_rejects_other_parameters_and_damaged_files(hd, tmp_path):
    ctx, lib, *_ = _lib(hd, n=800, n_q=10)
    path = str(tmp_path / "lib.hdl")
    hd.hd_library_save(lib, ctx, path)
    blob = open(path, "rb").read()
    other = hd.Ctx(2048, 16, synth.N_BINS, 1024, 4)          # another seed
    bad_cases = {"flip": bytearray(blob), "short": blob[:-9], "magic": b"XX" + blob[2:]}
    bad_cases["flip"][len(blob) // 2] ^= 0x40
    with pytest.raises(hd.HDError) as e:
        hd.hd_library_load(other, path)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
    for name, data in bad_cases.items():
        p = str(tmp_path / f"{name}.hdl")
        open(p, "wb").write(bytes(data))
        with pytest.raises(hd.HDError) as e:
            hd.hd_library_load(ctx, p)
        assert e.value.status == hd.HD_ERR_INVALID_ARG, name
    with pytest.raises(hd.HDError):
        hd.hd_library_load(ctx, str(tmp_path / "missing.hdl"))


def test_empty_library_round_trip(hd, tmp_path):
    ctx = hd.Ctx(1024, 8, 10, 512, 0)
    lib = hd.hd_build_library(ctx, torch.zeros((0, 16), dtype=torch.int64, device="cuda"),
                              torch.zeros(0, dtype=torch.float64, device="cuda"),
                              torch.zeros(0, dtype=torch.uint8, device="cuda"))
    path = str(tmp_path / "empty.hdl")
    hd.hd_library_save(lib, ctx, path)
    lib2 = hd.hd_library_load(ctx, path)
    assert lib2.n == 0
    q = torch.zeros((3, 16), dtype=torch.int64, device="cuda")
    i, d = hd.hd_search_open(lib2, q, dev(np.array([500.0, 600.0, 700.0])), dev(np.array([2, 2, 3], np.uint8)),
                             500.0, "da", 2)
    torch.cuda.synchronize()
    assert np.all(hd.as_u32(i) == 0xFFFFFFFF)
    assert os.path.getsize(path) > 0


@pytest.mark.parametrize("bits", [3, 4])
def test_multibit_round_trip(hd, tmp_path, bits):
    """A multi-bit library (Section 4.3 components) is saved with its component
    bits and loaded back row for row: the dot-product search on the loaded
    library equals the saved one's and the oracle's, the default tensor-core
    copy is rebuilt on load, and a file whose components were edited out of
    range (hash recomputed) is refused."""
    import oracle
    D, m = 512, 2 ** (bits - 1) - 1
    rng = np.random.default_rng(60 + bits)
    n, n_q = 3000, 200
    R = rng.integers(-m, m + 1, (n, D)).astype(np.int8)
    mz = rng.uniform(400.0, 420.0, n)
    z = rng.integers(2, 4, n).astype(np.uint8)
    Qv = rng.integers(-m, m + 1, (n_q, D)).astype(np.int8)
    q_mz, q_z = rng.uniform(400.0, 420.0, n_q), rng.integers(2, 4, n_q).astype(np.uint8)
    ctx = hd.Ctx(D, 8, 100, D // 2, 2)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(mz), dev(z), bits)
    path = str(tmp_path / f"mb{bits}.hdl")
    hd.hd_library_save(lib, ctx, path)
    lib2 = hd.hd_library_load(ctx, path)
    assert lib2.n == n and hd.hd_library_component_bits(lib2) == bits
    form = "tc_fp4" if bits <= 3 else "tc_fp8"
    a = hd.hd_search_dot(lib, dev(Qv), dev(q_mz), dev(q_z), 2.0, "da", 5, form)
    b = hd.hd_search_dot(lib2, dev(Qv), dev(q_mz), dev(q_z), 2.0, "da", 5, "auto")
    torch.cuda.synchronize()
    lib2.status()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    oi, osc = oracle.search_dot(R, mz, z, Qv, q_mz, q_z, 2.0, "da", 5)
    assert np.array_equal(b[0].cpu().numpy().view(np.uint32), oi) and np.array_equal(b[1].cpu().numpy(), osc)
    with pytest.raises(hd.HDError):                   # still refused by the binary entry points
        hd.hd_search_open(lib2, torch.zeros((4, D // 64), dtype=torch.int64, device="cuda"), dev(q_mz[:4]),
                          dev(q_z[:4]), 1.0, "da", 1)
    # component out of range, with a valid hash: the load's range check refuses it
    blob = bytearray(open(path, "rb").read())
    head = 8 + 4 * 4 + 8 + 4 * 4                      # magic, dim..alpha, seed, mode, encoder, n, flags
    blob[head + 7] = (m + 1) & 0xFF
    h = 1469598103934665603
    for byte in bytes(blob[:-8]):
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    blob[-8:] = h.to_bytes(8, "little")
    p2 = str(tmp_path / "bad.hdl")
    open(p2, "wb").write(bytes(blob))
    with pytest.raises(hd.HDError) as e:
        hd.hd_library_load(ctx, p2)
    assert e.value.status == hd.HD_ERR_INVALID_ARG
