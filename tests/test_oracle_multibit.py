"""Pins of the oracle's multi-bit components and their dot-product search
(Section 4.3: a higher precision per HV component raises the
identification rate; the quantiser is the reading stated in the oracle).

Encoder: the closed form of a one-peak spectrum (every component +-m),
invariance under duplicating every peak, sign agreement with the pinned
binary encoder, the round-half-up error bound against a numpy bundle of
Eq. 1 computed from unpacked bits, and the empty spectrum.  Search: +-1
components reduce it to the pinned Hamming search (S = D - 2 dist), a numpy
integer matrix-product brute force on windowed data, and Cauchy-Schwarz."""
import numpy as np
import pytest

import oracle
from tests.helpers import bits

D, Q, NB = 1024, 8, 300


@pytest.fixture(scope="module")
def im():
    F, L, _, _ = oracle.item_memory(D, Q, NB, D // 2, 21)
    return F, L


def random_csr(rng, n, max_peaks=40, min_peaks=1):
    counts = rng.integers(min_peaks, max_peaks + 1, n)
    off = np.r_[0, np.cumsum(counts)].astype(np.uint32)
    nnz = int(off[-1])
    return off, rng.integers(0, NB, nnz).astype(np.uint32), rng.integers(0, Q, nnz).astype(np.uint8)


def bundle(F, L, off, bins, levels, encoder):
    """Eq. 1's integer bundle from unpacked bits: sum over peaks of F_bin * L_level
    in bipolar form (encoder 0), or of (level + 1) * F_bin (encoder 1)."""
    Fb = 1 - 2 * bits(F).astype(np.int64)
    Lb = 1 - 2 * bits(L).astype(np.int64)
    out = np.zeros((off.size - 1, D), np.int64)
    for s in range(off.size - 1):
        for p in range(off[s], off[s + 1]):
            if encoder == 0:
                out[s] += Fb[bins[p]] * Lb[levels[p]]
            else:
                out[s] += (int(levels[p]) + 1) * Fb[bins[p]]
    return out


@pytest.mark.parametrize("encoder", [0, 1])
@pytest.mark.parametrize("nbits", [2, 3, 4])
def test_one_peak_closed_form(im, nbits, encoder):
    F, L = im
    m = 2 ** (nbits - 1) - 1
    rng = np.random.default_rng(nbits)
    off = np.arange(0, 11, dtype=np.uint32)
    b = rng.integers(0, NB, 10).astype(np.uint32)
    lv = rng.integers(0, Q, 10).astype(np.uint8)
    h = oracle.encode_multibit(D, F, L, off, b, lv, nbits, encoder=encoder)
    ref = bits(F[b] ^ L[lv]) if encoder == 0 else bits(F[b])
    assert np.array_equal(h, (m * (1 - 2 * ref.astype(np.int64))).astype(np.int8))


@pytest.mark.parametrize("encoder", [0, 1])
def test_duplicating_every_peak_keeps_components(im, encoder):
    F, L = im
    rng = np.random.default_rng(5)
    off, b, lv = random_csr(rng, 12)
    off2 = (2 * off).astype(np.uint32)
    b2, lv2 = np.repeat(b, 2), np.repeat(lv, 2)
    for nbits in (2, 3, 4):
        h1 = oracle.encode_multibit(D, F, L, off, b, lv, nbits, encoder=encoder)
        h2 = oracle.encode_multibit(D, F, L, off2, b2, lv2, nbits, encoder=encoder)
        assert np.array_equal(h1, h2)


@pytest.mark.parametrize("encoder", [0, 1])
def test_sign_range_and_rounding(im, encoder):
    F, L = im
    rng = np.random.default_rng(7 + encoder)
    off, b, lv = random_csr(rng, 20)
    I = bundle(F, L, off, b, lv, encoder)
    hb = bits(oracle.encode(D, F, L, off, b, lv, encoder=encoder)).astype(np.int64)
    M = np.abs(I).max(axis=1, keepdims=True)
    assert np.all(M > 0)
    for nbits in (2, 3, 4):
        m = 2 ** (nbits - 1) - 1
        h = oracle.encode_multibit(D, F, L, off, b, lv, nbits, encoder=encoder).astype(np.int64)
        assert np.all(np.abs(h) <= m) and np.all(np.abs(h).max(axis=1) == m)
        # the sign agrees with the binary HV: +1 <-> bit 0, -1 <-> bit 1
        assert np.all(hb[h > 0] == 0) and np.all(hb[h < 0] == 1)
        assert np.all(h[I == 0] == 0)
        assert np.all(np.sign(h[h != 0]) == np.sign(I[h != 0]))
        # |h| is m |I| / M rounded to the nearest integer: |2 M |h| - 2 m |I|| <= M ...
        err = 2 * M * np.abs(h) - 2 * m * np.abs(I)
        assert np.all(np.abs(err) <= M)
        # ... and an exact half is rounded up in magnitude
        half = np.abs(err) == M
        assert np.all(err[half] > 0)


def test_empty_spectrum_is_zero(im):
    F, L = im
    off = np.array([0, 0, 3], np.uint32)
    b = np.array([1, 2, 3], np.uint32)
    lv = np.array([1, 2, 3], np.uint8)
    h = oracle.encode_multibit(D, F, L, off, b, lv, 3)
    assert np.all(h[0] == 0) and np.abs(h[1]).max() == 3


def test_bad_arguments():
    F, L, _, _ = oracle.item_memory(D, Q, NB, D // 2, 1)
    off = np.array([0, 1], np.uint32)
    with pytest.raises(ValueError):
        oracle.encode_multibit(D, F, L, off, np.array([1], np.uint32), np.array([1], np.uint8), 1)
    with pytest.raises(ValueError):
        oracle.encode_multibit(D, F, L, off, np.array([1], np.uint32), np.array([1], np.uint8), 9)


def windowed_data(rng, n_ref, n_q):
    ref_mz = rng.uniform(400, 430, n_ref)
    ref_z = rng.integers(2, 4, n_ref).astype(np.uint8)
    q_mz = rng.uniform(400, 430, n_q)
    q_z = rng.integers(2, 4, n_q).astype(np.uint8)
    return ref_mz, ref_z, q_mz, q_z


def test_pm1_components_reduce_to_hamming_search(im):
    """bits = 2 on one-peak spectra gives +-1 components, and S = D - 2 dist."""
    F, L = im
    rng = np.random.default_rng(11)
    n_ref, n_q = 300, 40
    rb, rl = rng.integers(0, NB, n_ref).astype(np.uint32), rng.integers(0, Q, n_ref).astype(np.uint8)
    qb, ql = rng.integers(0, NB, n_q).astype(np.uint32), rng.integers(0, Q, n_q).astype(np.uint8)
    r_off, q_off = np.arange(n_ref + 1, dtype=np.uint32), np.arange(n_q + 1, dtype=np.uint32)
    r_h = oracle.encode_multibit(D, F, L, r_off, rb, rl, 2)
    q_h = oracle.encode_multibit(D, F, L, q_off, qb, ql, 2)
    r_b = oracle.encode(D, F, L, r_off, rb, rl)
    q_b = oracle.encode(D, F, L, q_off, qb, ql)
    assert np.all(np.abs(r_h) == 1)
    ref_mz, ref_z, q_mz, q_z = windowed_data(rng, n_ref, n_q)
    for unit, tol in (("da", 5.0), ("ppm", 20000.0), ("mass", 12.0)):
        i1, s1 = oracle.search_dot(r_h, ref_mz, ref_z, q_h, q_mz, q_z, tol, unit, k=7)
        i2, d2 = oracle.search(D, r_b, ref_mz, ref_z, q_b, q_mz, q_z, tol, unit, k=7)
        assert np.array_equal(i1, i2)
        ok = i2 != 0xFFFFFFFF
        assert np.array_equal(s1[ok], D - 2 * d2[ok].astype(np.int32))
        assert np.all(s1[~ok] == np.iinfo(np.int32).min)


def numpy_search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, tol, k):
    """Brute force: all dot products by an int64 matrix product, candidates by
    the plain window predicate, the k best by (score descending, index ascending)."""
    S = Qv.astype(np.int64) @ R.astype(np.int64).T
    idx = np.full((Qv.shape[0], k), 0xFFFFFFFF, np.uint32)
    sc = np.full((Qv.shape[0], k), np.iinfo(np.int32).min, np.int32)
    for q in range(Qv.shape[0]):
        cand = np.nonzero((ref_z == q_z[q]) & (np.abs(ref_mz - q_mz[q]) <= tol))[0]
        order = np.lexsort((cand, -S[q, cand]))[:k]
        idx[q, :order.size] = cand[order]
        sc[q, :order.size] = S[q, cand[order]]
    return idx, sc


@pytest.mark.parametrize("m", [1, 3, 7])
def test_search_dot_brute_force(m):
    rng = np.random.default_rng(m)
    n_ref, n_q, dim = 500, 60, 256
    R = rng.integers(-m, m + 1, (n_ref, dim)).astype(np.int8)
    Qv = rng.integers(-m, m + 1, (n_q, dim)).astype(np.int8)
    R[7] = R[3]                       # duplicate rows: equal scores, lower index first
    Qv[0] = R[3]
    ref_mz, ref_z, q_mz, q_z = windowed_data(rng, n_ref, n_q)
    ref_mz[7], ref_z[7] = ref_mz[3], ref_z[3]
    q_mz[0], q_z[0] = ref_mz[3], ref_z[3]
    for k in (1, 5, 40):
        i1, s1 = oracle.search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, 3.0, "da", k=k)
        i2, s2 = numpy_search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, 3.0, k)
        assert np.array_equal(i1, i2) and np.array_equal(s1, s2)
    i1, s1 = oracle.search_dot(R, ref_mz, ref_z, Qv, q_mz, q_z, 3.0, "da", k=2)
    assert i1[0, 0] == 3 and i1[0, 1] == 7 and s1[0, 0] == s1[0, 1] == int((R[3].astype(np.int64) ** 2).sum())


def test_encoded_scores_obey_cauchy_schwarz(im):
    F, L = im
    rng = np.random.default_rng(13)
    off, b, lv = random_csr(rng, 50)
    h = oracle.encode_multibit(D, F, L, off, b, lv, 3)
    mz = np.full(50, 500.0)
    z = np.full(50, 2, np.uint8)
    idx, sc = oracle.search_dot(h, mz, z, h, mz, z, 0.0, "da", k=50)
    norms = (h.astype(np.int64) ** 2).sum(axis=1)
    for q in range(50):
        s = np.zeros(50, np.int64)
        s[idx[q]] = sc[q]
        assert np.all(s.astype(np.float64) ** 2 <= norms[q] * norms.astype(np.float64) + 1e-9)
        assert s[q] == norms[q]
