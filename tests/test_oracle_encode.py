"""Pins of the oracle's encoder (Eq. 1 and the binarisation after it).

Bind = element-wise product (XOR of bits), bundle = sum, binarise: positive
-> +1 (bit 0), otherwise -1 (bit 1).  Closed forms that follow: one peak
gives F xor L; two peaks give the OR of the bound vectors (a zero sum maps to
-1); three give the bitwise majority; for any n the result is the majority of
the bound bits with ties going to bit 1.  Duplicating all peaks or reordering
them changes nothing."""
import numpy as np
import pytest

import oracle
from tests.helpers import bits, pack

D, Q, NB = 256, 8, 64


@pytest.fixture(scope="module")
def im():
    F, L, _, _ = oracle.item_memory(D, Q, NB, D // 2, seed=77)
    return F, L


def _enc(im, rows):
    F, L = im
    off = np.zeros(len(rows) + 1, np.uint32)
    off[1:] = np.cumsum([len(r) for r in rows])
    b = np.array([p[0] for r in rows for p in r], np.uint32)
    lv = np.array([p[1] for r in rows for p in r], np.uint8)
    return oracle.encode(D, F, L, off, b, lv)


def _bound(im, peaks):
    F, L = im
    return np.stack([bits(F[b] ^ L[l]) for b, l in peaks])


def test_empty_is_all_minus_one(im):
    out = _enc(im, [[]])
    assert np.all(bits(out) == 1)


def test_one_peak_is_bind(im):
    F, L = im
    out = _enc(im, [[(5, 3)], [(63, 0)]])
    assert np.array_equal(out[0], F[5] ^ L[3])
    assert np.array_equal(out[1], F[63] ^ L[0])


def test_two_peaks_or(im):
    F, L = im
    out = _enc(im, [[(1, 2), (40, 7)]])
    assert np.array_equal(out[0], (F[1] ^ L[2]) | (F[40] ^ L[7]))


def test_three_peaks_majority(im):
    F, L = im
    a, b, c = F[3] ^ L[1], F[30] ^ L[4], F[50] ^ L[6]
    out = _enc(im, [[(3, 1), (30, 4), (50, 6)]])
    assert np.array_equal(out[0], (a & b) | (a & c) | (b & c))


def test_tie_goes_to_minus_one(im):
    F, L = im
    a, b = F[2] ^ L[1], F[9] ^ L[5]
    # identical peaks never tie; a,a,b,b ties wherever a and b differ -> bit 1
    out = _enc(im, [[(0, 0), (0, 0)], [(2, 1), (2, 1), (9, 5), (9, 5)]])
    assert np.array_equal(out[0], F[0] ^ L[0])
    assert np.array_equal(out[1], a | b)
    assert np.any(a != b)


@pytest.mark.parametrize("n", list(range(1, 13)) + [49, 50, 51])
def test_majority_any_n(im, n):
    rng = np.random.default_rng(n)
    peaks = [(int(rng.integers(NB)), int(rng.integers(Q))) for _ in range(n)]
    ones = _bound(im, peaks).sum(0)
    # bit 1 (-1) unless the +1 components (zeros) outnumber the -1 ones
    expect = (2 * ones >= n).astype(np.uint8)
    out = _enc(im, [peaks])
    assert np.array_equal(bits(out[0]), expect)


def test_duplicate_and_reorder_invariant(im):
    rng = np.random.default_rng(3)
    for n in (4, 7, 50):
        peaks = [(int(rng.integers(NB)), int(rng.integers(Q))) for _ in range(n)]
        rev = peaks[::-1]
        dup = [p for p in peaks for _ in range(2)]
        out = _enc(im, [peaks, rev, dup])
        assert np.array_equal(out[0], out[1])
        assert np.array_equal(out[0], out[2])


def test_rejects_out_of_range(im):
    with pytest.raises(ValueError):
        _enc(im, [[(NB, 0)]])
    with pytest.raises(ValueError):
        _enc(im, [[(0, Q)]])
