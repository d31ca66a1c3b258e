"""Pins of the oracle's encoder variants (Section 4.2, "Encoding strategy":
HyperOMS encoding vs ID-Level HDC vs random-projection LSH; Section 3.3.1's
other reading of the position flips, a random walk).

Position walk: consecutive position HVs differ in exactly alpha components,
distance parity follows from the flip counts, and the walk decorrelates.
Random IDs: balanced, pairwise near-orthogonal, unrelated to the base
streams.  Projection encoder: closed forms for one and two peaks, the
weight-ratio invariance of a sign, and a numpy +-1 matrix-product brute
force."""
import numpy as np
import pytest

import oracle
from tests.helpers import bits, hamming_matrix


def test_walk_steps_flip_exactly_alpha():
    D, f = 512, 300
    for alpha in (1, 7, 64, 256):
        F, L, _, _ = oracle.item_memory(D, 4, f, alpha, 11, mode=1)
        d = np.array([hamming_matrix(F[i:i + 1], F[i + 1:i + 2])[0, 0] for i in range(f - 1)])
        assert np.all(d == alpha), alpha
        # F_0 is the nested mode's base vector (same stream), and the level HVs do not depend on the mode
        F0, L0, _, _ = oracle.item_memory(D, 4, f, 0, 11, mode=0)
        assert np.array_equal(F[0], F0[0]) and np.array_equal(L, L0)
        # parity: d(F_0, F_k) has the parity of k * alpha
        dk = hamming_matrix(F[:1], F)[0]
        assert np.all((dk % 2) == ((np.arange(f) * alpha) % 2))


def test_walk_decorrelates():
    D, f, alpha = 2048, 400, 32
    F, _, _, _ = oracle.item_memory(D, 4, f, alpha, 5, mode=1)
    dk = hamming_matrix(F[:1], F)[0].astype(np.float64)
    k = np.arange(f)
    # expected distance of a walk with alpha distinct flips per step: D/2 * (1 - (1 - 2 alpha / D)^k)
    expect = D / 2 * (1 - (1 - 2 * alpha / D) ** k)
    assert np.all(np.abs(dk - expect) <= 6 * np.sqrt(D / 4) + 1)
    assert np.all(dk <= k * alpha)


def test_random_ids_are_balanced_and_orthogonal():
    D, f = 4096, 64
    F, _, _, _ = oracle.item_memory(D, 4, f, 0, 9, mode=2)
    sigma = np.sqrt(D) / 2
    ones = bits(F).sum(axis=1)
    assert np.all(np.abs(ones - D / 2) <= 5 * sigma)
    dm = hamming_matrix(F, F)
    off = dm[~np.eye(f, dtype=bool)]
    assert np.all(np.abs(off - D / 2) <= 5 * sigma)
    F0, _, _, _ = oracle.item_memory(D, 4, f, D // 2, 9, mode=0)   # not the nested table
    assert np.all(np.abs(hamming_matrix(F, F0)[np.arange(f), np.arange(f)] - D / 2) <= 5 * sigma)
    F_b, _, _, _ = oracle.item_memory(D, 4, f, 0, 10, mode=2)       # another seed, another table
    assert np.all(np.abs(hamming_matrix(F, F_b)[np.arange(f), np.arange(f)] - D / 2) <= 5 * sigma)


def test_mode_arguments_checked():
    with pytest.raises(ValueError):
        oracle.item_memory(256, 4, 10, 257, 0, mode=1)     # more than 256 flips per step
    with pytest.raises(ValueError):
        oracle.item_memory(256, 4, 10, 8, 0, mode=3)


def _csr(rows):
    off = np.zeros(len(rows) + 1, np.uint32)
    b, lv = [], []
    for i, r in enumerate(rows):
        off[i + 1] = off[i] + len(r)
        for (bin_, level) in r:
            b.append(bin_)
            lv.append(level)
    return off, np.array(b, np.uint32), np.array(lv, np.uint8)


def test_projection_closed_forms():
    D, f, Q = 256, 40, 8
    F, L, _, _ = oracle.item_memory(D, Q, f, 0, 3, mode=2)
    rows = [[(5, 0)], [(5, 6)], [(3, 6), (9, 2)], [(3, 4), (9, 4)], []]
    hv = oracle.encode(D, F, L, *_csr(rows), encoder=1)
    assert np.array_equal(hv[0], F[5]) and np.array_equal(hv[1], F[5])     # one peak: its direction
    assert np.array_equal(hv[2], F[3])                                      # heavier peak dominates
    assert np.array_equal(hv[3], F[3] | F[9])                               # equal weights: ties -> -1
    assert np.all(hv[4] == np.uint64(0xFFFFFFFFFFFFFFFF))                   # empty: every sum is 0


def test_projection_matches_matrix_product():
    rng = np.random.default_rng(8)
    D, f, Q = 512, 300, 16
    F, L, _, _ = oracle.item_memory(D, Q, f, 0, 21, mode=2)
    R = 1 - 2 * bits(F).astype(np.int64)                  # [f, D] of +-1
    rows = []
    for _ in range(40):
        n = int(rng.integers(0, 30))
        bb = np.sort(rng.choice(f, n, replace=False))
        rows.append([(int(x), int(rng.integers(0, Q))) for x in bb])
    off, b, lv = _csr(rows)
    hv = oracle.encode(D, F, L, off, b, lv, encoder=1)
    for i, r in enumerate(rows):
        v = np.zeros(f, np.int64)
        for (bin_, level) in r:
            v[bin_] = level + 1
        s = v @ R
        assert np.array_equal(bits(hv[i:i + 1])[0], (s <= 0).astype(np.uint8))
    # doubling every weight ((l + 1) -> 2 (l + 1)) keeps every sign (levels up to 31 need Q = 32;
    # the random position table does not depend on Q)
    F2, L2, _, _ = oracle.item_memory(D, 2 * Q, f, 0, 21, mode=2)
    assert np.array_equal(F2, F)
    rows2 = [[(bin_, 2 * level + 1) for (bin_, level) in r] for r in rows]
    assert np.array_equal(oracle.encode(D, F2, L2, *_csr(rows2), encoder=1), hv)
