"""Pins of the oracle's item memory against what Section 3.3 fixes.

Section 3.3.1: position HVs are a random base with alpha components flipped
at random positions; similarity is highest on the diagonal and falls with the
bin distance, and far bins are near-orthogonal at alpha = D/2.
Section 3.3.2: level p (percent) flips (D/2)(p/100) components of L_0, so the
top level is orthogonal to L_0 and the level distance grows linearly.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import bits, hamming_matrix

D, Q, F_BINS = 512, 16, 300


@pytest.fixture(scope="module")
def im():
    return oracle.item_memory(D, Q, F_BINS, D // 2, seed=1234)


def test_ranks_are_permutations(im):
    _, _, rF, rL = im
    assert np.array_equal(np.sort(rF), np.arange(D))
    assert np.array_equal(np.sort(rL), np.arange(D))
    assert not np.array_equal(rF, rL)


def test_base_vectors_random(im):
    F, L, _, _ = im
    sigma = np.sqrt(D) / 2
    for v in (F[0], L[0]):
        assert abs(int(bits(v).sum()) - D / 2) < 5 * sigma
    assert abs(int(hamming_matrix(F[:1], L[:1])[0, 0]) - D / 2) < 5 * sigma


def test_position_flips_total_alpha_and_nested(im):
    F, _, _, _ = im
    dm = hamming_matrix(F, F)
    # the last bin carries all alpha flips: orthogonal to the first at alpha = D/2
    assert dm[0, -1] == D // 2
    # nested flips: the distance between two bins is the difference of their
    # distances to the first bin, so similarity falls monotonically with |i-j|
    d0 = dm[0]
    assert np.all(np.diff(d0) >= 0)
    i, j = np.triu_indices(F_BINS, 1)
    assert np.array_equal(dm[i, j], d0[j] - d0[i])
    assert np.all(np.diag(dm) == 0)
    # flips spread evenly: cumulative flips track i * alpha / (f-1) within one
    ideal = np.arange(F_BINS) * (D // 2) / (F_BINS - 1)
    assert np.all(np.abs(d0 - ideal) < 1.0)


def test_level_flips_linear(im):
    _, L, _, _ = im
    dm = hamming_matrix(L, L)
    assert dm[0, Q - 1] == D // 2
    for j in range(Q):
        # (D/2) * (p/100) flips with p = 100 j/(Q-1), floored
        assert dm[0, j] == int(Fraction(D, 2) * Fraction(j, Q - 1))
    a, b = np.triu_indices(Q, 1)
    assert np.array_equal(dm[a, b], dm[0, b] - dm[0, a])


def test_seeds_independent():
    F1, L1, _, _ = oracle.item_memory(D, Q, 8, D // 2, seed=1)
    F2, L2, _, _ = oracle.item_memory(D, Q, 8, D // 2, seed=2)
    sigma = np.sqrt(D) / 2
    assert abs(int(hamming_matrix(F1[:1], F2[:1])[0, 0]) - D / 2) < 5 * sigma
    assert abs(int(hamming_matrix(L1[:1], L2[:1])[0, 0]) - D / 2) < 5 * sigma


def test_small_alpha_keeps_locality():
    F, _, _, _ = oracle.item_memory(256, 4, 128, 32, seed=9)
    dm = hamming_matrix(F, F)
    assert dm[0, -1] == 32
    assert dm[0, 1] <= 1


def test_rejects_bad_args():
    with pytest.raises(ValueError):
        oracle.item_memory(100, Q, 4, 10, 0)
    with pytest.raises(ValueError):
        oracle.item_memory(D, 1, 4, 10, 0)
    with pytest.raises(ValueError):
        oracle.item_memory(D, Q, 4, D + 1, 0)
