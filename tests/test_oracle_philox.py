"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The paper draws its position and level HVs at random (Section 3.3.1-3.3.2)
without naming a generator; Philox4x32-10 is the reading.  No known-answer
vector is available here, so the generator is pinned by properties a correct
Philox has and a broken one (a dropped key word, too few rounds, a lost
counter word) loses: bit balance, distinct outputs for distinct counters,
and avalanche in every counter and key word."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _block(c, k):
    return oracle.philox4x32_10(c, k)


def _popc128(x):
    return int(np.unpackbits(np.asarray(x, np.uint32).view(np.uint8)).sum())


def test_bit_balance_and_distinct_outputs():
    n = 8192
    outs = np.stack([_block([i, 0, 0, 0], [7, 11]) for i in range(n)])
    b = np.unpackbits(outs.view(np.uint8))
    sigma = 0.5 / np.sqrt(b.size)
    assert abs(b.mean() - 0.5) < 5 * sigma
    for lane in range(4):
        bl = np.unpackbits(outs[:, lane].copy().view(np.uint8))
        assert abs(bl.mean() - 0.5) < 5 * 0.5 / np.sqrt(bl.size)
    assert len({tuple(o) for o in outs}) == n


@pytest.mark.parametrize("which", ["ctr0", "ctr1", "ctr2", "ctr3", "key0", "key1"])
def test_avalanche(which):
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(300):
        c = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        bit = np.uint32(1 << int(rng.integers(0, 32)))
        c2, k2 = c.copy(), k.copy()
        if which.startswith("ctr"):
            c2[int(which[-1])] ^= bit
        else:
            k2[int(which[-1])] ^= bit
        flips.append(_popc128(_block(c, k) ^ _block(c2, k2)))
    flips = np.asarray(flips, float)
    # a 128-bit output flips 64 +- 5.66 bits per sample when the input bit matters
    assert abs(flips.mean() - 64.0) < 5 * 5.66 / np.sqrt(flips.size)
    assert flips.min() > 20


def test_consecutive_counters_uncorrelated():
    outs = np.stack([_block([i, 3, 0, 0], [1, 2]) for i in range(4096)]).astype(np.float64)
    x = outs[:, 0] / 2**32
    r = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(r) < 5 / np.sqrt(x.size)
