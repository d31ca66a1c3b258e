"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The paper draws its position and level HVs at random (Section 3.3.1-3.3.2)
without naming a generator; Philox4x32-10 is the reading.  The generator is
pinned by the published known-answer vectors of the Random123 distribution
(its kat_vectors file, "philox4x32 10" lines: counter words, key words,
expected output words), which fix the round function, the key schedule, the
round count and the order of the output words; and by properties a correct
Philox has and a broken one (a dropped key word, too few rounds, a lost
counter word) loses: bit balance, distinct outputs for distinct counters,
and avalanche in every counter and key word."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")

# Random123 known-answer vectors for philox4x32_10: (ctr[4], key[2], out[4])
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_known_answer_vectors(ctr, key, want):
    assert [int(x) for x in oracle.philox4x32_10(ctr, key)] == list(want)


def test_word_stream_layout():
    """Word i of stream s under seed is component i%4 of the block at counter
    (i/4, s, 0, 0) with key (seed low, seed high); counter 0 of stream 0 under
    seed 0 is the first known-answer vector."""
    assert [int(x) for x in oracle.random_words(0, 0, 4)] == list(KAT[0][2])
    seed, stream = 0x0123456789ABCDEF, 3
    w = oracle.random_words(seed, stream, 4 * 37 + 3)
    for c in (0, 1, 17, 36, 37):
        blk = oracle.philox4x32_10([c, stream, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        n = min(4, w.size - 4 * c)
        assert np.array_equal(w[4 * c:4 * c + n], blk[:n])


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
