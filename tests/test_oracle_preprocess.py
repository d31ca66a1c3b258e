"""Pins of the oracle's preprocessing (Section 3.2, Table 1) on hand-worked
spectra.  Each expected value below follows from the steps by hand: m/z
values sit mid-bin so the binning is unambiguous."""
import math

import numpy as np
import pytest

import oracle

P = dict(mz_min=101.0, mz_max=1500.0, bin_width=0.05, n_bins=27981, max_peaks=50, n_levels=16)


def _run(spectra, **kw):
    p = dict(P)
    p.update(kw)
    off = np.zeros(len(spectra) + 1, np.uint32)
    off[1:] = np.cumsum([len(s) for s in spectra])
    mz = np.array([x[0] for s in spectra for x in s], float)
    it = np.array([x[1] for s in spectra for x in s], float)
    o, b, lv = oracle.preprocess(off, mz, it, **p)
    return [list(zip(b[o[i]:o[i + 1]].tolist(), lv[o[i]:o[i + 1]].tolist())) for i in range(len(spectra))]


def test_range_filter_and_binning():
    # 101.025 -> (0.025/0.05) = 0.5 -> bin 0; 750.025 -> 12980.5 -> 12980;
    # 100.99 and 1500.01 are outside 101-1500
    out = _run([[(100.99, 1.0), (101.025, 1.0), (750.025, 1.0), (1500.01, 1.0)]])
    assert [b for b, _ in out[0]] == [0, 12980]
    assert [l for _, l in out[0]] == [15, 15]


def test_upper_edge_stays_in_range():
    out = _run([[(1500.0, 1.0)]])
    assert 0 <= out[0][0][0] <= 27980


def test_same_bin_summed_then_quantised():
    # 200.01 and 200.02 share bin 1980 (99.01/0.05=1980.2, 99.02/0.05=1980.4):
    # sum 0.7 of max 1.0 -> floor(16*0.7)=11; the max bin -> 16 clamped to 15
    out = _run([[(300.025, 1.0), (200.02, 0.4), (200.01, 0.3)]])
    assert out[0] == [(1980, 11), (3980, 15)]


def test_relative_intensity_filter():
    # below 1% of the most intense peak is dropped; exactly 1% stays
    out = _run([[(150.025, 1.0), (160.025, 0.0099), (170.025, 0.01), (180.025, 0.5)]])
    assert [b for b, _ in out[0]] == [980, 1380, 1580]
    # levels: floor(16*1)=16->15, floor(16*0.01)=0, floor(16*0.5)=8
    assert [l for _, l in out[0]] == [15, 0, 8]


def test_top_peaks_with_ties():
    # keep 3 most intense; the 0.5 ties go to the lowest m/z (200.025)
    sp = [(500.025, 0.5), (400.025, 0.9), (300.025, 0.5), (600.025, 0.7), (200.025, 0.5)]
    out = _run([sp], max_peaks=3)
    assert [b for b, _ in out[0]] == [1980, 5980, 9980]


def test_exact_duplicate_peaks_sum():
    out = _run([[(250.025, 0.25), (250.025, 0.25), (900.025, 1.0)]])
    # 0.5 of max -> level 8
    assert out[0] == [(2980, 8), (15980, 15)]


def test_non_positive_and_non_finite_dropped():
    sp = [(150.025, 0.0), (160.025, -1.0), (170.025, math.nan), (math.inf, 1.0),
          (180.025, 0.4), (190.025, math.inf)]
    out = _run([sp])
    assert out[0] == [(1580, 15)]


def test_empty_and_all_dropped():
    out = _run([[], [(50.0, 1.0)], [(150.025, 1.0)]])
    assert out[0] == [] and out[1] == [] and out[2] == [(980, 15)]


def test_output_ascending_bins_and_levels_bounded():
    rng = np.random.default_rng(0)
    sp = [(float(m), float(i)) for m, i in zip(rng.uniform(101, 1500, 120), rng.random(120) + 0.01)]
    out = _run([sp], n_levels=32)[0]
    b = [x[0] for x in out]
    assert b == sorted(b) and len(set(b)) == len(b) and len(b) <= 50
    assert all(0 <= l < 32 for _, l in out)
    assert max(l for _, l in out) == 31


def test_rejects_bad_params():
    with pytest.raises(ValueError):
        _run([[(200.0, 1.0)]], n_levels=1)
    with pytest.raises(ValueError):
        _run([[(200.0, 1.0)]], bin_width=0.0)
