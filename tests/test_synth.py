"""The synthetic input recipe (stand-ins for the paper's datasets, Section 4.1
and Table 1): shapes and laws of references, decoys, queries and batch sizes.
Host logic only; no method arithmetic lives in the generator."""
import numpy as np

from paper_2211_16422_gb300 import synth


def test_references_and_decoys():
    rng = np.random.default_rng(3)
    n = 4000
    refs = synth.make_references(n, (2, 3, 4), (0.6, 0.3, 0.1), rng, decoy_fraction=0.5)
    assert refs.n == n and np.all(np.diff(refs.offsets.astype(np.int64)) == 50)
    assert np.all((refs.precursor_mz >= 400) & (refs.precursor_mz <= 1500))
    assert np.all((refs.mz >= 101) & (refs.mz <= 1500))
    it = refs.intensity.reshape(n, 50)
    assert np.allclose(it.max(axis=1), 1.0) and np.all(it > 0)
    # intensities sqrt(U(0.01, 1]) before normalisation: no ratio below 0.1
    assert np.all(it.min(axis=1) / it.max(axis=1) >= 0.1 - 1e-12)
    frac = np.bincount(refs.charge[:n // 2], minlength=5)[2:] / (n // 2)
    assert np.all(np.abs(frac - np.array([0.6, 0.3, 0.1])) < 0.04)
    # decoys: the second half, target k's precursor, charge and intensities, new fragment positions
    half = n // 2
    assert np.all(refs.decoy[:half] == 0) and np.all(refs.decoy[half:] == 1)
    assert np.array_equal(refs.precursor_mz[half:], refs.precursor_mz[:half])
    assert np.array_equal(refs.charge[half:], refs.charge[:half])
    mz = refs.mz.reshape(n, 50)
    assert np.array_equal(it[half:], it[:half])
    assert np.mean(mz[half:] != mz[:half]) > 0.99


def test_queries_follow_the_modification_recipe():
    rng = np.random.default_rng(4)
    refs = synth.make_references(3000, (2, 3), (0.5, 0.5), rng, decoy_fraction=0.5)
    qs = synth.make_queries(refs, 4000, rng)
    src = qs.source
    assert np.all(refs.decoy[src] == 0) and np.all(qs.charge == refs.charge[src])
    shift = (qs.precursor_mz - refs.precursor_mz[src]) * qs.charge.astype(np.float64)
    fixed = np.array(synth.FIXED_SHIFTS)
    is_fixed = np.min(np.abs(shift[:, None] - fixed[None, :]), axis=1) < 1e-9
    assert np.all(is_fixed | (np.abs(shift) <= 100.0))
    # five equally likely choices: four fixed shifts and one uniform draw
    assert abs(np.mean(is_fixed) - 0.8) < 0.03
    assert abs(np.mean(np.abs(shift) < 1e-12) - 0.2) < 0.03
    # 30% of the peaks move by shift / z (unless they would leave the range), 10% become noise
    q_mz = qs.mz.reshape(qs.n, 50)
    r_mz = refs.mz.reshape(refs.n, 50)[src]
    delta = q_mz - r_mz
    big = np.abs(shift) > 1.0
    moved = np.abs(delta - (shift / qs.charge)[:, None]) < 1e-9
    assert abs(np.mean(moved[big].sum(axis=1)) - 15) < 1.0
    unchanged = np.abs(delta) < 1e-12
    assert np.all(unchanged[big].sum(axis=1) + moved[big].sum(axis=1) <= 45)
    assert np.all((q_mz >= 101) & (q_mz <= 1500))
    assert np.allclose(qs.intensity.reshape(qs.n, 50).max(axis=1), 1.0)


def test_batch_sizes_log_uniform():
    rng = np.random.default_rng(5)
    s = synth.batch_sizes(20000, 10, 20000, rng)
    assert s.min() >= 10 and s.max() <= 20000
    # log-uniform: log10 of the sizes is about uniform on [1, 4.3]
    lg = np.log10(s)
    assert abs(np.median(lg) - (1 + np.log10(20001)) / 2) < 0.1
