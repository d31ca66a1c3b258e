"""Seeded synthetic MS/MS spectra: the inputs of every test and benchmark.

This module only draws raw spectra (fragment m/z, intensity, precursor m/z,
charge, decoy flag).  It holds none of the method's arithmetic: no binning,
no quantisation, no hypervectors.  Both the GPU path and the CPU oracle
consume what it produces, each with its own preprocessing.

The workloads stand in for the paper's real datasets (iPRG2012 / HEK293
queries against yeast+HCD and MassIVE-KB libraries, Section 4.1), which are
not available here.  Shapes and value laws follow the paper's
preprocessing settings (Table 1: 50 peaks, fragment m/z 101-1500):

* reference: precursor m/z ~ U(400, 1500); charge from a per-workload
  distribution; ``n_peaks`` fragment peaks with m/z ~ U(101, 1500) and
  intensity sqrt(U(0.01, 1]) normalised to a maximum of 1;
* decoy k (second half of the library): target k with its fragment peaks
  repositioned -- new m/z ~ U(101, 1500), same intensities, precursor and
  charge (the library's decoys come from shuffle-and-reposition, Section
  4.1, which moves the fragments);
* query: a copy of a uniformly drawn target; a mass shift drawn with equal
  probability from {0, +15.995, +42.011, +79.966, U(-100, 100)} Da is added
  to the precursor as shift/charge; 30% of the peaks move by shift/charge
  (a peak that would leave [101, 1500] stays); 10% are replaced by noise
  peaks; intensities are multiplied by U(0.8, 1.2) and renormalised.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

FRAG_MZ_LO, FRAG_MZ_HI = 101.0, 1500.0
PREC_MZ_LO, PREC_MZ_HI = 400.0, 1500.0
FIXED_SHIFTS = (0.0, 15.995, 42.011, 79.966)


@dataclass
class Spectra:
    """Raw spectra in CSR form (``offsets[n+1]`` over the peak arrays)."""
    offsets: np.ndarray        # uint32 [n+1]
    mz: np.ndarray             # float64 [nnz]
    intensity: np.ndarray      # float64 [nnz]
    precursor_mz: np.ndarray   # float64 [n]
    charge: np.ndarray         # uint8 [n]
    decoy: np.ndarray          # uint8 [n]
    source: np.ndarray = field(default=None)  # int64 [n]: copied target (queries)

    @property
    def n(self) -> int:
        return int(self.precursor_mz.shape[0])

    def subset(self, idx) -> "Spectra":
        idx = np.asarray(idx, dtype=np.int64)
        lens = (self.offsets[1:] - self.offsets[:-1]).astype(np.int64)[idx]
        off = np.zeros(idx.size + 1, dtype=np.uint32)
        np.cumsum(lens, out=off[1:])
        starts = self.offsets[:-1].astype(np.int64)[idx]
        gather = (np.repeat(starts - off[:-1].astype(np.int64), lens)
                  + np.arange(int(off[-1]), dtype=np.int64))
        return Spectra(off, self.mz[gather], self.intensity[gather],
                       self.precursor_mz[idx], self.charge[idx], self.decoy[idx],
                       None if self.source is None else self.source[idx])


def _dense_to_spectra(mz2d, int2d, prec, charge, decoy, source=None) -> Spectra:
    n, p = mz2d.shape
    off = (np.arange(n + 1, dtype=np.uint64) * p).astype(np.uint32)
    return Spectra(off, np.ascontiguousarray(mz2d.reshape(-1)),
                   np.ascontiguousarray(int2d.reshape(-1)),
                   prec.astype(np.float64), charge.astype(np.uint8),
                   decoy.astype(np.uint8), source)


def _intensities(rng, shape):
    raw = 1.0 - rng.random(shape) * 0.99          # U(0.01, 1]
    v = np.sqrt(raw)
    return v / v.max(axis=-1, keepdims=True)


def make_references(n, charges, weights, rng, n_peaks=50, decoy_fraction=0.0):
    """``n`` reference spectra; the last ``decoy_fraction`` of them are decoys."""
    n_dec = int(round(n * decoy_fraction))
    n_tgt = n - n_dec
    if n_dec > n_tgt:
        raise ValueError("decoy_fraction must be <= 0.5")
    w = np.asarray(weights, dtype=np.float64)
    charge_t = np.asarray(charges, dtype=np.uint8)[
        rng.choice(len(charges), size=n_tgt, p=w / w.sum())]
    prec_t = rng.uniform(PREC_MZ_LO, PREC_MZ_HI, n_tgt)
    mz_t = rng.uniform(FRAG_MZ_LO, FRAG_MZ_HI, (n_tgt, n_peaks))
    it_t = _intensities(rng, (n_tgt, n_peaks))
    if n_dec:
        mz_d = rng.uniform(FRAG_MZ_LO, FRAG_MZ_HI, (n_dec, n_peaks))
        mz = np.concatenate([mz_t, mz_d])
        it = np.concatenate([it_t, it_t[:n_dec]])
        prec = np.concatenate([prec_t, prec_t[:n_dec]])
        charge = np.concatenate([charge_t, charge_t[:n_dec]])
    else:
        mz, it, prec, charge = mz_t, it_t, prec_t, charge_t
    decoy = np.zeros(n, dtype=np.uint8)
    decoy[n_tgt:] = 1
    return _dense_to_spectra(mz, it, prec, charge, decoy)


def make_queries(refs: Spectra, n_q, rng, move_frac=0.30, noise_frac=0.10,
                 jitter=0.20):
    """Modified copies of random targets of ``refs`` (all rows must hold the
    same number of peaks)."""
    lens = np.diff(refs.offsets.astype(np.int64))
    p = int(lens[0])
    if not np.all(lens == p):
        raise ValueError("make_queries needs equal peak counts")
    n_tgt = int(np.count_nonzero(refs.decoy == 0))
    src = rng.integers(0, n_tgt, n_q)
    z = refs.charge[src].astype(np.float64)
    pick = rng.integers(0, len(FIXED_SHIFTS) + 1, n_q)
    shift = np.where(pick < len(FIXED_SHIFTS),
                     np.asarray(FIXED_SHIFTS + (0.0,))[pick],
                     rng.uniform(-100.0, 100.0, n_q))
    prec = refs.precursor_mz[src] + shift / z
    mz = refs.mz.reshape(-1, p)[src].copy()
    it = refs.intensity.reshape(-1, p)[src].copy()
    order = np.argsort(rng.random((n_q, p)), axis=1)
    n_move = int(round(move_frac * p))
    n_noise = int(round(noise_frac * p))
    rows = np.arange(n_q)[:, None]
    mv = order[:, :n_move]
    moved = mz[rows, mv] + (shift / z)[:, None]
    ok = (moved >= FRAG_MZ_LO) & (moved <= FRAG_MZ_HI)
    mz[rows, mv] = np.where(ok, moved, mz[rows, mv])
    nz = order[:, n_move:n_move + n_noise]
    mz[rows, nz] = rng.uniform(FRAG_MZ_LO, FRAG_MZ_HI, (n_q, n_noise))
    it[rows, nz] = np.sqrt(1.0 - rng.random((n_q, n_noise)) * 0.99)
    it = it * rng.uniform(1.0 - jitter, 1.0 + jitter, (n_q, p))
    it = it / it.max(axis=1, keepdims=True)
    return _dense_to_spectra(mz, it, prec, refs.charge[src],
                             np.zeros(n_q, dtype=np.uint8), src.astype(np.int64))


# Workloads: sizes and laws of the five configurations the benchmark and the
# parity tests use.  ``scale`` shrinks the library and query counts (the
# laws stay) so the CPU oracle can check a reduced copy in seconds.
WORKLOADS = {
    "tiny": dict(n_refs=1000, n_queries=100, charges=(2, 3), weights=(0.5, 0.5),
                 dim=2048, n_levels=16, tol=500.0, unit="da", k=1,
                 decoy_fraction=0.0, seed=0),
    "full": dict(n_refs=1_000_000, n_queries=50_000, charges=(2, 3, 4),
                 weights=(0.6, 0.3, 0.1), dim=8192, n_levels=32, tol=500.0,
                 unit="da", k=5, decoy_fraction=0.5, seed=1),
    "batched": dict(n_refs=2_000_000, n_batches=200, batch_lo=10, batch_hi=20_000,
                    charges=(1, 2, 3, 4, 5), weights=(0.05, 0.50, 0.30, 0.10, 0.05),
                    dims=(4096, 8192), n_levels=32,
                    windows=((20.0, "ppm"), (150.0, "da"), (500.0, "da")), k=5,
                    decoy_fraction=0.5, seed=3),
    "serving": dict(n_refs=1_000_000, charges=(2, 3, 4), weights=(0.6, 0.3, 0.1),
                    dim=8192, n_levels=32, tol=500.0, unit="da", k=5,
                    req_lo=1, req_hi=5000, decoy_fraction=0.5, seed=4),
}

# Binning of Table 1 (small-scale column): fragment m/z 101-1500, bin 0.05,
# 50 peaks; f = floor((1500 - 101) / 0.05) + 1 bins.
MZ_MIN, MZ_MAX, BIN_WIDTH, MAX_PEAKS, N_BINS = 101.0, 1500.0, 0.05, 50, 27981


def make_workload(name: str, scale: float = 1.0, seed=None):
    """(references, queries, spec) for the 'tiny' or 'full' workload."""
    spec = dict(WORKLOADS[name])
    rng = np.random.Generator(np.random.PCG64(spec["seed"] if seed is None else seed))
    n_r = max(2, int(round(spec["n_refs"] * scale)))
    n_q = max(1, int(round(spec["n_queries"] * scale)))
    refs = make_references(n_r, spec["charges"], spec["weights"], rng,
                           decoy_fraction=spec["decoy_fraction"])
    queries = make_queries(refs, n_q, rng)
    spec.update(n_refs=n_r, n_queries=n_q)
    return refs, queries, spec


def batch_sizes(n_batches, lo, hi, rng):
    """Log-uniform integer batch sizes floor(exp(U(ln lo, ln(hi+1))))."""
    s = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), n_batches)))
    return np.clip(s.astype(np.int64), lo, hi)


def raw_peak_soup(n, rng, max_len=200, p_bad=0.05):
    """Spectra with irregular peak lists for preprocessing edge cases: ragged
    lengths (including empty), out-of-range and non-positive peaks, exact
    duplicates and intensity ties."""
    lens = rng.integers(0, max_len + 1, n)
    lens[:: max(1, n // 7)] = 0
    off = np.zeros(n + 1, dtype=np.uint32)
    np.cumsum(lens, out=off[1:])
    nnz = int(off[-1])
    mz = rng.uniform(95.0, 1510.0, nnz)
    it = np.round(rng.random(nnz), 2) ** 2
    bad = rng.random(nnz) < p_bad
    it[bad] = -it[bad]
    dup = rng.random(nnz) < 0.05
    mz[1:][dup[1:]] = mz[:-1][dup[1:]]
    prec = rng.uniform(PREC_MZ_LO, PREC_MZ_HI, n)
    charge = rng.integers(1, 6, n).astype(np.uint8)
    return Spectra(off, mz, it, prec, charge, np.zeros(n, dtype=np.uint8))
