"""Oracle-side inputs for the parity tests: the oracle's own preprocessing and
encoding of the raw synthetic spectra, so no oracle input comes from the GPU
path."""
import functools

import oracle
from paper_2211_16422_gb300 import synth


@functools.lru_cache(maxsize=8)
def item_memory(D, Q, seed, n_bins=synth.N_BINS):
    F, L, _, _ = oracle.item_memory(D, Q, n_bins, D // 2, seed)
    return F, L


def pp_args(Q):
    return dict(mz_min=synth.MZ_MIN, mz_max=synth.MZ_MAX, bin_width=synth.BIN_WIDTH, n_bins=synth.N_BINS,
                max_peaks=synth.MAX_PEAKS, n_levels=Q)


def hvs(sp, D, Q, seed):
    """Oracle HVs [n, D/64] of raw spectra `sp` (synth.Spectra)."""
    F, L = item_memory(D, Q, seed)
    return oracle.encode(D, F, L, *oracle.preprocess(sp.offsets, sp.mz, sp.intensity, **pp_args(Q)))


@functools.lru_cache(maxsize=1)
def workload_ref_hvs(name, D, Q, seed):
    """Oracle HVs of a named workload's references (cached: several tests use
    the 1,000,000-reference library)."""
    refs, _, _ = synth.make_workload(name)
    return hvs(refs, D, Q, seed)
