"""CPU oracle of the HyperOMS hot path -- TEST INFRASTRUCTURE.

Python wrapper (ctypes) around ``hd_oracle.c``: a plain, slow C restatement
of the paper's encoding (Section 3.3, Eq. 1), candidate filter and Hamming
search (Section 3.4) and preprocessing (Section 3.2, Table 1), and the
multi-bit components and their dot-product search (Section 4.3); plus, in
plain numpy on top of that search, the target-decoy q-values (Section 2.1)
and the cascade search (Section 3.4).  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the GPU library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TOL_DA, TOL_PPM, TOL_MASS = 0, 1, 2
_UNITS = {"da": TOL_DA, "ppm": TOL_PPM, "mass": TOL_MASS}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no SIMD, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            u32, u64, dbl, i32 = C.c_uint32, C.c_uint64, C.c_double, C.c_int
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_random_words.argtypes = [u64, u32, u32, P]
            lib.orc_item_memory.argtypes = [u32, u32, u32, u32, u64, u32, P, P, P, P]
            lib.orc_preprocess.argtypes = [u32, P, P, P, dbl, dbl, dbl, u32, u32, dbl, u32, P, P, P]
            lib.orc_preprocess.restype = C.c_longlong
            lib.orc_encode.argtypes = [u32, P, u32, P, u32, u32, P, P, P, P, u32, u32]
            lib.orc_window_count.argtypes = [u32, P, P, u32, P, P, dbl, i32, P]
            lib.orc_library_order.argtypes = [u32, P, P, P]
            lib.orc_search.argtypes = [u32, u32, P, P, P, u32, P, P, P, dbl, i32, u32, P, u32, P, P, u32]
            lib.orc_encode_multibit.argtypes = [u32, P, u32, P, u32, u32, P, P, P, u32, P, u32, u32]
            lib.orc_search_dot.argtypes = [u32, u32, P, P, P, u32, P, P, P, dbl, i32, u32, P, u32, P, P, u32]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ``ctr`` 4 x uint32, ``key`` 2 x uint32."""
    c, k = _c(ctr, np.uint32), _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def random_words(seed, stream, n):
    """Words 0..n-1 of Philox word stream `stream` under `seed`: word i is
    component i%4 of the block at counter (i/4, stream, 0, 0), key (seed low,
    seed high) -- the random words the item memory draws from."""
    out = np.zeros(int(n), np.uint32)
    _load().orc_random_words(int(seed), int(stream), int(n), _p(out))
    return out


def item_memory(dim, n_levels, n_bins, alpha, seed, mode=0):
    """(F [f, D/64] u64, L [Q, D/64] u64, rank_F [D], rank_L [D]).  ``mode``: 0 nested
    position flips (alpha in total), 1 random walk (alpha flips per step), 2 independent
    random position HVs."""
    W = dim // 64
    F = np.zeros((n_bins, W), np.uint64)
    L = np.zeros((n_levels, W), np.uint64)
    rF = np.zeros(dim, np.uint32)
    rL = np.zeros(dim, np.uint32)
    rc = _load().orc_item_memory(dim, n_levels, n_bins, alpha, seed, mode, _p(F), _p(L), _p(rF), _p(rL))
    if rc:
        raise ValueError(f"orc_item_memory rc={rc}")
    return F, L, rF, rL


def preprocess(offsets, mz, intensity, *, mz_min, mz_max, bin_width, n_bins, max_peaks,
               n_levels, min_rel=0.01):
    """Raw peaks (CSR) -> (offsets u32, bins u32, levels u8)."""
    off = _c(offsets, np.uint32)
    n = off.size - 1
    mzs, its = _c(mz, np.float64), _c(intensity, np.float64)
    o_off = np.zeros(n + 1, np.uint32)
    cap = max(1, n * max_peaks)
    o_bin = np.zeros(cap, np.uint32)
    o_lvl = np.zeros(cap, np.uint8)
    nnz = _load().orc_preprocess(n, _p(off), _p(mzs), _p(its), mz_min, mz_max, bin_width, n_bins,
                                 max_peaks, min_rel, n_levels, _p(o_off), _p(o_bin), _p(o_lvl))
    if nnz < 0:
        raise ValueError(f"orc_preprocess rc={nnz}")
    return o_off, o_bin[:nnz].copy(), o_lvl[:nnz].copy()


def encode(dim, F, L, offsets, bins, levels, n_threads=None, encoder=0):
    """Binary HVs [n, D/64] u64 of CSR spectrum vectors: encoder 0 = Eq. 1 + sign,
    1 = random projection with weights level + 1."""
    off = _c(offsets, np.uint32)
    n = off.size - 1
    out = np.zeros((n, dim // 64), np.uint64)
    F, L = _c(F, np.uint64), _c(L, np.uint64)
    b, lv = _c(bins, np.uint32), _c(levels, np.uint8)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = _load().orc_encode(dim, _p(F), F.shape[0], _p(L), L.shape[0], n, _p(off), _p(b), _p(lv), _p(out),
                            n_threads, encoder)
    if rc:
        raise ValueError(f"orc_encode rc={rc}")
    return out


def encode_multibit(dim, F, L, offsets, bins, levels, bits, n_threads=None, encoder=0):
    """Multi-bit components [n, D] int8 in [-m, m], m = 2^(bits-1) - 1: the
    bundle I of ``encode`` (Eq. 1, or the projection sum for encoder 1)
    quantised with the spectrum's own step max|I| / m, halves rounded up in
    magnitude (reading of Section 4.3's higher-precision components)."""
    off = _c(offsets, np.uint32)
    n = off.size - 1
    out = np.zeros((n, dim), np.int8)
    F, L = _c(F, np.uint64), _c(L, np.uint64)
    b, lv = _c(bins, np.uint32), _c(levels, np.uint8)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = _load().orc_encode_multibit(dim, _p(F), F.shape[0], _p(L), L.shape[0], n, _p(off), _p(b), _p(lv),
                                     int(bits), _p(out), n_threads, encoder)
    if rc:
        raise ValueError(f"orc_encode_multibit rc={rc}")
    return out


def search_dot(ref, ref_mz, ref_z, qv, q_mz, q_z, tol, unit="da", k=1, which=None, n_threads=None):
    """Brute-force windowed top-k by the dot product of integer components:
    (idx [m, k] u32, score [m, k] i32), higher score first, the lower reference
    index on a tie; missing slots hold 0xFFFFFFFF / INT32_MIN."""
    rv, rm, rz = _c(ref, np.int8), _c(ref_mz, np.float64), _c(ref_z, np.uint8)
    qq, qm, qz = _c(qv, np.int8), _c(q_mz, np.float64), _c(q_z, np.uint8)
    dim = rv.shape[1] if rv.ndim == 2 and rv.shape[0] else qq.shape[1]
    w = None if which is None else _c(which, np.uint32)
    m = qm.size if w is None else w.size
    idx = np.zeros((m, k), np.uint32)
    score = np.zeros((m, k), np.int32)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = _load().orc_search_dot(dim, rm.size, _p(rv), _p(rm), _p(rz), qm.size, _p(qq), _p(qm), _p(qz),
                                float(tol), _UNITS[unit], k, _p(w), 0 if w is None else w.size,
                                _p(idx), _p(score), n_threads)
    if rc:
        raise ValueError(f"orc_search_dot rc={rc}")
    return idx, score


def window_count(ref_mz, ref_z, q_mz, q_z, tol, unit="da"):
    rm, rz = _c(ref_mz, np.float64), _c(ref_z, np.uint8)
    qm, qz = _c(q_mz, np.float64), _c(q_z, np.uint8)
    out = np.zeros(qm.size, np.uint32)
    _load().orc_window_count(rm.size, _p(rm), _p(rz), qm.size, _p(qm), _p(qz), float(tol),
                             _UNITS[unit], _p(out))
    return out


def library_order(mz, z):
    m, zz = _c(mz, np.float64), _c(z, np.uint8)
    out = np.zeros(m.size, np.uint32)
    _load().orc_library_order(m.size, _p(m), _p(zz), _p(out))
    return out


def search(dim, ref_hv, ref_mz, ref_z, q_hv, q_mz, q_z, tol, unit="da", k=1, which=None,
           n_threads=None):
    """Brute-force windowed top-k: (idx [m, k] u32, dist [m, k] u16).  ``unit``:
    "da" and "ppm" bound the precursor m/z difference, "mass" the neutral
    precursor mass difference (mz - 1.007276) * z, in Da."""
    rh, rm, rz = _c(ref_hv, np.uint64), _c(ref_mz, np.float64), _c(ref_z, np.uint8)
    qh, qm, qz = _c(q_hv, np.uint64), _c(q_mz, np.float64), _c(q_z, np.uint8)
    w = None if which is None else _c(which, np.uint32)
    m = qm.size if w is None else w.size
    idx = np.zeros((m, k), np.uint32)
    dist = np.zeros((m, k), np.uint16)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = _load().orc_search(dim, rm.size, _p(rh), _p(rm), _p(rz), qm.size, _p(qh), _p(qm), _p(qz),
                            float(tol), _UNITS[unit], k, _p(w), 0 if w is None else w.size,
                            _p(idx), _p(dist), n_threads)
    if rc:
        raise ValueError(f"orc_search rc={rc}")
    return idx, dist


def fdr_qvalues(scores, is_decoy):
    """Target-decoy q-values of spectrum-spectrum matches (SSMs), the FDR
    filter of Section 2.1 (the target-decoy strategy the paper cites).

    Plain definition, written out: order the SSMs by score, highest first.
    The threshold at score s accepts every SSM with score >= s; its FDR is
    (decoy SSMs with score >= s) / (target SSMs with score >= s), with the
    denominator taken as 1 when it is 0.  The q-value of an SSM with score s
    is the smallest FDR over all thresholds s' <= s.  Equal scores share one
    threshold.  Returns float64 q per SSM, in the input order.
    """
    s = np.asarray(scores, np.int64)
    d = np.asarray(is_decoy).astype(bool)
    n = s.size
    if n == 0:
        return np.zeros(0, np.float64)
    order = np.argsort(-s, kind="stable")
    s_sorted, d_sorted = s[order], d[order]
    n_dec = np.cumsum(d_sorted)
    n_tgt = np.cumsum(~d_sorted)
    last = np.r_[np.nonzero(np.diff(s_sorted))[0], n - 1]   # last SSM of each run of equal scores
    fdr = n_dec[last].astype(np.float64) / np.maximum(n_tgt[last], 1).astype(np.float64)
    q_run = np.minimum.accumulate(fdr[::-1])[::-1]           # min over this and every lower threshold
    run = np.searchsorted(last, np.arange(n))                 # run of each sorted position
    q = np.empty(n, np.float64)
    q[order] = q_run[run]
    return q


def cascade(dim, ref_hv, ref_mz, ref_z, ref_decoy, q_hv, q_mz, q_z, levels, fdr, n_threads=None):
    """Cascade search (Section 3.4, after the cascade strategy the paper
    cites): levels are searched in order, each with its own precursor window
    (tol, unit).  At a level, the queries not identified so far are searched
    (top-1, as ``search``); the level's SSMs -- those queries with at least one
    candidate -- get q-values among themselves (``fdr_qvalues`` on the score
    D - dist); an SSM whose reference is a target and whose q <= fdr
    identifies its query at that level, and the query leaves the cascade.

    Returns (idx u32 [n], dist u16 [n], level u8 [n], q f64 [n]): the SSM of
    the last level each query was searched at (idx 0xFFFFFFFF, dist 0xFFFF,
    q NaN when that level had no candidate), and the level that identified it
    (0xFF: none).
    """
    dec_flags = np.asarray(ref_decoy).astype(bool)
    n = int(np.asarray(q_mz).size)
    idx = np.full(n, 0xFFFFFFFF, np.uint32)
    dist = np.full(n, 0xFFFF, np.uint16)
    level = np.full(n, 0xFF, np.uint8)
    q = np.full(n, np.nan, np.float64)
    active = np.arange(n, dtype=np.uint32)
    for li, (tol, unit) in enumerate(levels):
        if active.size == 0:
            break
        i1, d1 = search(dim, ref_hv, ref_mz, ref_z, q_hv, q_mz, q_z, tol, unit, k=1, which=active,
                        n_threads=n_threads)
        i1, d1 = i1[:, 0], d1[:, 0]
        idx[active], dist[active], q[active] = i1, d1, np.nan
        has = i1 != 0xFFFFFFFF
        ssm = active[has]
        is_dec = dec_flags[i1[has]]
        qv = fdr_qvalues(dim - d1[has].astype(np.int64), is_dec)
        q[ssm] = qv
        hit = ssm[(~is_dec) & (qv <= fdr)]
        level[hit] = li
        active = np.setdiff1d(active, hit).astype(np.uint32)
    return idx, dist, level, q


def cascade_dot(ref_comp, ref_mz, ref_z, ref_decoy, q_comp, q_mz, q_z, levels, fdr, n_threads=None):
    """Cascade search of multi-bit components (Section 3.4's cascade with the
    target-decoy FDR of Section 2.1, scored by the dot product of Section
    4.3's higher-precision components).  The same steps as ``cascade``: at
    each level the queries not identified so far are searched top-1 (as
    ``search_dot``), the level's SSMs get q-values among themselves
    (``fdr_qvalues`` on the score S), and a target SSM with q <= fdr
    identifies its query at that level.

    Returns (idx u32 [n], score i32 [n], level u8 [n], q f64 [n]): the SSM of
    the last level each query was searched at (idx 0xFFFFFFFF, score
    INT32_MIN, q NaN when that level had no candidate), and the level that
    identified it (0xFF: none).
    """
    dec_flags = np.asarray(ref_decoy).astype(bool)
    n = int(np.asarray(q_mz).size)
    idx = np.full(n, 0xFFFFFFFF, np.uint32)
    score = np.full(n, np.iinfo(np.int32).min, np.int32)
    level = np.full(n, 0xFF, np.uint8)
    q = np.full(n, np.nan, np.float64)
    active = np.arange(n, dtype=np.uint32)
    for li, (tol, unit) in enumerate(levels):
        if active.size == 0:
            break
        i1, s1 = search_dot(ref_comp, ref_mz, ref_z, q_comp, q_mz, q_z, tol, unit, k=1, which=active,
                            n_threads=n_threads)
        i1, s1 = i1[:, 0], s1[:, 0]
        idx[active], score[active], q[active] = i1, s1, np.nan
        has = i1 != 0xFFFFFFFF
        ssm = active[has]
        is_dec = dec_flags[i1[has]]
        qv = fdr_qvalues(s1[has].astype(np.int64), is_dec)
        q[ssm] = qv
        hit = ssm[(~is_dec) & (qv <= fdr)]
        level[hit] = li
        active = np.setdiff1d(active, hit).astype(np.uint32)
    return idx, score, level, q
