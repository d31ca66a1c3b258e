"""CPU oracle of the HyperOMS hot path -- TEST INFRASTRUCTURE.

Python wrapper (ctypes) around ``hd_oracle.c``: a plain, slow C restatement
of the paper's encoding (Section 3.3, Eq. 1), candidate filter and Hamming
search (Section 3.4) and preprocessing (Section 3.2, Table 1).  Only the
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

TOL_DA, TOL_PPM = 0, 1


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
            lib.orc_item_memory.argtypes = [u32, u32, u32, u32, u64, P, P, P, P]
            lib.orc_preprocess.argtypes = [u32, P, P, P, dbl, dbl, dbl, u32, u32, dbl, u32, P, P, P]
            lib.orc_preprocess.restype = C.c_longlong
            lib.orc_encode.argtypes = [u32, P, u32, P, u32, u32, P, P, P, P, u32]
            lib.orc_window_count.argtypes = [u32, P, P, u32, P, P, dbl, i32, P]
            lib.orc_library_order.argtypes = [u32, P, P, P]
            lib.orc_search.argtypes = [u32, u32, P, P, P, u32, P, P, P, dbl, i32, u32, P, u32, P, P, u32]
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


def item_memory(dim, n_levels, n_bins, alpha, seed):
    """(F [f, D/64] u64, L [Q, D/64] u64, rank_F [D], rank_L [D])."""
    W = dim // 64
    F = np.zeros((n_bins, W), np.uint64)
    L = np.zeros((n_levels, W), np.uint64)
    rF = np.zeros(dim, np.uint32)
    rL = np.zeros(dim, np.uint32)
    rc = _load().orc_item_memory(dim, n_levels, n_bins, alpha, seed, _p(F), _p(L), _p(rF), _p(rL))
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


def encode(dim, F, L, offsets, bins, levels, n_threads=None):
    """Binary HVs [n, D/64] u64 of CSR spectrum vectors (Eq. 1 + sign)."""
    off = _c(offsets, np.uint32)
    n = off.size - 1
    out = np.zeros((n, dim // 64), np.uint64)
    F, L = _c(F, np.uint64), _c(L, np.uint64)
    b, lv = _c(bins, np.uint32), _c(levels, np.uint8)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = _load().orc_encode(dim, _p(F), F.shape[0], _p(L), L.shape[0], n, _p(off), _p(b), _p(lv), _p(out),
                            n_threads)
    if rc:
        raise ValueError(f"orc_encode rc={rc}")
    return out


def window_count(ref_mz, ref_z, q_mz, q_z, tol, unit="da"):
    rm, rz = _c(ref_mz, np.float64), _c(ref_z, np.uint8)
    qm, qz = _c(q_mz, np.float64), _c(q_z, np.uint8)
    out = np.zeros(qm.size, np.uint32)
    _load().orc_window_count(rm.size, _p(rm), _p(rz), qm.size, _p(qm), _p(qz), float(tol),
                             int(unit == "ppm"), _p(out))
    return out


def library_order(mz, z):
    m, zz = _c(mz, np.float64), _c(z, np.uint8)
    out = np.zeros(m.size, np.uint32)
    _load().orc_library_order(m.size, _p(m), _p(zz), _p(out))
    return out


def search(dim, ref_hv, ref_mz, ref_z, q_hv, q_mz, q_z, tol, unit="da", k=1, which=None,
           n_threads=None):
    """Brute-force windowed top-k: (idx [m, k] u32, dist [m, k] u16)."""
    rh, rm, rz = _c(ref_hv, np.uint64), _c(ref_mz, np.float64), _c(ref_z, np.uint8)
    qh, qm, qz = _c(q_hv, np.uint64), _c(q_mz, np.float64), _c(q_z, np.uint8)
    w = None if which is None else _c(which, np.uint32)
    m = qm.size if w is None else w.size
    idx = np.zeros((m, k), np.uint32)
    dist = np.zeros((m, k), np.uint16)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = _load().orc_search(dim, rm.size, _p(rh), _p(rm), _p(rz), qm.size, _p(qh), _p(qm), _p(qz),
                            float(tol), int(unit == "ppm"), k, _p(w), 0 if w is None else w.size,
                            _p(idx), _p(dist), n_threads)
    if rc:
        raise ValueError(f"orc_search rc={rc}")
    return idx, dist
