"""Python binding of libhd (ctypes): the same entry points as include/hd.h.

Argument marshalling only -- every step runs in libhd's CUDA kernels.  Device
buffers are torch CUDA tensors (PyTorch serves as the allocator and stream
provider); hypervectors are int64 tensors of shape [n, D/64] holding the
uint64 words bit for bit.  Loading fails loudly when libhd.so is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

HD_OK, HD_ERR_INVALID_ARG, HD_ERR_OOM, HD_ERR_CUDA, HD_ERR_TIMEOUT, HD_ERR_UNSUPPORTED = range(6)
HD_TOL_DA, HD_TOL_PPM, HD_TOL_MASS = 0, 1, 2
HD_FORM_AUTO, HD_FORM_POPC, HD_FORM_TC_FP8, HD_FORM_TC_BF16, HD_FORM_TC_FP4, HD_FORM_TC_MXF4 = 0, 1, 2, 3, 4, 5
FORMS = {"auto": HD_FORM_AUTO, "popc": HD_FORM_POPC, "tc_fp8": HD_FORM_TC_FP8, "tc_bf16": HD_FORM_TC_BF16,
         "tc_fp4": HD_FORM_TC_FP4, "tc_mxf4": HD_FORM_TC_MXF4}
NO_IDX, NO_DIST = 0xFFFFFFFF, 0xFFFF


class HDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class _Params(C.Structure):
    _fields_ = [("dim", C.c_uint32), ("n_levels", C.c_uint32), ("n_bins", C.c_uint32),
                ("alpha", C.c_uint32), ("seed", C.c_uint64), ("position_mode", C.c_uint32),
                ("encoder", C.c_uint32)]


class _PPParams(C.Structure):
    _fields_ = [("mz_min", C.c_double), ("mz_max", C.c_double), ("bin_width", C.c_double),
                ("min_rel_intensity", C.c_double), ("n_bins", C.c_uint32),
                ("max_peaks", C.c_uint32), ("n_levels", C.c_uint32)]


class _Window(C.Structure):
    _fields_ = [("tol", C.c_double), ("unit", C.c_int)]


class _TuneResult(C.Structure):
    _fields_ = [("form", C.c_int), ("tile_group", C.c_uint32), ("super_group", C.c_uint32),
                ("cluster", C.c_uint32), ("cta_group", C.c_uint32), ("tiles_per_stage", C.c_uint32),
                ("ms", C.c_double)]


def _windows(windows):
    """[(tol, 'da'|'ppm'), ...] -> ctypes array of hd_window."""
    arr = (_Window * len(windows))()
    for i, (tol, unit) in enumerate(windows):
        arr[i].tol, arr[i].unit = float(tol), _unit(unit)
    return arr


_lib = None
_lock = threading.Lock()
P, u32, u64, dbl, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_double, C.c_int

_SIGS = {
    "hd_status_string": ([i32], C.c_char_p),
    "hd_last_error_message": ([], C.c_char_p),
    "hd_version": ([], u32),
    "hd_ctx_create": ([P, P], i32),
    "hd_ctx_destroy": ([P], None),
    "hd_ctx_item_memory": ([P, P, P, P, P, P], i32),
    "hd_ctx_status": ([P], i32),
    "hd_random_words": ([u64, u32, u32, P, P], i32),
    "hd_preprocess": ([P, P, P, P, P, u32, P, P, P, P], i32),
    "hd_encode": ([P, P, P, P, u32, P, P], i32),
    "hd_build_library": ([P, P, P, P, u32, P], i32),
    "hd_library_free": ([P], None),
    "hd_library_info": ([P, P, P], i32),
    "hd_library_export": ([P, P, P, P, P, P], i32),
    "hd_library_status": ([P], i32),
    "hd_library_prepare": ([P, i32], i32),
    "hd_library_set_schedule": ([P, u32, u32, u32, u32], i32),
    "hd_library_set_stage_tiles": ([P, u32], i32),
    "hd_library_set_wait_limit": ([P, u64], i32),
    "hd_library_inject_stall": ([P, u32], i32),
    "hd_query_windows": ([P, P, P, u32, dbl, i32, P, P, P], i32),
    "hd_search_open": ([P, P, P, P, u32, dbl, i32, u32, P, P, P], i32),
    "hd_search_open_ex": ([P, P, P, P, u32, dbl, i32, u32, i32, P, P, P], i32),
    "hd_search_host": ([P, P, P, P, P, P, P, u32, dbl, i32, u32, P, P, P], i32),
    "hd_search_open_noalloc": ([P, P, P, P, u32, dbl, i32, u32, P, P, P], i32),
    "hd_search_open_multi": ([P, P, P, P, P, u32, P, u32, u32, i32, P, P, P], i32),
    "hd_library_set_decoys": ([P, P], i32),
    "hd_library_save": ([P, P, C.c_char_p], i32),
    "hd_library_load": ([P, C.c_char_p, P], i32),
    "hd_cascade_search": ([P, P, P, P, u32, P, u32, dbl, i32, P, P, P, P, P], i32),
    "hd_cascade_search_dot": ([P, P, P, P, u32, P, u32, dbl, i32, P, P, P, P, P], i32),
    "hd_plan_create": ([P, P, P, P, P, P, P, P, u32, P, u32, u32, i32, P, P, P, P], i32),
    "hd_plan_create_dot": ([P, P, P, P, P, P, P, P, u32, P, u32, u32, i32, P, P, P, P], i32),
    "hd_plan_launch": ([P, P], i32),
    "hd_plan_info": ([P, P], i32),
    "hd_plan_destroy": ([P], None),
    "hd_library_autotune": ([P, P, P, P, P, u32, P, u32, u32, P, P, u32, P], i32),
    "hd_library_autotune_dot": ([P, P, P, P, P, u32, P, u32, u32, P, P, u32, P], i32),
    "hd_server_create": ([P, P, P, P], i32),
    "hd_server_submit": ([P, P, P, P, P, P, u32, dbl, i32, P, P, P], i32),
    "hd_server_submit_dot": ([P, P, P, P, P, P, u32, dbl, i32, P, P, P], i32),
    "hd_server_wait": ([P, u64, dbl, P], i32),
    "hd_server_stats_get": ([P, P], i32),
    "hd_server_batch_log": ([P, P, u32, P], i32),
    "hd_server_destroy": ([P], None),
    "hd_profile_enable": ([i32], i32),
    "hd_profile_collect": ([i32, P, P], i32),
    "hd_launch_count": ([], u64),
    "hd_measure_peak": ([i32, u32, P], i32),
    "hd_encode_multibit": ([P, P, P, P, u32, u32, P, P], i32),
    "hd_build_library_multibit": ([P, P, P, P, u32, u32, P], i32),
    "hd_library_component_bits": ([P, P], i32),
    "hd_search_dot": ([P, P, P, P, u32, dbl, i32, u32, i32, P, P, P], i32),
    "hd_search_dot_multi": ([P, P, P, P, P, u32, P, u32, u32, i32, P, P, P], i32),
}
HD_KERNEL_ENCODE, HD_KERNEL_SEARCH = 0, 1


def library_path() -> str:
    return _build.LIB


def load():
    """The loaded libhd (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libhd.so not built ({path}); run __graft_entry__.build()")
            lib = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(status: int):
    if status != HD_OK:
        lib = load()
        raise HDError(status, lib.hd_last_error_message().decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr()) if t.numel() else C.c_void_p(0)
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    raise TypeError(type(t))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def _out(t, dtype, n_elems, name):
    """A caller's output tensor: written in place by the kernels, so it must be a
    contiguous CUDA tensor of `dtype` with room for n_elems elements (a copy made
    here would receive the results instead of the caller's tensor)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < n_elems:
        raise ValueError(f"{name} holds {t.numel()} elements, {n_elems} needed")
    return t


def _need(t, n_elems, name):
    """An input tensor must hold at least n_elems elements (the kernels read that many)."""
    if t.numel() < n_elems:
        raise ValueError(f"{name} holds {t.numel()} elements, {n_elems} needed")
    return t


def _results(n, k, out_idx, out_dist, dist_dtype=torch.int16, dist_name="out_dist"):
    """Output buffers of a top-k search: the caller's (checked) or new ones."""
    if out_idx is None:
        out_idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    if out_dist is None:
        out_dist = torch.empty((n, k), dtype=dist_dtype, device="cuda")
    return _out(out_idx, torch.int32, n * k, "out_idx"), _out(out_dist, dist_dtype, n * k, dist_name)


def _unit(unit) -> int:
    units = {"da": HD_TOL_DA, "ppm": HD_TOL_PPM, "mass": HD_TOL_MASS,
             HD_TOL_DA: HD_TOL_DA, HD_TOL_PPM: HD_TOL_PPM, HD_TOL_MASS: HD_TOL_MASS}
    if unit not in units:
        raise ValueError(f"unknown tolerance unit {unit!r}")
    return units[unit]


class Ctx:
    """Item memory (hd_ctx) on the current CUDA device."""

    POSITION_MODES = {"nested": 0, "walk": 1, "random": 2}
    ENCODERS = {"id_level": 0, "projection": 1}

    def __init__(self, dim, n_levels, n_bins, alpha=None, seed=0, position_mode="nested", encoder="id_level"):
        lib = load()
        self.dim, self.n_levels, self.n_bins = int(dim), int(n_levels), int(n_bins)
        self.alpha = self.dim // 2 if alpha is None else int(alpha)
        p = _Params(self.dim, self.n_levels, self.n_bins, self.alpha, int(seed),
                    self.POSITION_MODES[position_mode], self.ENCODERS[encoder])
        h = C.c_void_p()
        _check(lib.hd_ctx_create(C.byref(p), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().hd_ctx_destroy(self._h)
            self._h = None

    __del__ = close

    def status(self):
        _check(load().hd_ctx_status(self._h))


class Library:
    """Sorted, device-resident reference library (hd_library)."""

    def __init__(self, handle, n, dim):
        self._h, self.n, self.dim = handle, n, dim

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().hd_library_free(self._h)
            self._h = None

    __del__ = close

    def status(self):
        _check(load().hd_library_status(self._h))


def hd_ctx_create(dim, n_levels, n_bins, alpha=None, seed=0) -> Ctx:
    return Ctx(dim, n_levels, n_bins, alpha, seed)


def hd_ctx_item_memory(ctx: Ctx, stream=None):
    """(F [f, D/64] i64, L [Q, D/64] i64, rank_F [D] i32, rank_L [D] i32) on the device."""
    W = ctx.dim // 64
    F = torch.empty((ctx.n_bins, W), dtype=torch.int64, device="cuda")
    L = torch.empty((ctx.n_levels, W), dtype=torch.int64, device="cuda")
    rF = torch.empty(ctx.dim, dtype=torch.int32, device="cuda")
    rL = torch.empty(ctx.dim, dtype=torch.int32, device="cuda")
    _check(load().hd_ctx_item_memory(ctx.handle, _ptr(F), _ptr(L), _ptr(rF), _ptr(rL), _stream(stream)))
    return F, L, rF, rL


def hd_random_words(seed: int, stream_id: int, n: int, out=None, stream=None):
    """Words 0..n-1 of Philox4x32-10 word stream `stream_id` under `seed` (int32 [n] holding
    the uint32 words; read them with as_u32)."""
    if out is None:
        out = torch.empty(int(n), dtype=torch.int32, device="cuda")
    _out(out, torch.int32, int(n), "out")
    _check(load().hd_random_words(int(seed), int(stream_id), int(n), _ptr(out), _stream(stream)))
    return out


def hd_preprocess(ctx: Ctx, raw_off, raw_mz, raw_int, *, mz_min, mz_max, bin_width, n_bins, max_peaks,
                  n_levels, min_rel_intensity=0.01, stream=None):
    """Raw peak CSR on the device -> (offsets i32 [n+1], bins i32 [cap], levels u8 [cap]); the
    valid prefix of bins/levels is offsets[-1] long."""
    raw_off = _dev(raw_off, torch.int32, "raw_off")
    raw_mz = _dev(raw_mz, torch.float64, "raw_mz")
    raw_int = _dev(raw_int, torch.float64, "raw_int")
    n = raw_off.numel() - 1
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    cap = max(1, n * int(max_peaks))
    bins = torch.empty(cap, dtype=torch.int32, device="cuda")
    lv = torch.empty(cap, dtype=torch.uint8, device="cuda")
    pp = _PPParams(mz_min, mz_max, bin_width, min_rel_intensity, n_bins, max_peaks, n_levels)
    _check(load().hd_preprocess(ctx.handle, C.byref(pp), _ptr(raw_off), _ptr(raw_mz), _ptr(raw_int), n,
                                _ptr(off), _ptr(bins), _ptr(lv), _stream(stream)))
    return off, bins, lv


def hd_encode(ctx: Ctx, offsets, bins, levels, out=None, stream=None):
    offsets = _dev(offsets, torch.int32, "offsets")
    bins = _dev(bins, torch.int32, "bins")
    levels = _dev(levels, torch.uint8, "levels")
    n = offsets.numel() - 1
    if out is None:
        out = torch.empty((n, ctx.dim // 64), dtype=torch.int64, device="cuda")
    _out(out, torch.int64, n * (ctx.dim // 64), "out")
    _check(load().hd_encode(ctx.handle, _ptr(offsets), _ptr(bins), _ptr(levels), n, _ptr(out), _stream(stream)))
    return out


def hd_build_library(ctx: Ctx, hv, prec_mz, charge) -> Library:
    hv = _dev(hv, torch.int64, "hv")
    prec_mz = _dev(prec_mz, torch.float64, "prec_mz")
    charge = _dev(charge, torch.uint8, "charge")
    n = prec_mz.numel()
    torch.cuda.current_stream().synchronize()
    h = C.c_void_p()
    _check(load().hd_build_library(ctx.handle, _ptr(hv), _ptr(prec_mz), _ptr(charge), n, C.byref(h)))
    return Library(h, n, ctx.dim)


def hd_encode_multibit(ctx: Ctx, offsets, bins, levels, bits, out=None, stream=None):
    """Multi-bit components [n, D] int8 in [-m, m], m = 2^(bits-1) - 1 (bits 2..5)."""
    offsets = _dev(offsets, torch.int32, "offsets")
    bins = _dev(bins, torch.int32, "bins")
    levels = _dev(levels, torch.uint8, "levels")
    n = offsets.numel() - 1
    if out is None:
        out = torch.empty((n, ctx.dim), dtype=torch.int8, device="cuda")
    _out(out, torch.int8, n * ctx.dim, "out")
    _check(load().hd_encode_multibit(ctx.handle, _ptr(offsets), _ptr(bins), _ptr(levels), n, int(bits), _ptr(out),
                                     _stream(stream)))
    return out


def hd_build_library_multibit(ctx: Ctx, comp, prec_mz, charge, bits) -> Library:
    """Library of multi-bit component rows (int8 [n, D]); prepares its default tensor-core copy."""
    comp = _dev(comp, torch.int8, "comp")
    prec_mz = _dev(prec_mz, torch.float64, "prec_mz")
    charge = _dev(charge, torch.uint8, "charge")
    n = prec_mz.numel()
    torch.cuda.current_stream().synchronize()
    h = C.c_void_p()
    _check(load().hd_build_library_multibit(ctx.handle, _ptr(comp), _ptr(prec_mz), _ptr(charge), n, int(bits),
                                            C.byref(h)))
    return Library(h, n, ctx.dim)


def hd_library_component_bits(lib: Library) -> int:
    b = C.c_uint32()
    _check(load().hd_library_component_bits(lib.handle, C.byref(b)))
    return int(b.value)


def hd_search_dot(lib: Library, q_comp, q_mz, q_charge, tol, unit="da", k=1, form="auto",
                  out_idx=None, out_score=None, stream=None):
    """Dot-product top-k over multi-bit components: (idx i32 [n_q, k], score i32 [n_q, k]);
    padding idx -1 (0xFFFFFFFF) and score INT32_MIN."""
    q_comp = _dev(q_comp, torch.int8, "q_comp")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q_comp, n * lib.dim, "q_comp")
    _need(q_charge, n, "q_charge")
    out_idx, out_score = _results(n, k, out_idx, out_score, torch.int32, "out_score")
    _check(load().hd_search_dot(lib.handle, _ptr(q_comp), _ptr(q_mz), _ptr(q_charge), n, float(tol), _unit(unit),
                                int(k), FORMS[form], _ptr(out_idx), _ptr(out_score), _stream(stream)))
    return out_idx, out_score


def hd_search_dot_multi(lib: Library, q_comp, q_mz, q_charge, q_class, windows, k=1, form="auto",
                        out_idx=None, out_score=None, stream=None):
    """hd_search_dot with a window per query (query q uses windows[q_class[q]])."""
    q_comp = _dev(q_comp, torch.int8, "q_comp")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    if q_class is not None:
        q_class = _need(_dev(q_class, torch.uint8, "q_class"), n, "q_class")
    _need(q_comp, n * lib.dim, "q_comp")
    _need(q_charge, n, "q_charge")
    out_idx, out_score = _results(n, k, out_idx, out_score, torch.int32, "out_score")
    w = _windows(windows)
    _check(load().hd_search_dot_multi(lib.handle, _ptr(q_comp), _ptr(q_mz), _ptr(q_charge), _ptr(q_class), n, w,
                                      len(windows), int(k), FORMS[form], _ptr(out_idx), _ptr(out_score),
                                      _stream(stream)))
    return out_idx, out_score

def hd_library_prepare(lib: Library, form: str):
    """Build the library's copy for a tensor-core form ('tc_fp4' / 'tc_mxf4' share the e2m1
    copy; 'tc_fp8', 'tc_bf16')."""
    _check(load().hd_library_prepare(lib.handle, FORMS[form]))


def hd_library_set_schedule(lib: Library, tile_group: int = 0, super_group: int = 0, cluster: int = 0,
                            cta_group: int = 0):
    """Work-item shape and SM pairing of the tensor-core forms: (cluster,
    cta_group) = (2, 2) for SM pairs or (1, 1) for one SM (0 = default)."""
    _check(load().hd_library_set_schedule(lib.handle, int(tile_group), int(super_group), int(cluster),
                                          int(cta_group)))


def hd_library_set_stage_tiles(lib: Library, tiles_per_stage: int = 0):
    """Reference tiles per query stage of the kind::mxf4 form: 2 shares each staged
    query chunk between two tiles; 0 or 1 stages one tile (the default)."""
    _check(load().hd_library_set_stage_tiles(lib.handle, int(tiles_per_stage)))


def hd_library_set_wait_limit(lib: Library, seconds: float = 0.0):
    """Bound of every device wait of searches on `lib` (0: the 2 s default)."""
    _check(load().hd_library_set_wait_limit(lib.handle, int(seconds * 1e9)))


def hd_library_inject_stall(lib: Library, n_searches: int = 1):
    """Test hook: the next n searches on `lib` stall one stage until their bounded wait runs out."""
    _check(load().hd_library_inject_stall(lib.handle, int(n_searches)))


def hd_library_export(lib: Library, stream=None):
    """Sorted rows: (hv [n, D/64] i64, mz f64, charge u8, orig i32)."""
    n, W = lib.n, lib.dim // 64
    hv = torch.empty((n, W), dtype=torch.int64, device="cuda")
    mz = torch.empty(n, dtype=torch.float64, device="cuda")
    z = torch.empty(n, dtype=torch.uint8, device="cuda")
    orig = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().hd_library_export(lib.handle, _ptr(hv), _ptr(mz), _ptr(z), _ptr(orig), _stream(stream)))
    return hv, mz, z, orig


def hd_query_windows(lib: Library, q_mz, q_charge, tol, unit="da", stream=None):
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q_charge, n, "q_charge")
    lo = torch.empty(n, dtype=torch.int32, device="cuda")
    hi = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().hd_query_windows(lib.handle, _ptr(q_mz), _ptr(q_charge), n, float(tol), _unit(unit),
                                   _ptr(lo), _ptr(hi), _stream(stream)))
    return lo, hi


def hd_search_open(lib: Library, q_hv, q_mz, q_charge, tol, unit="da", k=1, form="auto",
                   out_idx=None, out_dist=None, stream=None):
    """(idx i32 [n_q, k] input reference indices, dist i16 [n_q, k]); padding 0xFFFFFFFF /
    0xFFFF (read them as unsigned)."""
    q_hv = _dev(q_hv, torch.int64, "q_hv")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q_hv, n * (lib.dim // 64), "q_hv")
    _need(q_charge, n, "q_charge")
    out_idx, out_dist = _results(n, k, out_idx, out_dist)
    _check(load().hd_search_open_ex(lib.handle, _ptr(q_hv), _ptr(q_mz), _ptr(q_charge), n, float(tol),
                                    _unit(unit), int(k), FORMS[form], _ptr(out_idx), _ptr(out_dist),
                                    _stream(stream)))
    return out_idx, out_dist


def hd_search_open_noalloc(lib: Library, q_hv, q_mz, q_charge, tol, unit="da", k=1, out_idx=None,
                           out_dist=None, stream=None):
    """hd_search_open without device allocation inside libhd (scratch from its fixed
    device buffer).  The outputs are the caller's: pass preallocated contiguous tensors
    (int32 / int16, at least n_q * k elements each) to keep the whole call
    allocation-free.  Calls that overlap on the GPU share the buffer and must be
    serialised by the caller."""
    q_hv = _dev(q_hv, torch.int64, "q_hv")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q_hv, n * (lib.dim // 64), "q_hv")
    _need(q_charge, n, "q_charge")
    out_idx, out_dist = _results(n, k, out_idx, out_dist)
    _check(load().hd_search_open_noalloc(lib.handle, _ptr(q_hv), _ptr(q_mz), _ptr(q_charge), n, float(tol),
                                         _unit(unit), int(k), _ptr(out_idx), _ptr(out_dist), _stream(stream)))
    return out_idx, out_dist


def hd_search_open_multi(lib: Library, q_hv, q_mz, q_charge, q_class, windows, k=1, form="auto",
                         out_idx=None, out_dist=None, stream=None):
    """Search with a window per query: query q uses windows[q_class[q]]; `windows` is a list of
    (tol, unit) pairs (at most 16); q_class a uint8 CUDA tensor or None."""
    q_hv = _dev(q_hv, torch.int64, "q_hv")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    if q_class is not None:
        q_class = _need(_dev(q_class, torch.uint8, "q_class"), n, "q_class")
    _need(q_hv, n * (lib.dim // 64), "q_hv")
    _need(q_charge, n, "q_charge")
    out_idx, out_dist = _results(n, k, out_idx, out_dist)
    w = _windows(windows)
    _check(load().hd_search_open_multi(lib.handle, _ptr(q_hv), _ptr(q_mz), _ptr(q_charge), _ptr(q_class), n, w,
                                       len(windows), int(k), FORMS[form], _ptr(out_idx), _ptr(out_dist),
                                       _stream(stream)))
    return out_idx, out_dist


def hd_library_save(lib: Library, ctx: Ctx, path: str):
    """Write the library (sorted rows, decoy flags, item-memory parameters) to `path`."""
    _check(load().hd_library_save(lib.handle, ctx.handle, os.fsencode(path)))


def hd_library_load(ctx: Ctx, path: str) -> "Library":
    """Read a library written by hd_library_save; ctx must have the same parameters."""
    h = C.c_void_p()
    _check(load().hd_library_load(ctx.handle, os.fsencode(path), C.byref(h)))
    n, dim = C.c_uint32(), C.c_uint32()
    _check(load().hd_library_info(h, C.byref(n), C.byref(dim)))
    return Library(h, n.value, dim.value)


def hd_library_set_decoys(lib: Library, is_decoy):
    """Decoy flags [n_refs] (uint8, input order, nonzero = decoy) for the cascade's FDR filter."""
    f = _dev(is_decoy, torch.uint8, "is_decoy")
    _check(load().hd_library_set_decoys(lib.handle, _ptr(f)))


def hd_cascade_search(lib: Library, q_hv, q_mz, q_charge, levels, fdr=0.01, form="auto", stream=None):
    """Cascade search with target-decoy FDR: `levels` is a list of (tol, unit) windows, narrow
    first.  Returns (idx int32 [n], dist int16 [n], q float64 [n], level uint8 [n]); level 255 =
    not identified."""
    q_hv = _dev(q_hv, torch.int64, "q_hv")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q_hv, n * (lib.dim // 64), "q_hv")
    _need(q_charge, n, "q_charge")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    dist = torch.empty(n, dtype=torch.int16, device="cuda")
    q = torch.empty(n, dtype=torch.float64, device="cuda")
    level = torch.empty(n, dtype=torch.uint8, device="cuda")
    w = _windows(levels)
    _check(load().hd_cascade_search(lib.handle, _ptr(q_hv), _ptr(q_mz), _ptr(q_charge), n, w, len(levels),
                                    float(fdr), FORMS[form], _ptr(idx), _ptr(dist), _ptr(q), _ptr(level),
                                    _stream(stream)))
    return idx, dist, q, level


def hd_cascade_search_dot(lib: Library, q_comp, q_mz, q_charge, levels, fdr=0.01, form="auto", stream=None):
    """Cascade search of a multi-bit library: q_comp int8 [n, D] components.  Returns
    (idx int32 [n], score int32 [n], q float64 [n], level uint8 [n]); score INT32_MIN without a
    candidate, level 255 = not identified."""
    q_comp = _dev(q_comp, torch.int8, "q_comp")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q_comp, n * lib.dim, "q_comp")
    _need(q_charge, n, "q_charge")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    score = torch.empty(n, dtype=torch.int32, device="cuda")
    q = torch.empty(n, dtype=torch.float64, device="cuda")
    level = torch.empty(n, dtype=torch.uint8, device="cuda")
    w = _windows(levels)
    _check(load().hd_cascade_search_dot(lib.handle, _ptr(q_comp), _ptr(q_mz), _ptr(q_charge), n, w, len(levels),
                                        float(fdr), FORMS[form], _ptr(idx), _ptr(score), _ptr(q), _ptr(level),
                                        _stream(stream)))
    return idx, score, q, level


class Plan:
    """Encode + multi-window search of a fixed query set, captured as one CUDA graph.
    Keeps references to every bound buffer; refill them in place and call launch()."""

    def __init__(self, ctx: Ctx, lib: Library, offsets, bins, levels, q_mz, q_charge, q_class, windows, k=1,
                 form="auto"):
        """On a multi-bit library the plan encodes components and runs the dot-product search:
        launch() then returns (idx, score int32)."""
        self.offsets = _dev(offsets, torch.int32, "offsets")
        self.bins = _dev(bins, torch.int32, "bins")
        self.levels = _dev(levels, torch.uint8, "levels")
        self.q_mz = _dev(q_mz, torch.float64, "q_mz")
        self.q_charge = _dev(q_charge, torch.uint8, "q_charge")
        self.q_class = None if q_class is None else _dev(q_class, torch.uint8, "q_class")
        n = self.q_mz.numel()
        self.multibit = hd_library_component_bits(lib) > 1
        self.out_idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
        self._keep = (ctx, lib)
        w = _windows(windows)
        h = C.c_void_p()
        torch.cuda.current_stream().synchronize()
        if self.multibit:
            self.q_comp = torch.empty((n, ctx.dim), dtype=torch.int8, device="cuda")
            self.out_score = torch.empty((n, k), dtype=torch.int32, device="cuda")
            _check(load().hd_plan_create_dot(ctx.handle, lib.handle, _ptr(self.offsets), _ptr(self.bins),
                                             _ptr(self.levels), _ptr(self.q_mz), _ptr(self.q_charge),
                                             _ptr(self.q_class), n, w, len(windows), int(k), FORMS[form],
                                             _ptr(self.q_comp), _ptr(self.out_idx), _ptr(self.out_score),
                                             C.byref(h)))
        else:
            self.q_hv = torch.empty((n, ctx.dim // 64), dtype=torch.int64, device="cuda")
            self.out_dist = torch.empty((n, k), dtype=torch.int16, device="cuda")
            _check(load().hd_plan_create(ctx.handle, lib.handle, _ptr(self.offsets), _ptr(self.bins),
                                         _ptr(self.levels), _ptr(self.q_mz), _ptr(self.q_charge),
                                         _ptr(self.q_class), n, w, len(windows), int(k), FORMS[form],
                                         _ptr(self.q_hv), _ptr(self.out_idx), _ptr(self.out_dist), C.byref(h)))
        self._h = h
        nodes = C.c_uint32()
        _check(load().hd_plan_info(h, C.byref(nodes)))
        self.kernel_nodes = nodes.value

    def launch(self, stream=None):
        _check(load().hd_plan_launch(self._h, _stream(stream)))
        return (self.out_idx, self.out_score) if self.multibit else (self.out_idx, self.out_dist)

    def close(self):
        if getattr(self, "_h", None):
            load().hd_plan_destroy(self._h)
            self._h = None

    __del__ = close


def hd_library_autotune(lib: Library, q_hv, q_mz, q_charge, q_class, windows, k=1):
    """Times every prepared form and schedule; keeps the fastest as the library's 'auto'.
    Returns (best, all) as dicts.  On a multi-bit library q_hv holds the queries' int8
    components [n, D] and the dot-product search is tuned (hd_library_autotune_dot)."""
    multibit = hd_library_component_bits(lib) > 1
    if multibit:
        q = _dev(q_hv, torch.int8, "q_comp")
    else:
        q = _dev(q_hv, torch.int64, "q_hv")
    q_mz = _dev(q_mz, torch.float64, "q_mz")
    q_charge = _dev(q_charge, torch.uint8, "q_charge")
    n = q_mz.numel()
    _need(q, n * (lib.dim if multibit else lib.dim // 64), "q_comp" if multibit else "q_hv")
    _need(q_charge, n, "q_charge")
    if q_class is not None:
        q_class = _need(_dev(q_class, torch.uint8, "q_class"), n, "q_class")
    torch.cuda.current_stream().synchronize()
    best = _TuneResult()
    allr = (_TuneResult * 128)()
    n_all = C.c_uint32()
    w = _windows(windows)
    fn = load().hd_library_autotune_dot if multibit else load().hd_library_autotune
    _check(fn(lib.handle, _ptr(q), _ptr(q_mz), _ptr(q_charge), _ptr(q_class), q_mz.numel(), w, len(windows),
              int(k), C.byref(best), allr, 128, C.byref(n_all)))
    names = {v: k_ for k_, v in FORMS.items()}
    conv = lambda r: {"form": names[r.form], "tile_group": r.tile_group, "super_group": r.super_group,
                      "cluster": r.cluster, "cta_group": r.cta_group, "tiles_per_stage": r.tiles_per_stage,
                      "ms": r.ms}
    return conv(best), [conv(allr[i]) for i in range(min(128, n_all.value))]


class _PeakResult(C.Structure):
    _fields_ = [("best_per_s", C.c_double), ("median_per_s", C.c_double), ("ms_best", C.c_double),
                ("ops_per_launch", C.c_uint64), ("sms", C.c_uint32), ("launches", C.c_uint32)]


PEAK_KINDS = {"tc_fp4": 0, "tc_fp8": 1, "tc_bf16": 2, "popc": 3, "lop3": 4, "tc_mxf4": 5}


def hd_measure_peak(kind: str, launches: int = 10):
    """Instruction-rate microbenchmark (hd_measure_peak): 'tc_fp4' / 'tc_fp8' / 'tc_bf16'
    (flops/s of the SM-pair tensor-core instruction), 'popc' (popcounts/s) or 'lop3'."""
    r = _PeakResult()
    _check(load().hd_measure_peak(PEAK_KINDS[kind], int(launches), C.byref(r)))
    return {f: getattr(r, f) for f, _ in _PeakResult._fields_}


class _ServerParams(C.Structure):
    _fields_ = [("slots", C.c_uint32), ("max_batch_queries", C.c_uint32), ("mem_budget_bytes", C.c_uint64),
                ("k", C.c_uint32), ("form", C.c_int)]


class _RequestInfo(C.Structure):
    _fields_ = [("latency_s", C.c_double), ("queue_s", C.c_double), ("n_queries", C.c_uint32),
                ("batch_queries", C.c_uint32)]


class _ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("queries", C.c_uint64),
                ("batches", C.c_uint64), ("max_inflight", C.c_uint32)]


class _BatchRecord(C.Structure):
    _fields_ = [("batch", C.c_uint64), ("slot", C.c_uint32), ("n_queries", C.c_uint32), ("n_requests", C.c_uint32),
                ("device_start_ms", C.c_double), ("device_end_ms", C.c_double)]


class Server:
    """Continuous-batching server (hd_server_*) on a resident library."""

    def __init__(self, ctx: Ctx, lib: Library, k=5, slots=3, max_batch_queries=8192, mem_budget_bytes=0,
                 form="auto"):
        self.k = int(k)
        self._keep = (ctx, lib)
        self._pending = {}
        self.multibit = hd_library_component_bits(lib) > 1
        p = _ServerParams(int(slots), int(max_batch_queries), int(mem_budget_bytes), self.k, FORMS[form])
        h = C.c_void_p()
        _check(load().hd_server_create(ctx.handle, lib.handle, C.byref(p), C.byref(h)))
        self._h = h

    def submit(self, offsets, bins, levels, q_mz, q_charge, tol, unit="da"):
        """Queue one request (host arrays); returns its id.  On a multi-bit library the
        request is scored by the dot product (wait() returns int32 scores)."""
        off = np.ascontiguousarray(offsets, np.uint32)
        b = np.ascontiguousarray(bins, np.uint32)
        lv = np.ascontiguousarray(levels, np.uint8)
        mz = np.ascontiguousarray(q_mz, np.float64)
        z = np.ascontiguousarray(q_charge, np.uint8)
        n = mz.size
        oi = np.empty((n, self.k), np.uint32)
        od = np.empty((n, self.k), np.int32 if self.multibit else np.uint16)
        rid = C.c_uint64()
        fn = load().hd_server_submit_dot if self.multibit else load().hd_server_submit
        _check(fn(self._h, _ptr(off), _ptr(b), _ptr(lv), _ptr(mz), _ptr(z), n, float(tol), _unit(unit), _ptr(oi),
                  _ptr(od), C.byref(rid)))
        self._pending[rid.value] = (oi, od)
        return rid.value

    def wait(self, rid, timeout_s=120.0):
        """(idx [n, k] u32, dist [n, k] u16 -- or score [n, k] int32 on a multi-bit
        library --, info dict) once the request is done."""
        info = _RequestInfo()
        oi, od = self._pending[rid]
        _check(load().hd_server_wait(self._h, C.c_uint64(rid), float(timeout_s), C.byref(info)))
        del self._pending[rid]
        return oi, od, {"latency_s": info.latency_s, "queue_s": info.queue_s, "n_queries": info.n_queries,
                        "batch_queries": info.batch_queries}

    def stats(self):
        st = _ServerStats()
        _check(load().hd_server_stats_get(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def batch_log(self, cap=4096):
        """Device-time intervals of the finished batches (oldest first), as dicts."""
        arr = (_BatchRecord * cap)()
        n = C.c_uint32()
        _check(load().hd_server_batch_log(self._h, arr, cap, C.byref(n)))
        return [{f: getattr(arr[i], f) for f, _ in _BatchRecord._fields_} for i in range(n.value)]

    def close(self):
        if getattr(self, "_h", None):
            load().hd_server_destroy(self._h)
            self._h = None

    __del__ = close


def hd_search_host(ctx: Ctx, lib: Library, offsets, bins, levels, q_mz, q_charge, tol, unit="da", k=1,
                   out_idx=None, out_dist=None, stream=None):
    """End to end from host arrays (numpy, or pinned CPU tensors); returns host arrays."""
    def host(a, dt):
        if isinstance(a, torch.Tensor):
            assert not a.is_cuda and a.is_contiguous()
            return a
        return np.ascontiguousarray(a, dtype=dt)
    offsets, bins = host(offsets, np.uint32), host(bins, np.uint32)
    levels, q_mz, q_charge = host(levels, np.uint8), host(q_mz, np.float64), host(q_charge, np.uint8)
    n = (offsets.numel() if isinstance(offsets, torch.Tensor) else offsets.size) - 1
    if out_idx is None:
        out_idx = np.empty((n, k), np.uint32)
    if out_dist is None:
        out_dist = np.empty((n, k), np.uint16)
    _check(load().hd_search_host(ctx.handle, lib.handle, _ptr(offsets), _ptr(bins), _ptr(levels), _ptr(q_mz),
                                 _ptr(q_charge), n, float(tol), _unit(unit), int(k), _ptr(out_idx),
                                 _ptr(out_dist), _stream(stream)))
    return out_idx, out_dist


def hd_profile_enable(on: bool = True):
    _check(load().hd_profile_enable(1 if on else 0))


def hd_profile_collect(kind: int):
    """(total milliseconds, launches) of the recorded launches of `kind`."""
    ms, n = C.c_double(), C.c_uint32()
    _check(load().hd_profile_collect(kind, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def hd_launch_count() -> int:
    return int(load().hd_launch_count())


def as_u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def as_u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def as_u16(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint16)
