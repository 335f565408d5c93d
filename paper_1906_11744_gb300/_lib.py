"""ctypes binding of the C ABI in include/kf.h (argument marshalling only).

Every function here has the name of its C entry point and forwards to it;
array arguments are torch CUDA tensors (device_ptrs = 1) or numpy arrays /
CPU tensors (device_ptrs = 0).  The library must have been built (see
``paper_1906_11744_gb300.build``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KF_OK = 0
KF_ERR_ARG = -1
KF_ERR_CUDA = -2
KF_ERR_CAPACITY = -3
KF_ERR_TIMEOUT = -4
KF_ERR_STATE = -5
KF_MAX_LAYERS = 32
KF_MAX_CANDS = 16
KF_FIT_FOUND = 0
KF_FIT_GIVEN = 1
KF_FIT_OK = 0
KF_FIT_SKIPPED = 1
KF_NOALLOC_MAX_TRACKS = 16384
KF_NOALLOC_MAX_HITS = 262144
KF_SEED_MAX_DETA = 1.0
KF_MAX_MATERIAL_NODES = 4096
KF_MAX_DISKS = 16
KF_N_COUNTERS = 11


class kf_detector(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("radius", ctypes.c_float * KF_MAX_LAYERS),
                ("x0", ctypes.c_float * KF_MAX_LAYERS), ("z_max", ctypes.c_float),
                ("bz", ctypes.c_float), ("sigma_rphi", ctypes.c_float), ("sigma_z", ctypes.c_float),
                ("eloss", ctypes.c_float * KF_MAX_LAYERS), ("field_cz", ctypes.c_float),
                ("field_cr", ctypes.c_float), ("n_disks", ctypes.c_int),
                ("disk_z", ctypes.c_float * KF_MAX_DISKS), ("disk_rmin", ctypes.c_float),
                ("disk_rmax", ctypes.c_float), ("disk_x0", ctypes.c_float), ("disk_eloss", ctypes.c_float),
                ("sigma_r", ctypes.c_float), ("eta_barrel", ctypes.c_float)]


class kf_config(ctypes.Structure):
    _fields_ = [("max_cands", ctypes.c_int), ("max_holes", ctypes.c_int), ("chi2_cut", ctypes.c_float),
                ("dup_shared_frac", ctypes.c_float), ("n_eta_bins", ctypes.c_int),
                ("n_phi_bins", ctypes.c_int), ("lanes_per_seed", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("persistent", ctypes.c_int),
                ("per_event", ctypes.c_int), ("ckpt_stride", ctypes.c_int), ("find_regcap", ctypes.c_int),
                ("dup_deta", ctypes.c_float), ("dup_dphi", ctypes.c_float), ("dup_dpt", ctypes.c_float),
                ("seed_clean", ctypes.c_int), ("seed_deta", ctypes.c_float), ("seed_dphi", ctypes.c_float),
                ("seed_dpt", ctypes.c_float), ("seed_min_shared", ctypes.c_int),
                ("resolve_max_rounds", ctypes.c_int)]


class KFError(RuntimeError):
    pass


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "kf_create": ([ctypes.POINTER(kf_detector), ctypes.POINTER(kf_config), ctypes.POINTER(_P)], _I),
    "kf_destroy": ([_P], _I),
    "kf_load_hits": ([_P, _I, _P, _P, _P, _P, _P, _I, _P], _I),
    "kf_load_seeds": ([_P, _I, _P, _P, _P, _P, _I, _P], _I),
    "kf_set_alignment": ([_P, _P, _I, _P], _I),
    "kf_set_material": ([_P, _I, _P, _I, _P], _I),
    "kf_find_tracks": ([_P, _P], _I),
    "kf_remove_duplicates": ([_P, _P], _I),
    "kf_fit_tracks": ([_P, _I, _P, _P, _I, _I, _P], _I),
    "kf_fit_adjoint": ([_P, _P, _P, _P, _I, _P], _I),
    "kf_get_tracks": ([_P, _P, _P, _P, _P, _P, _P, _I, _P], _I),
    "kf_get_fit": ([_P, _P, _P, _P, _P, _I, _P], _I),
    "kf_capture_graph": ([_P, _I, _P], _I),
    "kf_launch_graph": ([_P, _P], _I),
    "kf_autotune": ([_P, _P, _I, _P, _P], _I),
    "kf_get_counters": ([_P, _P, _P], _I),
    "kf_get_counters_n": ([_P, _P, _I, _P], _I),
    "kf_sync": ([_P, _P], _I),
    "kf_set_stage_timing": ([_P, _I], _I),
    "kf_get_stage_ms": ([_P, _P, _P], _I),
    "kf_graph_kernel_count": ([_P, _P], _I),
    "kf_last_error": ([_P], ctypes.c_char_p),
    "kf_get_gradient": ([_P, _P, _P, _P, _I, _P], _I),
    "kf_remove_duplicates_noalloc": ([_I, _I, _I, _P, _P, _P, ctypes.c_float, _P, _P, _P], _I),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libkf.so; raises if it was not built (there is no fallback)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise KFError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(ctx, rc, what):
    if rc != KF_OK:
        msg = load().kf_last_error(ctx).decode() if ctx else ""
        raise KFError(f"{what} failed ({rc}): {msg}")


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, dtype):
    """(pointer, keepalive, device flag) for a torch tensor or array-like."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        if a.is_cuda:
            return ctypes.c_void_p(a.data_ptr()), a, 1
        return ctypes.c_void_p(a.data_ptr()), a, 0
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), arr, 0


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _flag(*flags):
    fl = {f for f in flags if f is not None}
    if len(fl) > 1:
        raise KFError("mixed host and device arrays in one call")
    return fl.pop() if fl else 0


def kf_create(det: kf_detector, cfg: kf_config):
    ctx = _P()
    rc = load().kf_create(ctypes.byref(det), ctypes.byref(cfg), ctypes.byref(ctx))
    if rc != KF_OK:
        raise KFError(f"kf_create failed ({rc})")
    return ctx


def kf_destroy(ctx):
    _check(None, load().kf_destroy(ctx), "kf_destroy")


def kf_load_hits(ctx, ev_offsets, x, y, z, layer, stream=None):
    off = np.ascontiguousarray(ev_offsets, dtype=np.int32)
    px, kx, fx = _arg(x, np.float32)
    py, ky, fy = _arg(y, np.float32)
    pz, kz, fz = _arg(z, np.float32)
    pl, kl, fl = _arg(layer, np.int32)
    rc = load().kf_load_hits(ctx, off.size - 1, off.ctypes.data_as(_P), px, py, pz, pl,
                             _flag(fx, fy, fz, fl), _stream(stream))
    _check(ctx, rc, "kf_load_hits")


def kf_load_seeds(ctx, ev_offsets, params, cov, seed_hits, stream=None):
    off = np.ascontiguousarray(ev_offsets, dtype=np.int32)
    pp, kp, fp = _arg(params, np.float32)
    pc, kc, fc = _arg(cov, np.float32)
    ps, ks, fs = _arg(seed_hits, np.int32)
    rc = load().kf_load_seeds(ctx, off.size - 1, off.ctypes.data_as(_P), pp, pc, ps, _flag(fp, fc, fs),
                              _stream(stream))
    _check(ctx, rc, "kf_load_seeds")


def kf_set_alignment(ctx, offsets, stream=None):
    po, ko, fo = _arg(offsets, np.float32)
    _check(ctx, load().kf_set_alignment(ctx, po, _flag(fo), _stream(stream)), "kf_set_alignment")


def kf_set_material(ctx, x0_map=None, stream=None):
    """x0_map [n_layers][n_z] (None: back to the per-layer x0)."""
    if x0_map is None:
        _check(ctx, load().kf_set_material(ctx, 0, None, 0, _stream(stream)), "kf_set_material")
        return
    n_z = int(x0_map.shape[1])
    pm, km, fm = _arg(x0_map, np.float32)
    _check(ctx, load().kf_set_material(ctx, n_z, pm, _flag(fm), _stream(stream)), "kf_set_material")


def kf_find_tracks(ctx, stream=None):
    _check(ctx, load().kf_find_tracks(ctx, _stream(stream)), "kf_find_tracks")


def kf_remove_duplicates(ctx, stream=None):
    _check(ctx, load().kf_remove_duplicates(ctx, _stream(stream)), "kf_remove_duplicates")


def kf_fit_tracks(ctx, source=KF_FIT_FOUND, hit_lists=None, n_hits=None, stream=None):
    ph, kh, fh = _arg(hit_lists, np.int32)
    pn, kn, fn = _arg(n_hits, np.int32)
    max_len = 0 if hit_lists is None else int(hit_lists.shape[1])
    rc = load().kf_fit_tracks(ctx, source, ph, pn, max_len, _flag(fh, fn), _stream(stream))
    _check(ctx, rc, "kf_fit_tracks")


def kf_fit_adjoint(ctx, g_align, g_hits=None, g_seed=None, stream=None):
    pa, ka, fa = _arg(g_align, np.float32)
    ph, kh, fh = _arg(g_hits, np.float32)
    ps, ks, fs = _arg(g_seed, np.float32)
    rc = load().kf_fit_adjoint(ctx, pa, ph, ps, _flag(fa, fh, fs), _stream(stream))
    _check(ctx, rc, "kf_fit_adjoint")


def kf_get_gradient(ctx, g_align=None, g_hits=None, g_seed=None, stream=None):
    args = [_arg(g_align, np.float32), _arg(g_hits, np.float32), _arg(g_seed, np.float32)]
    rc = load().kf_get_gradient(ctx, *[a[0] for a in args], _flag(*[a[2] for a in args]), _stream(stream))
    _check(ctx, rc, "kf_get_gradient")


def kf_get_tracks(ctx, hits=None, n_found=None, chi2=None, params=None, cov=None, keep=None, stream=None):
    """Outputs are written into the given (preallocated) arrays/tensors."""
    args = [_arg(hits, np.int32), _arg(n_found, np.int32), _arg(chi2, np.float32),
            _arg(params, np.float32), _arg(cov, np.float32), _arg(keep, np.uint8)]
    rc = load().kf_get_tracks(ctx, *[a[0] for a in args], _flag(*[a[2] for a in args]), _stream(stream))
    _check(ctx, rc, "kf_get_tracks")


def kf_get_fit(ctx, params=None, cov=None, chi2=None, status=None, stream=None):
    args = [_arg(params, np.float32), _arg(cov, np.float32), _arg(chi2, np.float32), _arg(status, np.int32)]
    rc = load().kf_get_fit(ctx, *[a[0] for a in args], _flag(*[a[2] for a in args]), _stream(stream))
    _check(ctx, rc, "kf_get_fit")


def kf_capture_graph(ctx, with_adjoint=0, stream=None):
    _check(ctx, load().kf_capture_graph(ctx, int(with_adjoint), _stream(stream)), "kf_capture_graph")


def kf_launch_graph(ctx, stream=None):
    _check(ctx, load().kf_launch_graph(ctx, _stream(stream)), "kf_launch_graph")


def kf_autotune(ctx, stream=None, max_results=128):
    res = np.zeros((max_results, 5), np.float32)
    n = ctypes.c_int(0)
    rc = load().kf_autotune(ctx, res.ctypes.data_as(_P), max_results, ctypes.byref(n), _stream(stream))
    _check(ctx, rc, "kf_autotune")
    return res[:n.value]


def kf_get_counters(ctx, stream=None):
    """The finding's counters (kf_get_counters_n, all KF_N_COUNTERS of them)."""
    c = np.zeros(KF_N_COUNTERS, np.int64)
    _check(ctx, load().kf_get_counters_n(ctx, c.ctypes.data_as(_P), KF_N_COUNTERS, _stream(stream)),
           "kf_get_counters_n")
    return dict(steps=int(c[0]), updates=int(c[1]), chi2_evals=int(c[2]), seeds=int(c[3]),
                holes=int(c[4]), careful=int(c[5]), not_pd=int(c[6]), redone=int(c[7]),
                disk_steps=int(c[8]), disk_updates=int(c[9]), disk_holes=int(c[10]))


def kf_set_stage_timing(ctx, enable=True):
    _check(ctx, load().kf_set_stage_timing(ctx, int(enable)), "kf_set_stage_timing")


def kf_get_stage_ms(ctx, stream=None):
    """Stage durations of the last run (ms); stages that did not run are left out."""
    ms = np.zeros(6, np.float32)
    _check(ctx, load().kf_get_stage_ms(ctx, ms.ctypes.data_as(_P), _stream(stream)), "kf_get_stage_ms")
    names = ("bin", "find", "dedup", "fit", "adjoint", "seed_clean")
    return {k: float(v) for k, v in zip(names, ms) if v >= 0}


def kf_graph_kernel_count(ctx):
    n = ctypes.c_int(0)
    _check(ctx, load().kf_graph_kernel_count(ctx, ctypes.byref(n)), "kf_graph_kernel_count")
    return n.value


def kf_sync(ctx, stream=None):
    _check(ctx, load().kf_sync(ctx, _stream(stream)), "kf_sync")


def kf_last_error(ctx) -> str:
    return load().kf_last_error(ctx).decode()


def kf_remove_duplicates_noalloc(n_tracks, n_layers, n_hits, hits, n_found, chi2, dup_shared_frac, keep,
                                 status=None, stream=None):
    """Allocation-free duplicate removal of one event; all arrays are CUDA
    tensors (the caller owns them).  Returns the C return code."""
    args = [_arg(hits, np.int32), _arg(n_found, np.int32), _arg(chi2, np.float32), _arg(keep, np.uint8),
            _arg(status, np.int32)]
    for a in args:
        if a[2] == 0:
            raise KFError("kf_remove_duplicates_noalloc takes device arrays only")
    return load().kf_remove_duplicates_noalloc(int(n_tracks), int(n_layers), int(n_hits), args[0][0], args[1][0],
                                               args[2][0], float(dup_shared_frac), args[3][0], args[4][0],
                                               _stream(stream))
