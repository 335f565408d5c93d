"""FP64 CPU oracle of the Kalman-filter track finder (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  It wraps ``kf_oracle.cpp`` (plain double-precision
C++, full 6x6 matrices, no shared code with the CUDA path) through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (host code, any architecture)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Detector(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("radius", ctypes.c_double * 64),
                ("x0", ctypes.c_double * 64), ("z_max", ctypes.c_double), ("bz", ctypes.c_double),
                ("sigma_rphi", ctypes.c_double), ("sigma_z", ctypes.c_double),
                ("n_z", ctypes.c_int), ("x0_map", ctypes.c_void_p), ("eloss", ctypes.c_double * 64),
                ("field_cz", ctypes.c_double), ("field_cr", ctypes.c_double),
                ("n_disks", ctypes.c_int), ("disk_z", ctypes.c_double * 32), ("disk_rmin", ctypes.c_double),
                ("disk_rmax", ctypes.c_double), ("disk_x0", ctypes.c_double), ("disk_eloss", ctypes.c_double),
                ("sigma_r", ctypes.c_double), ("eta_barrel", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("max_cands", ctypes.c_int), ("max_holes", ctypes.c_int), ("chi2_cut", ctypes.c_double)]


_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.orc_propagate.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, ctypes.c_double, _P, _P]
            L.orc_path_length.argtypes = [ctypes.c_double, _P, ctypes.c_double, _P]
            L.orc_propagate_ad.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, ctypes.c_double, _P]
            L.orc_transport.argtypes = [_P, _P, _P]
            L.orc_update.argtypes = [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P, _P]
            L.orc_update_disk.argtypes = [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P, _P]
            L.orc_propagate_plane.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _P,
                                              ctypes.c_double, _P, _P]
            L.orc_propagate_plane_ad.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _P,
                                                 ctypes.c_double, _P]
            L.orc_eloss_disk.argtypes = [_P, _P, ctypes.c_double]
            L.orc_highland_disk.argtypes = [_P, ctypes.c_double]
            L.orc_highland_disk.restype = ctypes.c_double
            L.orc_highland.argtypes = [_P, ctypes.c_double]
            L.orc_x0_at.argtypes = [_P, ctypes.c_int, ctypes.c_double]
            L.orc_eloss.argtypes = [_P, _P, ctypes.c_double]
            L.orc_x0_at.restype = ctypes.c_double
            L.orc_highland.restype = ctypes.c_double
            L.orc_add_ms.argtypes = [_P, _P, ctypes.c_double]
            L.orc_fit.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_long, _P, _P, ctypes.c_int,
                                  _P, _P, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]
            L.orc_fit_grad.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_long, _P, _P, ctypes.c_int,
                                       _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
            L.orc_fit_grad32.argtypes = L.orc_fit_grad.argtypes
            L.orc_find_event.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P,
                                         ctypes.c_long, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                         _P, _P, _P, _P, _P, _P]
            L.orc_replay.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
            L.orc_select_children.argtypes = [ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int, _P]
            L.orc_census_step.argtypes = [_P, ctypes.c_double, _P, _P, ctypes.c_int, _P, _P, _P, _P]
            L.orc_census_disk_step.argtypes = [_P, ctypes.c_double, _P, _P, ctypes.c_int, _P, _P, _P]
            L.orc_census_fit.argtypes = [_P, _P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P]
            L.orc_census_transport.argtypes = [_P, _P, _P]
            L.orc_dedup.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double]
            L.orc_kinematics.argtypes = [ctypes.c_int, ctypes.c_double, _P, _P]
            L.orc_seed_clean.argtypes = [ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, _P]
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_detector(det) -> Detector:
    """ctypes detector from a synth.Detector; values rounded to float32 first,
    so the oracle sees exactly the numbers the float32 path is given."""
    d = Detector()
    d.n_layers = det.n_layers
    for i, r in enumerate(det.radius):
        d.radius[i] = float(np.float32(r))
        d.x0[i] = float(np.float32(det.x0[i]))
    d.z_max = float(np.float32(det.z_max))
    d.bz = float(np.float32(det.bz))
    d.sigma_rphi = float(np.float32(det.sigma_rphi))
    d.sigma_z = float(np.float32(det.sigma_z))
    for i, e in enumerate(getattr(det, "eloss", ()) or ()):
        d.eloss[i] = float(np.float32(e))
    d.field_cz = float(np.float32(getattr(det, "field_cz", 0.0)))
    d.field_cr = float(np.float32(getattr(det, "field_cr", 0.0)))
    dz = tuple(getattr(det, "disk_z", ()) or ())
    d.n_disks = len(dz)
    for i, v in enumerate(dz):
        d.disk_z[i] = float(np.float32(v))
    d.disk_rmin = float(np.float32(getattr(det, "disk_rmin", 0.0)))
    d.disk_rmax = float(np.float32(getattr(det, "disk_rmax", 0.0)))
    d.disk_x0 = float(np.float32(getattr(det, "disk_x0", 0.0)))
    d.disk_eloss = float(np.float32(getattr(det, "disk_eloss", 0.0)))
    d.sigma_r = float(np.float32(getattr(det, "sigma_r", 0.1)))
    d.eta_barrel = float(getattr(det, "eta_barrel", 0.9))
    m = getattr(det, "x0_map", None)
    if m is not None:  # float32-rounded like every other input; kept alive by the structure
        d._map = np.ascontiguousarray(np.asarray(m, np.float32).astype(np.float64).reshape(det.n_layers, -1))
        d.n_z = d._map.shape[1]
        d.x0_map = d._map.ctypes.data
    return d


def make_config(max_cands=6, max_holes=3, chi2_cut=30.0) -> Config:
    return Config(max_cands, max_holes, float(np.float32(chi2_cut)))


# ------------------------------------------------------------ single-state pins
def propagate(bz: float, p, R: float, cz: float = 0.0, cr: float = 0.0):
    """Helix to radius R in the axial field bz (1 + cz z^2 + cr r^2) taken at
    the starting point; J at that field held fixed."""
    p = _c(p, np.float64)
    q = np.zeros(6)
    J = np.zeros(36)
    ok = lib().orc_propagate(bz, cz, cr, _ptr(p), R, _ptr(q), _ptr(J))
    return bool(ok), q, J.reshape(6, 6)


def path_length(bz: float, p, R: float):
    p = _c(p, np.float64)
    s = np.zeros(1)
    ok = lib().orc_path_length(bz, _ptr(p), R, _ptr(s))
    return bool(ok), float(s[0])


def propagate_ad(bz: float, p, R: float, cz: float = 0.0, cr: float = 0.0):
    p = _c(p, np.float64)
    J = np.zeros(36)
    ok = lib().orc_propagate_ad(bz, cz, cr, _ptr(p), R, _ptr(J))
    return bool(ok), J.reshape(6, 6)


def transport(J, C):
    J = _c(J, np.float64)
    C = _c(C, np.float64)
    out = np.zeros(36)
    lib().orc_transport(_ptr(J), _ptr(C), _ptr(out))
    return out.reshape(6, 6)


def update(p, C, m, vr, vz):
    p = _c(p, np.float64); C = _c(C, np.float64); m = _c(m, np.float64)
    po, Co, c2, r = np.zeros(6), np.zeros(36), np.zeros(1), np.zeros(2)
    ok = lib().orc_update(_ptr(p), _ptr(C), _ptr(m), vr, vz, _ptr(po), _ptr(Co), _ptr(c2), _ptr(r))
    return bool(ok), po, Co.reshape(6, 6), float(c2[0]), r


def highland(p, x0):
    p = _c(p, np.float64)
    return lib().orc_highland(_ptr(p), x0)


def propagate_plane(bz: float, p, zd: float, cz: float = 0.0, cr: float = 0.0):
    """Helix to the plane z = zd (an endcap disk) in the field at the start;
    J at that field held fixed."""
    p = _c(p, np.float64)
    q = np.zeros(6)
    J = np.zeros(36)
    ok = lib().orc_propagate_plane(bz, cz, cr, _ptr(p), zd, _ptr(q), _ptr(J))
    return bool(ok), q, J.reshape(6, 6)


def propagate_plane_ad(bz: float, p, zd: float, cz: float = 0.0, cr: float = 0.0):
    p = _c(p, np.float64)
    J = np.zeros(36)
    ok = lib().orc_propagate_plane_ad(bz, cz, cr, _ptr(p), zd, _ptr(J))
    return bool(ok), J.reshape(6, 6)


def update_disk(p, C, m, vr, vrr):
    """One Kalman update on an endcap disk: residuals along r-phi and r."""
    p = _c(p, np.float64); C = _c(C, np.float64); m = _c(m, np.float64)
    po, Co, c2, r = np.zeros(6), np.zeros(36), np.zeros(1), np.zeros(2)
    ok = lib().orc_update_disk(_ptr(p), _ptr(C), _ptr(m), vr, vrr, _ptr(po), _ptr(Co), _ptr(c2), _ptr(r))
    return bool(ok), po, Co.reshape(6, 6), float(c2[0]), r


def highland_disk(p, x0):
    p = _c(p, np.float64)
    return lib().orc_highland_disk(_ptr(p), x0)


def eloss_disk(p, C, e):
    p = _c(p, np.float64).copy()
    C = _c(np.asarray(C, np.float64).reshape(36), np.float64).copy()
    lib().orc_eloss_disk(_ptr(p), _ptr(C), float(e))
    return p, C.reshape(6, 6)


def eloss(p, C, e):
    """Mean ionization energy loss step of one state (e: the layer's loss at
    normal incidence for beta -> 1, GeV): returns (p', C' [6][6])."""
    p = _c(p, np.float64).copy()
    C = _c(np.asarray(C, np.float64).reshape(36), np.float64).copy()
    lib().orc_eloss(_ptr(p), _ptr(C), float(e))
    return p, C.reshape(6, 6)


def x0_at(det, layer: int, z: float) -> float:
    """Thickness of a layer at z: the detector's material map, else its x0."""
    d = make_detector(det)
    return lib().orc_x0_at(ctypes.byref(d), int(layer), float(z))


def add_ms(p, C, x0):
    p = _c(p, np.float64)
    C = _c(C, np.float64).copy()
    lib().orc_add_ms(_ptr(p), _ptr(C), x0)
    return C.reshape(6, 6)


def sym_to_full(c21):
    c21 = np.asarray(c21)
    out = np.zeros(c21.shape[:-1] + (6, 6))
    k = 0
    for i in range(6):
        for j in range(i, 6):
            out[..., i, j] = c21[..., k]
            out[..., j, i] = c21[..., k]
            k += 1
    return out


# ------------------------------------------------------------ batch entry points
def fit(det, prior_p, prior_C, hit_lists, n_hits, hx, hy, hz, hlayer, align=None,
        ms_after_last=False, want_each=False):
    """Kalman fit of tracks (inputs promoted to float64): prior_p [6][n], prior_C [21][n] (SoA), hit_lists
    [n][max_len] indices into hx/hy/hz/hlayer.  Returns (p [n][6], C [n][21],
    chi2 [n], status [n]) and per-hit chi2 if want_each."""
    prior_p = _c(prior_p, np.float64); prior_C = _c(prior_C, np.float64)
    n = prior_p.shape[1]
    hit_lists = _c(hit_lists, np.int32); n_hits = _c(n_hits, np.int32)
    max_len = hit_lists.shape[1]
    hx, hy, hz = _c(hx, np.float64), _c(hy, np.float64), _c(hz, np.float64)
    hlayer = _c(hlayer, np.int32)
    align = _c(np.zeros((det.n_layers, 2)) if align is None else align, np.float64)
    p = np.zeros((n, 6)); C = np.zeros((n, 21)); c2 = np.zeros(n); st = np.zeros(n, np.int32)
    each = np.zeros((n, max_len)) if want_each else None
    d = make_detector(det)
    lib().orc_fit(ctypes.byref(d), n, _ptr(prior_p), _ptr(prior_C), n, _ptr(hit_lists),
                  _ptr(n_hits), max_len, _ptr(hx), _ptr(hy), _ptr(hz), _ptr(hlayer), _ptr(align),
                  int(ms_after_last), _ptr(p), _ptr(C), _ptr(c2),
                  _ptr(each) if want_each else None, _ptr(st))
    if want_each:
        return p, C, c2, st, each
    return p, C, c2, st


def fit_grad(det, prior_p, prior_C, hit_lists, n_hits, hx, hy, hz, hlayer, align=None, fp32=False):
    """Summed fit chi2 and its gradient (forward-mode dual numbers).
    Returns (chi2_total, g_align [L][2], g_hits [n_hit_arrays][3], g_seed [n][6], chi2 [n]).
    fp32: the same computation with every operation rounded to single
    precision (the FP32 rounding scale of each result)."""
    prior_p = _c(prior_p, np.float64); prior_C = _c(prior_C, np.float64)
    n = prior_p.shape[1]
    hit_lists = _c(hit_lists, np.int32); n_hits = _c(n_hits, np.int32)
    hx, hy, hz = _c(hx, np.float64), _c(hy, np.float64), _c(hz, np.float64)
    hlayer = _c(hlayer, np.int32)
    align = _c(np.zeros((det.n_layers, 2)) if align is None else align, np.float64)
    tot = np.zeros(1); ga = np.zeros((det.n_layers, 2)); gh = np.zeros((hx.size, 3))
    gs = np.zeros((n, 6)); each = np.zeros(n)
    d = make_detector(det)
    fn = lib().orc_fit_grad32 if fp32 else lib().orc_fit_grad
    rc = fn(ctypes.byref(d), n, _ptr(prior_p), _ptr(prior_C), n, _ptr(hit_lists),
                            _ptr(n_hits), hit_lists.shape[1], _ptr(hx), _ptr(hy), _ptr(hz),
                            _ptr(hlayer), _ptr(align), _ptr(tot), _ptr(ga), _ptr(gh), _ptr(gs),
                            _ptr(each))
    if rc != 0:
        raise RuntimeError(f"orc_fit_grad failed: {rc}")
    return float(tot[0]), ga, gh, gs, each


def find_event(batch, e: int, max_cands=None, chi2_cut=30.0, max_holes=3, seeds=None, brute=False,
               align=None):
    """Combinatorial finding for event e of a synth.Batch (optionally a subset
    of its seeds, event-local indices [a, b)).  Returns a dict with hits
    [n][L] (event-local, -1 padded), n_found, chi2, p [n][6], C [n][21] and
    counters."""
    det = batch.det
    L = getattr(det, "n_surfaces", det.n_layers)  # barrel layers, then endcap disks
    x, y, z, lay = batch.event_hits(e)
    prm, cov, sh = batch.event_seeds(e)
    prm = _c(prm, np.float64); cov = _c(cov, np.float64); sh = _c(sh, np.int32)
    ns = prm.shape[1]
    a, b = (0, ns) if seeds is None else seeds
    n = b - a
    out_hits = np.full((n, L), -1, np.int32)
    out_n = np.zeros(n, np.int32)
    out_c2 = np.zeros(n)
    out_p = np.zeros((n, 6))
    out_C = np.zeros((n, 21))
    cnt = np.zeros(13, np.int64)
    mc = batch.cfg["max_cands"] if max_cands is None else max_cands
    d = make_detector(det)
    cfg = make_config(mc, max_holes, chi2_cut)
    al = _c(batch.align if align is None else align, np.float64)
    x, y, z, lay = _c(x, np.float64), _c(y, np.float64), _c(z, np.float64), _c(lay, np.int32)
    lib().orc_find_event(ctypes.byref(d), ctypes.byref(cfg), x.size, _ptr(x), _ptr(y), _ptr(z),
                         _ptr(lay), _ptr(prm), _ptr(cov), _ptr(sh), ns, a, b, _ptr(al), int(brute),
                         _ptr(out_hits), _ptr(out_n), _ptr(out_c2), _ptr(out_p), _ptr(out_C),
                         _ptr(cnt))
    return dict(hits=out_hits, n_found=out_n, chi2=out_c2, p=out_p, C=out_C,
                counters=dict(steps=int(cnt[0]), prop_calls=int(cnt[1]), updates=int(cnt[2]),
                              ms=int(cnt[3]), chi2_evals=int(cnt[4]), seeds=int(cnt[5]),
                              children=int(cnt[6]), holes=int(cnt[7]), window_hits=int(cnt[8]),
                              disk_steps=int(cnt[9]), disk_updates=int(cnt[10]), disk_holes=int(cnt[11]),
                              disk_window_hits=int(cnt[12])))


def dedup(hits, n_hits, chi2, frac=0.5, brute=False, params=None, bz=0.0, deta=0.0, dphi=0.0, dpt=0.0):
    """Greedy duplicate removal over one event's tracks; returns keep flags (uint8).
    With params ([n][6] track states) a pair must also pass the pT, eta and phi
    pre-cuts (deta, dphi, dpt; a cut <= 0 is off)."""
    hits = _c(hits, np.int32); n_hits = _c(n_hits, np.int32); chi2 = _c(chi2, np.float64)
    n = n_hits.size
    keep = np.zeros(n, np.uint8)
    pp = None if params is None else _c(np.asarray(params, np.float64).reshape(n, 6), np.float64)
    lib().orc_dedup(n, _ptr(hits), _ptr(n_hits), _ptr(chi2), hits.shape[1] if n else 1,
                    float(frac), int(brute), _ptr(keep), None if pp is None else _ptr(pp), float(bz),
                    float(deta), float(dphi), float(dpt))
    return keep


def kinematics(bz, params):
    """(eta, |q/pT|, phi0) of track states params [n][6]; phi0 is the direction
    of motion at the point of the helix closest to the z axis."""
    pp = _c(np.asarray(params, np.float64).reshape(-1, 6), np.float64)
    out = np.zeros((pp.shape[0], 3))
    lib().orc_kinematics(pp.shape[0], float(bz), _ptr(pp), _ptr(out))
    return out


def seed_clean(params, hits, bz, deta, dphi=0.0, dpt=0.0, min_shared=0):
    """Seed cleaning of one event's seeds (params [n][6], hits [n][3]): keep
    flags (uint8) of the greedy walk in seed order."""
    pp = _c(np.asarray(params, np.float64).reshape(-1, 6), np.float64)
    hh = _c(np.asarray(hits).reshape(-1, 3), np.int32)
    keep = np.zeros(pp.shape[0], np.uint8)
    lib().orc_seed_clean(pp.shape[0], _ptr(pp), _ptr(hh), float(bz), float(deta), float(dphi), float(dpt),
                         int(min_shared), _ptr(keep))
    return keep


def replay_path(batch, e: int, seed: int, hits_row, align=None):
    """Replay, in the oracle, the finding path that produced the hit list
    `hits_row` (event-local indices, -1 padded) for event-local seed `seed`.
    Returns (status, chi2 sum, n_found, per-layer chi2)."""
    det = batch.det
    L = det.n_layers
    x, y, z, lay = batch.event_hits(e)
    prm, cov, sh = batch.event_seeds(e)
    x, y, z = _c(x, np.float64), _c(y, np.float64), _c(z, np.float64)
    lay = _c(lay, np.int32)
    hits = [h for h in hits_row if h >= 0]
    dec = np.full(L, -2, np.int32)
    last = int(lay[hits[2]])
    for h in hits[3:]:
        last = max(last, int(lay[h]))
    for l in range(int(lay[hits[2]]) + 1, last + 1):
        dec[l] = -1
    for h in hits[3:]:
        dec[int(lay[h])] = h
    p0 = _c(prm[:, seed], np.float64)
    c0 = _c(cov[:, seed], np.float64)
    s3 = _c(sh[:, seed], np.int32)
    al = _c(batch.align if align is None else align, np.float64)
    chi2l = np.zeros(L)
    tot = np.zeros(1)
    nf = np.zeros(1, np.int32)
    d = make_detector(det)
    st = lib().orc_replay(ctypes.byref(d), _ptr(x), _ptr(y), _ptr(z), _ptr(lay), _ptr(p0), _ptr(c0),
                          _ptr(s3), _ptr(dec), _ptr(al), _ptr(chi2l), _ptr(tot), _ptr(nf), None, None)
    return int(st), float(tot[0]), int(nf[0]), chi2l


def replay_decisions(batch, e: int, seed: int, decisions, align=None):
    """Replay a finding path given per layer: a hit index (update), -1 (hole)
    or -2 (stop; the path ends).  Returns (status, chi2 sum, n_found,
    per-layer chi2, final p [6], final C [21])."""
    det = batch.det
    x, y, z, lay = batch.event_hits(e)
    prm, cov, sh = batch.event_seeds(e)
    x, y, z = _c(x, np.float64), _c(y, np.float64), _c(z, np.float64)
    lay = _c(lay, np.int32)
    dec = _c(decisions, np.int32)
    p0 = _c(prm[:, seed], np.float64)
    c0 = _c(cov[:, seed], np.float64)
    s3 = _c(sh[:, seed], np.int32)
    al = _c(batch.align if align is None else align, np.float64)
    chi2l = np.zeros(det.n_layers)
    tot = np.zeros(1)
    nf = np.zeros(1, np.int32)
    pf = np.zeros(6)
    cf = np.zeros(21)
    d = make_detector(det)
    st = lib().orc_replay(ctypes.byref(d), _ptr(x), _ptr(y), _ptr(z), _ptr(lay), _ptr(p0), _ptr(c0),
                          _ptr(s3), _ptr(dec), _ptr(al), _ptr(chi2l), _ptr(tot), _ptr(nf), _ptr(pf), _ptr(cf))
    return int(st), float(tot[0]), int(nf[0]), chi2l, pf, cf


def select_children(n_found, chi2, parent, kind, hit, max_cands):
    """The finding's selection step on hand-made children (kind 0 hit, 1 hole,
    2 carried): indices of the kept children in rank order."""
    n = len(n_found)
    nf = _c(n_found, np.int32); c2 = _c(chi2, np.float64); pa = _c(parent, np.int32)
    kd = _c(kind, np.int32); ht = _c(hit, np.int32)
    out = np.zeros(max(n, 1), np.int32)
    k = lib().orc_select_children(n, _ptr(nf), _ptr(c2), _ptr(pa), _ptr(kd), _ptr(ht), int(max_cands), _ptr(out))
    return out[:k].tolist()


# ------------------------------------------------------------ operation census
CENSUS_PARTS = ("propagate_transport", "frame_window", "hit_chi2", "update", "scatter")


def census_step(det, p, C21, layer, m1, m2, align=(0.0, 0.0), chi2_cut=30.0):
    """Operations of one finding step (orc_census_step): a [5][4] array, rows
    CENSUS_PARTS, columns (adds, multiplies, divides, special functions);
    None when the state does not cross the layer or a hit is on the far side."""
    out = np.zeros(20, np.int64)
    d = make_detector(det)
    rc = lib().orc_census_step(ctypes.byref(d), float(chi2_cut), _ptr(_c(p, np.float64)), _ptr(_c(C21, np.float64)),
                               int(layer), _ptr(_c(m1, np.float64)), _ptr(_c(m2, np.float64)),
                               _ptr(_c(align, np.float64)), _ptr(out))
    return None if rc != 0 else out.reshape(5, 4)


def census_disk_step(det, p, C21, surface, m1, m2, chi2_cut=30.0):
    """Operations of one finding step onto an endcap disk (orc_census_disk_step),
    as census_step: a [5][4] array, rows CENSUS_PARTS (the window row: the
    frame and the r window of the chi2 < cut ellipse); None without a crossing
    or with a hit on the far side."""
    out = np.zeros(20, np.int64)
    d = make_detector(det)
    rc = lib().orc_census_disk_step(ctypes.byref(d), float(chi2_cut), _ptr(_c(p, np.float64)),
                                    _ptr(_c(C21, np.float64)), int(surface), _ptr(_c(m1, np.float64)),
                                    _ptr(_c(m2, np.float64)), _ptr(out))
    return None if rc != 0 else out.reshape(5, 4)


def census_fit(det, p0, C21, raw, layers, align, ms_after_last=False):
    """Operations of a Kalman fit over the hits raw [n][3] on layers [n]
    (orc_census_fit): (adds, multiplies, divides, special functions), or None
    when the fit fails."""
    out = np.zeros(4, np.int64)
    raw = _c(raw, np.float64)
    d = make_detector(det)
    rc = lib().orc_census_fit(ctypes.byref(d), _ptr(_c(p0, np.float64)), _ptr(_c(C21, np.float64)), raw.shape[0],
                              _ptr(raw), _ptr(_c(layers, np.int32)), _ptr(_c(align, np.float64)),
                              int(ms_after_last), _ptr(out))
    return None if rc != 0 else out


def census_transport(J, C21):
    """Operations of one covariance transport (orc_census_transport): entries
    of J exactly 0 or 1 are constants.  (adds, multiplies, divides, special)."""
    out = np.zeros(4, np.int64)
    lib().orc_census_transport(_ptr(_c(np.asarray(J, np.float64).reshape(36), np.float64)), _ptr(_c(C21, np.float64)),
                               _ptr(out))
    return out
