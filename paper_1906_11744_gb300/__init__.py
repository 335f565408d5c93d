"""GB300 batched Kalman-filter track finding and fitting (arXiv:1906.11744).

The compute path is the CUDA library behind the C ABI of ``include/kf.h``;
this package only marshals arguments (``_lib``) and offers a small object
wrapper (``Tracker``).  PyTorch supplies device memory and streams.  There is
no CPU fallback: without the built library every call raises ``KFError``.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (
    KF_FIT_FOUND,
    KF_FIT_GIVEN,
    KF_FIT_OK,
    KF_FIT_SKIPPED,
    KF_MAX_DISKS,
    KFError,
    kf_autotune,
    kf_capture_graph,
    kf_config,
    kf_create,
    kf_destroy,
    kf_detector,
    kf_find_tracks,
    kf_fit_adjoint,
    kf_fit_tracks,
    kf_get_counters,
    kf_get_fit,
    kf_get_gradient,
    kf_get_stage_ms,
    kf_get_tracks,
    kf_graph_kernel_count,
    kf_last_error,
    kf_launch_graph,
    kf_load_hits,
    kf_load_seeds,
    kf_remove_duplicates,
    kf_set_alignment,
    kf_set_material,
    kf_set_stage_timing,
    kf_sync,
)


def make_detector(radius, x0, z_max=120.0, bz=3.8, sigma_rphi=0.01, sigma_z=0.1, eloss=None,
                  field_cz=0.0, field_cr=0.0, disk_z=(), disk_rmin=15.0, disk_rmax=110.0, disk_x0=0.02,
                  disk_eloss=0.0, sigma_r=0.1, eta_barrel=0.9) -> kf_detector:
    """Detector geometry (include/kf.h, kf_detector); eloss: mean ionization
    loss per layer at normal incidence for beta -> 1 (GeV; None: none);
    field_cz, field_cr: Bz(r, z) = bz (1 + field_cz z^2 + field_cr r^2);
    disk_z: |z| of the endcap disks of each side (empty: a barrel detector),
    with their radii, thickness, loss, radial resolution and the |eta| from
    which a seed searches them."""
    d = kf_detector()
    if len(disk_z) > KF_MAX_DISKS:
        raise ValueError(f"at most {KF_MAX_DISKS} disks per side")
    d.n_disks = len(disk_z)
    for i, z in enumerate(disk_z):
        d.disk_z[i] = float(z)
    d.disk_rmin, d.disk_rmax, d.disk_x0 = float(disk_rmin), float(disk_rmax), float(disk_x0)
    d.disk_eloss, d.sigma_r, d.eta_barrel = float(disk_eloss), float(sigma_r), float(eta_barrel)
    d.n_layers = len(radius)
    for i, r in enumerate(radius):
        d.radius[i] = float(r)
        d.x0[i] = float(x0[i])
        d.eloss[i] = float(eloss[i]) if eloss is not None and len(eloss) else 0.0
    d.z_max, d.bz, d.sigma_rphi, d.sigma_z = float(z_max), float(bz), float(sigma_rphi), float(sigma_z)
    d.field_cz, d.field_cr = float(field_cz), float(field_cr)
    return d


def make_config(max_cands=6, max_holes=3, chi2_cut=30.0, dup_shared_frac=0.5, n_eta_bins=64,
                n_phi_bins=1024, lanes_per_seed=0, block_threads=0, persistent=1, per_event=0,
                ckpt_stride=1, find_regcap=0, dup_deta=0.0, dup_dphi=0.0, dup_dpt=0.0, seed_clean=0,
                seed_deta=0.05, seed_dphi=0.05, seed_dpt=0.0, seed_min_shared=1,
                resolve_max_rounds=0) -> kf_config:
    """Algorithm settings (include/kf.h, kf_config).  The kinematic cuts of
    duplicate removal are off by default; seed cleaning is off unless
    seed_clean=1, and then drops a seed within 0.05 in eta and phi0 of a kept
    lower-index seed that shares a hit with it."""
    return kf_config(max_cands, max_holes, chi2_cut, dup_shared_frac, n_eta_bins, n_phi_bins,
                     lanes_per_seed, block_threads, persistent, per_event, ckpt_stride, find_regcap,
                     dup_deta, dup_dphi, dup_dpt, seed_clean, seed_deta, seed_dphi, seed_dpt,
                     seed_min_shared, resolve_max_rounds)


class Tracker:
    """One library context: load events, find, remove duplicates, fit."""

    def __init__(self, det: kf_detector, cfg: kf_config):
        self.det = det
        self.cfg = cfg
        self.ctx = kf_create(det, cfg)
        self.n_seeds = 0
        self.n_hits = 0

    def close(self):
        if self.ctx is not None:
            kf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_layers(self):
        return self.det.n_layers

    @property
    def n_surfaces(self):
        """Barrel layers plus the endcap disks of both sides (a found track's hit-list row)."""
        return self.det.n_layers + 2 * self.det.n_disks

    def load_hits(self, ev_offsets, x, y, z, layer, stream=None):
        kf_load_hits(self.ctx, ev_offsets, x, y, z, layer, stream)
        self.n_hits = int(np.asarray(ev_offsets)[-1])

    def load_seeds(self, ev_offsets, params, cov, seed_hits, stream=None):
        kf_load_seeds(self.ctx, ev_offsets, params, cov, seed_hits, stream)
        self.n_seeds = int(np.asarray(ev_offsets)[-1])

    def set_alignment(self, offsets, stream=None):
        kf_set_alignment(self.ctx, offsets, stream)

    def set_material(self, x0_map=None, stream=None):
        """Thickness per layer at z nodes [n_layers][n_z] (None: per-layer x0)."""
        kf_set_material(self.ctx, x0_map, stream)

    def find_tracks(self, stream=None):
        kf_find_tracks(self.ctx, stream)

    def remove_duplicates(self, stream=None):
        kf_remove_duplicates(self.ctx, stream)

    def fit_tracks(self, source=KF_FIT_FOUND, hit_lists=None, n_hits=None, stream=None):
        kf_fit_tracks(self.ctx, source, hit_lists, n_hits, stream)

    def fit_adjoint(self, g_align, g_hits=None, g_seed=None, stream=None):
        kf_fit_adjoint(self.ctx, g_align, g_hits, g_seed, stream)

    def get_tracks(self, device=None, stream=None):
        """Found tracks as numpy arrays (device=None) or torch tensors on `device`."""
        n, L = self.n_seeds, self.n_surfaces
        out = self._alloc(device, hits=((n, L), "i4"), n_found=((n,), "i4"), chi2=((n,), "f4"),
                          params=((6, n), "f4"), cov=((21, n), "f4"), keep=((n,), "u1"))
        kf_get_tracks(self.ctx, **out, stream=stream)
        return out

    def get_fit(self, device=None, stream=None):
        n = self.n_seeds
        out = self._alloc(device, params=((6, n), "f4"), cov=((21, n), "f4"), chi2=((n,), "f4"),
                          status=((n,), "i4"))
        kf_get_fit(self.ctx, **out, stream=stream)
        return out

    def capture_graph(self, with_adjoint=False, stream=None):
        kf_capture_graph(self.ctx, int(with_adjoint), stream)

    def launch_graph(self, stream=None):
        kf_launch_graph(self.ctx, stream)

    def autotune(self, stream=None):
        return kf_autotune(self.ctx, stream)

    def counters(self, stream=None):
        return kf_get_counters(self.ctx, stream)

    def sync(self, stream=None):
        kf_sync(self.ctx, stream)

    def set_stage_timing(self, enable=True):
        kf_set_stage_timing(self.ctx, enable)

    def stage_ms(self, stream=None):
        return kf_get_stage_ms(self.ctx, stream)

    def graph_kernel_count(self):
        return kf_graph_kernel_count(self.ctx)

    @staticmethod
    def _alloc(device, **specs):
        out = {}
        for name, (shape, dt) in specs.items():
            if device is None:
                out[name] = np.zeros(shape, dtype=np.dtype(dt))
            else:
                import torch
                tdt = {"i4": torch.int32, "f4": torch.float32, "u1": torch.uint8}[dt]
                out[name] = torch.zeros(shape, dtype=tdt, device=device)
        return out
