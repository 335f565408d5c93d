"""Synthetic barrel-detector events (inputs only; see the package docstring).

Workloads follow the paper's setting (Sec. 3: Phase-I-like barrel, constant
3.8 T field; Sec. 4 and Sec. 5: simulated events at pileup 50 to 200) with the
shapes named per configuration in ``CONFIGS``:

* tracks from the origin (vertex smear 0.01 cm), pT uniform in 0.5-10 GeV,
  phi uniform, eta uniform in [-eta_max, eta_max], charge +-1;
* thin cylindrical layers at evenly spaced radii, |z| < 120 cm, 0.02 X0 each;
* one multiple-scattering kick per crossed layer (Highland width, independent
  Gaussian kicks in phi and theta, q/pT unchanged);
* hits smeared in r-phi (along the cylinder) and z; noise hits uniform in phi and z;
* seeds from the three true hits on layers 1-3, with a prior taken from the
  circle through the three points.

Random numbers come from numpy's Philox counter-based generator keyed by
(config seed, event index), so every machine draws the same events.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

#: Curvature constant: 1/rho [1/cm] = K_FIELD * B[T] / pT[GeV].
K_FIELD = 0.00299792458
#: Mass hypothesis used for the velocity in the scattering width (charged pion, GeV).
M_PION = 0.13957

#: Variances of the seed prior placed at the first seed hit, in the order
#: (x, y, z, q/pT, phi, theta).  The position is the first hit itself; the
#: direction and curvature widths are about two to three times the RMS error
#: of the three-hit circle estimate (q/pT 0.05 GeV^-1, phi 0.004 rad, theta
#: 0.007 rad in the 17-layer geometry), loose against the estimate while
#: keeping the information gain of each Kalman update within the range a
#: single-precision covariance resolves.
SEED_PRIOR_VAR = (1.0e-2, 1.0e-2, 1.0e-1, 1.0e-2, 1.0e-4, 4.0e-4)


@dataclasses.dataclass(frozen=True)
class Detector:
    radius: tuple
    z_max: float = 120.0
    x0: tuple = ()
    bz: float = 3.8
    sigma_rphi: float = 0.01
    sigma_z: float = 0.1
    # optional material map [n_layers][n_z]: thickness at z nodes spread evenly
    # over [-z_max, z_max] (the simulation itself uses x0)
    x0_map: object = None
    # optional mean ionization loss per layer at normal incidence for beta -> 1
    # (GeV); the simulation itself has none
    eloss: tuple = ()
    # axial field Bz(r, z) = bz (1 + field_cz z^2 + field_cr r^2) (cm^-2; 0, 0:
    # uniform); the simulation traces tracks through it in FIELD_SUBSTEPS
    # helix steps per layer, each in the field at its starting point
    field_cz: float = 0.0
    field_cr: float = 0.0
    # endcap disks (Sec. 2 and 3: barrel layers and endcap disks, the event
    # split into five eta regions): planes at z = +-disk_z[k] (|z| increasing)
    # covering disk_rmin <= r <= disk_rmax, each disk_x0 radiation lengths
    # thick (with disk_eloss mean ionization loss at normal incidence, GeV);
    # hits measured along r-phi (sigma_rphi) and r (sigma_r).  Surfaces are
    # numbered barrel layers 0..L-1, then the +z disks, then the -z disks.
    # Seeds with |eta| >= eta_barrel search the disks of their side after the
    # barrel layers.
    disk_z: tuple = ()
    disk_rmin: float = 15.0
    disk_rmax: float = 110.0
    disk_x0: float = 0.02
    disk_eloss: float = 0.0
    sigma_r: float = 0.1
    eta_barrel: float = 0.9

    @property
    def n_layers(self) -> int:
        return len(self.radius)

    @property
    def n_disks(self) -> int:
        return len(self.disk_z)

    @property
    def n_surfaces(self) -> int:
        return self.n_layers + 2 * self.n_disks


def detector_for(n_layers: int, r_min: float, r_max: float, bz: float = 3.8,
                 x0: float = 0.02, z_max: float = 120.0, field_cz: float = 0.0,
                 field_cr: float = 0.0) -> Detector:
    radius = tuple(r_min + (r_max - r_min) * i / (n_layers - 1) for i in range(n_layers))
    return Detector(radius=radius, z_max=z_max, x0=(x0,) * n_layers, bz=bz, field_cz=field_cz,
                    field_cr=field_cr)


#: helix steps per layer-to-layer crossing when the simulation traces tracks
#: through a field that varies
FIELD_SUBSTEPS = 8


def field_at(det: Detector, x, y, z):
    """Bz at (x, y, z) (T)."""
    return det.bz * (1.0 + det.field_cz * z * z + det.field_cr * (x * x + y * y))


# Workload configurations.  "tracks" may be an int or the string "pileup" for
# 50 tracks per unit of pileup drawn uniformly from pileup_range.
CONFIGS: Dict[str, dict] = {
    # 1 event, 100 tracks, 10 layers 4-100 cm, no noise, N = 6 candidates.
    "c0": dict(n_events=1, tracks=100, n_layers=10, r_max=100.0, eta_max=1.0,
               noise=0.0, max_cands=6, seed=1000),
    # PU-50-like: 2,500 tracks, 17 layers 4-110 cm, 10% noise, 64x1024 bins.
    "c1": dict(n_events=1, tracks=2500, n_layers=17, r_max=110.0, eta_max=1.5,
               noise=0.10, max_cands=6, seed=1001),
    # As c1 plus duplicate seeds for 10% of the tracks, built on layers 2-4.
    "c1b": dict(n_events=1, tracks=2500, n_layers=17, r_max=110.0, eta_max=1.5,
                noise=0.10, max_cands=6, dup_seed_frac=0.10, seed=1011),
    # 64 events of uneven pileup 20-200 (1,000-10,000 tracks each).
    "c2": dict(n_events=64, tracks="pileup", pileup_range=(20, 200), n_layers=17,
               r_max=110.0, eta_max=1.5, noise=0.10, max_cands=6, seed=1002),
    # Fit-only: 10,000 tracks, true hit assignment, layer misalignment 0.005 cm.
    "c3": dict(n_events=1, tracks=10000, n_layers=17, r_max=110.0, eta_max=1.5,
               noise=0.0, max_cands=6, misalign_sigma=0.005, seed=1003),
    # PU-200 HL-LHC-like batch: 100 events x 8,000 tracks, 20% noise, N = 10.
    "c4": dict(n_events=100, tracks=8000, n_layers=17, r_max=110.0, eta_max=1.5,
               noise=0.20, max_cands=10, seed=1004),
    # Barrel and endcaps: c1's barrel plus seven disks per side at |z| =
    # 130-250 cm (r 15-110 cm), tracks over |eta| < 2.4, so that about half of
    # the seeds lie in the forward eta regions.
    "c5": dict(n_events=1, tracks=2500, n_layers=17, r_max=110.0, eta_max=2.4,
               noise=0.10, max_cands=6, seed=1005,
               disk_z=(130.0, 150.0, 170.0, 190.0, 210.0, 230.0, 250.0)),
    # PU-200-like barrel plus endcaps: 20 events x 8,000 tracks over |eta| <
    # 2.4, 20% noise on every surface, N = 10 (the benchmark's endcap step).
    "c6": dict(n_events=20, tracks=8000, n_layers=17, r_max=110.0, eta_max=2.4,
               noise=0.20, max_cands=10, seed=1006,
               disk_z=(130.0, 150.0, 170.0, 190.0, 210.0, 230.0, 250.0)),
}


def _rng(seed: int, event: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, event]))


def _highland(kappa, theta, phi_dir, phi_pos, x0):
    """Highland scattering width for a thin layer of x0 radiation lengths."""
    sin_t = np.sin(theta)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = 1.0 / (np.abs(kappa) * sin_t)
        beta = p / np.sqrt(p * p + M_PION * M_PION)
        t = x0 / np.abs(sin_t * np.cos(phi_dir - phi_pos))
        th0 = 0.0136 / (beta * p) * np.sqrt(t) * (1.0 + 0.038 * np.log(t))
    return np.where(np.isfinite(th0), th0, 0.0)


def _cross_cylinder(x, y, z, kappa, phi, theta, R, bz):
    """Truth tracing: first crossing of the helix with the cylinder of radius R.

    The trajectory is a circle in the transverse plane with centre
    c = (x - sin(phi)/h, y + cos(phi)/h), h = -K_FIELD*bz*kappa (positive
    charges turn clockwise seen from +z when bz > 0), intersected with the
    circle of radius R about the origin.  Returns (ok, x, y, z, phi).
    """
    n = x.shape[0]
    h = -K_FIELD * bz * kappa
    cot = np.cos(theta) / np.sin(theta)
    ok = np.zeros(n, dtype=bool)
    s = np.full(n, np.nan)
    r02 = x * x + y * y
    straight = np.abs(h) < 1e-12
    # Straight line: |p + s t|^2 = R^2.
    if straight.any():
        b = x * np.cos(phi) + y * np.sin(phi)
        disc = b * b + R * R - r02
        root = -b + np.sqrt(np.maximum(disc, 0.0))
        good = straight & (disc >= 0) & (root > 0)
        s = np.where(good, root, s)
        ok |= good
    curved = ~straight
    if curved.any():
        with np.errstate(divide="ignore", invalid="ignore"):
            cx = x - np.sin(phi) / h
            cy = y + np.cos(phi) / h
            rho = 1.0 / np.abs(h)
            d = np.hypot(cx, cy)
            # d^2 - rho^2 without cancellation: |p|^2 + 2 (p . n)/h, n the left normal.
            pn = -x * np.sin(phi) + y * np.cos(phi)
            d2_m_rho2 = r02 + 2.0 * pn / h
            a = (R * R + d2_m_rho2) / (2.0 * d)
            hh2 = R * R - a * a
            hh = np.sqrt(np.maximum(hh2, 0.0))
            ex, ey = cx / d, cy / d
            best = np.full(n, np.inf)
            a0 = np.arctan2(y - cy, x - cx)
            sgn = np.sign(h)
            for side in (1.0, -1.0):
                px = a * ex - side * hh * ey
                py = a * ey + side * hh * ex
                ap = np.arctan2(py - cy, px - cx)
                turn = np.mod((ap - a0) * sgn, 2.0 * np.pi)
                turn = np.where(turn <= 1e-13, 2.0 * np.pi, turn)
                best = np.minimum(best, turn)
            good = curved & (hh2 >= 0) & np.isfinite(best)
            s = np.where(good, best * rho, s)
            ok |= good
    s = np.where(ok, s, 0.0)
    with np.errstate(invalid="ignore"):
        hs = h * s
        # Transverse displacement along the arc (exact for both branches).
        sin_term = np.where(straight, s, np.sin(hs) / np.where(straight, 1.0, h))
        cos_term = np.where(straight, 0.0, (1.0 - np.cos(hs)) / np.where(straight, 1.0, h))
    xn = x + np.cos(phi) * sin_term - np.sin(phi) * cos_term
    yn = y + np.sin(phi) * sin_term + np.cos(phi) * cos_term
    zn = z + s * cot
    phn = phi + hs
    return ok, xn, yn, zn, phn


def _cross_in_field(x, y, z, kappa, phi, theta, R, det: Detector):
    """Truth tracing to radius R: one helix in a uniform field; in a field
    that varies, FIELD_SUBSTEPS helices to radii spread evenly between the
    start and R, each in the field at its own starting point."""
    if det.field_cz == 0.0 and det.field_cr == 0.0:
        return _cross_cylinder(x, y, z, kappa, phi, theta, R, det.bz)
    r0 = np.hypot(x, y)
    ok = np.ones(x.shape[0], dtype=bool)
    for k in range(1, FIELD_SUBSTEPS + 1):
        Rk = R if k == FIELD_SUBSTEPS else r0 + (R - r0) * k / FIELD_SUBSTEPS
        okk, x, y, z, phi = _cross_cylinder(x, y, z, kappa, phi, theta, Rk, field_at(det, x, y, z))
        ok &= okk
    return ok, x, y, z, phi


def _cross_plane(x, y, z, kappa, phi, theta, zd, bz):
    """Truth tracing to the plane z = zd: the transverse arc s = (zd - z) tan
    theta (s > 0 and less than half a turn, |h s| < pi), then the helix there.
    Returns (ok, x, y, phi)."""
    cot = np.cos(theta) / np.sin(theta)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (zd - z) / cot
    ok = np.isfinite(s) & (s > 0)
    s = np.where(ok, s, 0.0)
    h = -K_FIELD * bz * kappa
    straight = np.abs(h) < 1e-12
    ok &= np.abs(h * s) < np.pi  # within half a turn (a looper would meet barrel layers again first)
    with np.errstate(invalid="ignore", divide="ignore"):
        hs = h * s
        sin_term = np.where(straight, s, np.sin(hs) / np.where(straight, 1.0, h))
        cos_term = np.where(straight, 0.0, (1.0 - np.cos(hs)) / np.where(straight, 1.0, h))
    xn = x + np.cos(phi) * sin_term - np.sin(phi) * cos_term
    yn = y + np.sin(phi) * sin_term + np.cos(phi) * cos_term
    return ok, xn, yn, phi + hs


def _cross_plane_in_field(x, y, z, kappa, phi, theta, zd, det: Detector):
    """Truth tracing to the plane z = zd: one helix in a uniform field; in a
    field that varies, FIELD_SUBSTEPS helices to planes spread evenly in z
    between the start and zd, each in the field at its own starting point,
    the whole arc within half a turn.  Returns (ok, x, y, phi)."""
    if det.field_cz == 0.0 and det.field_cr == 0.0:
        return _cross_plane(x, y, z, kappa, phi, theta, zd, det.bz)
    ok = np.ones(x.shape[0], dtype=bool)
    turn = np.zeros(x.shape[0])
    z0 = z.copy()
    for k in range(1, FIELD_SUBSTEPS + 1):
        zk = np.full_like(z0, zd) if k == FIELD_SUBSTEPS else z0 + (zd - z0) * k / FIELD_SUBSTEPS
        okk, xn, yn, phn = _cross_plane(x, y, z, kappa, phi, theta, zk, field_at(det, x, y, z))
        ok &= okk
        turn += np.where(okk, phn - phi, 0.0)
        x, y, z, phi = (np.where(okk, xn, x), np.where(okk, yn, y), np.where(okk, zk, z),
                        np.where(okk, phn, phi))
    ok &= np.abs(turn) < np.pi
    return ok, x, y, phi


def _highland_disk(kappa, theta, x0):
    """Highland width in a disk of x0 radiation lengths (path factor 1/|cos theta|)."""
    sin_t = np.sin(theta)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = 1.0 / (np.abs(kappa) * sin_t)
        beta = p / np.sqrt(p * p + M_PION * M_PION)
        t = x0 / np.abs(np.cos(theta))
        th0 = 0.0136 / (beta * p) * np.sqrt(t) * (1.0 + 0.038 * np.log(t))
    return np.where(np.isfinite(th0), th0, 0.0)


@dataclasses.dataclass
class Event:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    layer: np.ndarray
    sim: np.ndarray  # generating track index, -1 for noise
    track_hits: np.ndarray  # [n_tracks][n_surfaces] hit index or -1
    truth: np.ndarray  # [n_tracks][n_surfaces][6] state at each crossing, before the kick
    n_tracks: int


def simulate_event(det: Detector, n_tracks: int, eta_max: float, noise: float,
                   rng: np.random.Generator, misalign: Optional[np.ndarray] = None,
                   vertex_sigma: float = 0.01, pt_range=(0.5, 10.0)) -> Event:
    n = n_tracks
    L = det.n_layers
    vx, vy, vz = rng.normal(0.0, vertex_sigma, size=(3, n))
    pt = rng.uniform(pt_range[0], pt_range[1], size=n)
    phi = rng.uniform(-np.pi, np.pi, size=n)
    eta = rng.uniform(-eta_max, eta_max, size=n)
    q = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    theta = 2.0 * np.arctan(np.exp(-eta))
    kappa = q / pt

    x, y, z = vx.copy(), vy.copy(), vz.copy()
    ph, th = phi.copy(), theta.copy()
    alive = np.ones(n, dtype=bool)
    hx_l, hy_l, hz_l, sim_l, lay_l = [], [], [], [], []
    S = det.n_surfaces
    truth = np.full((n, S, 6), np.nan)
    local_index = np.full((n, S), -1, dtype=np.int64)  # index into this event's hit list (pre-shuffle)
    n_hits = 0
    for li in range(L):
        R = det.radius[li]
        ok, xn, yn, zn, phn = _cross_in_field(x, y, z, kappa, ph, th, R, det)
        ok &= alive & (np.abs(zn) <= det.z_max)
        alive = ok
        phi_pos = np.arctan2(yn, xn)
        d_rphi = rng.normal(0.0, det.sigma_rphi, size=n)
        d_z = rng.normal(0.0, det.sigma_z, size=n)
        kicks = rng.normal(size=(2, n))
        idx = np.nonzero(ok)[0]
        truth[idx, li, 0] = xn[idx]
        truth[idx, li, 1] = yn[idx]
        truth[idx, li, 2] = zn[idx]
        truth[idx, li, 3] = kappa[idx]
        truth[idx, li, 4] = phn[idx]
        truth[idx, li, 5] = th[idx]
        hphi = phi_pos + d_rphi / R
        hz = zn + d_z
        if misalign is not None:
            # The layer is displaced by (a_rphi, a_z): it reports hits rotated
            # by +a_rphi/R about z and shifted by +a_z.
            hphi = hphi + misalign[li, 0] / R
            hz = hz + misalign[li, 1]
        hx_l.append(R * np.cos(hphi[idx]))
        hy_l.append(R * np.sin(hphi[idx]))
        hz_l.append(hz[idx])
        sim_l.append(idx.astype(np.int32))
        lay_l.append(np.full(idx.size, li, dtype=np.int32))
        local_index[idx, li] = n_hits + np.arange(idx.size)
        n_hits += idx.size
        # Multiple scattering at the layer: q/pT kept, direction kicked.
        th0 = _highland(kappa, th, phn, phi_pos, det.x0[li])
        sin_t = np.sin(th)
        new_ph = phn + kicks[0] * th0 / sin_t
        new_th = th + kicks[1] * th0
        x = np.where(ok, xn, x)
        y = np.where(ok, yn, y)
        z = np.where(ok, zn, z)
        ph = np.where(ok, new_ph, ph)
        th = np.where(ok, new_th, th)
        # Noise hits for this layer.
        n_noise = int(round(noise * idx.size))
        if n_noise:
            nphi = rng.uniform(-np.pi, np.pi, size=n_noise)
            nz = rng.uniform(-det.z_max, det.z_max, size=n_noise)
            hx_l.append(R * np.cos(nphi))
            hy_l.append(R * np.sin(nphi))
            hz_l.append(nz)
            sim_l.append(np.full(n_noise, -1, dtype=np.int32))
            lay_l.append(np.full(n_noise, li, dtype=np.int32))
            n_hits += n_noise
    # Endcap disks on each track's side, from its last barrel crossing (a disk
    # whose plane the track does not reach, or reaches outside the disk's
    # radii, gives no hit and no scattering).
    side = np.sign(np.cos(th))
    for k in range(det.n_disks):
        for sgn, si in ((1.0, det.n_layers + k), (-1.0, det.n_layers + det.n_disks + k)):
            zd = sgn * det.disk_z[k]
            ok, xn, yn, phn = _cross_plane_in_field(x, y, z, kappa, ph, th, zd, det)
            rn = np.hypot(xn, yn)
            ok &= (side == sgn) & (rn >= det.disk_rmin) & (rn <= det.disk_rmax)
            idx = np.nonzero(ok)[0]
            phi_pos = np.arctan2(yn, xn)
            d_rphi = rng.normal(0.0, det.sigma_rphi, size=n)
            d_r = rng.normal(0.0, det.sigma_r, size=n)
            kicks = rng.normal(size=(2, n))
            truth[idx, si, 0] = xn[idx]
            truth[idx, si, 1] = yn[idx]
            truth[idx, si, 2] = zd
            truth[idx, si, 3] = kappa[idx]
            truth[idx, si, 4] = phn[idx]
            truth[idx, si, 5] = th[idx]
            hr = rn + d_r
            hphi = phi_pos + d_rphi / rn
            hx_l.append(hr[idx] * np.cos(hphi[idx]))
            hy_l.append(hr[idx] * np.sin(hphi[idx]))
            hz_l.append(np.full(idx.size, zd))
            sim_l.append(idx.astype(np.int32))
            lay_l.append(np.full(idx.size, si, dtype=np.int32))
            local_index[idx, si] = n_hits + np.arange(idx.size)
            n_hits += idx.size
            th0 = _highland_disk(kappa, th, det.disk_x0)
            sin_t = np.sin(th)
            x = np.where(ok, xn, x)
            y = np.where(ok, yn, y)
            z = np.where(ok, zd, z)
            ph = np.where(ok, phn + kicks[0] * th0 / sin_t, ph)
            th = np.where(ok, th + kicks[1] * th0, th)
            n_noise = int(round(noise * idx.size))
            if n_noise:
                nphi = rng.uniform(-np.pi, np.pi, size=n_noise)
                nr = np.sqrt(rng.uniform(det.disk_rmin ** 2, det.disk_rmax ** 2, size=n_noise))
                hx_l.append(nr * np.cos(nphi))
                hy_l.append(nr * np.sin(nphi))
                hz_l.append(np.full(n_noise, zd))
                sim_l.append(np.full(n_noise, -1, dtype=np.int32))
                lay_l.append(np.full(n_noise, si, dtype=np.int32))
                n_hits += n_noise
    hx = np.concatenate(hx_l)
    hy = np.concatenate(hy_l)
    hz = np.concatenate(hz_l)
    sim = np.concatenate(sim_l)
    lay = np.concatenate(lay_l)
    # Shuffle so that the hit index carries no truth information.
    perm = rng.permutation(n_hits)
    inv = np.empty(n_hits, dtype=np.int64)
    inv[perm] = np.arange(n_hits)
    track_hits = np.where(local_index >= 0, inv[np.maximum(local_index, 0)], -1).astype(np.int32)
    return Event(x=hx[perm].astype(np.float32), y=hy[perm].astype(np.float32),
                 z=hz[perm].astype(np.float32), layer=lay[perm].astype(np.int32),
                 sim=sim[perm], track_hits=track_hits, truth=truth, n_tracks=n)


def _upper_index():
    return [(i, j) for i in range(6) for j in range(i, 6)]


def seed_priors(hx, hy, hz, seed_hits, bz):
    """Prior state at the first seed hit from the circle through the three hits.

    Returns params [n][6] and the diagonal prior covariance [n][21] (upper
    triangle, row-major).  Inputs are the stored float32 hit coordinates.
    """
    h1, h2, h3 = seed_hits[:, 0], seed_hits[:, 1], seed_hits[:, 2]
    ax, ay, az = hx[h1].astype(np.float64), hy[h1].astype(np.float64), hz[h1].astype(np.float64)
    bx, by = hx[h2].astype(np.float64), hy[h2].astype(np.float64)
    cx, cy, cz = hx[h3].astype(np.float64), hy[h3].astype(np.float64), hz[h3].astype(np.float64)
    n = ax.size
    params = np.zeros((n, 6))
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    cross = (bx - ax) * (cy - by) - (by - ay) * (cx - bx)
    with np.errstate(divide="ignore", invalid="ignore"):
        a2, b2, c2 = ax * ax + ay * ay, bx * bx + by * by, cx * cx + cy * cy
        ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d
        uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d
        rho = np.hypot(ax - ux, ay - uy)
        sgn = np.where(cross >= 0, 1.0, -1.0)
        tx = -sgn * (ay - uy) / rho
        ty = sgn * (ax - ux) / rho
        v1x, v1y, v3x, v3y = ax - ux, ay - uy, cx - ux, cy - uy
        ang = np.arctan2(v1x * v3y - v1y * v3x, v1x * v3x + v1y * v3y) * sgn
        ang = np.mod(ang, 2.0 * np.pi)
        s13 = ang * rho
        curv = sgn / rho
    straight = ~np.isfinite(curv) | (np.abs(d) < 1e-12) | (bz == 0.0)
    # Straight-line fallback: direction from hit 1 to hit 3.
    lx, ly = cx - ax, cy - ay
    chord = np.hypot(lx, ly)
    phi = np.where(straight, np.arctan2(ly, lx), np.arctan2(ty, tx))
    s13 = np.where(straight, chord, s13)
    curv = np.where(straight, 0.0, curv)
    cot = (cz - az) / s13
    theta = np.arctan2(1.0, cot)
    kappa = np.zeros(n) if bz == 0.0 else -curv / (K_FIELD * bz)
    params[:, 0], params[:, 1], params[:, 2] = ax, ay, az
    params[:, 3], params[:, 4], params[:, 5] = kappa, phi, theta
    cov = np.zeros((n, 21))
    ui = _upper_index()
    for k, (i, j) in enumerate(ui):
        if i == j:
            cov[:, k] = SEED_PRIOR_VAR[i]
    return params, cov


@dataclasses.dataclass
class Batch:
    """A batch of events in the flat layout the C ABI takes.

    Hit and seed arrays are concatenated over events; ``hit_off`` and
    ``seed_off`` hold the CSR offsets.  ``seed_hits`` are event-local hit
    indices.  ``params``/``cov`` are structure-of-arrays ([6][n], [21][n]).
    """
    det: Detector
    cfg: dict
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    layer: np.ndarray
    hit_off: np.ndarray
    params: np.ndarray
    cov: np.ndarray
    seed_hits: np.ndarray
    seed_off: np.ndarray
    align: np.ndarray  # [n_layers][2] true misalignment (a_rphi, a_z)
    hit_sim: np.ndarray
    seed_sim: np.ndarray
    track_hits: List[np.ndarray]  # per event [n_tracks][n_layers]
    truth: List[np.ndarray]  # per event [n_tracks][n_layers][6]

    @property
    def n_events(self) -> int:
        return len(self.hit_off) - 1

    @property
    def n_hits(self) -> int:
        return int(self.hit_off[-1])

    @property
    def n_seeds(self) -> int:
        return int(self.seed_off[-1])

    def event_hits(self, e: int):
        a, b = self.hit_off[e], self.hit_off[e + 1]
        return self.x[a:b], self.y[a:b], self.z[a:b], self.layer[a:b]

    def event_seeds(self, e: int):
        a, b = self.seed_off[e], self.seed_off[e + 1]
        return self.params[:, a:b], self.cov[:, a:b], self.seed_hits[:, a:b]


def make_batch(name: str, n_events: Optional[int] = None, tracks: Optional[int] = None,
               bz: Optional[float] = None, **overrides) -> Batch:
    """Build the seeded batch for configuration ``name`` (see ``CONFIGS``).

    ``n_events`` and ``tracks`` shrink a configuration for tests; ``bz``
    replaces the field (0 gives straight tracks).
    """
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    if n_events is not None:
        cfg["n_events"] = n_events
    if tracks is not None:
        cfg["tracks"] = tracks
    det = detector_for(cfg["n_layers"], 4.0, cfg["r_max"], bz=3.8 if bz is None else bz,
                       field_cz=cfg.get("field_cz", 0.0), field_cr=cfg.get("field_cr", 0.0))
    disk_keys = ("disk_z", "disk_rmin", "disk_rmax", "disk_x0", "disk_eloss", "sigma_r", "eta_barrel")
    if any(k in cfg for k in disk_keys):
        det = dataclasses.replace(det, **{k: cfg[k] for k in disk_keys if k in cfg})
    L = det.n_layers
    align = np.zeros((L, 2), dtype=np.float32)
    if cfg.get("misalign_sigma"):
        ar = _rng(cfg["seed"], 1 << 20)
        align = ar.normal(0.0, cfg["misalign_sigma"], size=(L, 2)).astype(np.float32)
    xs, ys, zs, ls, sims = [], [], [], [], []
    hit_off = [0]
    prm, cov, sh, seed_off, ssim = [], [], [], [0], []
    thits, truths = [], []
    for e in range(cfg["n_events"]):
        rng = _rng(cfg["seed"], e)
        if cfg["tracks"] == "pileup":
            lo, hi = cfg["pileup_range"]
            n_trk = 50 * int(rng.integers(lo, hi + 1))
        else:
            n_trk = int(cfg["tracks"])
        ev = simulate_event(det, n_trk, cfg["eta_max"], cfg["noise"], rng,
                            misalign=align.astype(np.float64) if cfg.get("misalign_sigma") else None)
        th = ev.track_hits
        layers = [(0, 1, 2)]
        sel = [np.nonzero((th[:, 0] >= 0) & (th[:, 1] >= 0) & (th[:, 2] >= 0))[0]]
        if cfg.get("dup_seed_frac"):
            cand = np.nonzero((th[:, 1] >= 0) & (th[:, 2] >= 0) & (th[:, 3] >= 0))[0]
            k = int(round(cfg["dup_seed_frac"] * n_trk))
            pick = np.sort(rng.choice(cand, size=min(k, cand.size), replace=False))
            layers.append((1, 2, 3))
            sel.append(pick)
        s_hits, s_sim = [], []
        for lay3, trk in zip(layers, sel):
            s_hits.append(np.stack([th[trk, lay3[0]], th[trk, lay3[1]], th[trk, lay3[2]]], axis=1))
            s_sim.append(trk)
        s_hits = np.concatenate(s_hits).astype(np.int32)
        s_sim = np.concatenate(s_sim).astype(np.int32)
        p, c = seed_priors(ev.x, ev.y, ev.z, s_hits, det.bz)
        xs.append(ev.x); ys.append(ev.y); zs.append(ev.z); ls.append(ev.layer); sims.append(ev.sim)
        hit_off.append(hit_off[-1] + ev.x.size)
        prm.append(p); cov.append(c); sh.append(s_hits); ssim.append(s_sim)
        seed_off.append(seed_off[-1] + s_hits.shape[0])
        thits.append(th); truths.append(ev.truth)
    return Batch(
        det=det, cfg=cfg,
        x=np.concatenate(xs), y=np.concatenate(ys), z=np.concatenate(zs),
        layer=np.concatenate(ls).astype(np.int32), hit_off=np.asarray(hit_off, dtype=np.int32),
        params=np.ascontiguousarray(np.concatenate(prm).T.astype(np.float32)),
        cov=np.ascontiguousarray(np.concatenate(cov).T.astype(np.float32)),
        seed_hits=np.ascontiguousarray(np.concatenate(sh).T.astype(np.int32)),
        seed_off=np.asarray(seed_off, dtype=np.int32), align=align,
        hit_sim=np.concatenate(sims), seed_sim=np.concatenate(ssim),
        track_hits=thits, truth=truths,
    )


def true_hit_lists(batch: Batch, e: int, max_len: int):
    """Per generated track of event e: its hit indices in layer order, padded with -1."""
    th = batch.track_hits[e]
    out = np.full((th.shape[0], max_len), -1, dtype=np.int32)
    n = np.zeros(th.shape[0], dtype=np.int32)
    for t in range(th.shape[0]):
        hs = th[t][th[t] >= 0]
        out[t, :hs.size] = hs
        n[t] = hs.size
    return out, n
