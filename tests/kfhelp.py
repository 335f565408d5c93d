"""Shared helpers of the GPU parity tests (test code only)."""
import numpy as np

# Parameter tolerance |dp_i| <= TOL * max(|p_i|, SCALE_i) (1e-4 relative in FP32);
# covariance |dC_ij| <= TOL * sqrt(C_ii C_jj) (correlation-scaled).
TOL = 1e-4
SCALE = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
# Near-tie bounds for found hit lists, derived from FP32 rounding of
# positions near 100 cm (ulp 7.6e-6 cm against 0.01 cm resolution): a chi2
# term carries about 1e-3 relative error, a 15-hit chi2 sum about 5e-4.
TIE_REL = 2e-3
CUT_ABS = 0.1


def tracker_for(batch, device=None, **cfg):
    import torch

    from paper_1906_11744_gb300 import Tracker, make_config, make_detector

    d = batch.det
    disks = dict(disk_z=tuple(d.disk_z), disk_rmin=d.disk_rmin, disk_rmax=d.disk_rmax, disk_x0=d.disk_x0,
                 disk_eloss=d.disk_eloss, sigma_r=d.sigma_r, eta_barrel=d.eta_barrel) if getattr(d, "disk_z", ()) else {}
    det = make_detector(d.radius, d.x0, d.z_max, d.bz, d.sigma_rphi, d.sigma_z, eloss=getattr(d, "eloss", None),
                        field_cz=getattr(d, "field_cz", 0.0), field_cr=getattr(d, "field_cr", 0.0), **disks)
    c = dict(max_cands=batch.cfg["max_cands"])
    c.update(cfg)
    t = Tracker(det, make_config(**c))
    if device is None:
        t.load_hits(batch.hit_off, batch.x, batch.y, batch.z, batch.layer)
        t.load_seeds(batch.seed_off, batch.params, batch.cov, batch.seed_hits)
    else:
        tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
        t.load_hits(batch.hit_off, tt(batch.x), tt(batch.y), tt(batch.z), tt(batch.layer))
        t.load_seeds(batch.seed_off, tt(batch.params), tt(batch.cov), tt(batch.seed_hits))
    t.set_alignment(batch.align)
    if getattr(d, "x0_map", None) is not None:
        t.set_material(np.asarray(d.x0_map, np.float32))
    return t


def param_close(gpu_p, ref_p):
    """gpu_p, ref_p [n][6]; returns (ok mask, max scaled error)."""
    scale = np.maximum(np.abs(ref_p), SCALE)
    err = np.abs(gpu_p - ref_p) / scale
    return np.all(err <= TOL, axis=1), float(err.max()) if err.size else 0.0


def local_frame(ref_p):
    """[n][6][5] map from the local parameters (r-phi along the tangent of
    the cylinder, z, q/pT, phi, theta) to the global state, at each state's
    position; plus the radial unit vectors [n][6]."""
    phi = np.arctan2(ref_p[:, 1], ref_p[:, 0])
    n = ref_p.shape[0]
    B = np.zeros((n, 6, 5))
    B[:, 0, 0], B[:, 1, 0] = -np.sin(phi), np.cos(phi)
    B[:, 2, 1] = B[:, 3, 2] = B[:, 4, 3] = B[:, 5, 4] = 1.0
    rad = np.zeros((n, 6))
    rad[:, 0], rad[:, 1] = np.cos(phi), np.sin(phi)
    return B, rad




def cov_close(gpu_c21, ref_c21, ref_p):
    """Covariance comparison in the local frame, where it is positive definite.

    After the first propagation the 6x6 covariance has rank 5: its radial
    direction is structurally null, so correlation-scaling the global x/y
    block divides FP32 rounding by near-zero variances.  The comparison uses
    the 5x5 local block, correlation-scaled (|dC_ij| <= TOL sqrt(C_ii C_jj)),
    and the radial variance (zero on the cylinder, but for the update's
    tangential step, which both sides share) within TOL of the oracle's
    tangential variance."""
    import oracle
    g = oracle.sym_to_full(gpu_c21)
    r = oracle.sym_to_full(ref_c21)
    B, rad = local_frame(ref_p)
    gl = np.einsum("nia,nij,njb->nab", B, g, B)
    rl = np.einsum("nia,nij,njb->nab", B, r, B)
    d = np.sqrt(np.abs(np.einsum("nii->ni", rl)))
    norm = d[:, :, None] * d[:, None, :]
    err = np.abs(gl - rl) / np.maximum(norm, 1e-30)
    ok = np.all(err <= TOL, axis=(1, 2))
    tang = rl[:, 0, 0]
    radg = np.einsum("ni,nij,nj->n", rad, g, rad)
    radr = np.einsum("ni,nij,nj->n", rad, r, rad)
    ok &= np.abs(radg - radr) <= TOL * tang
    return ok, float(err.max()) if err.size else 0.0


def audit_mismatch(batch, e, s_local, gpu_row, ref_row):
    """Classify a hit-list mismatch by replaying both paths in the oracle.

    Returns (explained, kind, rel) where kind is 'tie' (equal hit counts,
    chi2 sums within TIE_REL), 'cut' (a hit chi2 within CUT_ABS of the cut) or
    'unexplained'; rel is the relative chi2-sum difference."""
    import oracle
    sg, cg, ng, lg = oracle.replay_path(batch, e, s_local, gpu_row)
    so, co, no, lo = oracle.replay_path(batch, e, s_local, ref_row)
    rel = abs(cg - co) / max(abs(co), 1.0)
    cut = 30.0
    near_cut = np.any(np.abs(lg[lg > 0] - cut) < CUT_ABS) or np.any(np.abs(lo[lo > 0] - cut) < CUT_ABS)
    if sg == 0 and ng == no and rel <= TIE_REL:
        return True, "tie", rel
    if near_cut:
        return True, "cut", rel
    return False, "unexplained", rel


def oracle_find_events(batch, events, chunk=250, **kw):
    """The oracle's finding on whole events, seed chunks spread over the host
    cores (the C++ calls release the interpreter lock).  Returns {event: dict
    of hits, n_found, chi2, p, C} and the summed counters."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    jobs = []
    for e in events:
        ns = int(batch.seed_off[e + 1] - batch.seed_off[e])
        jobs += [(e, lo, min(lo + chunk, ns)) for lo in range(0, ns, chunk)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(lambda j: (j, oracle.find_event(batch, j[0], seeds=(j[1], j[2]), **kw)), jobs))
    out, counters = {}, {}
    for (e, lo, hi), r in res:
        d = out.setdefault(e, {k: [] for k in ("hits", "n_found", "chi2", "p", "C")})
        for k in d:
            d[k].append((lo, r[k]))
        for k, v in r["counters"].items():
            counters[k] = counters.get(k, 0) + v
    for e, d in out.items():
        for k in d:
            d[k] = np.concatenate([v for _, v in sorted(d[k], key=lambda t: t[0])])
    return out, counters


class _EventView:
    """One event of a batch with its hit coordinates replaced (for replays)."""

    def __init__(self, batch, e, x, y, z):
        self.det, self.align = batch.det, batch.align
        self._hits = (x, y, z, batch.event_hits(e)[3])
        self._seeds = batch.event_seeds(e)

    def event_hits(self, e):
        return self._hits

    def event_seeds(self, e):
        return self._seeds


# One FP32 ulp of relative jitter on the hit coordinates: the resolution at
# which the single-precision path sees the inputs.
JITTER_REL = 2.0 ** -23


def jitter_audit(batch, e, s_local, gpu_row, ref_row, trials=8, seed=0, cut=30.0):
    """Whether a hit-list mismatch is a tie at FP32 resolution.

    Both paths are replayed in FP64 on copies of the event whose hit
    coordinates are jittered by up to one FP32 ulp (relative 2^-23, uniform).
    A chi2-sum tie is resolved within FP32 resolution when the difference of
    the two sums changes sign under jitter or stays within 3 standard
    deviations of its jitter spread; a hit at the cut likewise when its chi2
    crosses the cut or stays within 3 standard deviations of it.  Returns
    (ok, nominal relative difference, spread relative to the sum)."""
    import oracle
    x, y, z, _ = batch.event_hits(e)
    rng = np.random.default_rng(seed)
    sg, cg, ng, lg = oracle.replay_path(batch, e, s_local, gpu_row)
    so, co, no, lo = oracle.replay_path(batch, e, s_local, ref_row)
    d0 = cg - co
    near = [np.nonzero((np.abs(lg - cut) < CUT_ABS) & (lg > 0))[0], np.nonzero((np.abs(lo - cut) < CUT_ABS) & (lo > 0))[0]]
    ds, cuts = [], []
    for _ in range(trials):
        jx, jy, jz = (a.astype(np.float64) * (1.0 + JITTER_REL * rng.uniform(-1, 1, a.size)) for a in (x, y, z))
        v = _EventView(batch, e, jx, jy, jz)
        a = oracle.replay_path(v, 0, s_local, gpu_row)
        b = oracle.replay_path(v, 0, s_local, ref_row)
        ds.append(a[1] - b[1])
        cuts.append(np.concatenate([a[3][near[0]], b[3][near[1]]]))
    ds = np.array(ds)
    scale = max(abs(co), 1.0)
    spread = float(ds.std())
    tie_ok = ng == no and (ds.min() <= 0.0 <= ds.max() or abs(d0) <= 3.0 * spread)
    cut_ok = False
    if near[0].size or near[1].size:
        c = np.array(cuts)  # trials x near hits
        nominal = np.concatenate([lg[near[0]], lo[near[1]]])
        for k in range(c.shape[1]):
            if (c[:, k].min() < cut <= c[:, k].max()) or abs(nominal[k] - cut) <= 3.0 * c[:, k].std():
                cut_ok = True
    return tie_ok or cut_ok, abs(d0) / scale, spread / scale


def crossing_cos(ref_p):
    """|cos| of the angle between the direction of motion and the radial
    direction at each state's position (1 = radial, 0 = tangent)."""
    r = np.hypot(ref_p[:, 0], ref_p[:, 1])
    return np.abs(ref_p[:, 0] * np.cos(ref_p[:, 4]) + ref_p[:, 1] * np.sin(ref_p[:, 4])) / np.maximum(r, 1e-30)


def found_cov_close(gpu_c21, ref_c21, ref_p):
    """Covariance of found-track states: the local-frame comparison of
    cov_close at 1e-4 where the last crossing has cos(alpha) >= 0.5, scaled by
    (0.5 / cos alpha)^4 below it.  The finder runs crossings down to
    cos(alpha) = 0.2 in FP32 (the re-fit only down to 0.5), and the FP32 error
    of the transported covariance grows as 1/cos^4 of that angle; the radial
    variance is compared with the oracle's at the same bound, relative to the
    tangential variance.  Returns (ok mask, (largest error over its
    bound, largest radial ratio over its bound))."""
    import oracle
    g = oracle.sym_to_full(gpu_c21)
    r = oracle.sym_to_full(ref_c21)
    B, rad = local_frame(ref_p)
    gl = np.einsum("nia,nij,njb->nab", B, g, B)
    rl = np.einsum("nia,nij,njb->nab", B, r, B)
    d = np.sqrt(np.abs(np.einsum("nii->ni", rl)))
    err = (np.abs(gl - rl) / np.maximum(d[:, :, None] * d[:, None, :], 1e-30)).reshape(len(rl), -1).max(1)
    amp = np.maximum(1.0, (0.5 / np.maximum(crossing_cos(ref_p), 1e-3)) ** 4)
    tol = TOL * amp
    ok = err <= tol
    tang = rl[:, 0, 0]
    radg = np.einsum("ni,nij,nj->n", rad, g, rad)
    radr = np.einsum("ni,nij,nj->n", rad, r, rad)
    rad_ratio = np.abs(radg - radr) / (tol * np.maximum(tang, 1e-300))
    ok &= rad_ratio <= 1.0
    if not err.size:
        return ok, (0.0, 0.0)
    return ok, (float((err / tol).max()), float(rad_ratio.max()))
