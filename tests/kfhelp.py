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
    if any(getattr(d, "eloss", ()) or ()):
        raise ValueError("the CUDA path does not apply energy loss; this detector sets it")
    det = make_detector(d.radius, d.x0, d.z_max, d.bz, d.sigma_rphi, d.sigma_z)
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


RADIAL_TOL = 1e-3


def cov_close(gpu_c21, ref_c21, ref_p):
    """Covariance comparison in the local frame, where it is positive definite.

    After the first propagation the 6x6 covariance has rank 5: its radial
    direction is structurally null, so correlation-scaling the global x/y
    block divides FP32 rounding by near-zero variances.  The comparison uses
    the 5x5 local block, correlation-scaled (|dC_ij| <= TOL sqrt(C_ii C_jj)),
    and requires the radial variance of both to stay below RADIAL_TOL of the
    tangential one."""
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
    for c in (g, r):
        radv = np.abs(np.einsum("ni,nij,nj->n", rad, c, rad))
        ok &= radv <= RADIAL_TOL * tang
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
