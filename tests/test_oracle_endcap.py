"""Pins of the oracle's endcap disks and eta regions (Sec. 2: the event is
split into five eta regions, barrel, transition and endcap on each side, each
searched over its own layers; Sec. 3: the geometry has barrel layers and
endcap disks).

Reading pinned here: a disk is the plane z = +-z_k between radii r_min and
r_max; a propagation to it is the helix over the transverse arc
s = (z_k - z) tan(theta) > 0, with the exact Jacobian (its z row vanishes); a
disk hit is measured along r-phi and r; scattering and energy loss use the
path factor 1/|cos(theta)|.  A seed with |eta| >= eta_barrel (the transition
and endcap regions) searches the barrel layers after its seed and then the
disks of its side; a candidate that does not cross a surface within its
bounds passes it (carried, still searching, no hole).  Barrel-region seeds
search the barrel layers only.  The pins: Runge-Kutta integration of the
Lorentz force to the plane, the straight line at B = 0, the Jacobian against
central differences and forward-mode differentiation, a disk update against
the normal equations of least squares, the disk path factor of scattering and
energy loss, unit-width pulls on disks, the dual fit gradient with disk hits,
and the finding on a barrel-plus-endcap event.
"""
import math

import numpy as np
import pytest

import oracle
from synth import make_batch
from synth.events import true_hit_lists

C_LIGHT = 0.00299792458
BZ = 3.8


def _forward_states(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ang = rng.uniform(-np.pi, np.pi)
        r0 = rng.uniform(5.0, 40.0)
        eta = rng.choice([-1, 1]) * rng.uniform(1.0, 2.4)
        out.append(np.array([r0 * math.cos(ang), r0 * math.sin(ang), rng.uniform(-20, 20),
                             rng.uniform(-1.5, 1.5), rng.uniform(-np.pi, np.pi), 2 * math.atan(math.exp(-eta))]))
    return out


def _rk4_to_plane(p, zd, bz, step=0.02):
    """Lorentz force in 3D path length until z reaches zd (bisection on the
    last step); returns (x, y, z, phi of the direction)."""
    x, y, z, kap, phi, th = [float(v) for v in p]
    a = C_LIGHT * kap * math.sin(th)

    def deriv(s):
        return np.array([s[3], s[4], s[5], a * s[4] * bz, -a * s[3] * bz, 0.0])

    def rk4(s, h):
        k1 = deriv(s)
        k2 = deriv(s + 0.5 * h * k1)
        k3 = deriv(s + 0.5 * h * k2)
        k4 = deriv(s + h * k3)
        return s + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)

    s = np.array([x, y, z, math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)])
    sgn = 1.0 if zd > z else -1.0
    for _ in range(400000):
        nxt = rk4(s, step)
        if sgn * (nxt[2] - zd) >= 0:
            lo, hi = 0.0, step
            for _ in range(70):
                mid = 0.5 * (lo + hi)
                if sgn * (rk4(s, mid)[2] - zd) >= 0:
                    hi = mid
                else:
                    lo = mid
            e = rk4(s, hi)
            return e[0], e[1], e[2], math.atan2(e[4], e[3])
        s = nxt
    raise AssertionError("no crossing")


def test_plane_propagation_matches_lorentz_force():
    for p in _forward_states(6, 31):
        zd = 140.0 if p[5] < math.pi / 2 else -140.0
        ok, q, _ = oracle.propagate_plane(BZ, p, zd)
        assert ok
        x, y, z, ph = _rk4_to_plane(p, zd, BZ)
        assert abs(q[0] - x) < 1e-8 and abs(q[1] - y) < 1e-8 and abs(q[2] - zd) < 1e-12
        assert abs((q[4] - ph + math.pi) % (2 * math.pi) - math.pi) < 1e-9
        assert q[3] == p[3] and q[5] == p[5]
        # moving away from the plane: no crossing
        assert not oracle.propagate_plane(BZ, p, -zd)[0]


def test_plane_straight_line_at_zero_field():
    for p in _forward_states(10, 32):
        zd = 150.0 if p[5] < math.pi / 2 else -150.0
        ok, q, _ = oracle.propagate_plane(0.0, p, zd)
        s = (zd - p[2]) * math.tan(p[5])
        assert ok and abs(q[0] - (p[0] + s * math.cos(p[4]))) < 1e-10 and abs(q[1] - (p[1] + s * math.sin(p[4]))) < 1e-10
        assert q[4] == p[4]


@pytest.mark.parametrize("bz,cz,cr", [(3.8, 0.0, 0.0), (0.0, 0.0, 0.0), (3.8, -3e-5, -2e-5)])
def test_plane_jacobian_against_finite_differences_and_ad(bz, cz, cr):
    scale = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
    for p in _forward_states(8, 33):
        zd = 160.0 if p[5] < math.pi / 2 else -160.0
        ok, q, J = oracle.propagate_plane(bz, p, zd, cz, cr)
        assert ok
        b0 = bz * (1 + cz * p[2] ** 2 + cr * (p[0] ** 2 + p[1] ** 2))
        Jfix, Jfull = np.zeros((6, 6)), np.zeros((6, 6))
        for j in range(6):
            h = 1e-6 * scale[j]
            pp, pm = p.copy(), p.copy()
            pp[j] += h
            pm[j] -= h
            Jfix[:, j] = (oracle.propagate_plane(b0, pp, zd)[1] - oracle.propagate_plane(b0, pm, zd)[1]) / (2 * h)
            Jfull[:, j] = (oracle.propagate_plane(bz, pp, zd, cz, cr)[1] - oracle.propagate_plane(bz, pm, zd, cz, cr)[1]) / (2 * h)
        assert np.all(np.abs(Jfix - J) <= 1e-6 * np.maximum(1.0, np.abs(J)))
        ok, Jad = oracle.propagate_plane_ad(bz, p, zd, cz, cr)
        assert ok and np.all(np.abs(Jfull - Jad) <= 1e-6 * np.maximum(1.0, np.abs(Jad)))
        assert np.allclose(J[2], 0.0, atol=1e-12)  # the state stays on the plane
        assert np.array_equal(J[3], np.eye(6)[3]) and np.array_equal(J[5], np.eye(6)[5])


def test_disk_update_equals_normal_equations():
    """One update on a disk == the weighted least-squares posterior with
    H = ((-sin phi_p, cos phi_p, 0...), (cos phi_p, sin phi_p, 0...))."""
    rng = np.random.default_rng(34)
    for _ in range(20):
        A = rng.normal(size=(6, 6))
        C = A @ A.T * 1e-3 + np.eye(6) * 1e-4
        ang = rng.uniform(-np.pi, np.pi)
        r = rng.uniform(15, 110)
        p = np.array([r * math.cos(ang), r * math.sin(ang), 150.0, 0.3, ang + 0.1, 0.4])
        m = np.array([(r + 0.05) * math.cos(ang + 0.001), (r + 0.05) * math.sin(ang + 0.001), 150.0])
        vr, vrr = 1e-4, 1e-2
        ok, po, Co, chi2, res = oracle.update_disk(p, C, m, vr, vrr)
        assert ok
        H = np.zeros((2, 6))
        H[0, 0], H[0, 1] = -math.sin(ang), math.cos(ang)
        H[1, 0], H[1, 1] = math.cos(ang), math.sin(ang)
        d = m[:2] - p[:2]
        assert np.allclose(res, H[:, :2] @ d, rtol=1e-12, atol=1e-14)
        V = np.diag([vr, vrr])
        P = np.linalg.inv(np.linalg.inv(C) + H.T @ np.linalg.inv(V) @ H)
        mean = p + P @ H.T @ np.linalg.inv(V) @ res
        assert np.allclose(Co, P, rtol=1e-8, atol=1e-14)
        assert np.allclose(po, mean, rtol=1e-10, atol=1e-12)
        S = H @ C @ H.T + V
        assert abs(chi2 - res @ np.linalg.solve(S, res)) < 1e-9 * max(1, chi2)


def test_disk_path_factor_of_scattering_and_energy_loss():
    """On a disk the material is crossed along z: Highland width at
    t = x0/|cos(theta)|, energy loss e/|cos(theta)|/beta^2 (first order
    dp = dE/beta), and the loss's Jacobian against central differences."""
    p = np.array([30.0, 5.0, 150.0, 1.0, 0.4, 0.5])  # pT 1 GeV, theta 0.5
    pm = 1.0 / math.sin(0.5)
    beta = pm / math.sqrt(pm * pm + 0.13957 ** 2)
    t = 0.02 / abs(math.cos(0.5))
    expected = 0.0136 / (beta * pm) * math.sqrt(t) * (1 + 0.038 * math.log(t))
    assert abs(oracle.highland_disk(p, 0.02) - expected) < 1e-15
    # the width does not depend on the position or on phi
    p2 = p.copy()
    p2[0], p2[4] = -10.0, 2.0
    assert oracle.highland_disk(p2, 0.02) == oracle.highland_disk(p, 0.02)
    e = 1e-3
    C = np.eye(6) * 1e-4
    q, _ = oracle.eloss_disk(p, C, e)
    dE = e / abs(math.cos(0.5)) / beta ** 2
    p_new = 1.0 / (abs(q[3]) * math.sin(0.5))
    assert abs((pm - p_new) - dE / beta) < 2e-3 * dE
    h = 1e-6
    F = np.eye(6)
    for j in range(6):
        pp, pq = p.copy(), p.copy()
        pp[j] += h * (0.1 if j == 3 else 1.0)
        pq[j] -= h * (0.1 if j == 3 else 1.0)
        F[3, j] = (oracle.eloss_disk(pp, C, e)[0][3] - oracle.eloss_disk(pq, C, e)[0][3]) / (2 * h * (0.1 if j == 3 else 1.0))
    _, C1 = oracle.eloss_disk(p, C, e)
    assert np.allclose(C1, F @ C @ F.T, rtol=1e-6, atol=1e-12)
    assert abs(F[3, 0]) < 1e-9 and abs(F[3, 1]) < 1e-9 and abs(F[3, 4]) < 1e-9


def _fit_true_forward(b):
    S = b.det.n_surfaces
    x, y, z, lay = b.event_hits(0)
    prm, cov, _ = b.event_seeds(0)
    lists, n = true_hit_lists(b, 0, S)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    p, C21, chi2, st = oracle.fit(b.det, prm, cov, lists, n, x, y, z, lay, align=b.align)
    return p, C21, st, lists, n, lay


def test_pulls_on_disks_are_unit_width():
    """Fits of the true hit lists of tracks that end on a disk: pulls against
    generator truth in the disk's local frame (r-phi, r, q/pT, phi, theta)
    have mean ~0 and RMS within 5%."""
    b = make_batch("c5", tracks=8000, noise=0.0)
    p, C21, st, lists, n, lay = _fit_true_forward(b)
    L = b.det.n_layers
    last = np.array([lists[i, n[i] - 1] for i in range(len(n))])
    on_disk = (st == 0) & (lay[last] >= L)
    p, C, last = p[on_disk], oracle.sym_to_full(C21[on_disk]), last[on_disk]
    truth = b.truth[0][b.seed_sim[on_disk], lay[last]]
    phip = np.arctan2(truth[:, 1], truth[:, 0])
    ut = np.stack([-np.sin(phip), np.cos(phip)], 1)
    wt = np.stack([np.cos(phip), np.sin(phip)], 1)
    d = p[:, :2] - truth[:, :2]
    pulls = {
        "rphi": np.einsum("ij,ij->i", ut, d) / np.sqrt(np.einsum("ij,ijk,ik->i", ut, C[:, :2, :2], ut)),
        "r": np.einsum("ij,ij->i", wt, d) / np.sqrt(np.einsum("ij,ijk,ik->i", wt, C[:, :2, :2], wt)),
        "kappa": (p[:, 3] - truth[:, 3]) / np.sqrt(C[:, 3, 3]),
        "phi": ((p[:, 4] - truth[:, 4] + np.pi) % (2 * np.pi) - np.pi) / np.sqrt(C[:, 4, 4]),
        "theta": (p[:, 5] - truth[:, 5]) / np.sqrt(C[:, 5, 5]),
    }
    N = on_disk.sum()
    assert N > 3000
    assert np.allclose(p[:, 2], truth[:, 2], atol=1e-9) and np.all(np.abs(C[:, 2, 2]) < 1e-12)  # on the plane
    for k, v in pulls.items():
        assert abs(v.mean()) < 4 / math.sqrt(N), (k, v.mean())
        assert abs(v.std() - 1.0) < 0.05, (k, v.std())


def test_dual_gradient_with_disk_hits_against_finite_differences():
    b = make_batch("c5", tracks=60, noise=0.0)
    S = b.det.n_surfaces
    L = b.det.n_layers
    x, y, z, lay = b.event_hits(0)
    prm, cov, _ = b.event_seeds(0)
    lists, n = true_hit_lists(b, 0, S)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    fwd = [i for i in range(len(n)) if lay[lists[i, n[i] - 1]] >= L][:4]
    assert len(fwd) == 4
    lists, n = lists[fwd], n[fwd]
    prm, cov = prm[:, fwd].astype(np.float64), cov[:, fwd].astype(np.float64)
    x, y, z = x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)
    al = b.align.astype(np.float64)
    tot, ga, gh, gs, _ = oracle.fit_grad(b.det, prm, cov, lists, n, x, y, z, lay, al)

    def total(prm_, x_, y_):
        return oracle.fit(b.det, prm_, cov, lists, n, x_, y_, z, lay, align=al)[2].sum()

    assert abs(total(prm, x, y) - tot) < 1e-9 * tot
    h = 1e-6
    disk_hits = [int(hh) for hh in lists[0, :n[0]] if lay[hh] >= L][:3]
    assert disk_hits
    for hidx in disk_hits + [int(lists[0, 1])]:
        for arr_i in range(2):
            a1, a2 = [x.copy(), y.copy()], [x.copy(), y.copy()]
            a1[arr_i][hidx] += h
            a2[arr_i][hidx] -= h
            fd = (total(prm, *a1) - total(prm, *a2)) / (2 * h)
            assert abs(fd - gh[hidx, arr_i]) < 1e-5 * max(1.0, abs(fd)), (hidx, arr_i, fd, gh[hidx, arr_i])
    for t in range(2):
        for k in range(6):
            p1, p2 = prm.copy(), prm.copy()
            p1[k, t] += h
            p2[k, t] -= h
            fd = (total(p1, x, y) - total(p2, x, y)) / (2 * h)
            assert abs(fd - gs[t, k]) < 1e-5 * max(1.0, abs(fd)), (t, k, fd, gs[t, k])


def _plan_truth(b, s, prm):
    """The true hits of seed s on the surfaces its eta region searches."""
    L = b.det.n_layers
    eta = -math.log(math.tan(0.5 * prm[5, s]))
    t = b.track_hits[0][b.seed_sim[s]].copy()
    if abs(eta) < b.det.eta_barrel:
        t[L:] = -1
    return t[t >= 0], eta


@pytest.mark.parametrize("noise", [0.0, 0.10])
def test_endcap_finding_recovers_true_hits(noise):
    """The barrel-plus-endcap event: at least 99% of the seeds find exactly
    their true hits on the surfaces of their region's plan; barrel-region
    seeds find no disk hit, forward seeds only disk hits of their own side;
    forward seeds do find disk hits."""
    b = make_batch("c5", noise=noise)
    r = oracle.find_event(b, 0)
    prm, _, _ = b.event_seeds(0)
    x, y, z, lay = b.event_hits(0)
    L, D = b.det.n_layers, b.det.n_disks
    good, with_disk = 0, 0
    for s in range(b.n_seeds):
        tt, eta = _plan_truth(b, s, prm)
        f = r["hits"][s, :r["n_found"][s]]
        good += r["n_found"][s] == tt.size and np.array_equal(f, tt)
        surf = lay[f]
        if abs(eta) < b.det.eta_barrel:
            assert np.all(surf < L)
        elif eta > 0:
            assert np.all((surf < L) | ((surf >= L) & (surf < L + D)))
        else:
            assert np.all((surf < L) | (surf >= L + D))
        with_disk += (surf >= L).any()
    assert good >= 0.99 * b.n_seeds, good
    assert with_disk > 0.5 * b.n_seeds


def test_barrel_only_detector_unchanged_by_the_plans():
    """Without disks every seed's plan is the barrel: the finding equals the
    brute-force scan of every hit of each layer (no z pre-selection)."""
    b = make_batch("c1", tracks=400)
    r1 = oracle.find_event(b, 0)
    r2 = oracle.find_event(b, 0, brute=True)
    assert np.array_equal(r1["hits"], r2["hits"]) and np.array_equal(r1["chi2"], r2["chi2"])


def test_plane_reached_only_within_half_a_turn():
    """A looper reaches the plane z = z_d after the transverse arc s = (z_d -
    z) tan(theta): within half a turn (|h s| < pi) the step exists, beyond it
    (or with the plane behind the track) it does not; the crossing lies on
    the plane and at the closed-form helix position."""
    kb = C_LIGHT * BZ
    th = 2 * math.atan(math.exp(-1.5))  # eta 1.5, cot(theta) = sinh(1.5)
    cot = math.cos(th) / math.sin(th)
    # (q/pT, plane): 3.98 rad of arc; 0.02; 0.04; the plane behind the track
    for kap, zd, expect in ((3.0, 250.0, False), (0.05, 130.0, True), (1.0, 10.0, True), (0.5, -50.0, False)):
        p = np.array([3.0, 1.0, 2.0, kap, 0.4, th])
        ok, q, _ = oracle.propagate_plane(BZ, p, zd)
        s = (zd - p[2]) / cot
        assert ok == (s > 0 and abs(kb * kap * s) < math.pi), (kap, zd)
        assert ok == expect, (kap, zd)
        if ok:
            h = -kb * kap
            phi1 = p[4] + h * s
            x = p[0] + (math.sin(phi1) - math.sin(p[4])) / h
            y = p[1] - (math.cos(phi1) - math.cos(p[4])) / h
            assert abs(q[2] - zd) < 1e-9 and abs(q[0] - x) < 1e-9 and abs(q[1] - y) < 1e-9


def test_passes_are_neither_holes_nor_stops():
    """Forward seeds pass the barrel layers beyond their reach (a dozen for
    |eta| near 2) and the disks they meet outside the disks' radii.  Were a
    pass a hole or a stop, a candidate allowed no hole would stop at its
    first one and never reach the disks: with max_holes = 0 the noise-free
    forward seeds still find their true hits (as with 3 holes allowed) and
    the disks' hits."""
    b = make_batch("c5", tracks=400, noise=0.0)
    r0 = oracle.find_event(b, 0, max_holes=0)
    r3 = oracle.find_event(b, 0, max_holes=3)
    prm, _, _ = b.event_seeds(0)
    x, y, z, lay = b.event_hits(0)
    L = b.det.n_layers
    fwd = same = with_disk = equal_holes = 0
    for s in range(b.n_seeds):
        tt, eta = _plan_truth(b, s, prm)
        if abs(eta) < b.det.eta_barrel:
            continue
        fwd += 1
        f = r0["hits"][s, :r0["n_found"][s]]
        same += np.array_equal(f, tt)
        with_disk += (lay[f] >= L).any()
        equal_holes += np.array_equal(r0["hits"][s], r3["hits"][s])
    assert fwd > 200
    assert same >= 0.98 * fwd and with_disk >= 0.9 * fwd and equal_holes >= 0.99 * fwd, (fwd, same, with_disk,
                                                                                         equal_holes)


def test_endcap_finding_in_a_parameterized_field():
    """The barrel-plus-endcap event simulated in the moderate parameterized
    field (the truth traced in eight helix steps per surface, each in the
    field at its own start; Bz 10% weaker at |z| = 120 cm, 43% at 250 cm):
    the oracle, whose steps take the field at their start, still finds the
    true hits of the plan for at least 99% of the seeds.  (Its q/pT pull on
    tracks that end on a disk widens to about 4 there: one helix per step in
    a field that changes by several percent along the step.)"""
    field = dict(field_cz=-0.10 / 120.0 ** 2, field_cr=-0.05 / 110.0 ** 2)
    b = make_batch("c5", noise=0.10, **field)
    r = oracle.find_event(b, 0)
    prm, _, _ = b.event_seeds(0)
    good = sum(np.array_equal(r["hits"][s, :r["n_found"][s]], _plan_truth(b, s, prm)[0])
               for s in range(b.n_seeds))
    assert good >= 0.99 * b.n_seeds, good
