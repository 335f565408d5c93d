"""Pins of the FP64 oracle against facts fixed by geometry and mathematics.

Each test pins one function of the oracle against something other than
itself: Runge-Kutta integration of the Lorentz force, the straight-line
closed form, the maximum reach of a circle through the origin, finite
differences, forward-mode automatic differentiation, the normal equations of
least squares, positive semi-definiteness, pull widths against generator truth,
brute-force search and brute-force duplicate removal.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from synth import make_batch
from synth.events import true_hit_lists

C_LIGHT = 0.00299792458


def _rk4_to_cylinder(p, R, bz, step=0.05):
    """Integrate dr/dl = t, dt/dl = (q/|p|) c (t x B) in 3D path length l until
    the transverse radius reaches R; the last step is solved by bisection."""
    x, y, z, kap, phi, th = [float(v) for v in p]
    a = C_LIGHT * kap * math.sin(th)  # q c / |p|

    def deriv(s):
        px, py, pz, tx, ty, tz = s
        # t x B with B = (0, 0, bz)
        return (tx, ty, tz, a * ty * bz, -a * tx * bz, 0.0)

    def rk4(s, h):
        k1 = deriv(s)
        k2 = deriv(tuple(si + 0.5 * h * ki for si, ki in zip(s, k1)))
        k3 = deriv(tuple(si + 0.5 * h * ki for si, ki in zip(s, k2)))
        k4 = deriv(tuple(si + h * ki for si, ki in zip(s, k3)))
        return tuple(si + h / 6.0 * (a1 + 2 * a2 + 2 * a3 + a4)
                     for si, a1, a2, a3, a4 in zip(s, k1, k2, k3, k4))

    s = (x, y, z, math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th))
    for _ in range(200000):
        nxt = rk4(s, step)
        if math.hypot(nxt[0], nxt[1]) >= R:
            lo, hi = 0.0, step
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                m = rk4(s, mid)
                if math.hypot(m[0], m[1]) >= R:
                    hi = mid
                else:
                    lo = mid
            return rk4(s, hi)
        s = nxt
    raise AssertionError("no crossing")


def _random_states(n, seed, r0=0.5):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ang = rng.uniform(-np.pi, np.pi)
        out.append(np.array([r0 * math.cos(ang), r0 * math.sin(ang), rng.uniform(-5, 5),
                             rng.uniform(-2.0, 2.0), rng.uniform(-np.pi, np.pi),
                             rng.uniform(0.5, 2.6)]))
    return out


def test_helix_matches_lorentz_force_integration():
    """Closed-form propagation == RK4 integration of the Lorentz force (sign of
    the bending, curvature constant, z advance, direction)."""
    for p in _random_states(6, 1):
        ok, q, _ = oracle.propagate(3.8, p, 30.0)
        assert ok
        s = _rk4_to_cylinder(p, 30.0, 3.8)
        assert abs(q[0] - s[0]) < 1e-8 and abs(q[1] - s[1]) < 1e-8 and abs(q[2] - s[2]) < 1e-8
        dphi = (q[4] - math.atan2(s[4], s[3]) + math.pi) % (2 * math.pi) - math.pi
        assert abs(dphi) < 1e-9
        assert q[3] == p[3] and q[5] == p[5]


def test_straight_line_at_zero_field():
    """B = 0: s = -b + sqrt(b^2 + R^2 - r0^2), b = p_xy . t (exact line solution)."""
    for p in _random_states(20, 2, r0=3.0):
        for R in (10.0, 55.5, 110.0):
            ok, s = oracle.path_length(0.0, p, R)
            b = p[0] * math.cos(p[4]) + p[1] * math.sin(p[4])
            exact = -b + math.sqrt(b * b + R * R - p[0] ** 2 - p[1] ** 2)
            assert ok and abs(s - exact) < 1e-12 * R
            ok, q, _ = oracle.propagate(0.0, p, R)
            assert abs(math.hypot(q[0], q[1]) - R) < 1e-12 * R
            assert q[4] == p[4]


def test_small_curvature_continuity():
    """The curved branch tends to the straight line as q/pT -> 0."""
    for p in _random_states(10, 3, r0=2.0):
        p = p.copy()
        p[3] = 1e-9
        ok1, s1 = oracle.path_length(3.8, p, 50.0)
        ok0, s0 = oracle.path_length(0.0, p, 50.0)
        assert ok1 and ok0 and abs(s1 - s0) < 1e-9


def test_max_reach_is_twice_the_radius():
    """A track through the origin reaches at most 2 rho (pT = 0.5 GeV: 87.78 cm)."""
    rho = 0.5 / (C_LIGHT * 3.8)
    for kap in (2.0, -2.0):
        p = np.array([0.0, 0.0, 0.0, kap, 0.3, 1.2])
        assert oracle.propagate(3.8, p, 2 * rho * (1 - 1e-6))[0]
        assert not oracle.propagate(3.8, p, 2 * rho * (1 + 1e-6))[0]
    assert abs(2 * rho - 87.78) < 0.01


def test_arc_length_closed_forms():
    """Track from the origin with radius rho: the arc to radius R is
    2 rho asin(R / 2 rho) (chord theorem), and from that crossing the track
    comes back through radius R after the rest of the circle,
    2 pi rho - 2 s_out."""
    for kap in (1.5, -0.7):
        rho = 1.0 / (C_LIGHT * 3.8 * abs(kap))
        p = np.array([0.0, 0.0, 0.0, kap, 0.4, math.pi / 2])
        ok, s_out = oracle.path_length(3.8, p, 20.0)
        assert ok and abs(s_out - 2 * rho * math.asin(20.0 / (2 * rho))) < 1e-10
        ok, q, _ = oracle.propagate(3.8, p, 20.0)
        ok, s_back = oracle.path_length(3.8, q, 20.0 - 1e-7)
        assert ok and abs(s_back - (2 * math.pi * rho - 2 * s_out)) < 1e-4
        # propagating by the full circle brings the direction back to the start
        ok, q2, _ = oracle.propagate(3.8, q, 20.0 - 1e-7)
        ok, q3, _ = oracle.propagate(3.8, q2, 1e-3)
        assert ok and abs(((q3[4] - p[4]) + math.pi) % (2 * math.pi) - math.pi) < 1e-3


@pytest.mark.parametrize("bz", [3.8, 0.0])
def test_jacobian_against_finite_differences_and_ad(bz):
    scale = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
    for p in _random_states(8, 4, r0=5.0):
        for R in (12.0, 40.0):
            ok, q, J = oracle.propagate(bz, p, R)
            assert ok
            Jfd = np.zeros((6, 6))
            for j in range(6):
                h = 1e-6 * scale[j]
                pp, pm = p.copy(), p.copy()
                pp[j] += h
                pm[j] -= h
                okp, qp, _ = oracle.propagate(bz, pp, R)
                okm, qm, _ = oracle.propagate(bz, pm, R)
                Jfd[:, j] = (qp - qm) / (2 * h)
            assert np.all(np.abs(Jfd - J) <= 1e-6 * np.maximum(1.0, np.abs(J)))
            ok, Jad = oracle.propagate_ad(bz, p, R)
            assert ok and np.allclose(Jad, J, rtol=1e-10, atol=1e-10)
            # the state stays on the cylinder to first order: radial row combination vanishes
            assert np.allclose(q[0] * J[0] + q[1] * J[1], 0.0, atol=1e-9 * R)
            # 20 structural non-zeros at most; kappa and theta rows are identity
            assert np.count_nonzero(np.abs(J) > 0) <= 20
            assert np.array_equal(J[3], np.eye(6)[3]) and np.array_equal(J[5], np.eye(6)[5])


def test_update_equals_normal_equations():
    """One Kalman update == the weighted least-squares posterior with the
    prediction as a pseudo-measurement: P = (C^-1 + H^T V^-1 H)^-1."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        A = rng.normal(size=(6, 6))
        C = A @ A.T * 1e-3 + np.eye(6) * 1e-4
        ang = rng.uniform(-np.pi, np.pi)
        R = rng.uniform(4, 110)
        p = np.array([R * math.cos(ang), R * math.sin(ang), rng.uniform(-50, 50), 0.3, ang + 0.1, 1.0])
        m = np.array([R * math.cos(ang + 0.001), R * math.sin(ang + 0.001), p[2] + 0.05])
        vr, vz = 1e-4, 1e-2
        ok, po, Co, chi2, r = oracle.update(p, C, m, vr, vz)
        assert ok
        H = np.zeros((2, 6))
        H[0, 0], H[0, 1], H[1, 2] = -math.sin(ang), math.cos(ang), 1.0
        V = np.diag([vr, vz])
        P = np.linalg.inv(np.linalg.inv(C) + H.T @ np.linalg.inv(V) @ H)
        mean = p + P @ H.T @ np.linalg.inv(V) @ r
        assert np.allclose(Co, P, rtol=1e-8, atol=1e-14)
        assert np.allclose(po, mean, rtol=1e-10, atol=1e-12)
        S = H @ C @ H.T + V
        assert abs(chi2 - r @ np.linalg.solve(S, r)) < 1e-9 * max(1, chi2)
    # a hit on the far half of the cylinder is not compatible
    ok, *_ = oracle.update(p, C, -m, vr, vz)
    assert not ok


def test_highland_width():
    """Highland width for a 1 GeV/c relativistic track at normal incidence in
    0.02 X0: 0.0136 * sqrt(0.02) * (1 + 0.038 ln 0.02) ~= 1.6375e-3 rad
    (beta from the pion mass changes it by 1%)."""
    p = np.array([10.0, 0.0, 0.0, 1.0, 0.0, math.pi / 2])  # pT = p = 1 GeV, radial
    beta = 1.0 / math.sqrt(1.0 + 0.13957 ** 2)
    expected = 0.0136 / beta * math.sqrt(0.02) * (1 + 0.038 * math.log(0.02))
    assert abs(oracle.highland(p, 0.02) - expected) < 1e-15
    assert abs(expected - 1.6375e-3 / beta) < 1e-6
    # oblique incidence in phi at fixed momentum lengthens the path:
    # t = x0 / (sin(theta) cos(phi - phi_p))
    p2 = p.copy()
    p2[4] = 0.6
    assert oracle.highland(p2, 0.02) > oracle.highland(p, 0.02)


def _fit_true(batch, e=0, ms_after_last=False, want_each=False):
    L = batch.det.n_layers
    x, y, z, lay = batch.event_hits(e)
    prm, cov, sh = batch.event_seeds(e)
    sims = batch.seed_sim[batch.seed_off[e]:batch.seed_off[e + 1]]
    lists, n = true_hit_lists(batch, e, L)
    lists, n = lists[sims], n[sims]
    res = oracle.fit(batch.det, prm, cov, lists, n, x, y, z, lay, align=batch.align,
                     ms_after_last=ms_after_last, want_each=want_each)
    return res, lists, n, sims


def test_pulls_are_unit_width():
    """Fitted parameters at the last hit against generator truth: pulls in the
    local frame (r-phi, z, q/pT, phi, theta) have mean ~0 (within 4 standard
    errors) and RMS within 3%."""
    b = make_batch("c3", misalign_sigma=0.0)
    (p, C21, chi2, st), lists, n, sims = _fit_true(b)
    # a looper whose fitted curvature no longer reaches its last layer may stop
    good = st == 0
    assert good.mean() > 0.999
    p, C21, lists, n, sims = p[good], C21[good], lists[good], n[good], sims[good]
    C = oracle.sym_to_full(C21)
    last = np.array([lists[i, n[i] - 1] for i in range(len(n))])
    lay = b.layer[last]
    truth = b.truth[0][sims, lay]
    phip = np.arctan2(truth[:, 1], truth[:, 0])
    ut = np.stack([-np.sin(phip), np.cos(phip)], 1)
    d_rphi = np.einsum("ij,ij->i", ut, p[:, :2] - truth[:, :2])
    v_rphi = np.einsum("ij,ijk,ik->i", ut, C[:, :2, :2], ut)
    pulls = {
        "rphi": d_rphi / np.sqrt(v_rphi),
        "z": (p[:, 2] - truth[:, 2]) / np.sqrt(C[:, 2, 2]),
        "kappa": (p[:, 3] - truth[:, 3]) / np.sqrt(C[:, 3, 3]),
        "phi": ((p[:, 4] - truth[:, 4] + np.pi) % (2 * np.pi) - np.pi) / np.sqrt(C[:, 4, 4]),
        "theta": (p[:, 5] - truth[:, 5]) / np.sqrt(C[:, 5, 5]),
    }
    N = len(n)
    assert N > 9000
    for k, v in pulls.items():
        assert abs(v.mean()) < 4 / math.sqrt(N), (k, v.mean())
        assert abs(v.std() - 1.0) < 0.03, (k, v.std())


def test_chi2_per_hit_has_two_degrees_of_freedom():
    """Predicted-residual chi2 of a consistent filter is chi2(2) distributed per
    2D hit once the prior no longer matters (hits 5 onward)."""
    b = make_batch("c3", misalign_sigma=0.0)
    (p, C21, chi2, st, each), lists, n, sims = _fit_true(b, want_each=True)
    vals = np.concatenate([each[i, 4:n[i]] for i in range(len(n)) if st[i] == 0])
    assert vals.size > 50000
    assert abs(vals.mean() - 2.0) < 0.04
    # chi2(2) is exponential with mean 2: P(chi2 > 2 ln 10) = 0.1
    assert abs((vals > 2 * math.log(10)).mean() - 0.1) < 0.01


def test_covariance_symmetric_psd_rank5():
    """After propagation the covariance is PSD of rank 5 (the radial direction
    is projected out); the local 5x5 block is positive definite."""
    b = make_batch("c1", tracks=300)
    (p, C21, chi2, st), lists, n, sims = _fit_true(b)
    C = oracle.sym_to_full(C21)
    for i in np.nonzero(st == 0)[0]:
        w = np.linalg.eigvalsh(C[i])
        nrm = np.abs(w).max()
        assert w.min() > -1e-12 * nrm
        assert np.sum(w < 1e-9 * nrm) == 1
        phi = math.atan2(p[i, 1], p[i, 0])
        B = np.zeros((6, 5))
        B[0, 0], B[1, 0] = -math.sin(phi), math.cos(phi)
        B[2, 1] = B[3, 2] = B[4, 3] = B[5, 4] = 1.0
        assert np.linalg.eigvalsh(B.T @ C[i] @ B).min() > 0


def test_config0_finds_true_tracks():
    """No noise, 100 tracks: at least 99% of seeds find exactly their true hits."""
    b = make_batch("c0")
    r = oracle.find_event(b, 0)
    th = b.track_hits[0]
    good = 0
    for s in range(b.n_seeds):
        t = th[b.seed_sim[s]]
        t = t[t >= 0]
        good += (r["n_found"][s] == t.size) and np.array_equal(r["hits"][s, :t.size], t)
    assert good >= 0.99 * b.n_seeds


def test_z_preselection_equals_brute_force():
    """Finding with the exact z pre-selection == testing every hit of the layer."""
    b = make_batch("c1", tracks=400)
    r1 = oracle.find_event(b, 0)
    r2 = oracle.find_event(b, 0, brute=True)
    assert np.array_equal(r1["hits"], r2["hits"])
    assert np.array_equal(r1["n_found"], r2["n_found"])
    assert np.array_equal(r1["chi2"], r2["chi2"])


def test_dedup_index_equals_brute_force():
    b = make_batch("c1b", tracks=600)
    r = oracle.find_event(b, 0)
    k1 = oracle.dedup(r["hits"], r["n_found"], r["chi2"], 0.5)
    k2 = oracle.dedup(r["hits"], r["n_found"], r["chi2"], 0.5, brute=True)
    assert np.array_equal(k1, k2)
    # duplicate seeds exist in c1b, so something is removed, and no kept pair
    # shares more than half of the shorter track
    assert k1.sum() < k1.size
    kept = np.nonzero(k1)[0]
    sets = [set(r["hits"][i, :r["n_found"][i]]) for i in kept]
    for a in range(len(kept)):
        for c in range(a + 1, len(kept)):
            sh = len(sets[a] & sets[c])
            assert sh <= 0.5 * min(len(sets[a]), len(sets[c]))


def test_dedup_greedy_order_small_case():
    """Hand-made case.  Visiting order is (more hits, lower chi2, index):
    A (5 hits, 1.0), B (5, 2.0), D (4, 0.5), C (4, 3.0)."""
    hits = np.full((4, 6), -1, np.int32)
    hits[0, :5] = [1, 2, 3, 4, 5]      # A
    hits[1, :5] = [1, 2, 3, 4, 9]      # B: 4 shared with A > 2.5 -> removed
    hits[2, :4] = [4, 5, 20, 21]       # C: 2 shared with A (not > 2), 2 with D -> kept
    hits[3, :4] = [20, 21, 22, 30]     # D: nothing shared with A -> kept
    n = np.array([5, 5, 4, 4], np.int32)
    chi2 = np.array([1.0, 2.0, 3.0, 0.5])
    assert list(oracle.dedup(hits, n, chi2)) == [1, 0, 1, 1]
    # D now shares 3 hits with C; D is visited first, so C is the one removed
    hits[3, :4] = [20, 21, 4, 30]
    assert list(oracle.dedup(hits, n, chi2)) == [1, 0, 0, 1]
    assert list(oracle.dedup(hits, n, chi2, brute=True)) == [1, 0, 0, 1]


def _material_map(det, n_z=9, seed=11):
    """A strongly varying map: thickness 0.005-0.06 X0 at n_z z nodes per layer."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.005, 0.06, size=(det.n_layers, n_z)).astype(np.float32)


@pytest.mark.parametrize("with_map,with_eloss", [(False, False), (True, False), (True, True)])
def test_dual_gradient_against_finite_differences(with_map, with_eloss):
    """d(sum chi2)/d(alignment, hits, seed parameters) by dual numbers ==
    central finite differences of the fit (FP64); with a material map the
    scattering thickness also depends on the state's z; with energy loss q/pT
    changes after every layer."""
    b = make_batch("c3", tracks=40)
    if with_map:
        b.det = dataclasses.replace(b.det, x0_map=_material_map(b.det))
    if with_eloss:
        b.det = dataclasses.replace(b.det, eloss=(2e-4,) * b.det.n_layers)
    L = b.det.n_layers
    x, y, z, lay = b.event_hits(0)
    prm, cov, sh = b.event_seeds(0)
    sims = b.seed_sim
    lists, n = true_hit_lists(b, 0, L)
    lists, n = lists[sims][:5], n[sims][:5]
    prm, cov = prm[:, :5].astype(np.float64), cov[:, :5].astype(np.float64)
    x, y, z = x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)
    al = b.align.astype(np.float64)
    tot, ga, gh, gs, _ = oracle.fit_grad(b.det, prm, cov, lists, n, x, y, z, lay, al)

    def total(prm_, x_, y_, z_, al_):
        return oracle.fit(b.det, prm_, cov, lists, n, x_, y_, z_, lay, align=al_)[2].sum()

    assert abs(total(prm, x, y, z, al) - tot) < 1e-9 * tot
    h = 1e-6
    for (li, c) in [(3, 0), (3, 1), (10, 0), (16, 1)]:
        a1, a2 = al.copy(), al.copy()
        a1[li, c] += h
        a2[li, c] -= h
        fd = (total(prm, x, y, z, a1) - total(prm, x, y, z, a2)) / (2 * h)
        assert abs(fd - ga[li, c]) < 1e-5 * max(1.0, abs(fd)), (li, c, fd, ga[li, c])
    for hidx in lists[0, [0, 2, 7]]:
        for arr_i in range(3):
            arrs = [x.copy(), y.copy(), z.copy()]
            arrs2 = [x.copy(), y.copy(), z.copy()]
            arrs[arr_i][hidx] += h
            arrs2[arr_i][hidx] -= h
            fd = (total(prm, *arrs, al) - total(prm, *arrs2, al)) / (2 * h)
            assert abs(fd - gh[hidx, arr_i]) < 1e-5 * max(1.0, abs(fd)), (hidx, arr_i, fd, gh[hidx, arr_i])
    for t in range(2):
        for k in range(6):
            p1, p2 = prm.copy(), prm.copy()
            p1[k, t] += h
            p2[k, t] -= h
            fd = (total(p1, x, y, z, al) - total(p2, x, y, z, al)) / (2 * h)
            assert abs(fd - gs[t, k]) < 1e-5 * max(1.0, abs(fd)), (t, k, fd, gs[t, k])


def test_golden_closed_forms():
    """Hand-derived closed-form cases stored under tests/golden/."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")
    n = 0
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        kind, bz = f[0], float(f[1])
        p = np.array([float(v) for v in f[2:8]])
        R, expected = float(f[8]), float(f[9])
        if kind == "path":
            ok, s = oracle.path_length(bz, p, R)
            assert ok and abs(s - expected) < 1e-9, (line, s)
        else:
            ok, _, _ = oracle.propagate(bz, p, R)
            assert int(ok) == int(expected), line
        n += 1
    assert n == 4


def test_oracle_threads_give_sequential_results():
    """The oracle's calls run on several host threads at once (the timed CPU
    baseline does so); the dual-number width is per thread, so concurrent
    gradients equal sequential ones."""
    from concurrent.futures import ThreadPoolExecutor
    b = make_batch("c1", tracks=200)
    x, y, z, lay = b.event_hits(0)
    prm, cov, sh = b.event_seeds(0)
    r = oracle.find_event(b, 0)
    ks = [np.arange(i, prm.shape[1], 4) for i in range(4)]

    def run(k):
        return oracle.fit_grad(b.det, prm[:, k], cov[:, k], r["hits"][k], r["n_found"][k], x, y, z, lay, b.align)

    seq = [run(k) for k in ks]
    with ThreadPoolExecutor(4) as ex:
        par = list(ex.map(run, ks))
    for s_, p_ in zip(seq, par):
        for a, c in zip(s_, p_):
            assert np.array_equal(np.asarray(a), np.asarray(c))


# ------------------------------------------------- kinematic duplicate criteria

def _state(eta, phi, kappa, x=0.0, y=0.0, z=0.0):
    return [x, y, z, kappa, phi, 2.0 * math.atan(math.exp(-eta))]


def test_phi0_is_the_direction_at_closest_approach_brute_force():
    """phi0 against a brute-force search for the point of the helix closest to
    the z axis (dense sampling of one turn, then a bounded 1D minimisation),
    the helix written out from its parametric form."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(7)
    for bz in (3.8, -2.0):
        for _ in range(40):
            x, y = rng.uniform(-60, 60, 2)
            kap = rng.choice([-1, 1]) * rng.uniform(0.05, 2.0)
            phi = rng.uniform(-math.pi, math.pi)
            p = [x, y, rng.uniform(-50, 50), kap, phi, rng.uniform(0.3, 2.8)]
            h = -C_LIGHT * bz * kap
            turn = 2 * math.pi / abs(h)

            def r2(s):
                xs = x + (math.sin(phi + h * s) - math.sin(phi)) / h
                ys = y - (math.cos(phi + h * s) - math.cos(phi)) / h
                return xs * xs + ys * ys

            grid = np.linspace(0.0, turn, 20001)
            xs = x + (np.sin(phi + h * grid) - math.sin(phi)) / h
            ys = y - (np.cos(phi + h * grid) - math.cos(phi)) / h
            i = int(np.argmin(xs * xs + ys * ys))
            d = turn / 20000
            res = minimize_scalar(r2, bounds=(grid[i] - d, grid[i] + d), method="bounded",
                                  options={"xatol": 1e-12 * turn})
            want = math.atan2(math.sin(phi + h * res.x), math.cos(phi + h * res.x))
            got = oracle.kinematics(bz, [p])[0, 2]
            diff = abs(got - want)
            assert min(diff, 2 * math.pi - diff) < 1e-6


def test_phi0_straight_line_and_invariance_along_the_helix():
    # zero field: the direction does not change along the line
    p = [30.0, -4.0, 1.0, 0.7, 2.5, 1.1]
    assert abs(oracle.kinematics(0.0, [p])[0, 2] - 2.5) < 1e-15
    # a track from the origin: phi0 is its initial direction at every radius
    rng = np.random.default_rng(3)
    for _ in range(20):
        phi = rng.uniform(-math.pi, math.pi)
        eta = rng.uniform(-1.5, 1.5)
        kap = rng.choice([-1, 1]) * rng.uniform(0.1, 2.0)
        p0 = _state(eta, phi, kap)
        for R in (4.0, 30.0, 80.0):
            ok, q, _ = oracle.propagate(3.8, p0, R)
            if not ok:
                continue
            k = oracle.kinematics(3.8, [q])[0]
            d = abs(k[2] - phi)
            assert min(d, 2 * math.pi - d) < 1e-12
            assert abs(k[0] - eta) < 1e-12          # theta is constant along the helix
            assert abs(k[1] - abs(kap)) < 1e-15
    # eta = asinh(cot theta)
    for th in (0.3, 1.0, math.pi / 2, 2.0, 2.9):
        k = oracle.kinematics(3.8, [[0, 0, 0, 0.5, 0.0, th]])[0]
        assert abs(k[0] - math.asinh(math.cos(th) / math.sin(th))) < 1e-14


def test_seed_clean_small_cases():
    hits = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 9]], np.int32)
    # A~B and B~C in eta, A and C not: greedy keeps A, drops B, keeps C
    p = [_state(0.0, 0.1, 0.5), _state(0.03, 0.1, 0.5), _state(0.06, 0.1, 0.5)]
    assert list(oracle.seed_clean(p, hits, 3.8, 0.05)) == [1, 0, 1]
    # shared hits required: none shared -> nothing dropped; one shared -> dropped
    assert list(oracle.seed_clean(p, hits, 3.8, 0.05, min_shared=1)) == [1, 1, 1]
    h2 = hits.copy(); h2[1, 2] = 1
    assert list(oracle.seed_clean(p, h2, 3.8, 0.05, min_shared=1)) == [1, 0, 1]
    assert list(oracle.seed_clean(p, h2, 3.8, 0.05, min_shared=2)) == [1, 1, 1]
    # phi difference taken on the circle
    q = [_state(0.0, math.pi - 0.01, 0.5), _state(0.0, -math.pi + 0.01, 0.5)]
    assert list(oracle.seed_clean(q, hits[:2], 3.8, 0.05, dphi=0.05)) == [1, 0]
    assert list(oracle.seed_clean(q, hits[:2], 3.8, 0.05, dphi=0.015)) == [1, 1]
    # relative pT: |0.5 - 0.55| / 0.55 = 0.0909
    r = [_state(0.0, 0.0, 0.5), _state(0.0, 0.0, -0.55)]
    assert list(oracle.seed_clean(r, hits[:2], 3.8, 0.05, dpt=0.1)) == [1, 0]
    assert list(oracle.seed_clean(r, hits[:2], 3.8, 0.05, dpt=0.09)) == [1, 1]


def _np_kin(bz, p):
    """eta, |q/pT| and phi0 by other formulas: asinh(cot theta), and phi0 from
    h times the circle centre, which needs no division by h."""
    p = np.asarray(p, np.float64)
    h = -C_LIGHT * bz * p[:, 3]
    vx = h * p[:, 0] - np.sin(p[:, 4])
    vy = h * p[:, 1] + np.cos(p[:, 4])
    return np.stack([np.arcsinh(np.cos(p[:, 5]) / np.sin(p[:, 5])), np.abs(p[:, 3]),
                     np.arctan2(-vx, vy)], axis=1)


def _np_close(ka, kb, deta, dphi, dpt):
    ok = np.ones(np.broadcast(ka[..., 0], kb[..., 0]).shape, bool)
    if deta > 0:
        ok &= np.abs(ka[..., 0] - kb[..., 0]) < deta
    if dphi > 0:
        d = np.abs(ka[..., 2] - kb[..., 2])
        ok &= np.minimum(d, 2 * np.pi - d) < dphi
    if dpt > 0:
        ok &= np.abs(ka[..., 1] - kb[..., 1]) <= dpt * np.maximum(ka[..., 1], kb[..., 1])
    return ok


@pytest.mark.parametrize("cuts", [(0.05, 0.05, 0.0, 1), (0.02, 0.02, 0.5, 0)])
def test_seed_clean_c1b_fixed_point(cuts):
    """On the duplicate-seed workload: the kept set is the fixed point of the
    greedy rule (a seed is kept iff no kept lower-index seed is its duplicate),
    checked with an independently written pair predicate; the injected
    duplicates (two shared hits) are removed."""
    deta, dphi, dpt, ms = cuts
    b = make_batch("c1b")
    p = b.params.T.astype(np.float64)
    sh = b.seed_hits.T
    keep = oracle.seed_clean(p, sh, b.det.bz, deta, dphi, dpt, ms)
    k = _np_kin(b.det.bz, p)
    n = p.shape[0]
    close = _np_close(k[:, None, :], k[None, :, :], deta, dphi, dpt)
    shared = (sh[:, None, :, None] == sh[None, :, None, :]).sum(axis=(2, 3))
    dup = close & (shared >= ms)
    kept = keep.astype(bool)
    for j in range(n):
        assert kept[j] == (not np.any(kept[:j] & dup[:j, j])), j
    n_orig = np.unique(b.seed_sim).size
    if ms == 1:  # exactly the injected duplicates go
        assert kept[:n_orig].all() and (~kept[n_orig:]).sum() >= 0.98 * (n - n_orig)


def test_dedup_kinematic_precuts():
    hits = np.full((2, 5), -1, np.int32)
    hits[0] = [1, 2, 3, 4, 5]
    hits[1] = [1, 2, 3, 4, 6]
    n = np.array([5, 5], np.int32)
    chi2 = np.array([1.0, 2.0])
    p = [_state(0.0, 0.2, 0.5), _state(0.3, 0.2, 0.5)]
    assert list(oracle.dedup(hits, n, chi2)) == [1, 0]
    assert list(oracle.dedup(hits, n, chi2, params=p, bz=3.8, deta=0.1)) == [1, 1]
    assert list(oracle.dedup(hits, n, chi2, params=p, bz=3.8, deta=0.5)) == [1, 0]
    assert list(oracle.dedup(hits, n, chi2, brute=True, params=p, bz=3.8, deta=0.1)) == [1, 1]
    # a track without hits is never kept
    assert list(oracle.dedup(hits, np.array([5, 0], np.int32), chi2)) == [1, 0]


def test_dedup_kinematic_index_equals_brute_force():
    b = make_batch("c1b", tracks=600)
    r = oracle.find_event(b, 0)
    for cuts in [(0.01, 0.01, 0.2), (0.002, 0.0, 0.0), (0.0, 0.003, 0.05)]:
        k1 = oracle.dedup(r["hits"], r["n_found"], r["chi2"], 0.5, params=r["p"], bz=b.det.bz,
                          deta=cuts[0], dphi=cuts[1], dpt=cuts[2])
        k2 = oracle.dedup(r["hits"], r["n_found"], r["chi2"], 0.5, brute=True, params=r["p"],
                          bz=b.det.bz, deta=cuts[0], dphi=cuts[1], dpt=cuts[2])
        assert np.array_equal(k1, k2)
        # no kept pair is a duplicate under both criteria
        kin = _np_kin(b.det.bz, np.asarray(r["p"]).reshape(-1, 6))
        kept = np.nonzero(k1)[0]
        sets = [set(r["hits"][i, :r["n_found"][i]]) for i in kept]
        for a in range(len(kept)):
            for c in range(a + 1, len(kept)):
                over = len(sets[a] & sets[c]) > 0.5 * min(len(sets[a]), len(sets[c]))
                assert not (over and _np_close(kin[kept[a]], kin[kept[c]], *cuts))


# ------------------------------------------------------------- material map

def test_material_map_interpolation():
    """Thickness at z: linear between the nodes, constant beyond the ends
    (against numpy's interpolation); without a map, the per-layer value."""
    b = make_batch("c1", tracks=10)
    det = dataclasses.replace(b.det, x0_map=_material_map(b.det))
    nodes = np.linspace(-det.z_max, det.z_max, 9)
    rng = np.random.default_rng(5)
    for layer in (0, 7, 16):
        for z in np.concatenate([rng.uniform(-1.3 * det.z_max, 1.3 * det.z_max, 50), nodes]):
            want = np.interp(z, nodes, det.x0_map[layer].astype(np.float64))
            assert abs(oracle.x0_at(det, layer, z) - want) < 1e-12
        assert oracle.x0_at(b.det, layer, 33.0) == float(np.float32(b.det.x0[layer]))


def test_material_map_constant_equals_per_layer():
    """A map holding each layer's x0 at every node gives the per-layer fit and
    finding (the interpolation of equal nodes is that value)."""
    b = make_batch("c1", tracks=300)
    flat = np.repeat(np.asarray(b.det.x0, np.float32)[:, None], 5, axis=1)
    r0 = oracle.find_event(b, 0)
    b.det = dataclasses.replace(b.det, x0_map=flat)
    r1 = oracle.find_event(b, 0)
    assert np.array_equal(r0["hits"], r1["hits"])
    assert np.allclose(r0["chi2"], r1["chi2"], rtol=1e-12, atol=0)
    assert np.allclose(r0["p"], r1["p"], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------ energy loss

MPI = 0.13957


def _pmag(p):
    return 1.0 / (abs(p[3]) * math.sin(p[5]))


def test_eloss_momentum_change_and_path_factor():
    """dE = beta dp to first order; the loss doubles at half the normal
    component of the direction (cos(phi - phi_p) = 0.5) and grows as 1/beta^2
    at low momentum; the charge is kept."""
    e = 1e-6
    for kap in (0.5, -2.0, 5.0):
        p = np.array([40.0, 0.0, 3.0, kap, 0.0, math.pi / 2])
        q, _ = oracle.eloss(p, np.eye(6), e)
        pm, pm1 = _pmag(p), _pmag(q)
        beta = pm / math.hypot(pm, MPI)
        de = e / beta ** 2
        assert abs((pm - pm1) - de / beta) < 1e-5 * de  # second order: m^2 beta dE / (2 p^3)
        assert np.sign(q[3]) == np.sign(kap)
        # oblique: cos(phi - phi_p) = 0.5 -> twice the path
        p2 = p.copy(); p2[4] = math.pi / 3
        q2, _ = oracle.eloss(p2, np.eye(6), e)
        assert abs((pm - _pmag(q2)) / (pm - pm1) - 2.0) < 1e-5
    # 1/beta^2: at p = 0.2 GeV the loss is (1 + m^2/p^2) times the beta -> 1 value
    p = np.array([40.0, 0.0, 3.0, 5.0, 0.0, math.pi / 2])
    q, _ = oracle.eloss(p, np.eye(6), e)
    pm = _pmag(p)
    dE = (math.hypot(pm, MPI) - math.hypot(_pmag(q), MPI))
    assert abs(dE / e - (1 + MPI ** 2 / pm ** 2)) < 1e-5


def test_eloss_jacobian_against_finite_differences():
    """The covariance map C' = F C F^T with F = d p'/d p: the hand-written q/pT
    row against central differences of the state map."""
    rng = np.random.default_rng(4)
    e = 3e-4
    for _ in range(20):
        p = np.array([rng.uniform(-50, 50), rng.uniform(-50, 50), rng.uniform(-30, 30),
                      rng.choice([-1, 1]) * rng.uniform(0.1, 3.0), rng.uniform(-3, 3), rng.uniform(0.5, 2.6)])
        phip = math.atan2(p[1], p[0])
        if abs(math.cos(p[4] - phip)) < 0.2:
            continue
        F = np.zeros((6, 6))
        for j in range(6):
            h = 1e-6 * max(1.0, abs(p[j]))
            a, b = p.copy(), p.copy()
            a[j] += h
            b[j] -= h
            F[:, j] = (oracle.eloss(a, np.eye(6), e)[0] - oracle.eloss(b, np.eye(6), e)[0]) / (2 * h)
        A = rng.normal(size=(6, 6))
        C = A @ A.T
        q, C1 = oracle.eloss(p, C, e)
        want = F @ C @ F.T
        assert np.abs(C1 - want).max() < 1e-6 * np.abs(want).max()
