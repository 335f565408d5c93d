"""Pins of the oracle's parameterized axial field (Sec. 3: the method takes a
constant or a parameterized field).

Reading pinned here: Bz(r, z) = bz (1 + cz z^2 + cr r^2), and each
propagation to a layer is a helix in the field at its starting point; the
propagation Jacobian is that of the helix with the field held fixed, while
derivatives taken through the fit (the adjoint) also see the field move with
the starting point.  The pins:
  * the propagation equals the uniform-field propagation in Bz(start);
  * Runge-Kutta integration of the Lorentz force with the field frozen at the
    start point gives the same crossing; with the field varying along the
    path the crossing moves by no more than the curvature change allows;
  * J equals central differences at fixed field; forward-mode derivatives of
    the whole map equal central differences of the map, and differ from J by
    exactly the rank-one field term (p3 / kb) J[:, 3] (grad kb)^T;
  * the dual-number gradient of a fit in such a field equals central
    differences of the fit;
  * finding in such a field (tracks simulated in fine helix steps) recovers
    the true hits.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from synth import make_batch
from synth.events import true_hit_lists

C_LIGHT = 0.00299792458
BZ = 3.8
CZ, CR = -3.0e-5, -2.0e-5  # strong for the single-step pins: Bz 0.57-1 of bz in |z| < 80, r < 40


def _fac(p, cz, cr):
    return 1.0 + cz * p[2] ** 2 + cr * (p[0] ** 2 + p[1] ** 2)


def _states(n, seed, r0=6.0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ang = rng.uniform(-np.pi, np.pi)
        out.append(np.array([r0 * math.cos(ang), r0 * math.sin(ang), rng.uniform(-60, 60),
                             rng.uniform(-1.5, 1.5), rng.uniform(-np.pi, np.pi), rng.uniform(0.5, 2.6)]))
    return out


def _rk4_crossing(p, R, bfun, step=0.02):
    """Lorentz force in 3D path length l, dt/dl = (q c/|p|) t x B(r), B = (0, 0,
    bfun(x, y, z)), until the transverse radius reaches R (bisection on the
    last step).  Returns (x, y, z, phi) at the crossing and the 3D path."""
    x, y, z, kap, phi, th = [float(v) for v in p]
    a = C_LIGHT * kap * math.sin(th)

    def deriv(s):
        _, _, _, tx, ty, _ = s
        b = bfun(s[0], s[1], s[2])
        return np.array([tx, ty, s[5], a * ty * b, -a * tx * b, 0.0])

    def rk4(s, h):
        k1 = deriv(s)
        k2 = deriv(s + 0.5 * h * k1)
        k3 = deriv(s + 0.5 * h * k2)
        k4 = deriv(s + h * k3)
        return s + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)

    s = np.array([x, y, z, math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)])
    path = [s[:3].copy()]
    for _ in range(400000):
        nxt = rk4(s, step)
        if math.hypot(nxt[0], nxt[1]) >= R:
            lo, hi = 0.0, step
            for _ in range(70):
                mid = 0.5 * (lo + hi)
                if math.hypot(*rk4(s, mid)[:2]) >= R:
                    hi = mid
                else:
                    lo = mid
            e = rk4(s, hi)
            path.append(e[:3].copy())
            return (e[0], e[1], e[2], math.atan2(e[4], e[3])), np.array(path)
        s = nxt
        path.append(s[:3].copy())
    raise AssertionError("no crossing")


def test_propagation_is_the_helix_in_the_field_at_the_start():
    for p in _states(12, 21):
        for R in (20.0, 45.0):
            ok, q, J = oracle.propagate(BZ, p, R, CZ, CR)
            ok0, q0, J0 = oracle.propagate(BZ * _fac(p, CZ, CR), p, R)
            assert ok == ok0
            if ok:
                assert np.allclose(q, q0, rtol=1e-13, atol=1e-12) and np.allclose(J, J0, rtol=1e-12, atol=1e-12)


def test_rk4_with_the_field_frozen_at_the_start():
    for p in _states(4, 22):
        ok, q, _ = oracle.propagate(BZ, p, 40.0, CZ, CR)
        assert ok
        b0 = BZ * _fac(p, CZ, CR)
        (x, y, z, ph), _ = _rk4_crossing(p, 40.0, lambda *_: b0)
        assert abs(q[0] - x) < 1e-8 and abs(q[1] - y) < 1e-8 and abs(q[2] - z) < 1e-8
        assert abs((q[4] - ph + math.pi) % (2 * math.pi) - math.pi) < 1e-9


def test_single_step_error_in_a_varying_field_is_bounded_by_the_curvature_change():
    """With the field varying along the path, the transverse path bends by
    curvature kappa(l) instead of kappa(0): the crossing moves by at most
    |h0| max|B/B0 - 1| s^2 / 2 (s the transverse arc), to first order; and
    it does move (the pin sees the field vary)."""
    moved = 0
    for p in _states(6, 23):
        R = 40.0
        ok, q, _ = oracle.propagate(BZ, p, R, CZ, CR)
        assert ok
        bfun = lambda x, y, z: BZ * (1.0 + CZ * z * z + CR * (x * x + y * y))  # noqa: E731
        (x, y, z, _), path = _rk4_crossing(p, R, bfun)
        b0 = bfun(*p[:3])
        dev = max(abs(bfun(*pt) / b0 - 1.0) for pt in path)
        ok, s = oracle.path_length(b0, p, R)
        h0 = abs(C_LIGHT * b0 * p[3])
        bound = 1.3 * h0 * dev * s * s / 2.0 + 1e-7
        d = math.sqrt((q[0] - x) ** 2 + (q[1] - y) ** 2)
        assert d <= bound, (d, bound)
        moved += d > 0.05 * bound
    assert moved >= 3


def test_jacobian_at_fixed_field_and_the_field_term():
    scale = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
    for p in _states(8, 24):
        R = 30.0
        ok, q, J = oracle.propagate(BZ, p, R, CZ, CR)
        if not ok:
            continue
        b0 = BZ * _fac(p, CZ, CR)
        Jfix = np.zeros((6, 6))
        Jfull = np.zeros((6, 6))
        for j in range(6):
            h = 1e-6 * scale[j]
            pp, pm = p.copy(), p.copy()
            pp[j] += h
            pm[j] -= h
            Jfix[:, j] = (oracle.propagate(b0, pp, R)[1] - oracle.propagate(b0, pm, R)[1]) / (2 * h)
            Jfull[:, j] = (oracle.propagate(BZ, pp, R, CZ, CR)[1] - oracle.propagate(BZ, pm, R, CZ, CR)[1]) / (2 * h)
        assert np.all(np.abs(Jfix - J) <= 1e-6 * np.maximum(1.0, np.abs(J)))
        ok, Jad = oracle.propagate_ad(BZ, p, R, CZ, CR)
        assert ok and np.all(np.abs(Jfull - Jad) <= 1e-6 * np.maximum(1.0, np.abs(Jad)))
        # the field term: q depends on kb and q/pT only through their product
        kb = -C_LIGHT * b0
        u = p[3] / kb * J[:, 3]
        u[3] = 0.0
        grad_kb = -C_LIGHT * BZ * np.array([2 * CR * p[0], 2 * CR * p[1], 2 * CZ * p[2], 0.0, 0.0, 0.0])
        assert np.allclose(Jad - J, np.outer(u, grad_kb), rtol=1e-9, atol=1e-11)
        assert np.abs(Jad - J).max() > 1e-4  # the term is not negligible here


FIELD_CFG = dict(field_cz=-0.10 / 120.0 ** 2, field_cr=-0.05 / 110.0 ** 2)  # 10% lower at |z| = 120 cm


def test_dual_gradient_with_field_against_finite_differences():
    b = make_batch("c3", tracks=40, **FIELD_CFG)
    assert b.det.field_cz != 0.0
    L = b.det.n_layers
    x, y, z, lay = b.event_hits(0)
    prm, cov, _ = b.event_seeds(0)
    lists, n = true_hit_lists(b, 0, L)
    lists, n = lists[b.seed_sim][:5], n[b.seed_sim][:5]
    prm, cov = prm[:, :5].astype(np.float64), cov[:, :5].astype(np.float64)
    x, y, z = x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)
    al = b.align.astype(np.float64)
    tot, ga, gh, gs, _ = oracle.fit_grad(b.det, prm, cov, lists, n, x, y, z, lay, al)

    def total(prm_, x_, y_, z_, al_, det=b.det):
        return oracle.fit(det, prm_, cov, lists, n, x_, y_, z_, lay, align=al_)[2].sum()

    assert abs(total(prm, x, y, z, al) - tot) < 1e-9 * tot
    # the field changes the fit: the chi2 in the uniform field differs
    uni = dataclasses.replace(b.det, field_cz=0.0, field_cr=0.0)
    assert abs(total(prm, x, y, z, al, uni) - tot) > 1e-3 * tot
    h = 1e-6
    for hidx in lists[0, [0, 4, 9]]:
        for arr_i in range(3):
            a1 = [x.copy(), y.copy(), z.copy()]
            a2 = [x.copy(), y.copy(), z.copy()]
            a1[arr_i][hidx] += h
            a2[arr_i][hidx] -= h
            fd = (total(prm, *a1, al) - total(prm, *a2, al)) / (2 * h)
            assert abs(fd - gh[hidx, arr_i]) < 1e-5 * max(1.0, abs(fd)), (hidx, arr_i, fd, gh[hidx, arr_i])
    for t in range(2):
        for k in range(6):
            p1, p2 = prm.copy(), prm.copy()
            p1[k, t] += h
            p2[k, t] -= h
            fd = (total(p1, x, y, z, al) - total(p2, x, y, z, al)) / (2 * h)
            assert abs(fd - gs[t, k]) < 1e-5 * max(1.0, abs(fd)), (t, k, fd, gs[t, k])
    for li, c in [(5, 0), (12, 1)]:
        a1, a2 = al.copy(), al.copy()
        a1[li, c] += h
        a2[li, c] -= h
        fd = (total(prm, x, y, z, a1) - total(prm, x, y, z, a2)) / (2 * h)
        assert abs(fd - ga[li, c]) < 1e-5 * max(1.0, abs(fd))


def test_finding_in_a_parameterized_field():
    """No noise, 100 tracks simulated through the field in fine steps: the
    single-step model finds at least 98% of the seeds' true hits exactly."""
    b = make_batch("c0", eta_max=1.5, **FIELD_CFG)
    r = oracle.find_event(b, 0)
    th = b.track_hits[0]
    good = 0
    for s in range(b.n_seeds):
        t = th[b.seed_sim[s]]
        t = t[t >= 0]
        good += (r["n_found"][s] == t.size) and np.array_equal(r["hits"][s, :t.size], t)
    assert good >= 0.98 * b.n_seeds
