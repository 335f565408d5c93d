"""Parity at the benchmark's full size and launch configuration.

The PU-200-like batch (100 events x 8,000 tracks, 20% noise, N = 10) runs as
the benchmark runs it: the finding kernel's launch shape chosen by the
autotuner, then one captured graph with binning, finding, duplicate removal,
fit and adjoint.  The oracle checks every seed of ten whole events (80,000 seeds, on all host
cores), duplicate flags of one whole event, fits and seed gradients of sampled
kept tracks, and the work counters of one whole event.
"""
import numpy as np
import pytest

import oracle
from kfhelp import TOL, audit_mismatch, cov_close, found_cov_close, jitter_audit, oracle_find_events, param_close, tracker_for
from synth import make_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pu200():
    import torch
    from paper_1906_11744_gb300 import kf_get_gradient
    b = make_batch("c4")
    dev = torch.device("cuda:0")
    t = tracker_for(b, device=dev)
    s = torch.cuda.Stream()
    t.autotune(s)
    t.capture_graph(with_adjoint=True, stream=s)
    t.launch_graph(stream=s)
    s.synchronize()
    trk = t.get_tracks()
    fit = t.get_fit()
    g_seed = np.zeros((6, b.n_seeds), np.float32)
    kf_get_gradient(t.ctx, g_seed=g_seed)
    counters = t.counters()
    t.close()
    return b, trk, fit, g_seed, counters


def test_sampled_found_tracks(pu200):
    b, trk, fit, g_seed, counters = pu200
    assert counters["seeds"] == b.n_seeds
    n_cmp = 0
    mism = []
    for e in (0, 37, 99):
        a = b.seed_off[e]
        ns = b.seed_off[e + 1] - a
        for lo in (0, ns // 2, ns - 100):
            ref = oracle.find_event(b, e, seeds=(lo, lo + 100))
            for i in range(100):
                n_cmp += 1
                if not np.array_equal(trk["hits"][a + lo + i], ref["hits"][i]):
                    mism.append((e, lo + i, trk["hits"][a + lo + i], ref["hits"][i]))
    assert n_cmp == 900
    assert len(mism) <= 0.005 * n_cmp, len(mism)
    for e, s, g, r in mism:
        ok, kind, rel = audit_mismatch(b, e, s, g, r)
        assert ok, (e, s, kind, rel)


def _most_tangent_seeds(b, events, per_event):
    """Seeds whose circle (from the seed parameters, centred at distance d with
    radius rho) crosses a searched layer R at the smallest cos(angle to the
    radial direction) = d sin(gamma) / R, cos(gamma) = (d^2 + rho^2 - R^2) / (2 d rho)."""
    K = 0.00299792458
    R = np.asarray(b.det.radius, np.float64)
    out = []
    for e in events:
        a, c = b.seed_off[e], b.seed_off[e + 1]
        p = b.params[:, a:c].astype(np.float64)
        h = -K * b.det.bz * p[3]
        cx = p[0] - np.sin(p[4]) / h
        cy = p[1] + np.cos(p[4]) / h
        d, rho = np.hypot(cx, cy), 1 / np.abs(h)
        cg = (d[:, None] ** 2 + rho[:, None] ** 2 - R[None, 3:] ** 2) / (2 * d[:, None] * rho[:, None])
        cos = np.where(np.abs(cg) <= 1, d[:, None] * np.sqrt(np.clip(1 - cg * cg, 0, 1)) / R[None, 3:], np.inf)
        order = np.argsort(cos.min(axis=1))[:per_event]
        out += [(e, int(s)) for s in order]
    return out


def test_near_tangent_loopers(pu200):
    """Low-pT loopers crossing outer layers close to tangentially: the finding
    redoes them with double-precision prediction, frame and update on those
    layers; their hit lists must equal the oracle's.  Seeds 391026, 581377 and
    741665 of this batch once accepted hits with FP64 chi2 above 1000."""
    b, trk, fit, g_seed, counters = pu200
    assert counters["not_pd"] == 0
    assert counters["careful"] > 0
    cases = [(int(np.searchsorted(b.seed_off, s, side="right") - 1), None, s) for s in (391026, 581377, 741665)]
    cases = [(e, s - b.seed_off[e]) for e, _, s in cases] + _most_tangent_seeds(b, (5, 50), 15)
    for e, ls in cases:
        ref = oracle.find_event(b, e, seeds=(ls, ls + 1))
        g = trk["hits"][b.seed_off[e] + ls]
        if not np.array_equal(g, ref["hits"][0]):
            ok, kind, rel = audit_mismatch(b, e, ls, g, ref["hits"][0])
            assert ok, (e, ls, kind, rel)


def test_whole_event_duplicate_flags(pu200):
    b, trk, fit, g_seed, counters = pu200
    e = 57
    a, c = b.seed_off[e], b.seed_off[e + 1]
    keep = oracle.dedup(trk["hits"][a:c], trk["n_found"][a:c], trk["chi2"][a:c].astype(np.float64), 0.5)
    assert np.array_equal(keep, trk["keep"][a:c])


def test_sampled_fits_and_seed_gradients(pu200):
    b, trk, fit, g_seed, counters = pu200
    for e in (3, 71):
        a = b.seed_off[e]
        x, y, z, lay = b.event_hits(e)
        idx = np.arange(a, a + 400, 2)
        kept = idx[(trk["keep"][idx] == 1) & (fit["status"][idx] == 0)]
        p, C, c2, st = oracle.fit(b.det, b.params[:, kept], b.cov[:, kept], trk["hits"][kept],
                                  trk["n_found"][kept], x, y, z, lay, align=b.align)
        ok = st == 0
        okp, ep = param_close(fit["params"][:, kept].T[ok], p[ok])
        okc, ec = cov_close(fit["cov"][:, kept].T[ok], C[ok], p[ok])
        assert okp.all(), ep
        assert okc.all(), ec
        sel = kept[ok][:60]
        tot, ga, gh, gs, each = oracle.fit_grad(b.det, b.params[:, sel], b.cov[:, sel], trk["hits"][sel],
                                                trk["n_found"][sel], x, y, z, lay, b.align)
        err = np.abs(g_seed[:, sel].T - gs).max() / np.abs(gs).max()
        assert err < 1e-3, err
    assert TOL == 1e-4


def test_ten_whole_events_against_oracle(pu200):
    """Every seed of ten whole PU-200 events: hit lists identical for at least
    99.5% of seeds; parameters and covariances of the identical ones within
    the fit tolerances.  Each mismatch is classified: a chi2-sum tie within
    1e-5 relative (the stated near-tie bound), or else a tie or a hit at the
    cut that one-ulp jitter of the hit coordinates shows to be unresolved at
    FP32 resolution (jitter_audit); none may be left unexplained."""
    b, trk, fit, g_seed, counters = pu200
    events = list(range(0, 100, 10))
    ref, _ = oracle_find_events(b, events)
    n_all = n_same = 0
    classes = {"tie<=1e-5": 0, "fp32-tie": 0}
    worst = 0.0
    for e in events:
        a = b.seed_off[e]
        r = ref[e]
        ns = r["hits"].shape[0]
        gh = trk["hits"][a:a + ns]
        same = np.all(gh == r["hits"], axis=1)
        n_all += ns
        n_same += int(same.sum())
        okp, ep = param_close(trk["params"][:, a:a + ns].T[same], r["p"][same])
        okc, ec = found_cov_close(trk["cov"][:, a:a + ns].T[same], r["C"][same], r["p"][same])
        assert okp.all(), (e, ep)
        assert okc.all(), (e, ec)
        for i in np.nonzero(~same)[0]:
            ok, kind, rel = audit_mismatch(b, e, i, gh[i], r["hits"][i])
            if kind == "tie" and rel <= 1e-5:
                classes["tie<=1e-5"] += 1
                continue
            ok2, rel2, spread = jitter_audit(b, e, i, gh[i], r["hits"][i])
            assert ok2, (e, i, kind, rel, spread)
            classes["fp32-tie"] += 1
            worst = max(worst, rel)
    rate = n_same / n_all
    print(f"ten PU-200 events: {n_same}/{n_all} seeds identical ({rate:.5f}); mismatches {classes}, "
          f"largest relative chi2-sum difference among the FP32 ties {worst:.2e}")
    assert n_all == 80000
    assert rate >= 0.995


def test_counters_equal_oracle_whole_event():
    """The kernels' work counters on one whole PU-200 event equal the oracle's
    (where a near-tie sends a candidate along another path the counts may
    differ by that path's steps; bounded at 1e-4 relative)."""
    b = make_batch("c4", n_events=1)
    t = tracker_for(b)
    t.find_tracks()
    g = t.counters()
    t.close()
    _, c = oracle_find_events(b, [0])
    for k in ("steps", "updates", "holes", "seeds"):
        assert abs(g[k] - c[k]) <= 1e-4 * c[k], (k, g[k], c[k])
    print("PU-200 event 0 counters (GPU, oracle):", {k: (g[k], c[k]) for k in ("steps", "updates", "holes", "seeds")})
