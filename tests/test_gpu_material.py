"""GPU parity with a material map (thickness per barrel layer at z nodes,
linear between them; Sec. 3's r-z material arrays): finding, fit and the
adjoint of the fit against the FP64 oracle given the same map.  The
tolerances are those of the runs without a map (test_gpu_parity.py,
test_gpu_adjoint.py); a map whose nodes all hold the layer's x0 must give
bit-identical results to no map.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from kfhelp import audit_mismatch, cov_close, param_close, tracker_for
from synth import make_batch
from synth.events import true_hit_lists

pytestmark = pytest.mark.gpu


def _with_map(b, n_z=9, seed=11):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.005, 0.06, size=(b.det.n_layers, n_z)).astype(np.float32)
    b.det = dataclasses.replace(b.det, x0_map=m)
    return b


def _close(g, ref):
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    scale = np.abs(ref).max()
    big = np.abs(ref) >= 1e-2 * scale
    comp = float((np.abs(g - ref)[big] / np.abs(ref)[big]).max()) if big.any() else 0.0
    return float(np.abs(g - ref).max() / scale), comp


def test_find_with_material_map():
    b = _with_map(make_batch("c1", tracks=600))
    t = tracker_for(b)
    t.find_tracks()
    trk = t.get_tracks()
    t.close()
    ref = oracle.find_event(b, 0)
    n = b.n_seeds
    mism = [i for i in range(n) if not np.array_equal(trk["hits"][i], ref["hits"][i])]
    unexplained = []
    for i in mism:
        ok, kind, rel = audit_mismatch(b, 0, i, trk["hits"][i], ref["hits"][i])
        if not ok:
            unexplained.append((i, rel))
    assert (n - len(mism)) / n >= 0.995
    assert not unexplained, unexplained[:10]
    same = np.array([i for i in range(n) if i not in set(mism)])
    okp, ep = param_close(trk["params"].T[same], ref["p"][same])
    assert okp.all(), ep


def test_fit_and_adjoint_with_material_map():
    from paper_1906_11744_gb300 import KF_FIT_GIVEN
    b = _with_map(make_batch("c3", tracks=300, seed=1003))
    L = b.det.n_layers
    lists, n = true_hit_lists(b, 0, L)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    t = tracker_for(b, ckpt_stride=2)
    t.fit_tracks(KF_FIT_GIVEN, lists, n)
    fit = t.get_fit()
    ok = fit["status"] == 0
    x, y, z, lay = b.event_hits(0)
    p, C, c2, st = oracle.fit(b.det, b.params, b.cov, lists, n, x, y, z, lay, align=b.align)
    both = ok & (st == 0)
    okp, ep = param_close(fit["params"].T[both], p[both])
    okc, ec = cov_close(fit["cov"].T[both], C[both], p[both])
    assert okp.all(), ep
    assert okc.all(), ec
    g_align = np.zeros((L, 2), np.float32)
    g_hits = np.zeros((b.n_hits, 3), np.float32)
    g_seed = np.zeros((6, b.n_seeds), np.float32)
    t.fit_adjoint(g_align, g_hits, g_seed)
    t.close()
    sel = np.nonzero(ok)[0]
    _, ga, gh, gs, _ = oracle.fit_grad(b.det, b.params[:, sel], b.cov[:, sel], lists[sel], n[sel],
                                       x, y, z, lay, b.align)
    for g, r in ((g_align, ga), (g_hits, gh), (g_seed[:, sel].T, gs)):
        e, c = _close(g, r)
        assert e < 1e-3 and c < 1e-2, (e, c)
    # the map's slope reaches the hit z gradient: without it the gradient differs
    flat = dataclasses.replace(b.det, x0_map=None)
    _, _, gh0, _, _ = oracle.fit_grad(flat, b.params[:, sel], b.cov[:, sel], lists[sel], n[sel],
                                      x, y, z, lay, b.align)
    assert np.abs(gh0 - gh).max() > 1e-2 * np.abs(gh).max()


def test_constant_map_equals_per_layer_thickness():
    """Nodes all holding the layer's x0: bit-identical tracks and fit."""
    b = make_batch("c1", tracks=400)
    t0 = tracker_for(b)
    t0.find_tracks()
    t0.fit_tracks()
    a_trk, a_fit = t0.get_tracks(), t0.get_fit()
    t0.close()
    flat = np.repeat(np.asarray(b.det.x0, np.float32)[:, None], 6, axis=1)
    b.det = dataclasses.replace(b.det, x0_map=flat)
    t1 = tracker_for(b)
    t1.find_tracks()
    t1.fit_tracks()
    b_trk, b_fit = t1.get_tracks(), t1.get_fit()
    t1.close()
    for k in ("hits", "n_found", "chi2", "params", "cov"):
        assert np.array_equal(a_trk[k], b_trk[k]), k
    for k in ("params", "cov", "chi2", "status"):
        assert np.array_equal(a_fit[k], b_fit[k]), k


def test_set_material_drops_the_graph_and_checks_arguments():
    import torch
    from paper_1906_11744_gb300 import KFError, kf_set_material
    b = make_batch("c0")
    t = tracker_for(b)
    s = torch.cuda.Stream()
    t.capture_graph(stream=s)
    t.launch_graph(s)
    s.synchronize()
    t.set_material(np.full((b.det.n_layers, 4), 0.02, np.float32))
    with pytest.raises(KFError):
        t.launch_graph(s)
    t.capture_graph(stream=s)  # capture again: works
    t.launch_graph(s)
    s.synchronize()
    with pytest.raises(KFError):
        kf_set_material(t.ctx, np.full((b.det.n_layers, 1), 0.02, np.float32))
    with pytest.raises(KFError):
        kf_set_material(t.ctx, np.full((b.det.n_layers, 4), -0.02, np.float32))
    t.set_material(None)
    t.close()
