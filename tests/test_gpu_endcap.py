"""Endcap disks and eta regions on the GPU against the oracle (Sec. 2: the
detector's barrel layers and endcap disks, each event split into eta regions;
the oracle's reading is pinned by tests/test_oracle_endcap.py).

The fit over barrel and disk hits (plane steps, (r-phi, r) measurements, the
disks' scattering and energy loss) must meet the barrel fit's tolerances; the
finding over the region plans (barrel seeds: barrel layers; forward seeds:
barrel layers, then their side's disks, passing surfaces they do not cross)
must give the oracle's hit lists; the adjoint of the fit over disk hits must
match the oracle's dual-number gradient."""
import dataclasses

import numpy as np
import pytest

import oracle
from kfhelp import TIE_REL, cov_close, found_cov_close, param_close, tracker_for
from synth import make_batch
from synth.events import true_hit_lists

pytestmark = pytest.mark.gpu


def _disk_local_close(gpu_c21, ref_c21, ref_p):
    """Covariances after a disk: compared in the plane's frame (x, y, q/pT,
    phi, theta; the z row is structurally zero), correlation-scaled."""
    from kfhelp import TOL
    g = oracle.sym_to_full(gpu_c21)
    r = oracle.sym_to_full(ref_c21)
    idx = [0, 1, 3, 4, 5]
    gl, rl = g[:, idx][:, :, idx], r[:, idx][:, :, idx]
    d = np.sqrt(np.abs(np.einsum("nii->ni", rl)))
    err = np.abs(gl - rl) / np.maximum(d[:, :, None] * d[:, None, :], 1e-30)
    ok = np.all(err <= TOL, axis=(1, 2)) & (np.abs(g[:, 2, :]).max(axis=1) == 0.0)
    return ok, float(err.max()) if err.size else 0.0


@pytest.mark.parametrize("eloss", [0.0, 2e-3])
def test_fit_over_barrel_and_disk_hits(eloss):
    """True hit lists of the barrel-plus-endcap event (forward tracks end on
    disks), fitted on the GPU and in the oracle: parameters within 1e-4,
    covariances within 1e-4 correlation-scaled (in the plane's frame for tracks
    that end on a disk), chi2 within 1e-3."""
    from paper_1906_11744_gb300 import KF_FIT_GIVEN
    b = make_batch("c5")
    if eloss:
        b = dataclasses.replace(b, det=dataclasses.replace(b.det, disk_eloss=eloss))
    S, L = b.det.n_surfaces, b.det.n_layers
    lists, n = true_hit_lists(b, 0, S)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    t = tracker_for(b)
    t.fit_tracks(KF_FIT_GIVEN, lists, n)
    g = t.get_fit()
    x, y, z, lay = b.event_hits(0)
    p, C, c2, st = oracle.fit(b.det, b.params, b.cov, lists, n, x, y, z, lay, align=b.align)
    both = (st == 0) & (g["status"] == 0)
    assert both.mean() > 0.999
    last = lay[lists[np.arange(len(n)), n - 1]]
    on_disk = both & (last >= L)
    on_layer = both & (last < L)
    assert on_disk.sum() > 0.3 * len(n)
    okp, ep = param_close(g["params"].T[both], p[both])
    okc, ec = cov_close(g["cov"].T[on_layer], C[on_layer], p[on_layer])
    okd, ed = _disk_local_close(g["cov"].T[on_disk], C[on_disk], p[on_disk])
    print(f"disk fit: {on_disk.sum()} end on a disk, params {ep:.2e}, cov {ec:.2e} / disk {ed:.2e}")
    assert okp.all(), ep
    assert okc.all(), ec
    assert okd.all(), ed
    assert np.allclose(g["chi2"][both], c2[both], rtol=1e-3, atol=1e-2)
    assert np.all(g["status"][st != 0] != 0)


def _find_case(noise=0.10, **cfg):
    b = make_batch("c5", noise=noise)
    t = tracker_for(b, **cfg)
    t.find_tracks()
    return b, t.get_tracks(), t


def _audit(b, trk, ref):
    """Identical hit lists, else an equal-length tie of chi2 sums on both
    sides (each side's own sum) within TIE_REL."""
    same = np.all(trk["hits"] == ref["hits"], axis=1)
    bad = []
    for i in np.nonzero(~same)[0]:
        tie = trk["n_found"][i] == ref["n_found"][i] and \
            abs(trk["chi2"][i] - ref["chi2"][i]) <= TIE_REL * max(abs(ref["chi2"][i]), 1.0)
        if not tie:
            bad.append((int(i), int(trk["n_found"][i]), int(ref["n_found"][i]), float(trk["chi2"][i]),
                        float(ref["chi2"][i])))
    return same, bad


def test_find_over_region_plans():
    """The barrel-plus-endcap event (2,500 tracks, |eta| < 2.4, 10% noise):
    hit lists identical to the oracle's for at least 99.5% of the seeds, every
    other one an equal-length chi2 tie; found parameters within 1e-4;
    barrel-region seeds hold no disk hit, forward seeds only their own side's."""
    b, trk, _ = _find_case()
    ref = oracle.find_event(b, 0)
    same, bad = _audit(b, trk, ref)
    print(f"endcap find: {same.sum()}/{b.n_seeds} identical, unexplained {bad[:5]}")
    assert not bad, bad[:10]
    assert same.mean() >= 0.995
    okp, ep = param_close(trk["params"].T[same], ref["p"][same])
    assert okp.all(), ep
    prm, _, _ = b.event_seeds(0)
    x, y, z, lay = b.event_hits(0)
    L, D = b.det.n_layers, b.det.n_disks
    eta = -np.log(np.tan(0.5 * prm[5].astype(np.float64)))
    n_disk = 0
    for s in range(b.n_seeds):
        f = trk["hits"][s, :trk["n_found"][s]]
        surf = lay[f]
        if abs(eta[s]) < b.det.eta_barrel:
            assert np.all(surf < L)
        elif eta[s] > 0:
            assert np.all(surf < L + D)
        else:
            assert np.all((surf < L) | (surf >= L + D))
        n_disk += (surf >= L).any()
    assert n_disk > 0.5 * b.n_seeds


def test_pu200_endcap_events_in_the_graph():
    """Two whole PU-200-like barrel-plus-endcap events (16,000 seeds, |eta| <
    2.4, 20% noise, N = 10: the benchmark's endcap workload) through the
    benchmark's graph (binning, finding over the region plans, duplicate
    removal, fit, adjoint): hit lists identical to the oracle's for at least
    99.5% of the seeds, every other one an equal-length chi2 tie; found
    parameters within 1e-4."""
    import torch
    from kfhelp import oracle_find_events
    b = make_batch("c6", n_events=2)
    t = tracker_for(b, device=torch.device("cuda:0"))
    s = torch.cuda.Stream()
    t.capture_graph(with_adjoint=True, stream=s)
    t.launch_graph(stream=s)
    s.synchronize()
    trk = t.get_tracks()
    t.close()
    ref, _ = oracle_find_events(b, [0, 1])
    n_same, n_all, bad = 0, 0, []
    for e in (0, 1):
        a, c = b.seed_off[e], b.seed_off[e + 1]
        g = {k: trk[k][a:c] for k in ("hits", "n_found", "chi2")}
        same, bad_e = _audit(b, g, ref[e])
        n_same += int(same.sum())
        n_all += c - a
        bad += [(e,) + x for x in bad_e]
        okp, ep = param_close(trk["params"].T[a:c][same], ref[e]["p"][same])
        assert okp.all(), ep
    print(f"PU-200 endcap: {n_same}/{n_all} identical, unexplained {bad[:5]}")
    assert not bad, bad[:10]
    assert n_same >= 0.995 * n_all


def test_find_endcap_variants_agree():
    """Lanes per seed 6 and 16, the register-capped kernel and the per-event
    (plain) form give identical tracks on the endcap event; so does a
    captured graph (finding, duplicate removal and fit)."""
    import torch
    b, base, _ = _find_case(noise=0.05)
    for cfg in (dict(lanes_per_seed=16), dict(find_regcap=1), dict(per_event=1)):
        _, trk, _ = _find_case(noise=0.05, **cfg)
        for k in ("hits", "n_found", "chi2", "params"):
            assert np.array_equal(trk[k], base[k]), (cfg, k)
    t = tracker_for(b, device=torch.device("cuda:0"))
    s = torch.cuda.Stream()
    t.capture_graph(with_adjoint=False, stream=s)
    t.launch_graph(stream=s)
    s.synchronize()
    g = t.get_tracks()
    for k in ("hits", "n_found", "chi2", "params"):
        assert np.array_equal(g[k], base[k]), k


def _adjoint_helpers():
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location("adj", os.path.join(os.path.dirname(__file__), "test_gpu_adjoint.py"))
    adj = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(adj)
    return adj


@pytest.mark.parametrize("case", ["plain", "eloss", "field"])
def test_adjoint_over_disk_hits(case):
    """The adjoint of the fit over barrel and disk hits (plane steps, (r-phi,
    r) measurements, disk scattering; with energy loss on the disks; in a
    parameterized field, whose term moves with each plane step's starting
    point) against the oracle's dual-number gradient: norm-wise within 1e-3
    and per component within 1e-3 relative plus 8 FP32 rounding scales (as
    tests/test_gpu_adjoint.py), also per hit vector.  Disk hits get no z
    gradient and no alignment gradient.  1,000 tracks: about ten loopers
    whose step onto a disk runs in double, and hits next to the x or y axis,
    whose small lab-frame gradient component needs the library sine of the
    fit (with the hardware sine, a direction 0.01 rad from an axis moved the
    prediction across it by 4e-7 of the step and such a component left the
    bound four-fold)."""
    from paper_1906_11744_gb300 import KF_FIT_GIVEN
    adj = _adjoint_helpers()
    b = make_batch("c5", tracks=1000)
    if case == "eloss":
        b = dataclasses.replace(b, det=dataclasses.replace(b.det, disk_eloss=2e-3))
    if case == "field":
        b = dataclasses.replace(b, det=dataclasses.replace(b.det, field_cz=-3.0e-6, field_cr=-5.0e-6))
    S, L = b.det.n_surfaces, b.det.n_layers
    lists, n = true_hit_lists(b, 0, S)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    t = tracker_for(b)
    t.fit_tracks(KF_FIT_GIVEN, lists, n)
    ok = t.get_fit()["status"] == 0
    x, y, z, lay = b.event_hits(0)
    sel = np.nonzero(ok)[0]
    on_disk = np.array([lay[lists[i, n[i] - 1]] >= L for i in sel])
    assert on_disk.sum() > 50
    g_align = np.zeros((L, 2), np.float32)
    g_hits = np.zeros((b.n_hits, 3), np.float32)
    g_seed = np.zeros((6, b.n_seeds), np.float32)
    t.fit_adjoint(g_align, g_hits, g_seed)
    (tot, ga, gh, gs, each), sig = adj._fp32_sigma(b, sel, lists, n)
    errs = [adj._close(g_align, ga)[0], adj._close(g_hits, gh)[0], adj._close(g_seed[:, sel].T, gs)[0]]
    comp = [adj._component_ok(g_align, ga, sig[0]), adj._component_ok(g_hits, gh, sig[1]),
            adj._component_ok(g_seed[:, sel].T, gs, sig[2])]
    dh = np.linalg.norm(g_hits.astype(np.float64) - gh, axis=1)
    bh = 1e-3 * np.linalg.norm(gh, axis=1) + 8.0 * np.linalg.norm(sig[1], axis=1)
    hit_ratio = float((dh / np.maximum(bh, 1e-300)).max())
    print(f"disk adjoint ({case}): norm-wise {errs}, inside plain 1e-3 {[c[1] for c in comp]}, "
          f"component bound ratios {[c[2] for c in comp]}, hit-vector bound ratio {hit_ratio:.2f}")
    assert max(errs) < 1e-3
    assert all(c[0] for c in comp), comp
    assert hit_ratio <= 1.0
    assert np.all(g_hits[lay >= L, 2] == 0.0)
    assert np.abs(g_hits[lay >= L, :2]).max() > 0.0


def test_duplicate_handling_on_endcap_tracks():
    """Seed cleaning and duplicate removal with the pT/eta/phi pre-cuts on
    the barrel-plus-endcap event with duplicate seeds for 10% of the tracks
    (Sec. 4.2): the seeds dropped and the tracks kept equal the oracle's on
    the same inputs (each decision first shown unique under 1e-5 changes of
    the cuts); duplicates are removed in the forward regions too."""
    import importlib.util
    import os
    import torch
    spec = importlib.util.spec_from_file_location("clean", os.path.join(os.path.dirname(__file__),
                                                                         "test_gpu_clean.py"))
    clean = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(clean)
    b = make_batch("c5", dup_seed_frac=0.10)
    seed_cuts = (0.05, 0.05, 0.0, 1)
    dup_cuts = (0.02, 0.02, 0.3)
    t = tracker_for(b, device=torch.device("cuda:0"), seed_clean=1, seed_deta=seed_cuts[0],
                    seed_dphi=seed_cuts[1], seed_dpt=seed_cuts[2], seed_min_shared=seed_cuts[3],
                    dup_deta=dup_cuts[0], dup_dphi=dup_cuts[1], dup_dpt=dup_cuts[2])
    t.find_tracks()
    t.remove_duplicates()
    trk = t.get_tracks()
    t.close()
    ref_seeds = clean._seed_clean_ref(b, 0, seed_cuts)
    assert np.array_equal((trk["n_found"] > 0).astype(np.uint8), ref_seeds)
    ref_keep = clean._dedup_ref(b, trk, 0, trk["n_found"].size, dup_cuts)
    assert np.array_equal(trk["keep"], ref_keep), np.nonzero(trk["keep"] != ref_keep)[0][:10]
    prm, _, _ = b.event_seeds(0)
    eta = -np.log(np.tan(0.5 * prm[5].astype(np.float64)))
    fwd = np.abs(eta) >= b.det.eta_barrel
    removed = (trk["n_found"] > 0) & (trk["keep"] == 0)
    print(f"endcap duplicates: {int((ref_seeds == 0).sum())} seeds cleaned, {int(removed.sum())} tracks "
          f"removed ({int((removed & fwd).sum())} forward)")
    assert (removed & fwd).sum() > 0


def test_endcap_work_counters_equal_the_oracles():
    """The finding's work counters on the barrel-plus-endcap event equal the
    oracle's on the same inputs (the multipliers of the endcap step's
    algorithmic flop count): candidate-layer steps, seeds and the steps onto
    disks exactly; updates and holes, with their disk parts, within 1e-4
    (near-tied children of candidates that do not win may move)."""
    b = make_batch("c5")
    t = tracker_for(b)
    t.find_tracks()
    c = t.counters()
    r = oracle.find_event(b, 0)["counters"]
    print("endcap counters:", {k: (c[k], r[k]) for k in ("steps", "disk_steps", "updates", "disk_updates",
                                                         "holes", "disk_holes", "seeds")})
    for k in ("steps", "seeds", "disk_steps"):
        assert c[k] == r[k], (k, c[k], r[k])
    for k in ("updates", "holes", "disk_updates", "disk_holes"):
        assert abs(c[k] - r[k]) <= 1e-4 * r[k] + 2, (k, c[k], r[k])
    assert r["disk_steps"] > 0.2 * r["steps"]
