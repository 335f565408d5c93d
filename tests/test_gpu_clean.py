"""GPU parity of duplicate handling beyond the shared-hit fraction (Sec. 4.2):
seed cleaning before finding and the pT/eta/phi pre-cuts of duplicate
removal, against the FP64 oracle.

The cuts decide integers (which seeds and tracks survive) from FP32 inputs:
the oracle evaluates them in double, the kernels in FP32.  Every comparison
below first checks that the decision is unique: the oracle gives the same
keep flags with each cut shrunk and grown by 1e-5 relative, so no pair lies
within rounding distance of a cut.  The flags must then agree exactly.
"""
import numpy as np
import pytest

import oracle
from kfhelp import tracker_for
from synth import make_batch

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _seed_clean_ref(b, e, cuts):
    deta, dphi, dpt, ms = cuts
    prm, _, sh = b.event_seeds(e)
    p = prm.T.astype(np.float64)
    keeps = [oracle.seed_clean(p, sh.T, float(np.float32(b.det.bz)), deta * f, dphi * f, dpt * f, ms)
             for f in (1.0, 1.0 - EPS, 1.0 + EPS)]
    assert all(np.array_equal(keeps[0], k) for k in keeps[1:]), "a seed pair lies on a cut"
    return keeps[0]


def _dedup_ref(b, trk, a, c, cuts):
    deta, dphi, dpt = cuts
    p = trk["params"][:, a:c].T.astype(np.float64)
    keeps = [oracle.dedup(trk["hits"][a:c], trk["n_found"][a:c], trk["chi2"][a:c].astype(np.float64), 0.5,
                          params=p, bz=float(np.float32(b.det.bz)), deta=deta * f, dphi=dphi * f, dpt=dpt * f)
             for f in (1.0, 1.0 - EPS, 1.0 + EPS)]
    assert all(np.array_equal(keeps[0], k) for k in keeps[1:]), "a track pair lies on a cut"
    return keeps[0]


SEED_CUTS = [(0.05, 0.05, 0.0, 1), (0.02, 0.02, 0.5, 0), (0.01, 0.0, 0.3, 2)]


@pytest.mark.parametrize("cuts", SEED_CUTS)
@pytest.mark.parametrize("per_event", [0, 1])
def test_seed_clean_duplicate_seeds(cuts, per_event):
    """Duplicate-seed workload (10% of the tracks seeded twice, on layers 1-3
    and 2-4): the seeds the GPU drops are those the oracle drops, a dropped
    seed gives an empty track that is not kept, and every kept seed's track
    is the one found without cleaning."""
    import torch
    b = make_batch("c1b")
    deta, dphi, dpt, ms = cuts
    t = tracker_for(b, device=torch.device("cuda:0"), per_event=per_event, seed_clean=1, seed_deta=deta,
                    seed_dphi=dphi, seed_dpt=dpt, seed_min_shared=ms)
    t.find_tracks()
    trk = t.get_tracks()
    cnt = t.counters()
    t.close()
    ref = _seed_clean_ref(b, 0, cuts)
    got = (trk["n_found"] > 0).astype(np.uint8)
    assert np.array_equal(got, ref), np.nonzero(got != ref)[0][:10]
    assert ref.sum() < ref.size
    assert np.all(trk["keep"][ref == 0] == 0)
    assert np.all(trk["hits"][ref == 0] == -1)
    assert cnt["seeds"] == int(ref.sum())
    t0 = tracker_for(b, device=torch.device("cuda:0"), per_event=per_event)
    t0.find_tracks()
    base = t0.get_tracks()
    t0.close()
    k = ref == 1
    assert np.array_equal(trk["hits"][k], base["hits"][k])
    assert np.array_equal(trk["n_found"][k], base["n_found"][k])
    assert np.array_equal(trk["chi2"][k], base["chi2"][k])


def test_seed_clean_pileup_events():
    """Three PU-200 events (8,000 seeds each), cleaning on kinematics alone
    (no shared hit required): the dropped seeds match the oracle per event."""
    import torch
    b = make_batch("c4", n_events=3)
    cuts = (0.01, 0.01, 0.2, 0)
    t = tracker_for(b, device=torch.device("cuda:0"), lanes_per_seed=10, seed_clean=1, seed_deta=cuts[0],
                    seed_dphi=cuts[1], seed_dpt=cuts[2], seed_min_shared=cuts[3])
    t.find_tracks()
    trk = t.get_tracks()
    t.close()
    dropped = 0
    for e in range(3):
        a, c = b.seed_off[e], b.seed_off[e + 1]
        ref = _seed_clean_ref(b, e, cuts)
        got = (trk["n_found"][a:c] > 0).astype(np.uint8)
        assert np.array_equal(got, ref), (e, np.nonzero(got != ref)[0][:10])
        dropped += int((ref == 0).sum())
    assert dropped > 0


@pytest.mark.parametrize("cuts", [(0.01, 0.01, 0.2), (0.002, 0.0, 0.0), (0.0, 0.003, 0.05)])
@pytest.mark.parametrize("per_event", [0, 1])
def test_dedup_kinematic_precuts(cuts, per_event):
    """Duplicate removal with the pT/eta/phi pre-cuts on the found tracks of
    the duplicate-seed workload: keep flags equal the oracle's greedy walk on
    the same tracks; the pre-cuts keep pairs that the shared fraction alone
    would remove."""
    import torch
    b = make_batch("c1b")
    t = tracker_for(b, device=torch.device("cuda:0"), per_event=per_event, dup_deta=cuts[0], dup_dphi=cuts[1],
                    dup_dpt=cuts[2])
    t.find_tracks()
    t.remove_duplicates()
    trk = t.get_tracks()
    t.close()
    ref = _dedup_ref(b, trk, 0, trk["n_found"].size, cuts)
    assert np.array_equal(trk["keep"], ref), np.nonzero(trk["keep"] != ref)[0][:10]
    plain = oracle.dedup(trk["hits"], trk["n_found"], trk["chi2"].astype(np.float64), 0.5)
    assert ref.sum() >= plain.sum()


def test_clean_dedup_fit_graph_pipeline():
    """Seed cleaning + duplicate removal with pre-cuts + fit + adjoint in one
    captured graph over a multi-event batch: the same tracks, keep flags and
    fit as the eager calls; the stage timer reports the cleaning stage."""
    import torch
    b = make_batch("c4", n_events=4)
    kw = dict(lanes_per_seed=10, seed_clean=1, seed_deta=0.01, seed_dphi=0.01, seed_dpt=0.2,
              seed_min_shared=0, dup_deta=0.02, dup_dphi=0.02, dup_dpt=0.3)
    dev = torch.device("cuda:0")
    t = tracker_for(b, device=dev, **kw)
    t.find_tracks()
    t.remove_duplicates()
    t.fit_tracks()
    eager_trk, eager_fit = t.get_tracks(), t.get_fit()
    t.close()
    g = tracker_for(b, device=dev, **kw)
    s = torch.cuda.Stream()
    g.set_stage_timing(True)
    g.capture_graph(with_adjoint=True, stream=s)
    g.launch_graph(s)
    st = g.stage_ms(s)
    trk, fit = g.get_tracks(), g.get_fit()
    g.close()
    assert "seed_clean" in st and st["seed_clean"] > 0
    for k in ("hits", "n_found", "chi2", "keep"):
        assert np.array_equal(trk[k], eager_trk[k]), k
    # the graph fits beside duplicate removal and clears the removed tracks
    # afterwards: every fit output equals the eager calls'
    for k in ("status", "chi2", "params", "cov"):
        assert np.array_equal(fit[k], eager_fit[k]), k
    assert (trk["n_found"] == 0).sum() > 0
    assert (~trk["keep"].astype(bool)).sum() > 0 and np.all(fit["params"][:, ~trk["keep"].astype(bool)] == 0)
    g = tracker_for(b, device=dev, **kw)  # the same without the adjoint (careful fit in the graph's main branch)
    g.capture_graph(with_adjoint=False, stream=s)
    g.launch_graph(s)
    s.synchronize()
    fit2 = g.get_fit()
    g.close()
    for k in ("status", "chi2", "params", "cov"):
        assert np.array_equal(fit2[k], eager_fit[k]), k
    for e in range(4):
        a, c = b.seed_off[e], b.seed_off[e + 1]
        ref = _dedup_ref(b, trk, a, c, (0.02, 0.02, 0.3))
        assert np.array_equal(trk["keep"][a:c], ref), e


def test_seed_clean_capacity_error_and_empty_event():
    """More than 16 lower-index duplicates of one seed is a capacity error
    (reported through the status word, not a fault); an event without seeds
    is cleaned without error."""
    from paper_1906_11744_gb300 import KFError, Tracker, make_config, make_detector
    b = make_batch("c1", tracks=200)
    prm = b.params.copy()
    sh = b.seed_hits.copy()
    prm[:, 1:20] = prm[:, :1]   # 20 copies of seed 0
    sh[:, 1:20] = sh[:, :1]
    d = b.det
    det = make_detector(d.radius, d.x0, d.z_max, d.bz, d.sigma_rphi, d.sigma_z)
    t = Tracker(det, make_config(max_cands=6, seed_clean=1, seed_min_shared=3))
    t.load_hits(b.hit_off, b.x, b.y, b.z, b.layer)
    t.load_seeds(b.seed_off, prm, b.cov, sh)
    t.find_tracks()
    with pytest.raises(KFError, match="seed cleaning"):
        t.get_tracks()
    t.close()
    # two events, the second without seeds
    hit_off = np.array([0, b.x.size, 2 * b.x.size], np.int32)
    seed_off = np.array([0, b.seed_off[1], b.seed_off[1]], np.int32)
    t = Tracker(det, make_config(max_cands=6, seed_clean=1))
    t.load_hits(hit_off, np.tile(b.x, 2), np.tile(b.y, 2), np.tile(b.z, 2), np.tile(b.layer, 2))
    t.load_seeds(seed_off, b.params, b.cov, b.seed_hits)
    t.find_tracks()
    trk = t.get_tracks()
    t.close()
    assert (trk["n_found"] > 0).all()


def _chain_of_seeds(n=400):
    """One event whose seeds form a chain: seed k uses hits (k, k+1, k+2) and
    all seeds have one state, so with two shared hits required seed k
    conflicts only with seed k - 1; the greedy walk keeps every other seed."""
    b = make_batch("c1", tracks=200)
    x, y, z, lay = (a[: n + 2].copy() for a in b.event_hits(0))
    prm = np.repeat(b.params[:, :1], n, axis=1)
    cov = np.repeat(b.cov[:, :1], n, axis=1)
    sh = np.stack([np.arange(n), np.arange(n) + 1, np.arange(n) + 2]).astype(np.int32)
    return b.det, x, y, z, lay, prm, cov, sh


def _clean_chain(resolve_max_rounds):
    from paper_1906_11744_gb300 import Tracker, make_config, make_detector
    d, x, y, z, lay, prm, cov, sh = _chain_of_seeds()
    det = make_detector(d.radius, d.x0, d.z_max, d.bz, d.sigma_rphi, d.sigma_z)
    t = Tracker(det, make_config(max_cands=6, seed_clean=1, seed_deta=0.01, seed_dphi=0.01, seed_min_shared=2,
                                 resolve_max_rounds=resolve_max_rounds))
    t.load_hits(np.array([0, x.size], np.int32), x, y, z, lay)
    t.load_seeds(np.array([0, prm.shape[1]], np.int32), prm, cov, sh)
    t.find_tracks()
    return t, d, prm, sh


def test_resolution_round_cap_reports_a_timeout():
    """The bounded device-side loop of seed cleaning (and duplicate removal)
    gives up after resolve_max_rounds rounds: the next synchronizing call
    returns KF_ERR_TIMEOUT, and the context stays usable.  Without a cap the
    same chain settles to the oracle's greedy result (every other seed)."""
    from paper_1906_11744_gb300 import KFError
    from paper_1906_11744_gb300._lib import KF_ERR_TIMEOUT
    t, d, prm, sh = _clean_chain(0)
    dropped = t.get_tracks()["n_found"] == 0
    t.close()
    ref = oracle.seed_clean(prm.T.astype(np.float64), sh.T, float(np.float32(d.bz)), 0.01, 0.01, 0.0, 2)
    assert np.array_equal(dropped, ref == 0)
    assert np.array_equal(ref, (np.arange(prm.shape[1]) % 2 == 0).astype(np.uint8))
    t, d, prm, sh = _clean_chain(1)
    with pytest.raises(KFError, match=f"\\({KF_ERR_TIMEOUT}\\).*seed cleaning"):
        t.get_tracks()
    # the status was reported once and cleared: the context works again
    t.find_tracks()
    with pytest.raises(KFError, match="seed cleaning"):
        t.get_tracks()
    t.close()
