"""Pins of the oracle's candidate selection in the finding (Sec. 2 building,
Sec. 4.3 candidate scores; readings recorded in the design notes).

The ranking key of a child, most significant first:
  1. more hits;
  2. lower chi2 sum;
  3. lower parent rank;
  4. kind: hit before hole before carried;
  5. lower hit index.
The best N children become the next candidates.  A live candidate makes one
child per compatible hit (chi2 < cut) and a hole child while it has fewer
than max_holes holes.  A candidate with neither stops and is carried
unchanged.  A candidate that does not cross the layer inside |z| <= z_max is
carried too.

Two kinds of test:
  * hand-made child lists in which each key level alone decides the order;
  * tiny events (four layers after the seed; extra hits beside true hits,
    exact duplicate hits, missing hits) where a brute-force beam written here
    from the definition must equal the oracle's finding exactly, for several
    N and max_holes.  The brute force expands every child of every kept path
    and recomputes each path's chi2 from scratch through the oracle's replay
    of a decision list, so it shares no incremental state with the finder.
"""
import dataclasses
from collections import Counter

import numpy as np
import pytest

import oracle
from synth import make_batch

HIT, HOLE, CARRIED = 0, 1, 2


def _sel(children, n):
    """children: list of (n_found, chi2, parent, kind, hit)."""
    cols = list(zip(*children))
    return oracle.select_children(*cols, n)


def test_each_key_level_decides_alone():
    # 1. more hits beats a lower chi2 sum
    assert _sel([(4, 1.0, 0, HIT, 3), (5, 20.0, 1, HIT, 9)], 2) == [1, 0]
    # 2. lower chi2 sum beats a lower parent rank
    assert _sel([(5, 3.0, 0, HIT, 1), (5, 2.0, 3, HIT, 9)], 2) == [1, 0]
    # 3. lower parent rank beats kind (a hole of parent 1 before a hit of parent 2)
    assert _sel([(5, 2.0, 2, HIT, 1), (5, 2.0, 1, HOLE, -1)], 2) == [1, 0]
    # 4. kind: hit before hole before carried, whatever the hit index
    assert _sel([(5, 2.0, 1, CARRIED, -1), (5, 2.0, 1, HOLE, -1), (5, 2.0, 1, HIT, 999)], 3) == [2, 1, 0]
    # 5. lower hit index
    assert _sel([(5, 2.0, 1, HIT, 12), (5, 2.0, 1, HIT, 7)], 2) == [1, 0]


def test_truncation_keeps_the_best_n_in_rank_order():
    ch = [(4, 9.0, 0, HOLE, -1), (5, 7.5, 1, HIT, 4), (5, 7.5, 0, HIT, 8), (3, 0.5, 2, CARRIED, -1),
          (5, 1.0, 2, HIT, 2), (4, 2.0, 1, HOLE, -1)]
    expect = [4, 2, 1, 5, 0, 3]  # by (hits desc, chi2, parent, kind, hit)
    for n in range(1, 7):
        assert _sel(ch, n) == expect[:n]
    assert _sel(ch, 16) == expect


# ---------------------------------------------------------------- brute force
def _tiny_event(seed, n_tracks=8):
    """One event, 7 layers (seed on 0-2, four layers searched), |eta| < 1.2.
    Edits: beside a third of the true hits on layers 3-6 an extra hit at
    1.5-4 sigma in r-phi and z; an exact copy of a fifth of them (equal chi2,
    so the parent-rank and hit-index levels decide); a sixth removed (holes,
    stops).  z_max = 30 cm, so that steep tracks leave the barrel."""
    b = make_batch("c1", n_events=1, tracks=n_tracks, n_layers=7, r_max=40.0, eta_max=1.2, noise=0.0,
                   seed=seed)
    rng = np.random.default_rng(seed)
    x, y, z, lay = (a.astype(np.float64) for a in b.event_hits(0))
    lay = lay.astype(np.int32)
    keep = np.ones(x.size, bool)
    seed_hits = set(b.seed_hits.ravel().tolist())
    extra = []
    for h in range(x.size):
        if lay[h] < 3 or h in seed_hits:
            continue
        u = rng.uniform()
        R = np.hypot(x[h], y[h])
        if u < 0.33:
            dphi = rng.choice([-1, 1]) * rng.uniform(1.5, 4.0) * b.det.sigma_rphi / R
            ph = np.arctan2(y[h], x[h]) + dphi
            dz = rng.choice([-1, 1]) * rng.uniform(1.5, 4.0) * b.det.sigma_z
            extra.append((R * np.cos(ph), R * np.sin(ph), z[h] + dz, lay[h]))
        elif u < 0.53:
            extra.append((x[h], y[h], z[h], lay[h]))
        elif u < 0.70:
            keep[h] = False
    # Removing hits renumbers the event: keep the seed hits' indices valid by
    # moving removed hits far away (another layer side) instead of deleting.
    x[~keep] = -x[~keep]
    y[~keep] = -y[~keep]
    ex = np.array(extra, np.float64).reshape(-1, 4)
    X = np.concatenate([x, ex[:, 0]]).astype(np.float32)
    Y = np.concatenate([y, ex[:, 1]]).astype(np.float32)
    Z = np.concatenate([z, ex[:, 2]]).astype(np.float32)
    Lay = np.concatenate([lay, ex[:, 3].astype(np.int32)]).astype(np.int32)
    det = dataclasses.replace(b.det, z_max=30.0)
    return dataclasses.replace(b, det=det, x=X, y=Y, z=Z, layer=Lay,
                               hit_off=np.array([0, X.size], np.int32))


def _brute_beam(b, s, N, max_holes, stats, cut=30.0):
    det = b.det
    L = det.n_layers
    x, y, z, lay = b.event_hits(0)
    _, _, sh = b.event_seeds(0)
    start = int(lay[sh[2, s]]) + 1
    bz = float(np.float32(det.bz))
    z_max = float(np.float32(det.z_max))
    by_layer = {l: np.nonzero(lay == l)[0] for l in range(L)}

    def replay(dec_list):
        dec = np.full(L, -2, np.int32)
        dec[start:start + len(dec_list)] = dec_list
        st, c2, nf, chl, p, _ = oracle.replay_decisions(b, 0, s, dec)
        return st, c2, nf, chl, p

    st, c2, nf, _, p = replay([])
    cands = [dict(dec=[], nf=nf, holes=0, chi2=c2, fin=st != 0, p=p)]
    for l in range(start, L):
        R = float(np.float32(det.radius[l]))
        children = []
        for r, c in enumerate(cands):
            carried = dict(c, dec=c["dec"] + [-2], fin=True)
            if c["fin"]:
                children.append(((c["nf"], c["chi2"], r, CARRIED, -1), carried))
                continue
            ok, q, _ = oracle.propagate(bz, c["p"], R)
            if not ok or abs(q[2]) > z_max:
                stats["left"] += 1
                children.append(((c["nf"], c["chi2"], r, CARRIED, -1), carried))
                continue
            n_ch = 0
            for h in by_layer[l]:
                st, c2, nf, chl, p = replay(c["dec"] + [int(h)])
                stats["near_cut"] += st == 0 and cut <= chl[l] < cut + 1.0
                if st == 0 and chl[l] < cut:
                    children.append(((nf, c2, r, HIT, int(h)),
                                     dict(dec=c["dec"] + [int(h)], nf=nf, holes=c["holes"], chi2=c2, fin=False, p=p)))
                    n_ch += 1
            if c["holes"] < max_holes:
                st, c2, nf, chl, p = replay(c["dec"] + [-1])
                children.append(((c["nf"], c["chi2"], r, HOLE, -1),
                                 dict(dec=c["dec"] + [-1], nf=c["nf"], holes=c["holes"] + 1, chi2=c["chi2"],
                                      fin=False, p=p)))
                n_ch += 1
            if n_ch == 0:
                stats["stop"] += 1
                children.append(((c["nf"], c["chi2"], r, CARRIED, -1), carried))
        children.sort(key=lambda t: (-t[0][0], t[0][1], t[0][2], t[0][3], t[0][4]))
        keys = [k for k, _ in children]
        stats["truncated"] += len(children) > N
        stats["chi2_tie"] += sum(1 for a, c in zip(keys, keys[1:]) if a[0] == c[0] and a[1] == c[1])
        stats["parent_tie_decides"] += sum(1 for a, c in zip(keys[:N], keys[1:N + 1])
                                           if a[:2] == c[:2] and a[2] != c[2])
        stats["at_hole_limit"] += sum(1 for _, d in children[:N] if d["holes"] == max_holes)
        cands = [d for _, d in children[:N]]
    best = cands[0]
    hits = [int(h) for h in sh[:, s]] + [h for h in best["dec"] if h >= 0]
    return hits, best["nf"], best["chi2"]


@pytest.mark.parametrize("ev_seed", [11, 12, 13])
def test_finding_equals_brute_force_beam(ev_seed):
    b = _tiny_event(ev_seed)
    n_seeds = b.seed_off[1]
    stats = Counter()
    cases = [(N, holes, 30.0) for N in (1, 2, 3, 6) for holes in (0, 1, 3)]
    cases += [(N, holes, 8.0) for N in (2, 6) for holes in (1, 3)]  # many hits near this cut
    for N, max_holes, cut in cases:
        ref = oracle.find_event(b, 0, max_cands=N, max_holes=max_holes, chi2_cut=cut)
        for s in range(n_seeds):
            hits, nf, c2 = _brute_beam(b, s, N, max_holes, stats, cut=cut)
            row = ref["hits"][s]
            assert row[:nf].tolist() == hits and np.all(row[nf:] == -1), (N, max_holes, cut, s)
            assert ref["n_found"][s] == nf
            assert ref["chi2"][s] == pytest.approx(c2, rel=1e-12, abs=0.0)
    # the events exercise every rule
    assert stats["truncated"] > 0 and stats["chi2_tie"] > 0 and stats["stop"] > 0
    assert stats["at_hole_limit"] > 0 and stats["left"] > 0 and stats["near_cut"] > 0


def test_brute_force_events_have_parent_rank_ties():
    """Exact duplicate hits make two candidates with equal states; their
    children then tie on hits and chi2 and the parent rank decides."""
    stats = Counter()
    for ev_seed in (11, 12, 13):
        b = _tiny_event(ev_seed)
        for s in range(b.seed_off[1]):
            _brute_beam(b, s, 3, 3, stats)
    assert stats["parent_tie_decides"] > 0
