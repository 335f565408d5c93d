"""Per-unit operation counts of the finding and fitting steps, from the
oracle's operation census (test infrastructure; see orc_census_step).

The counts come from the oracle's own step functions run on a counting
scalar, on states sampled along true tracks of a seeded PU-200-like event
(the benchmark's workload): trivial operations (by a constant 0 or 1) are not
counted, identical ones once, symmetric results once (upper triangle).  Each
add, multiply, divide and special function (sine, cosine, arctangent,
square root, logarithm) counts one operation.  The benchmark multiplies them
by the work counters, which tests pin to the oracle's, so that its
algorithmic flop count depends on neither the kernels nor hand counts.

The steps onto endcap disks (the plane step, the (r-phi, r) frame and r
window, the disk's update and scattering) are counted apart, on the disk
steps of true forward tracks of a barrel-plus-endcap PU-200-like event.

Writes flop_census.json beside this file:  python oracle/flop_census.py
"""
from __future__ import annotations

import json
import os
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "flop_census.json")

N_TRACKS = 300        # sampled true tracks (every 25th seed of event 0)
SECOND_HIT_DZ = 0.05  # cm: the second hit of a step lies this far along z from the first


def census(n_tracks: int = N_TRACKS) -> dict:
    import oracle
    from synth import make_batch
    b = make_batch("c4", n_events=1)
    det = b.det
    L = det.n_layers
    x, y, z, lay = b.event_hits(0)
    prm, cov, sh = b.event_seeds(0)
    th = b.track_hits[0]
    seeds = np.arange(0, b.n_seeds, max(1, b.n_seeds // n_tracks))[:n_tracks]
    align = np.full((L, 2), 1e-3)  # inputs of the count whatever their values
    steps, seed_fit, fit_hit = [], [], []
    for s in seeds:
        true = th[b.seed_sim[s]]
        s3 = [int(h) for h in sh[:, s]]
        start = int(lay[s3[2]]) + 1
        dec = np.full(L, -2, np.int32)
        for l in range(start, L):
            h = int(true[l])
            if h < 0:
                break
            st, _, _, _, p, C = oracle.replay_decisions(b, 0, s, dec)
            if st != 0:
                break
            m1 = np.array([x[h], y[h], z[h]], np.float64)
            m2 = m1 + np.array([0.0, 0.0, SECOND_HIT_DZ])
            c = oracle.census_step(det, p, C, l, m1, m2, align[l])
            if c is not None:
                steps.append(c)
            dec[l] = h
        raw3 = np.array([[x[h], y[h], z[h]] for h in s3])
        c = oracle.census_fit(det, prm[:, s], cov[:, s], raw3, lay[s3], align, ms_after_last=True)
        if c is not None:
            seed_fit.append(c)
        hs = [int(h) for h in true if h >= 0]
        rawn = np.array([[x[h], y[h], z[h]] for h in hs])
        c = oracle.census_fit(det, prm[:, s], cov[:, s], rawn, lay[hs], align, ms_after_last=False)
        if c is not None:
            fit_hit.append(c / len(hs))
    steps = np.array(steps, np.float64)       # [samples][5][4]
    mean = steps.mean(axis=0)
    parts = dict(zip(oracle.CENSUS_PARTS, mean))
    # hits in the method's search window per candidate-layer step, on a
    # quarter of the seeds of the same event (250 of every 1,000)
    ns = b.n_seeds
    chunks = [(lo, min(lo + 250, ns)) for lo in range(0, ns, 1000)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        cnts = list(ex.map(lambda c: oracle.find_event(b, 0, seeds=c)["counters"], chunks))
    n_steps = sum(c["steps"] for c in cnts)
    n_win = sum(c["window_hits"] for c in cnts)
    kinds = ["adds", "multiplies", "divides", "special"]
    return {
        "what": "operations per unit of the finding and fitting steps (oracle operation census)",
        "sample": f"{len(steps)} candidate-layer steps along {len(seeds)} true tracks of PU-200-like event 0 "
                  f"(100 x 8,000 tracks configuration), seeds and fits of the same tracks",
        "per_step_parts": {k: {kk: float(v) for kk, v in zip(kinds, parts[k])} for k in parts},
        "flops": {
            "F_STEP": float(parts["propagate_transport"].sum() + parts["frame_window"].sum()),
            "F_HIT": float(parts["hit_chi2"].sum()),
            "F_UPDATE": float(parts["update"].sum()),
            "F_MS": float(parts["scatter"].sum()),
            "F_SEED": float(np.mean(seed_fit, axis=0).sum()),
            "F_FIT_HIT": float(np.mean(fit_hit, axis=0).sum()),
        },
        "spread": {
            "F_STEP_min_max": [float((steps[:, 0] + steps[:, 1]).sum(axis=1).min()),
                               float((steps[:, 0] + steps[:, 1]).sum(axis=1).max())],
        },
        # hits inside the bounding box of each prediction's chi2 < cut ellipse
        # (the method's search window), per candidate-layer step
        "window_hits_per_step": n_win / n_steps,
        "window_hits_sample": f"{n_steps} oracle candidate-layer steps of event 0, seeds [lo, lo + 250) every 1,000",
    }


def census_disks(n_tracks: int = N_TRACKS) -> dict:
    """Per-unit counts of the steps onto endcap disks: every disk step of the
    true hit lists of forward seeds of event 0 of the barrel-plus-endcap
    configuration (20 x 8,000 tracks, |eta| < 2.4), from the fitted state
    before the step; window hits per disk step from the oracle's finding on
    a quarter of the event's seeds."""
    import oracle
    from synth import make_batch
    from synth.events import true_hit_lists
    b = make_batch("c6", n_events=1)
    det = b.det
    S, L = det.n_surfaces, det.n_layers
    x, y, z, lay = b.event_hits(0)
    prm, cov, _ = b.event_seeds(0)
    lists, n = true_hit_lists(b, 0, S)
    eta = -np.log(np.tan(0.5 * prm[5].astype(np.float64)))
    fwd = np.nonzero(np.abs(eta) >= det.eta_barrel)[0]
    seeds = fwd[np.arange(0, fwd.size, max(1, fwd.size // n_tracks))[:n_tracks]]
    steps = []
    for s in seeds:
        hl = lists[b.seed_sim[s]][None, :]
        nh = int(n[b.seed_sim[s]])
        for j in range(3, nh):
            h = int(hl[0, j])
            if lay[h] < L:
                continue
            p, C, _, st = oracle.fit(det, prm[:, s:s + 1], cov[:, s:s + 1], hl, np.array([j]), x, y, z, lay,
                                     align=b.align, ms_after_last=True)
            if st[0] != 0:
                break
            m1 = np.array([x[h], y[h], z[h]], np.float64)
            c = oracle.census_disk_step(det, p[0], C[0], int(lay[h]), m1, m1 + np.array([SECOND_HIT_DZ, 0.0, 0.0]))
            if c is not None:
                steps.append(c)
    steps = np.array(steps, np.float64)
    mean = steps.mean(axis=0)
    parts = dict(zip(oracle.CENSUS_PARTS, mean))
    ns = b.n_seeds
    chunks = [(lo, min(lo + 250, ns)) for lo in range(0, ns, 1000)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        cnts = list(ex.map(lambda c: oracle.find_event(b, 0, seeds=c)["counters"], chunks))
    n_dsteps = sum(c["disk_steps"] for c in cnts)
    n_dwin = sum(c["disk_window_hits"] for c in cnts)
    kinds = ["adds", "multiplies", "divides", "special"]
    return {
        "sample": f"{len(steps)} disk steps along {len(seeds)} true forward tracks of barrel-plus-endcap event 0 "
                  f"(20 x 8,000 tracks, |eta| < 2.4, seven disks per side)",
        "per_step_parts": {k: {kk: float(v) for kk, v in zip(kinds, parts[k])} for k in parts},
        "flops": {
            "F_DISK_STEP": float(parts["propagate_transport"].sum() + parts["frame_window"].sum()),
            "F_DISK_HIT": float(parts["hit_chi2"].sum()),
            "F_DISK_UPDATE": float(parts["update"].sum()),
            "F_DISK_MS": float(parts["scatter"].sum()),
        },
        "window_hits_per_disk_step": n_dwin / n_dsteps,
        "window_hits_sample": f"{n_dsteps} oracle disk steps of event 0, seeds [lo, lo + 250) every 1,000",
    }


def load() -> dict:
    with open(OUT) as f:
        return json.load(f)


if __name__ == "__main__":
    res = census()
    res["disks"] = census_disks()
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")
    print(json.dumps(res["flops"], indent=1), res["window_hits_per_step"])
    print(json.dumps(res["disks"]["flops"], indent=1), res["disks"]["window_hits_per_disk_step"])
