"""Hit binning forms give the same found tracks.

Grids of at most 65,536 cells per layer take the layer-grouped form (hits
grouped by event and layer, then one block per layer of an event counting
cells in shared memory); larger grids take the general form (atomic counts per
cell, global scan).  Windows are exact supersets of the chi2 ellipse, so the
found tracks do not depend on the grid; a layer of one event with more than
65,535 hits is handled by its block with global counters.
"""
import numpy as np
import pytest

import oracle
from kfhelp import audit_mismatch, tracker_for
from synth import make_batch

pytestmark = pytest.mark.gpu


def _hits(b, **cfg):
    t = tracker_for(b, **cfg)
    t.find_tracks()
    r = t.get_tracks()
    t.close()
    return r


def test_grouped_form_equals_general_form():
    b = make_batch("c2", n_events=4)
    grouped = _hits(b, n_eta_bins=64, n_phi_bins=1024)
    general = _hits(b, n_eta_bins=64, n_phi_bins=2048)
    for k in ("hits", "n_found", "chi2"):
        assert np.array_equal(grouped[k], general[k]), k


def test_layer_above_16_bit_hit_count():
    b = make_batch("c1", tracks=70000)
    counts = np.bincount(b.layer, minlength=b.det.n_layers)
    assert counts.max() > 65535
    grouped = _hits(b, n_eta_bins=64, n_phi_bins=1024)
    general = _hits(b, n_eta_bins=64, n_phi_bins=2048)
    for k in ("hits", "n_found", "chi2"):
        assert np.array_equal(grouped[k], general[k]), k
    mism = []
    for s in range(0, b.n_seeds, b.n_seeds // 40)[:40]:
        ref = oracle.find_event(b, 0, seeds=(s, s + 1))
        if not np.array_equal(grouped["hits"][s], ref["hits"][0]):
            mism.append(s)
    for s in mism:
        ok, kind, rel = audit_mismatch(b, 0, s, grouped["hits"][s], oracle.find_event(b, 0, seeds=(s, s + 1))["hits"][0])
        assert ok, (s, kind, rel)
