"""Call-order and replay rules of the C ABI (include/kf.h).

Loading hits unloads the seeds, because the seeds' hit indices were checked
against the previous hits.  A captured graph holds buffer addresses, sizes
and event offsets.  A replay after a load that changed any of them is
refused with KF_ERR_STATE.  A load that keeps them may change the values.
"""
import numpy as np
import pytest

from kfhelp import tracker_for
from synth import make_batch

pytestmark = pytest.mark.gpu


def _rc(fn, *args):
    from paper_1906_11744_gb300 import _lib
    return getattr(_lib.load(), fn)(*args)


def test_reloading_hits_requires_seeds_again():
    from paper_1906_11744_gb300 import _lib
    b = make_batch("c1b")
    t = tracker_for(b)
    # reload a smaller event: the seeds' hit indices may now point past it
    keep = b.hit_off[1] // 2
    off = np.array([0, keep], np.int32)
    t.load_hits(off, b.x[:keep], b.y[:keep], b.z[:keep], b.layer[:keep])
    assert _rc("kf_find_tracks", t.ctx, None) == _lib.KF_ERR_STATE
    assert _rc("kf_fit_tracks", t.ctx, _lib.KF_FIT_FOUND, None, None, 0, 1, None) == _lib.KF_ERR_STATE
    assert _rc("kf_autotune", t.ctx, None, 0, None, None) == _lib.KF_ERR_STATE
    # the original hits and seeds again: finding works
    t.load_hits(b.hit_off, b.x, b.y, b.z, b.layer)
    t.load_seeds(b.seed_off, b.params, b.cov, b.seed_hits)
    t.find_tracks()
    assert (t.get_tracks()["n_found"] >= 3).any()
    t.close()


def test_graph_replay_refused_after_a_size_change():
    import torch
    from paper_1906_11744_gb300 import _lib
    b = make_batch("c1b")
    t = tracker_for(b)
    s = torch.cuda.Stream()
    t.capture_graph(stream=s)
    t.launch_graph(s)
    s.synchronize()
    ref = t.get_tracks()
    # same sizes and offsets, values reloaded: the replay is allowed and equal
    t.load_hits(b.hit_off, b.x, b.y, b.z, b.layer)
    assert _rc("kf_launch_graph", t.ctx, ctypes_stream(s)) == _lib.KF_ERR_STATE  # seeds not reloaded
    t.load_seeds(b.seed_off, b.params, b.cov, b.seed_hits)
    t.launch_graph(s)
    s.synchronize()
    again = t.get_tracks()
    assert np.array_equal(ref["hits"], again["hits"])
    # a larger batch (two copies of the event): buffers grow, the replay is refused
    two = lambda a: np.concatenate([a, a], axis=-1)  # noqa: E731
    n_h, n_s = b.hit_off[1], b.seed_off[1]
    t.load_hits(np.array([0, n_h, 2 * n_h], np.int32), two(b.x), two(b.y), two(b.z), two(b.layer))
    t.load_seeds(np.array([0, n_s, 2 * n_s], np.int32), two(b.params), two(b.cov), two(b.seed_hits))
    assert _rc("kf_launch_graph", t.ctx, ctypes_stream(s)) == _lib.KF_ERR_STATE
    # a smaller load (no reallocation) with other offsets is refused too
    t.load_hits(np.array([0, n_h - 1], np.int32), b.x[:n_h - 1], b.y[:n_h - 1], b.z[:n_h - 1],
                b.layer[:n_h - 1])
    bad = b.seed_hits[:, :n_s].max(axis=0) < n_h - 1
    sh = np.ascontiguousarray(b.seed_hits[:, :n_s][:, bad])
    t.load_seeds(np.array([0, sh.shape[1]], np.int32), np.ascontiguousarray(b.params[:, :n_s][:, bad]),
                 np.ascontiguousarray(b.cov[:, :n_s][:, bad]), sh)
    assert _rc("kf_launch_graph", t.ctx, ctypes_stream(s)) == _lib.KF_ERR_STATE
    # capturing again makes the replay valid
    t.capture_graph(stream=s)
    t.launch_graph(s)
    s.synchronize()
    t.close()


def ctypes_stream(s):
    import ctypes
    return ctypes.c_void_p(s.cuda_stream)
