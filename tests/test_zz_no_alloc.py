"""The allocation-free duplicate-removal entry point.

Callers that cannot allocate device memory (a host framework that owns all
device allocations, a pipeline where cudaMalloc is banned from the hot path)
use kf_remove_duplicates_noalloc, which runs on a static scratch array.  This
file is collected last on purpose.  It checks, through the C ABI, that the
entry point returns exactly the keep flags of the context-based
kf_remove_duplicates on the same tracks, on two calls in a row (the second
call reuses the scratch the first one left behind), and that oversized events
are rejected before anything is launched.
"""
import ctypes

import numpy as np
import pytest

from kfhelp import tracker_for
from synth import make_batch

pytestmark = pytest.mark.gpu


def _found_tracks(name, **kw):
    b = make_batch(name, **kw)
    t = tracker_for(b)
    t.find_tracks()
    t.remove_duplicates()
    trk = t.get_tracks()
    t.close()
    return b, trk


def test_noalloc_matches_context_entry_point_twice():
    import torch

    from paper_1906_11744_gb300 import _lib
    dev = torch.device("cuda:0")
    cases = [_found_tracks("c1b"), _found_tracks("c1b", tracks=900, seed=77)]
    for b, trk in cases + cases[:1]:  # three calls; the third repeats the first on stale scratch
        n, L = trk["hits"].shape
        hits = torch.from_numpy(trk["hits"]).to(dev)
        n_found = torch.from_numpy(trk["n_found"]).to(dev)
        chi2 = torch.from_numpy(trk["chi2"]).to(dev)
        for _ in range(2):
            keep = torch.full((n,), 7, dtype=torch.uint8, device=dev)
            status = torch.full((1,), -9, dtype=torch.int32, device=dev)
            rc = _lib.kf_remove_duplicates_noalloc(n, L, b.n_hits, hits, n_found, chi2, 0.5, keep, status)
            assert rc == _lib.KF_OK
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert np.array_equal(keep.cpu().numpy(), trk["keep"])
        assert trk["keep"].sum() < n  # the duplicate seeds were removed


def test_noalloc_zero_tracks_clears_status():
    """An event without tracks launches no kernel but still writes 0 to the
    status word, so a caller never reads what an earlier call left there."""
    import torch

    from paper_1906_11744_gb300 import _lib
    dev = torch.device("cuda:0")
    status = torch.full((1,), -9, dtype=torch.int32, device=dev)
    empty_i = torch.zeros((1,), dtype=torch.int32, device=dev)
    rc = _lib.kf_remove_duplicates_noalloc(0, 17, 0, empty_i, empty_i, torch.zeros(1, device=dev), 0.5,
                                           torch.zeros(1, dtype=torch.uint8, device=dev), status)
    assert rc == _lib.KF_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_noalloc_rejects_events_beyond_its_limits():
    from paper_1906_11744_gb300 import _lib
    lib = _lib.load()
    null = ctypes.c_void_p(0)
    rc = lib.kf_remove_duplicates_noalloc(_lib.KF_NOALLOC_MAX_TRACKS + 1, 17, 100, null, null, null, 0.5,
                                          null, null, null)
    assert rc == _lib.KF_ERR_CAPACITY
    rc = lib.kf_remove_duplicates_noalloc(10, 17, _lib.KF_NOALLOC_MAX_HITS + 1, null, null, null, 0.5,
                                          null, null, null)
    assert rc == _lib.KF_ERR_CAPACITY
