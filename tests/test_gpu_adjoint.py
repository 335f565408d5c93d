"""Adjoint of the fit on the GPU against the FP64 oracle.

The oracle's gradient comes from forward-mode dual numbers through the same
fit definition (pinned against finite differences in test_oracle_pins.py);
here the GPU adjoint (FP32, checkpointed reverse sweep) must match it within
1e-3 relative, and the alignment gradient must also match FP64 central finite
differences of the oracle's summed chi2.

"1e-3 relative" is read two ways, both asserted:
  * per gradient array, against its largest component:
    max|g - g_ref| <= 1e-3 max|g_ref|;
  * per component: |g - g_ref| <= 1e-3 |g_ref| + 8 sigma, where sigma is that
    component's FP32 rounding scale: the RMS change when the oracle runs the
    same gradient with every operation rounded to single precision, on
    inputs jittered by up to one FP32 ulp (four trials).  The emulation
    rounds correctly (0.5 ulp per operation); the CUDA path takes its
    reciprocals, sines and logarithms from the hardware approximations (up to
    about 2 ulp), so its rounding scale is up to 4 sigma: the bound is two of
    those.  Components far
    below their array's scale are sums of much larger terms of both signs
    (residual times inverse covariance, ~1/sigma^2), so their FP32 error is
    set by those terms, not by their own size.  The fraction of components
    inside the plain 1e-3 relative bound is printed beside it.
"""
import numpy as np
import pytest

import oracle
from kfhelp import tracker_for
from synth import make_batch
from synth.events import true_hit_lists

pytestmark = pytest.mark.gpu

REL = 1e-3


def _close(g, ref):
    """max|g - ref| / max|ref| over the array, and the largest elementwise
    relative error among components above 1% of the array's scale."""
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    scale = np.abs(ref).max()
    big = np.abs(ref) >= 1e-2 * scale
    comp = float((np.abs(g - ref)[big] / np.abs(ref)[big]).max()) if big.any() else 0.0
    return float(np.abs(g - ref).max() / scale), comp


def _fp32_sigma(b, sel, lists, n, trials=16, seed=7):
    """The oracle's gradients (align, hits, seed) and, per component, the RMS
    over `trials` of their change when the same computation runs with every
    operation rounded to single precision, on inputs (hit coordinates, seed
    parameters) jittered by up to one FP32 ulp: the FP32 rounding scale of
    each component.  Sixteen trials: with four, the RMS of a component can
    fall to a third of its scale by chance (a chi-square with four degrees of
    freedom), and one of thousands of components then left the 8-sigma bound
    while more trials put it at 0.6-0.8 of it.  The trials run on threads (the
    oracle releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    from kfhelp import JITTER_REL
    x, y, z, lay = b.event_hits(0)
    rng = np.random.default_rng(seed)
    base = oracle.fit_grad(b.det, b.params[:, sel], b.cov[:, sel], lists[sel], n[sel], x, y, z, lay, b.align)
    j = lambda a: a.astype(np.float64) * (1.0 + JITTER_REL * rng.uniform(-1, 1, a.shape))  # noqa: E731
    inputs = [(j(b.params[:, sel]), j(x), j(y), j(z)) for _ in range(trials)]

    def one(inp):
        pp, xx, yy, zz = inp
        return oracle.fit_grad(b.det, pp, b.cov[:, sel], lists[sel], n[sel], xx, yy, zz, lay, b.align, fp32=True)

    acc = [np.zeros_like(base[1]), np.zeros_like(base[2]), np.zeros_like(base[3])]
    with ThreadPoolExecutor(max_workers=min(trials, 16)) as ex:
        for g in ex.map(one, inputs):
            for k in range(3):
                acc[k] += (g[k + 1] - base[k + 1]) ** 2
    return base, [np.sqrt(a / trials) for a in acc]


def _component_ok(g, ref, sigma):
    """Per-component bound |g - ref| <= 1e-3 |ref| + 8 sigma; returns (all
    inside, fraction inside the plain 1e-3 relative bound, largest ratio)."""
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    d = np.abs(g - ref)
    bound = REL * np.abs(ref) + 8.0 * sigma
    plain = d <= REL * np.abs(ref)
    return bool(np.all(d <= bound)), float(plain.mean()), float((d / np.maximum(bound, 1e-300)).max())


def _setup(n_tracks=300, stride=4, seed=1003):
    from paper_1906_11744_gb300 import KF_FIT_GIVEN
    b = make_batch("c3", tracks=n_tracks, seed=seed)
    L = b.det.n_layers
    lists, n = true_hit_lists(b, 0, L)
    lists, n = lists[b.seed_sim], n[b.seed_sim]
    t = tracker_for(b, ckpt_stride=stride)
    t.fit_tracks(KF_FIT_GIVEN, lists, n)
    return b, t, lists, n


@pytest.mark.parametrize("stride", [4, 2, 8, 1])
def test_adjoint_matches_oracle_dual_gradient(stride):
    b, t, lists, n = _setup(stride=stride)
    fit = t.get_fit()
    ok = fit["status"] == 0
    L = b.det.n_layers
    g_align = np.zeros((L, 2), np.float32)
    g_hits = np.zeros((b.n_hits, 3), np.float32)
    g_seed = np.zeros((6, b.n_seeds), np.float32)
    t.fit_adjoint(g_align, g_hits, g_seed)
    sel = np.nonzero(ok)[0]
    (tot, ga, gh, gs, each), sig = _fp32_sigma(b, sel, lists, n)
    ea, ca = _close(g_align, ga)
    eh, ch = _close(g_hits, gh)
    es, cs = _close(g_seed[:, sel].T, gs)
    comp = [_component_ok(g_align, ga, sig[0]), _component_ok(g_hits, gh, sig[1]),
            _component_ok(g_seed[:, sel].T, gs, sig[2])]
    print(f"stride {stride}: norm-wise align {ea:.2e} hits {eh:.2e} seed {es:.2e}; "
          f"components above 1% of scale: {ca:.2e} {ch:.2e} {cs:.2e}; "
          f"inside plain 1e-3: {comp[0][1]:.4f} {comp[1][1]:.4f} {comp[2][1]:.4f}; "
          f"largest |dg| / (1e-3 |g| + 8 sigma): {comp[0][2]:.2f} {comp[1][2]:.2f} {comp[2][2]:.2f}")
    assert ea < REL and eh < REL and es < REL
    assert all(c[0] for c in comp), comp
    assert np.all(g_seed[:, ~ok] == 0)


def test_alignment_gradient_against_fp64_finite_differences():
    b, t, lists, n = _setup(n_tracks=100)
    L = b.det.n_layers
    g_align = np.zeros((L, 2), np.float32)
    t.fit_adjoint(g_align)
    x, y, z, lay = b.event_hits(0)
    al = b.align.astype(np.float64)
    ok = t.get_fit()["status"] == 0
    sel = np.nonzero(ok)[0]

    def total(a):
        return oracle.fit(b.det, b.params[:, sel], b.cov[:, sel], lists[sel], n[sel], x, y, z, lay, align=a)[2].sum()

    h = 1e-6
    fd = np.zeros((L, 2))
    for li in range(L):
        for c in range(2):
            a1, a2 = al.copy(), al.copy()
            a1[li, c] += h
            a2[li, c] -= h
            fd[li, c] = (total(a1) - total(a2)) / (2 * h)
    err, comp = _close(g_align, fd)
    print(f"alignment vs FP64 finite differences: norm-wise {err:.2e}, components {comp:.2e}")
    assert err < REL, err


def test_graph_with_adjoint_equals_direct_call():
    import torch
    from paper_1906_11744_gb300 import KF_FIT_FOUND, kf_get_gradient
    b = make_batch("c2", n_events=2)
    L = b.det.n_layers
    t1 = tracker_for(b)
    t1.find_tracks()
    t1.remove_duplicates()
    t1.fit_tracks(KF_FIT_FOUND)
    ga1 = np.zeros((L, 2), np.float32)
    gs1 = np.zeros((6, b.n_seeds), np.float32)
    t1.fit_adjoint(ga1, None, gs1)
    s = torch.cuda.Stream()
    t2 = tracker_for(b)
    t2.capture_graph(with_adjoint=True, stream=s)
    t2.launch_graph(stream=s)
    s.synchronize()
    ga2 = np.zeros((L, 2), np.float32)
    gs2 = np.zeros((6, b.n_seeds), np.float32)
    kf_get_gradient(t2.ctx, ga2, None, gs2)
    # the seed gradients are per-track and deterministic; the alignment sums
    # are accumulated with atomics in double, equal to float rounding
    assert np.array_equal(gs1, gs2)
    assert np.allclose(ga1, ga2, rtol=1e-6, atol=1e-6 * np.abs(ga1).max())


def test_autograd_function_backward():
    import torch
    from paper_1906_11744_gb300.autograd import KFFitChi2
    b, t, lists, n = _setup(n_tracks=200)
    dev = torch.device("cuda:0")
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    t.hit_offsets = b.hit_off
    t.seed_offsets = b.seed_off
    t.layer_dev = tt(b.layer)
    t.cov_dev = tt(b.cov)
    t.seed_hits_dev = tt(b.seed_hits)
    align = tt(b.align).requires_grad_(True)
    hits = tt(np.stack([b.x, b.y, b.z], 1)).requires_grad_(True)
    seeds = tt(b.params).requires_grad_(True)
    chi2 = KFFitChi2.apply(t, align, hits, seeds, tt(lists), tt(n))
    chi2.backward()
    x, y, z, lay = b.event_hits(0)
    ok = t.get_fit()["status"] == 0
    sel = np.nonzero(ok)[0]
    tot, ga, gh, gs, each = oracle.fit_grad(b.det, b.params[:, sel], b.cov[:, sel], lists[sel], n[sel],
                                            x, y, z, lay, b.align)
    assert abs(chi2.item() - tot) / tot < 1e-4
    assert _close(align.grad.cpu().numpy(), ga)[0] < REL
    assert _close(hits.grad.cpu().numpy(), gh)[0] < REL
