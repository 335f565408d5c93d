"""torch.autograd.Function over the fit: forward = summed chi2 of the Kalman
re-fit, backward = the adjoint kernel (kf_fit_adjoint).  Argument marshalling
only; both directions run in the CUDA library."""
from __future__ import annotations

import torch

from . import KF_FIT_GIVEN, kf_fit_adjoint, kf_get_fit, kf_load_hits, kf_load_seeds, kf_set_alignment, kf_fit_tracks


class KFFitChi2(torch.autograd.Function):
    """chi2 = KFFitChi2.apply(tracker, align [L,2], hits [n_hits,3], seed_params
    [6,n_seeds], hit_lists [n_seeds,max_len] int32, n_hits [n_seeds] int32).

    The tracker's seed covariances and event offsets must already be loaded
    (Tracker.load_seeds); this call reloads hit positions, seed parameters and
    alignment from the given CUDA tensors.  Tracks whose fit fails contribute
    nothing."""

    @staticmethod
    def forward(ctx, tracker, align, hits, seed_params, hit_lists, n_hits):
        stream = torch.cuda.current_stream()
        h = hits.detach().float()
        kf_load_hits(tracker.ctx, tracker.hit_offsets, h[:, 0].contiguous(), h[:, 1].contiguous(),
                     h[:, 2].contiguous(), tracker.layer_dev, stream)
        kf_load_seeds(tracker.ctx, tracker.seed_offsets, seed_params.detach().float().contiguous(),
                      tracker.cov_dev, tracker.seed_hits_dev, stream)
        kf_set_alignment(tracker.ctx, align.detach().float().contiguous(), stream)
        kf_fit_tracks(tracker.ctx, KF_FIT_GIVEN, hit_lists, n_hits, stream)
        n = seed_params.shape[1]
        chi2 = torch.empty(n, dtype=torch.float32, device=hits.device)
        status = torch.empty(n, dtype=torch.int32, device=hits.device)
        kf_get_fit(tracker.ctx, chi2=chi2, status=status, stream=stream)
        ctx.tracker = tracker
        ctx.shapes = (align.shape, hits.shape, seed_params.shape)
        return torch.where(status == 0, chi2, torch.zeros_like(chi2)).double().sum()

    @staticmethod
    def backward(ctx, grad_out):
        stream = torch.cuda.current_stream()
        a_shape, h_shape, s_shape = ctx.shapes
        dev = grad_out.device
        g_align = torch.empty(a_shape, dtype=torch.float32, device=dev)
        g_hits = torch.empty(h_shape, dtype=torch.float32, device=dev)
        g_seed = torch.empty(s_shape, dtype=torch.float32, device=dev)
        kf_fit_adjoint(ctx.tracker.ctx, g_align, g_hits, g_seed, stream)
        go = grad_out.float()
        return None, go * g_align, go * g_hits, go * g_seed, None, None
