"""Shared helpers of the test suite: seeded cases, layout conversion, metrics."""
from __future__ import annotations

import numpy as np

import synth

N_PARAMS = 59


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def tiny_case():
    """BASELINE tiny workload: 1,000 Gaussians, 8 views of 64x64, targets from a perturbed copy."""
    from oracle import jacobian as J
    wl = synth.WORKLOADS["tiny"]
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    tgt = J.render(synth.perturbed_copy(wl, P).astype(np.float64), cams)
    tgt = (tgt + synth.pixel_noise(wl, tgt.size)).astype(np.float32)
    return wl, P, cams, tgt


def ragged_case(n=2000, views=4, W=72, H=56, seed=321, log_scale_mean=-3.0, radius=3.5):
    """Ragged tiles (W, H not multiples of 16), several tiles per view."""
    wl = synth.small_workload("ragged", seed, n, views, W, H, cam_radius=radius, log_scale_mean=log_scale_mean)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(seed, cams)]).astype(np.float32)
    return wl, P, cams, tgt


def pixel_mask(lin, threshold=1e-4):
    """True for pixels where no blending decision is within float32 reach of flipping.

    alpha-skip, alpha-clamp and T-stop decisions must be more than `threshold`
    (relative) from their thresholds; depth-order and tile-rect decisions are
    flagged by the oracle itself (ViewRaster.flip).
    """
    return np.concatenate([(vl.ras.margin >= threshold) & ~vl.ras.flip for vl in lin])
