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


def pcg_noise_spread(sys_, lam: float, n_iters: int, x_ref, eps: float = 1e-5, seeds=(0, 1)) -> float:
    """How far float32-level rounding can move a solve of this system: twice the
    largest relative L2 distance from x_ref (the oracle's solve) of the oracle's
    own Algorithm 1 run for n_iters iterations without break test with relative
    noise eps on b and on every J p and J^T u product. eps = 1e-5 is the float32
    products' error against the oracle (J p and J^T u within 1e-5 relative L2 on
    the paper crop).

    Algorithm 1 starts from x0 = M^-1 b, which overshoots the solution (by about
    4x in norm on these scenes), so the iterations cancel most of x0 and amplify
    the products' rounding with every iteration, whatever the damping: on the
    tiny case the spread is 1.3e-4 after 2 iterations, 2.7e-4 after 3 and 1.7e-3
    after 8 (at lambda = 1e-3 and at lambda = 1 alike). The PCG parity tests
    therefore hold x to the 1e-3 tolerance after an iteration count at which
    this spread is at most 5e-4, and report the spread and the distance after
    the paper's 8 iterations beside it.
    """
    from oracle import jacobian as jac, solver
    N = sys_.b.shape[0]
    n_res = sys_.F.shape[0]
    worst = 0.0
    for seed in seeds:
        rng = np.random.default_rng(seed)

        def noisy_JTJ(v):
            u = jac.apply_J(sys_.lin, v, n_res)
            u = u * (1.0 + eps * rng.standard_normal(u.shape))
            if sys_.W is not None:
                u = sys_.W * u
            g = jac.apply_JT(sys_.lin, u, N)
            return g * (1.0 + eps * rng.standard_normal(g.shape))

        b = sys_.b * (1.0 + eps * rng.standard_normal(sys_.b.shape))
        x = solver.pcg(noisy_JTJ, b, sys_.M, lam, n_iters, 0.0)[0]
        worst = max(worst, rel_l2(x, x_ref))
    return 2.0 * worst


# PCG solutions are held to this relative L2 distance from the oracle's, on
# systems whose noise spread (pcg_noise_spread) is at most PCG_SPREAD_MAX.
PCG_TOL = 1e-3
PCG_SPREAD_MAX = 5e-4
