"""Residuals of the L1 + SSIM objective and their weights (Eq. gn-loss; Sec. C,
"Precomputation Of Residual-To-Pixel Weights").

Test infrastructure: this module is part of the FP64 oracle; only tests/,
__graft_entry__.smoke() and bench.py's CPU legs use it.

The objective keeps, for every pixel i and colour channel, two residuals

    r1 = sqrt(lambda1 |c - C|),     r2 = sqrt(lambda2 (1 - SSIM_i))

with lambda1 = 0.8 and lambda2 = 0.2 (the weights of the 3DGS loss the paper
restates next to Eq. sgd-loss). Their Jacobian rows factor as
(dr/dc)(dc/dx), Eq. res-sq-root-weights, and the two residuals of a pixel
channel share dc/dx, so (Eq. apply-jtj-simplified, res-sq-root-weights-sum)

    J^T J p       = (dc/dx)^T (w . (dc/dx) p),   w = (dr1/dc)^2 + (dr2/dc)^2
    J^T F         = (dc/dx)^T e,                 e = (dr1/dc) r1 + (dr2/dc) r2
    diag(J^T J)_k = sum over pixel channels of w (dc/dx_k)^2
    E             = sum of r1^2 + r2^2 = sum of lambda1 |c - C| + lambda2 (1 - SSIM)

and the Gauss-Newton model of E after a step with u = (dc/dx) Delta is
E + 2 e.u + w.u^2.

Readings (the paper defers SSIM to the 3DGS loss and is silent on the rest):
  - SSIM per colour channel as in Wang et al. 2004: local statistics from an
    11 x 11 Gaussian window (standard deviation 1.5, normalised to sum 1)
    applied with zero padding outside the image ("same"-size correlation),
    C1 = 0.01^2, C2 = 0.03^2;
  - dSSIM_i/dc_i keeps only the centre pixel's own effect on SSIM_i (Sec. C:
    the per-pixel score is propagated back to the centre pixel, ignoring the
    window's other pixels);
  - both square roots have a derivative that is unbounded at zero; the
    derivatives use max(|c - C|, eps) and max(1 - SSIM, eps) under the root,
    eps = 1e-4, and dr1/dc = 0 where c = C exactly;
  - r2 uses max(1 - SSIM, 0) (SSIM <= 1 holds in exact arithmetic).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import ndimage

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
WINDOW = 11
WINDOW_SIGMA = 1.5


@dataclass
class Objective:
    """The L1 + SSIM objective of Eq. gn-loss."""
    lambda1: float = 0.8
    lambda2: float = 0.2
    eps: float = 1e-4


def window(size: int = WINDOW, sigma: float = WINDOW_SIGMA) -> np.ndarray:
    """1D Gaussian window, normalised to sum 1; the 2D window is its outer product."""
    t = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-t * t / (2.0 * sigma * sigma))
    return g / g.sum()


def local_mean(img: np.ndarray) -> np.ndarray:
    """Window-weighted local mean of an (H, W) or (H, W, 3) image, zero outside."""
    g = window()
    out = ndimage.correlate1d(np.asarray(img, np.float64), g, axis=0, mode="constant", cval=0.0)
    return ndimage.correlate1d(out, g, axis=1, mode="constant", cval=0.0)


@dataclass
class SSIMTerms:
    mu_x: np.ndarray
    mu_y: np.ndarray
    var_x: np.ndarray
    var_y: np.ndarray
    cov: np.ndarray
    ssim: np.ndarray


def ssim_terms(x: np.ndarray, y: np.ndarray) -> SSIMTerms:
    """Local statistics and the SSIM map of rendered x against target y (same shape)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = local_mean(x), local_mean(y)
    vx = local_mean(x * x) - mx * mx
    vy = local_mean(y * y) - my * my
    cxy = local_mean(x * y) - mx * my
    num = (2.0 * mx * my + SSIM_C1) * (2.0 * cxy + SSIM_C2)
    den = (mx * mx + my * my + SSIM_C1) * (vx + vy + SSIM_C2)
    return SSIMTerms(mx, my, vx, vy, cxy, num / den)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    return ssim_terms(x, y).ssim


def ssim_center_grad(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d SSIM_i / d x_i with only the centre pixel varying: it enters each local
    statistic of its own window with the centre weight w0 = g_mid^2, so
    d mu_x = w0, d var_x = 2 w0 (x_i - mu_x), d cov = w0 (y_i - mu_y); the
    quotient rule on SSIM = A1 A2 / (B1 B2) gives the rest."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    t = ssim_terms(x, y)
    w0 = window()[WINDOW // 2] ** 2
    A1 = 2.0 * t.mu_x * t.mu_y + SSIM_C1
    A2 = 2.0 * t.cov + SSIM_C2
    B1 = t.mu_x ** 2 + t.mu_y ** 2 + SSIM_C1
    B2 = t.var_x + t.var_y + SSIM_C2
    dA1 = 2.0 * w0 * t.mu_y
    dA2 = 2.0 * w0 * (y - t.mu_y)
    dB1 = 2.0 * w0 * t.mu_x
    dB2 = 2.0 * w0 * (x - t.mu_x)
    return (dA1 * A2 + A1 * dA2) / (B1 * B2) - t.ssim * (dB1 / B1 + dB2 / B2)


@dataclass
class Weights:
    e: np.ndarray       # (dr1/dc) r1 + (dr2/dc) r2, flat in residual order
    w: np.ndarray       # (dr1/dc)^2 + (dr2/dc)^2
    cost: float         # sum of r1^2 + r2^2
    r1: np.ndarray
    r2: np.ndarray
    dr1: np.ndarray
    dr2: np.ndarray


def view_weights(img: np.ndarray, tgt: np.ndarray, obj: Objective) -> Weights:
    """Residuals, their derivatives and the weights of one view, (H, W, 3) arrays in,
    flat (H * W * 3) arrays out."""
    img = np.asarray(img, np.float64)
    tgt = np.asarray(tgt, np.float64)
    d = img - tgt
    ad = np.abs(d)
    S = ssim_map(img, tgt)
    dS = ssim_center_grad(img, tgt)
    r1 = np.sqrt(obj.lambda1 * ad)
    dr1 = np.sqrt(obj.lambda1) * np.sign(d) / (2.0 * np.sqrt(np.maximum(ad, obj.eps)))
    one_minus = 1.0 - S
    r2 = np.sqrt(obj.lambda2 * np.maximum(one_minus, 0.0))
    dr2 = -np.sqrt(obj.lambda2) * dS / (2.0 * np.sqrt(np.maximum(one_minus, obj.eps)))
    e = dr1 * r1 + dr2 * r2
    w = dr1 * dr1 + dr2 * dr2
    cost = float(np.sum(r1 * r1) + np.sum(r2 * r2))
    f = lambda a: a.ravel()
    return Weights(f(e), f(w), cost, f(r1), f(r2), f(dr1), f(dr2))


def weights(img_flat: np.ndarray, tgt_flat: np.ndarray, cams: list, obj: Objective) -> Weights:
    """view_weights over the views of a call, concatenated in view order."""
    parts, o = [], 0
    for c in cams:
        n = c.width * c.height * 3
        parts.append(view_weights(img_flat[o:o + n].reshape(c.height, c.width, 3),
                                  tgt_flat[o:o + n].reshape(c.height, c.width, 3), obj))
        o += n
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts]) if parts else np.zeros(0)
    return Weights(cat("e"), cat("w"), float(sum(p.cost for p in parts)), cat("r1"), cat("r2"), cat("dr1"),
                   cat("dr2"))


def cost(img_flat: np.ndarray, tgt_flat: np.ndarray, cams: list, obj: Objective) -> float:
    """E of Eq. gn-loss over the views of a call."""
    return weights(img_flat, tgt_flat, cams, obj).cost
