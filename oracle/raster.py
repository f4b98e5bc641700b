"""Tile-ordered alpha blending of one view, with the per-pixel records of Sec. 3.3.

Eq. alpha-blending (Sec. 3.1): c = sum_i c_i alpha_i T_i, T_i = prod_{j<i} (1 - alpha_j).
For every (pixel, splat) pair that contributes to the pixel colour, the record
holds what the paper's gradient cache holds (Sec. 3.3, "T_s, dc/dalpha_s,
dc/dc_s"), computed here from their definitions:

    T_s            transmittance in front of splat s
    dc/dc_s        = alpha_s T_s
    dc/dalpha_s    = T_s c_s - (sum_{j > s} c_j alpha_j T_j) / (1 - alpha_s)

The colour behind s is an exact suffix sum over the pixel's later contributors.
Constants and the blending order are in ``oracle.conventions``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import conventions as cv
from .projection import Projection


@dataclass
class ViewRaster:
    width: int
    height: int
    image: np.ndarray        # (H, W, 3)
    rec_pix: np.ndarray      # (R,) flat pixel index y*W + x
    rec_splat: np.ndarray    # (R,) index into the Projection's splat arrays
    rec_T: np.ndarray        # (R,) transmittance in front of the splat
    rec_alpha: np.ndarray    # (R,) alpha used in blending
    rec_G: np.ndarray        # (R,) Gaussian weight exp(power)
    rec_clamped: np.ndarray  # (R,) True where alpha hit ALPHA_MAX
    rec_dcda: np.ndarray     # (R, 3) dc/dalpha
    rec_d: np.ndarray        # (R, 2) pixel centre minus splat mean
    margin: np.ndarray       # (H*W,) smallest relative distance of an alpha/T decision to its threshold
    n_contrib: np.ndarray    # (H*W,) contributing splats per pixel
    flip: np.ndarray = None  # (H*W,) a depth-order or tile-rect decision within float32 reach touches the pixel


def blend_order(proj: Projection) -> np.ndarray:
    """Splat order of Eq. alpha-blending: ascending (float32 depth, Gaussian index)."""
    return np.lexsort((proj.idx, proj.depth.astype(np.float32)))


def rasterize(proj: Projection, cam, smooth: bool = False, tiles=None) -> ViewRaster:
    """Blend every 16x16 tile of the view, or only the (tx, ty) tiles listed in
    `tiles` (the other pixels stay black and carry no records)."""
    W, H = int(cam.width), int(cam.height)
    T_ = cv.TILE
    tiles_x, tiles_y = (W + T_ - 1) // T_, (H + T_ - 1) // T_
    image = np.zeros((H, W, 3))
    margin = np.full(H * W, np.inf)
    flip = np.zeros(H * W, bool)
    n_contrib = np.zeros(H * W, np.int64)
    recs = {k: [] for k in ("pix", "splat", "T", "alpha", "G", "clamped", "dcda", "d")}
    order = blend_order(proj)
    rect = proj.rect
    y = proj.y
    depth32 = proj.depth.astype(np.float32).astype(np.float64)
    rect_flip = proj.rect_flip if proj.rect_flip is not None else np.zeros(proj.idx.shape[0], bool)

    only = None if tiles is None else {(int(a), int(b)) for a, b in tiles}
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            if only is not None and (tx, ty) not in only:
                continue
            xs = np.arange(tx * T_, min(W, tx * T_ + T_))
            ys = np.arange(ty * T_, min(H, ty * T_ + T_))
            gy, gx = np.meshgrid(ys, xs, indexing="ij")
            pix = (gy * W + gx).ravel()
            px = gx.ravel() + 0.5
            py = gy.ravel() + 0.5
            r = rect[order]
            sel = order[(r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])]
            # a rect decision near a flip can add or drop the splat in the tiles
            # between its inner and outer rects: flag the pixels it would reach
            if not smooth and rect_flip.any():
                ro, ri = proj.rect_outer[order], proj.rect_inner[order]
                in_o = (ro[:, 0] <= tx) & (tx < ro[:, 2]) & (ro[:, 1] <= ty) & (ty < ro[:, 3])
                in_i = (ri[:, 0] <= tx) & (tx < ri[:, 2]) & (ri[:, 1] <= ty) & (ty < ri[:, 3])
                ring = order[in_o & ~in_i & rect_flip[order]]
                for s_ in ring:
                    yr = y[s_]
                    ddx, ddy = px - yr[0], py - yr[1]
                    ar = yr[5] * np.exp(-0.5 * (yr[2] * ddx * ddx + yr[4] * ddy * ddy) - yr[3] * ddx * ddy)
                    flip[pix] |= ar >= cv.ALPHA_MIN * (1.0 - 1e-3)
            L = sel.shape[0]
            if L == 0:
                continue
            ys_ = y[sel]
            dx = px[:, None] - ys_[None, :, 0]
            dy = py[:, None] - ys_[None, :, 1]
            A, B, C, o = ys_[:, 2], ys_[:, 3], ys_[:, 4], ys_[:, 5]
            power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
            G = np.exp(power)
            a_raw = o * G
            if smooth:
                alpha = a_raw
                valid = np.ones_like(a_raw, bool)
                clamped = np.zeros_like(a_raw, bool)
            else:
                alpha = np.minimum(cv.ALPHA_MAX, a_raw)
                valid = alpha >= cv.ALPHA_MIN
                clamped = a_raw > cv.ALPHA_MAX
            om = np.where(valid, 1.0 - alpha, 1.0)
            Tinc = np.cumprod(om, axis=1)
            Tbef = np.concatenate([np.ones((Tinc.shape[0], 1)), Tinc[:, :-1]], axis=1)
            col_idx = np.arange(L)[None, :]
            if smooth:
                contrib = valid
                stop_at = np.full(pix.shape[0], L)
            else:
                stop = valid & (Tbef * (1.0 - alpha) < cv.T_MIN)
                has = stop.any(axis=1)
                stop_at = np.where(has, stop.argmax(axis=1), L)
                contrib = valid & (col_idx < stop_at[:, None])
                # decision margins over every splat the pixel examined (up to the stop)
                seen = col_idx <= stop_at[:, None]
                m_skip = np.abs(a_raw - cv.ALPHA_MIN) / cv.ALPHA_MIN
                m_clamp = np.abs(a_raw - cv.ALPHA_MAX) / cv.ALPHA_MAX
                m_stop = np.where(valid, np.abs(Tbef * (1.0 - alpha) - cv.T_MIN) / cv.T_MIN, np.inf)
                m = np.minimum(np.minimum(m_skip, m_clamp), m_stop)
                m = np.where(seen, m, np.inf).min(axis=1)
                margin[pix] = np.minimum(margin[pix], m)
                # depth-order near-ties (float32 depths within 2e-6 relative) between
                # consecutive splats that both reach the pixel
                if L > 1:
                    dd = np.abs(np.diff(depth32[sel])) / np.maximum(depth32[sel][:-1], 1e-30)
                    both = valid[:, :-1] & valid[:, 1:] & seen[:, 1:]
                    flip[pix] |= (both & (dd[None, :] < 2e-6)).any(axis=1)
            w = np.where(contrib, alpha * Tbef, 0.0)              # dc/dc_s = alpha_s T_s
            rgb = ys_[:, 6:9]
            wc = w[:, :, None] * rgb[None, :, :]                  # (P, L, 3)
            colour = wc.sum(axis=1)
            behind = np.cumsum(wc[:, ::-1, :], axis=1)[:, ::-1, :] - wc   # sum over j > s
            with np.errstate(divide="ignore", invalid="ignore"):
                dcda = Tbef[:, :, None] * rgb[None, :, :] - behind / (1.0 - alpha)[:, :, None]
            image[gy, gx] = colour.reshape(gy.shape + (3,))
            n_contrib[pix] = contrib.sum(axis=1)
            pi, si = np.nonzero(contrib)
            recs["pix"].append(pix[pi])
            recs["splat"].append(sel[si])
            recs["T"].append(Tbef[pi, si])
            recs["alpha"].append(alpha[pi, si])
            recs["G"].append(G[pi, si])
            recs["clamped"].append(clamped[pi, si])
            recs["dcda"].append(dcda[pi, si])
            recs["d"].append(np.stack([dx[pi, si], dy[pi, si]], axis=1))

    def cat(k, shape):
        return np.concatenate(recs[k]) if recs[k] else np.zeros(shape)

    return ViewRaster(
        W, H, image,
        cat("pix", (0,)).astype(np.int64), cat("splat", (0,)).astype(np.int64), cat("T", (0,)),
        cat("alpha", (0,)), cat("G", (0,)), cat("clamped", (0,)).astype(bool), cat("dcda", (0, 3)),
        cat("d", (0, 2)), margin, n_contrib, flip,
    )
