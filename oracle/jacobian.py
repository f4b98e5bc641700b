"""J p, J^T u and diag(J^T J) by the explicit per-pixel chain rule.

Sec. 3.3, Eq. backward-pass: dr/dx_i = (dr/dc)(dc/ds)(ds/dx_i). For the
sum-of-squares pixel residual r = c - C the first factor is the identity
(Sec. C, "for the L2 loss they take a trivial form of dr/dc = 1").
Per contributing (pixel, splat) record, dc/dy (3 x 9) is written out from the
blending definition; dy/dx (9 x 59) comes from ``projection`` (exact, forward
mode). Then, following Eq. apply-j, Eq. apply-jt and Eq. diag-jtj:

    (J p)_pixel     = sum over the pixel's records of (dc/dy)(dy/dx) p_gaussian
    (J^T u)_gauss   = sum over the Gaussian's records of (dy/dx)^T (dc/dy)^T u_pixel
    diag(J^T J)_k   = sum over records and channels of ((dc/dy)(dy/dx))[:, k]^2

Vectors over parameters are (N, 59) arrays (AoS); vectors over residuals are
per-view (H, W, 3) images concatenated in view order, flattened.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import conventions as cv
from .projection import Projection, project
from .raster import ViewRaster, rasterize


@dataclass
class ViewLin:
    """Linearisation of one view around the current parameters."""
    proj: Projection
    ras: ViewRaster
    a: np.ndarray        # (R, 3, 9) dc/dy for every record
    gauss: np.ndarray    # (R,) Gaussian index of every record
    pix_off: int         # offset of this view's first pixel in the subset's residual vector


def dc_dy(proj: Projection, ras: ViewRaster) -> np.ndarray:
    """dc/dy (3 x 9) of every record, from the blending definition (Sec. 3.3)."""
    R = ras.rec_pix.shape[0]
    y = proj.y[ras.rec_splat]
    A, B, C, o = y[:, 2], y[:, 3], y[:, 4], y[:, 5]
    dx, dy = ras.rec_d[:, 0], ras.rec_d[:, 1]
    free = ~ras.rec_clamped
    da_dpow = np.where(free, o * ras.rec_G, 0.0)      # alpha = o * exp(power)
    da_do = np.where(free, ras.rec_G, 0.0)
    dpow = np.stack([A * dx + B * dy,                  # d power / d mu_x (d = pixel - mu)
                     B * dx + C * dy,                  # d power / d mu_y
                     -0.5 * dx * dx,                   # d power / d A
                     -dx * dy,                         # d power / d B
                     -0.5 * dy * dy], axis=1)          # d power / d C
    a = np.zeros((R, 3, 9))
    for ch in range(3):
        g = ras.rec_dcda[:, ch]
        a[:, ch, 0:5] = (g * da_dpow)[:, None] * dpow
        a[:, ch, 5] = g * da_do
        a[:, ch, 6 + ch] = ras.rec_alpha * ras.rec_T
    return a


def linearise_view(params: np.ndarray, cam, pix_off: int = 0, smooth: bool = False) -> ViewLin:
    proj = project(params, cam, smooth=smooth)
    ras = rasterize(proj, cam, smooth=smooth)
    return ViewLin(proj, ras, dc_dy(proj, ras), proj.idx[ras.rec_splat], pix_off)


def linearise_view_tiles(params: np.ndarray, cam, tiles, pix_off: int = 0, smooth: bool = False) -> ViewLin:
    """linearise_view restricted to the listed (tx, ty) tiles, for scenes too large
    to linearise whole: every Gaussian is projected without derivatives, those
    whose splat rect (outer rect, to keep the near-flip flags) meets a listed tile
    are projected again with derivatives, and only the listed tiles are blended.
    Records, pixel indices and Gaussian indices are those of linearise_view."""
    P = np.asarray(params, np.float64)
    pv = project(P, cam, smooth=smooth, want_jac=False)
    r = pv.rect_outer if pv.rect_outer is not None else pv.rect
    hit = np.zeros(pv.idx.shape[0], bool)
    for tx, ty in tiles:
        hit |= (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
    keep = np.unique(pv.idx[hit])
    proj = project(P[keep], cam, smooth=smooth)
    proj.idx = keep[proj.idx]              # back to the scene's Gaussian indices (depth tie-break)
    proj.n = P.shape[0]
    vis = np.zeros(P.shape[0], bool)
    vis[proj.idx] = True
    proj.visible = vis
    ras = rasterize(proj, cam, smooth=smooth, tiles=tiles)
    return ViewLin(proj, ras, dc_dy(proj, ras), proj.idx[ras.rec_splat], pix_off)


def linearise(params: np.ndarray, cams: list, smooth: bool = False) -> list:
    out, off = [], 0
    for cam in cams:
        out.append(linearise_view(params, cam, off, smooth))
        off += cam.width * cam.height * 3
    return out


def render(params: np.ndarray, cams: list, smooth: bool = False) -> np.ndarray:
    """Concatenated flattened images of the views (no derivatives)."""
    out = []
    for cam in cams:
        proj = project(params, cam, smooth=smooth, want_jac=False)
        out.append(rasterize(proj, cam, smooth=smooth).image.ravel())
    return np.concatenate(out)


def n_residuals(cams: list) -> int:
    return sum(c.width * c.height * 3 for c in cams)


def apply_J(lin: list, p: np.ndarray, n_res: int) -> np.ndarray:
    """u = J p (Eq. apply-j). p: (N, 59). Returns the flat residual-space vector."""
    u = np.zeros(n_res)
    for vl in lin:
        ydot = np.einsum("sij,sj->si", vl.proj.jac, p[vl.proj.idx])     # (dy/dx) p per splat
        contrib = np.einsum("rcj,rj->rc", vl.a, ydot[vl.ras.rec_splat])  # (dc/dy) ydot per record
        rows = vl.pix_off + vl.ras.rec_pix[:, None] * 3 + np.arange(3)[None, :]
        np.add.at(u, rows.ravel(), contrib.ravel())
    return u


def apply_JT(lin: list, u: np.ndarray, n_gauss: int) -> np.ndarray:
    """g = J^T u (Eq. apply-jt). Returns (N, 59)."""
    g = np.zeros((n_gauss, 59))
    for vl in lin:
        rows = vl.pix_off + vl.ras.rec_pix[:, None] * 3 + np.arange(3)[None, :]
        ur = u[rows]                                                     # (R, 3)
        ybar_rec = np.einsum("rcj,rc->rj", vl.a, ur)
        S = vl.proj.idx.shape[0]
        ybar = np.zeros((S, 9))
        np.add.at(ybar, vl.ras.rec_splat, ybar_rec)
        gs = np.einsum("sij,si->sj", vl.proj.jac, ybar)
        np.add.at(g, vl.proj.idx, gs)
    return g


def _record_rows(vl: ViewLin, lo: int, hi: int) -> np.ndarray:
    """Full partials dc/dx (records lo..hi, 3, 59) = (dc/dy)(dy/dx)."""
    return np.einsum("rcj,rjk->rck", vl.a[lo:hi], vl.proj.jac[vl.ras.rec_splat[lo:hi]])


def jacobi_diag(lin: list, n_gauss: int, chunk: int = 50000, weights: np.ndarray | None = None) -> np.ndarray:
    """M = diag(J^T J) (Eq. diag-jtj): sum of squared full partials. Returns (N, 59).
    weights (flat, residual order): per pixel channel factors (dr/dc)^2 of a
    non-L2 residual (Eq. res-sq-root-weights-sum); None means 1."""
    d = np.zeros((n_gauss, 59))
    for vl in lin:
        R = vl.a.shape[0]
        for lo in range(0, R, chunk):
            hi = min(R, lo + chunk)
            rows = _record_rows(vl, lo, hi)
            sq = rows * rows
            if weights is not None:
                res = vl.pix_off + vl.ras.rec_pix[lo:hi, None] * 3 + np.arange(3)[None, :]
                sq = sq * weights[res][:, :, None]
            np.add.at(d, vl.gauss[lo:hi], sq.sum(axis=1))
    return d


def explicit_J(lin: list, n_res: int, n_gauss: int) -> sp.csr_matrix:
    """The sparse Jacobian itself, rows = residuals, columns = g*59 + k (tiny scenes only)."""
    ri, ci, vv = [], [], []
    for vl in lin:
        R = vl.a.shape[0]
        if R == 0:
            continue
        rows = _record_rows(vl, 0, R)                                   # (R, 3, 59)
        r = vl.pix_off + vl.ras.rec_pix[:, None, None] * 3 + np.arange(3)[None, :, None]
        c = vl.gauss[:, None, None] * 59 + np.arange(59)[None, None, :]
        r, c = np.broadcast_arrays(r, c)
        nz = rows != 0.0
        ri.append(r[nz])
        ci.append(c[nz])
        vv.append(rows[nz])
    if not ri:
        return sp.csr_matrix((n_res, n_gauss * 59))
    return sp.coo_matrix((np.concatenate(vv), (np.concatenate(ri), np.concatenate(ci))),
                         shape=(n_res, n_gauss * 59)).tocsr()


def residual(image_flat: np.ndarray, target_flat: np.ndarray) -> np.ndarray:
    """F = c - C per pixel and channel (sum-of-squares residual)."""
    return image_flat - target_flat


def cost(F: np.ndarray) -> float:
    """E = ||F||^2 (no normalisation)."""
    return float(np.dot(F, F))
