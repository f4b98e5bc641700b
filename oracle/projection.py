"""Projection of 3D Gaussians to 2D splats, with the exact per-splat Jacobian dy/dx.

Follows Sec. 3.1 ("all Gaussians are first projected into 2D Gaussian splats",
Eq. alpha-blending) and the splat attributes named in Sec. A (Eq. apply-jt:
"y_k ... the 2D mean, color, and opacity attributes"). The 2D conic (inverse
covariance) is part of y as well, since it is what the blending weight G uses.

Splat attribute vector y (9 values), in this order:
    0,1  2D mean (mu_x, mu_y) in pixels
    2,3,4  conic (A, B, C) = inverse of the 2D covariance [[a, b], [b, c]]
    5    opacity o = sigmoid(opacity logit)
    6,7,8  colour (r, g, b) = max(0, SH(dir) + 0.5)

The forward function is evaluated on ``ad.Dual`` numbers seeded with the 59
parameters of each Gaussian, so ``jac[s]`` is the exact 9 x 59 matrix dy/dx of
splat s (the factor ds/dx_i of Eq. backward-pass).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import ad, conventions as cv, sh


@dataclass
class Projection:
    n: int                   # Gaussians in the scene
    visible: np.ndarray      # (N,) bool
    idx: np.ndarray          # (S,) Gaussian index of each visible splat
    y: np.ndarray            # (S, 9) splat attributes
    jac: np.ndarray          # (S, 9, 59) dy/dx
    depth: np.ndarray        # (S,) camera-space z (float64)
    radius: np.ndarray       # (S,) integer pixel radius
    rect: np.ndarray         # (S, 4) tile rect [x0, y0, x1, y1) (exclusive ends)
    raw_rgb: np.ndarray      # (S, 3) SH(dir) + 0.5 before the clamp
    rect_margin: np.ndarray  # (S,) relative distance of the rect/radius decisions to a flip
    depth_raw: np.ndarray    # (N,) camera-space z of every Gaussian
    rect_flip: np.ndarray = None  # (S,) a radius or tile-rect decision lies within float32 reach
    rect_outer: np.ndarray = None  # (S, 4) union of the rects float32 rounding could produce
    rect_inner: np.ndarray = None  # (S, 4) their intersection


def camera_center(cam) -> np.ndarray:
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    return -R.T @ t


def _quat_rot(w, x, y, z):
    """Rotation matrix of a unit quaternion (w, x, y, z) as nested lists."""
    return [
        [1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)],
        [2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)],
        [2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)],
    ]


def project(params: np.ndarray, cam, smooth: bool = False, want_jac: bool = True,
            chunk: int = 20000) -> Projection:
    """Project every Gaussian into camera `cam` (one view).

    params: (N, 59) array (any float type; evaluated in float64). Work is split
    into chunks of Gaussians only to bound memory; chunks are independent.
    """
    P = np.asarray(params, np.float64)
    N = P.shape[0]
    if N > chunk:
        parts = [_project(P[s:s + chunk], cam, smooth, want_jac) for s in range(0, N, chunk)]
        offs = list(range(0, N, chunk))
        cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
        return Projection(
            n=N, visible=cat("visible"),
            idx=np.concatenate([p.idx + o for p, o in zip(parts, offs)]),
            y=cat("y"), jac=cat("jac"), depth=cat("depth"), radius=cat("radius"), rect=cat("rect"),
            raw_rgb=cat("raw_rgb"), rect_margin=cat("rect_margin"), depth_raw=cat("depth_raw"),
            rect_flip=cat("rect_flip"), rect_outer=cat("rect_outer"), rect_inner=cat("rect_inner"))
    return _project(P, cam, smooth, want_jac)


def _project(P: np.ndarray, cam, smooth: bool, want_jac: bool) -> Projection:
    N = P.shape[0]
    W, H = int(cam.width), int(cam.height)
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    fx, fy, cx, cy = (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy))

    # Visibility by depth first (value only); derivatives only for the kept splats.
    tz_all = P[:, 0:3] @ R[2] + t[2]
    keep = tz_all > cv.NEAR
    idx = np.nonzero(keep)[0]
    Pk = P[idx]
    S = idx.shape[0]
    nseed = 59 if want_jac else 1

    def var(col):
        if want_jac:
            return ad.Dual.seed(Pk[:, col], col, 59)
        return ad.Dual(Pk[:, col].copy(), np.zeros((S, 1)))

    x = [var(c) for c in range(59)]
    mu = x[0:3]
    # camera-space mean: t_c = R mu + t
    tc = [mu[0] * R[i, 0] + mu[1] * R[i, 1] + mu[2] * R[i, 2] + t[i] for i in range(3)]
    tx, ty, tz = tc
    # 2D mean (pinhole)
    mx = tx * fx / tz + cx
    my = ty * fy / tz + cy
    # 3D covariance Sigma = R(q) S S^T R(q)^T with S = diag(exp(log-scale))
    qn_len = ad.sqrt(x[6] * x[6] + x[7] * x[7] + x[8] * x[8] + x[9] * x[9])
    qw, qx, qy, qz = (x[6] / qn_len, x[7] / qn_len, x[8] / qn_len, x[9] / qn_len)
    Rq = _quat_rot(qw, qx, qy, qz)
    sc = [ad.exp(x[3 + j]) for j in range(3)]
    M = [[Rq[i][j] * sc[j] for j in range(3)] for i in range(3)]
    Sig = [[M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2] for j in range(3)] for i in range(3)]
    # Jacobian of the perspective map (EWA), T = Jp R, Sigma2 = T Sigma T^T + dilation
    j00 = fx / tz
    j02 = -(tx * fx) / (tz * tz)
    j11 = fy / tz
    j12 = -(ty * fy) / (tz * tz)
    T0 = [j00 * R[0, k] + j02 * R[2, k] for k in range(3)]
    T1 = [j11 * R[1, k] + j12 * R[2, k] for k in range(3)]

    def quad(U, V):
        acc = None
        for i in range(3):
            for j in range(3):
                term = U[i] * Sig[i][j] * V[j]
                acc = term if acc is None else acc + term
        return acc

    a = quad(T0, T0) + cv.DILATION
    b = quad(T0, T1)
    c = quad(T1, T1) + cv.DILATION
    det = a * c - b * b
    A = c / det
    B = -b / det
    C = a / det
    o = ad.sigmoid(x[10])
    # view direction and SH colour
    cc = camera_center(cam)
    dv = [mu[i] - cc[i] for i in range(3)]
    dlen = ad.sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2])
    dx_, dy_, dz_ = (dv[0] / dlen, dv[1] / dlen, dv[2] / dlen)
    Y = sh.basis(dx_, dy_, dz_)
    rgb_raw = []
    for ch in range(3):
        acc = None
        for k in range(16):
            term = Y[k] * x[11 + 3 * k + ch]
            acc = term if acc is None else acc + term
        rgb_raw.append(acc + cv.SH_OFFSET)
    rgb = rgb_raw if smooth else [ad.relu(v) for v in rgb_raw]

    ys = [mx, my, A, B, C, o, rgb[0], rgb[1], rgb[2]]
    yv = np.stack([q.v for q in ys], axis=1)
    jac = np.stack([q.d for q in ys], axis=1) if want_jac else np.zeros((S, 9, 0))

    # radius from the largest eigenvalue of the 2D covariance; tile rect
    av, bv, cvv = a.v, b.v, c.v
    mid = 0.5 * (av + cvv)
    lam_max = mid + np.sqrt(np.maximum(0.25 * (av - cvv) ** 2 + bv * bv, 0.0))
    r_real = cv.RADIUS_SIG * np.sqrt(lam_max)
    radius = np.ceil(r_real)
    tiles_x = (W + cv.TILE - 1) // cv.TILE
    tiles_y = (H + cv.TILE - 1) // cv.TILE
    ex = [(yv[:, 0] - radius) / cv.TILE, (yv[:, 1] - radius) / cv.TILE,
          (yv[:, 0] + radius) / cv.TILE, (yv[:, 1] + radius) / cv.TILE]
    x0 = np.clip(np.floor(ex[0]), 0, tiles_x).astype(np.int64)
    y0 = np.clip(np.floor(ex[1]), 0, tiles_y).astype(np.int64)
    x1 = np.clip(np.floor(ex[2]) + 1, 0, tiles_x).astype(np.int64)
    y1 = np.clip(np.floor(ex[3]) + 1, 0, tiles_y).astype(np.int64)
    if smooth:
        x0[:] = 0
        y0[:] = 0
        x1[:] = tiles_x
        y1[:] = tiles_y
    rect = np.stack([x0, y0, x1, y1], axis=1)

    # margins of the integer decisions (radius ceil, rect floors), relative; and
    # the rects float32 arithmetic could produce instead: a radius within 1e-5
    # (relative) of an integer may round to its neighbour, a rect edge within
    # 1e-3 px of a tile edge may floor to the neighbouring tile.
    frac = lambda v: np.abs(v - np.round(v))
    m = frac(r_real) / np.maximum(r_real, 1e-30)
    for e in ex:
        m = np.minimum(m, frac(e) / np.maximum(np.abs(e), 1.0))
    m = np.minimum(m, np.abs(tz.v - cv.NEAR) / cv.NEAR)

    def rect_of(rad, shift=(0, 0, 0, 0)):
        e = [(yv[:, 0] - rad) / cv.TILE, (yv[:, 1] - rad) / cv.TILE,
             (yv[:, 0] + rad) / cv.TILE, (yv[:, 1] + rad) / cv.TILE]
        lim = (tiles_x, tiles_y, tiles_x, tiles_y)
        out = []
        for i in range(4):
            f = np.floor(e[i]) + (1 if i >= 2 else 0) + shift[i]
            out.append(np.clip(f, 0, lim[i]).astype(np.int64))
        return np.stack(out, axis=1)

    alts = [rect]
    near_r = frac(r_real) < 1e-5 * np.maximum(r_real, 1.0)
    r_alt = np.where(r_real - np.floor(r_real) < 0.5, radius - 1, radius + 1)
    alts.append(np.where(near_r[:, None], rect_of(r_alt), rect))
    for i, e in enumerate(ex):
        near = frac(e) * cv.TILE < 1e-3
        step = np.where(e - np.floor(e) < 0.5, -1, 1)
        shift_v = [0, 0, 0, 0]
        alt = rect.copy()
        for sgn in (-1, 1):
            shift_v[i] = sgn
            cand = rect_of(radius, tuple(shift_v))
            alt = np.where(((step == sgn) & near)[:, None], cand, alt)
        alts.append(alt)
    A_ = np.stack(alts)
    r_outer = np.concatenate([A_[:, :, 0:2].min(0), A_[:, :, 2:4].max(0)], axis=1)
    r_inner = np.concatenate([A_[:, :, 0:2].max(0), A_[:, :, 2:4].min(0)], axis=1)
    if smooth:
        r_outer, r_inner = rect, rect
    flip = np.any(r_outer != r_inner, axis=1) | (np.abs(tz.v - cv.NEAR) < 1e-5)

    # A splat is drawn only if its covariance chain fits the renderer's float32
    # arithmetic: scales, 3D and 2D covariance (with the products of the
    # determinant), conic and mean must stay finite in float32. Decided here in
    # that precision, as the renderer decides it; float64 would keep splats
    # whose float32 covariance overflows.
    f32max = float(np.finfo(np.float32).max)
    fits = np.ones(S, bool)
    with np.errstate(over="ignore", invalid="ignore"):
        for v in ([q.v for q in sc] + [Sig[i][j].v for i in range(3) for j in range(i, 3)]
                  + [a.v, b.v, c.v, a.v * c.v, b.v * b.v, det.v, A.v, B.v, C.v, mx.v, my.v]):
            fits &= np.isfinite(v) & (np.abs(v) <= f32max)
    ok = (det.v > 0) & fits & (x1 > x0) & (y1 > y0)
    sel = np.nonzero(ok)[0]
    visible = np.zeros(N, bool)
    visible[idx[sel]] = True
    return Projection(
        n=N, visible=visible, idx=idx[sel], y=yv[sel], jac=jac[sel] if want_jac else jac,
        depth=tz.v[sel], radius=radius[sel].astype(np.int64), rect=rect[sel],
        raw_rgb=np.stack([q.v for q in rgb_raw], axis=1)[sel], rect_margin=m[sel],
        depth_raw=tz_all, rect_flip=flip[sel], rect_outer=r_outer[sel], rect_inner=r_inner[sel],
    )
