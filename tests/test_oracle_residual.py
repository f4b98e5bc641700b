"""Pins of the oracle's L1 + SSIM residuals (Eq. gn-loss, Sec. C) against the
mathematics (CPU only): closed forms of the window and of SSIM, a brute-force
SSIM over the explicit 11 x 11 window, central differences of the centre-pixel
derivative and of both square-root residuals, the weighted J^T J and diagonal
against the explicit Jacobian, and b = -J^T F as half the gradient of the L1
energy.
"""
import math

import numpy as np
import pytest

from oracle import jacobian as J
from oracle import residual as R
from oracle import solver
from test_oracle_pins import small_scene, two_cams


def _images(seed=4, H=17, W=23):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    x = np.empty((H, W, 3))
    y = np.empty((H, W, 3))
    for c in range(3):
        x[..., c] = 0.5 + 0.2 * np.sin(0.3 * xx + 0.2 * yy + c) + 0.05 * rng.standard_normal((H, W))
        y[..., c] = 0.5 + 0.2 * np.sin(0.31 * xx + 0.17 * yy + c + 0.3) + 0.05 * rng.standard_normal((H, W))
    return x, y


def _ssim_bruteforce(x, y, i, j, c):
    """SSIM at pixel (i, j), channel c, from the explicit 2D window, zero outside."""
    g = R.window()
    H, W = x.shape[:2]
    s = {k: 0.0 for k in ("x", "y", "xx", "yy", "xy")}
    for a in range(-5, 6):
        for b in range(-5, 6):
            ii, jj = i + a, j + b
            if 0 <= ii < H and 0 <= jj < W:
                wgt = g[a + 5] * g[b + 5]
                xv, yv = x[ii, jj, c], y[ii, jj, c]
                s["x"] += wgt * xv
                s["y"] += wgt * yv
                s["xx"] += wgt * xv * xv
                s["yy"] += wgt * yv * yv
                s["xy"] += wgt * xv * yv
    mx, my = s["x"], s["y"]
    vx, vy, cxy = s["xx"] - mx * mx, s["yy"] - my * my, s["xy"] - mx * my
    return ((2 * mx * my + R.SSIM_C1) * (2 * cxy + R.SSIM_C2)) / \
        ((mx * mx + my * my + R.SSIM_C1) * (vx + vy + R.SSIM_C2))


def test_window_is_a_normalised_gaussian_of_sd_1_5():
    g = R.window()
    assert g.shape == (11,) and abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    for t in range(1, 6):
        assert abs(g[5 + t] / g[5] - math.exp(-t * t / (2 * 1.5 ** 2))) < 1e-14


def test_local_mean_of_a_constant_image_and_its_zero_padded_corner():
    img = np.full((20, 20), 0.7)
    m = R.local_mean(img)
    assert abs(m[10, 10] - 0.7) < 1e-14
    g = R.window()
    assert abs(m[0, 0] - 0.7 * g[5:].sum() ** 2) < 1e-14          # only the in-image quarter of the window
    assert abs(m[0, 10] - 0.7 * g[5:].sum()) < 1e-14


def test_ssim_of_an_image_with_itself_is_one():
    x, _ = _images()
    np.testing.assert_allclose(R.ssim_map(x, x), 1.0, atol=1e-12)


def test_ssim_of_constant_images_is_the_luminance_term():
    a, b = 0.3, 0.8
    S = R.ssim_map(np.full((21, 21, 3), a), np.full((21, 21, 3), b))
    assert abs(S[10, 10, 1] - (2 * a * b + R.SSIM_C1) / (a * a + b * b + R.SSIM_C1)) < 1e-12


@pytest.mark.parametrize("pix", [(0, 0, 0), (0, 11, 1), (8, 12, 2), (16, 22, 0), (5, 1, 1)])
def test_ssim_map_matches_the_explicit_window(pix):
    x, y = _images()
    i, j, c = pix
    assert abs(R.ssim_map(x, y)[i, j, c] - _ssim_bruteforce(x, y, i, j, c)) < 1e-12


@pytest.mark.parametrize("pix", [(0, 0, 0), (3, 7, 1), (8, 12, 2), (16, 22, 0), (10, 0, 2)])
def test_centre_gradient_matches_central_differences(pix):
    x, y = _images()
    i, j, c = pix
    h = 1e-6
    xp, xm = x.copy(), x.copy()
    xp[i, j, c] += h
    xm[i, j, c] -= h
    fd = (R.ssim_map(xp, y)[i, j, c] - R.ssim_map(xm, y)[i, j, c]) / (2 * h)
    an = R.ssim_center_grad(x, y)[i, j, c]
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd))


def test_residual_derivatives_match_central_differences():
    x, y = _images(seed=9, H=12, W=13)
    obj = R.Objective()
    wt = R.view_weights(x, y, obj)
    S = R.ssim_map(x, y)
    H, W = x.shape[:2]
    checked = 0
    for (i, j, c) in [(0, 0, 0), (5, 6, 1), (11, 12, 2), (3, 9, 0), (7, 2, 2)]:
        k = (i * W + j) * 3 + c
        d = x[i, j, c] - y[i, j, c]
        assert abs(d) > 1e-3 and 1 - S[i, j, c] > 1e-3      # away from the eps floors
        h = 1e-7
        r1 = lambda v: math.sqrt(obj.lambda1 * abs(v - y[i, j, c]))
        def r2(v):
            xx = x.copy()
            xx[i, j, c] = v
            return math.sqrt(obj.lambda2 * (1.0 - R.ssim_map(xx, y)[i, j, c]))
        v0 = x[i, j, c]
        fd1 = (r1(v0 + h) - r1(v0 - h)) / (2 * h)
        fd2 = (r2(v0 + h) - r2(v0 - h)) / (2 * h)
        assert abs(fd1 - wt.dr1[k]) <= 1e-6 * max(1.0, abs(fd1))
        assert abs(fd2 - wt.dr2[k]) <= 1e-6 * max(1.0, abs(fd2))
        assert abs(wt.r1[k] - r1(v0)) < 1e-14 and abs(wt.r2[k] - r2(v0)) < 1e-12
        assert abs(wt.e[k] - (fd1 * r1(v0) + fd2 * r2(v0))) <= 1e-6 * max(1.0, abs(wt.e[k]))
        assert abs(wt.w[k] - (fd1 * fd1 + fd2 * fd2)) <= 1e-6 * max(1.0, wt.w[k])
        checked += 1
    assert checked == 5
    # the energy is the sum of squared residuals, and L1 + SSIM per pixel channel
    assert abs(wt.cost - float(np.sum(obj.lambda1 * np.abs(x - y) + obj.lambda2 * (1 - S)))) < 1e-9


def test_eps_floor_bounds_the_l1_weight():
    x = np.full((12, 12, 3), 0.5)
    y = x.copy()
    y[6, 6, 0] += 1e-6
    obj = R.Objective()
    wt = R.view_weights(x, y, obj)
    k = (6 * 12 + 6) * 3
    assert abs(wt.dr1[k] + math.sqrt(obj.lambda1) / (2 * math.sqrt(obj.eps))) < 1e-12
    assert wt.dr1[k + 1] == 0.0                             # c = C exactly: no L1 derivative
    assert np.isfinite(wt.w).all() and np.isfinite(wt.e).all()


def _tiny_l1ssim(seed=21):
    P = small_scene(8, seed)
    cams = two_cams()
    rng = np.random.default_rng(seed)
    n = rng.standard_normal(J.n_residuals(cams))
    tgt = J.render(P, cams) + np.sign(n) * (0.01 + 0.05 * np.abs(n))   # |c - C| >= 0.01 (default mode)
    return P, cams, tgt


def test_weighted_products_and_diag_equal_the_explicit_jacobian():
    P, cams, tgt = _tiny_l1ssim()
    sys_ = solver.build_subset(P, cams, tgt, objective=R.Objective())
    n_res = J.n_residuals(cams)
    Jx = J.explicit_J(sys_.lin, n_res, P.shape[0]).toarray()
    A = Jx.T @ (sys_.W[:, None] * Jx)
    v = np.random.default_rng(5).standard_normal(P.shape)
    np.testing.assert_allclose(solver.apply_JTJ(sys_, v).ravel(), A @ v.ravel(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(sys_.M.ravel(), np.diag(A), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(sys_.b.ravel(), -Jx.T @ sys_.F, rtol=1e-10, atol=1e-12)


def test_b_is_minus_half_the_gradient_of_the_l1_energy():
    """With lambda2 = 0 the energy is sum lambda1 |c - C| and e = lambda1 sign(c - C) / 2
    exactly, so b = -J^T e = -grad E / 2 (smooth mode: no blending decisions)."""
    P, cams, tgt = _tiny_l1ssim(seed=33)
    obj = R.Objective(lambda1=0.8, lambda2=0.0)
    img = J.render(P, cams, smooth=True)
    assert np.min(np.abs(img - tgt)) > 1e-5
    sys_ = solver.build_subset(P, cams, tgt, smooth=True, objective=obj)
    E = lambda Q: R.cost(J.render(Q, cams, smooth=True), tgt, cams, obj)
    rng = np.random.default_rng(8)
    for _ in range(3):
        v = rng.standard_normal(P.shape)
        h = 1e-7
        fd = (E(P + h * v) - E(P - h * v)) / (2 * h)
        assert abs(fd - (-2.0 * float(np.sum(sys_.b * v)))) <= 1e-5 * max(1.0, abs(fd))


def test_l1ssim_lm_step_pred_is_the_gauss_newton_model():
    """pred = E + 2 gamma e.u + gamma^2 w.u^2 (u = (dc/dx) Delta) and the model is
    tangent to the L1 energy at gamma = 0 (lambda2 = 0, smooth mode)."""
    P, cams, tgt = _tiny_l1ssim(seed=44)
    obj = R.Objective(lambda2=0.0)
    res = solver.lm_step(P, [cams], [tgt], 1e-2, n_iters=6, smooth=True, objective=obj)
    sys_ = solver.build_subset(P, cams, tgt, smooth=True, objective=obj)
    u = J.apply_J(sys_.lin, res.delta, J.n_residuals(cams))
    assert abs(res.pred - (sys_.cost + 2 * np.dot(sys_.F, u) + np.dot(sys_.W, u * u))) <= 1e-9 * sys_.cost
    E = lambda g: R.cost(J.render(P + g * res.delta, cams, smooth=True), tgt, cams, obj)
    h = 1e-6
    assert abs((E(h) - E(-h)) / (2 * h) - 2 * np.dot(sys_.F, u)) <= 1e-4 * abs(2 * np.dot(sys_.F, u))


# ----------------------------------------------------------------------------- planted mistakes
def _pins_fail(checks) -> bool:
    """True if any of the given pin checks raises an AssertionError."""
    for check in checks:
        try:
            check()
        except AssertionError:
            return True
    return False


def _centre_grad_pins():
    for pix in [(0, 0, 0), (3, 7, 1), (8, 12, 2), (16, 22, 0), (10, 0, 2)]:
        test_centre_gradient_matches_central_differences(pix)


def _window_pins():
    test_local_mean_of_a_constant_image_and_its_zero_padded_corner()
    for pix in [(0, 0, 0), (0, 11, 1), (8, 12, 2), (16, 22, 0), (5, 1, 1)]:
        test_ssim_map_matches_the_explicit_window(pix)


def _mistaken_centre_grad(kind):
    def grad(x, y):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        t = R.ssim_terms(x, y)
        w0 = 1.0 if kind == "no_centre_weight" else R.window()[R.WINDOW // 2] ** 2
        A1 = 2.0 * t.mu_x * t.mu_y + R.SSIM_C1
        A2 = 2.0 * t.cov + R.SSIM_C2
        B1 = t.mu_x ** 2 + t.mu_y ** 2 + R.SSIM_C1
        B2 = t.var_x + t.var_y + R.SSIM_C2
        dA1 = 2.0 * w0 * t.mu_y
        dA2 = 2.0 * w0 * (y - t.mu_y)
        dB1 = 2.0 * w0 * t.mu_x
        dB2 = 2.0 * w0 * (x - t.mu_x) * (-1.0 if kind == "variance_sign" else 1.0)
        if kind == "dropped_covariance":
            dA2 = 0.0 * dA2
        return (dA1 * A2 + A1 * dA2) / (B1 * B2) - t.ssim * (dB1 / B1 + dB2 / B2)
    return grad


@pytest.mark.parametrize("kind", ["no_centre_weight", "variance_sign", "dropped_covariance"])
def test_planted_centre_gradient_mistakes_are_caught(monkeypatch, kind):
    monkeypatch.setattr(R, "ssim_center_grad", _mistaken_centre_grad(kind))
    assert _pins_fail([_centre_grad_pins, test_residual_derivatives_match_central_differences])


@pytest.mark.parametrize("mode", ["reflect", "nearest"])
def test_planted_padding_mistakes_are_caught(monkeypatch, mode):
    from scipy import ndimage

    def local_mean(img):
        g = R.window()
        out = ndimage.correlate1d(np.asarray(img, np.float64), g, axis=0, mode=mode)
        return ndimage.correlate1d(out, g, axis=1, mode=mode)
    monkeypatch.setattr(R, "local_mean", local_mean)
    assert _pins_fail([_window_pins])


def test_planted_residual_mistakes_are_caught(monkeypatch):
    real = R.view_weights

    def no_ssim_in_e(img, tgt, obj):
        w = real(img, tgt, obj)
        w.e = w.dr1 * w.r1               # the SSIM residual's share of J^T F dropped
        return w
    monkeypatch.setattr(R, "view_weights", no_ssim_in_e)
    assert _pins_fail([test_residual_derivatives_match_central_differences])
    monkeypatch.setattr(R, "view_weights", real)

    def weights_not_squared(img, tgt, obj):
        w = real(img, tgt, obj)
        w.w = np.abs(w.dr1) + np.abs(w.dr2)   # sum of |dr/dc| instead of their squares
        return w
    monkeypatch.setattr(R, "view_weights", weights_not_squared)
    assert _pins_fail([test_residual_derivatives_match_central_differences])
