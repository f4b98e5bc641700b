"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them; the
planted-mistake tests at the end check that for a few such slips.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as ss

import synth
from oracle import jacobian as J
from oracle import conventions as cv
from oracle import projection, raster, sh, solver

HERE = os.path.dirname(__file__)


# ----------------------------------------------------------------------------- helpers
def cam_at(pos, W=32, H=32, hfov=60.0, target=(0, 0, 0)):
    R, t = synth.look_at(np.asarray(pos, np.float64), target)
    f = (W / 2) / math.tan(math.radians(hfov) / 2)
    return synth.Camera(R, t, f, f, W / 2, H / 2, W, H)


def gaussian(pos, log_scale=-1.5, quat=(1, 0, 0, 0), logit=0.0, dc=(0.3, -0.2, 0.1), rest=0.0, rng=None):
    p = np.zeros(59)
    p[0:3] = pos
    p[3:6] = log_scale
    p[6:10] = quat
    p[10] = logit
    p[11:14] = dc
    if rng is not None:
        p[14:] = rest * rng.standard_normal(45)
    return p


def small_scene(n=5, seed=3, log_scale=-1.4, spread=0.5):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 59))
    P[:, 0:3] = rng.uniform(-spread, spread, (n, 3))
    P[:, 3:6] = rng.normal(log_scale, 0.2, (n, 3))
    q = rng.standard_normal((n, 4))
    P[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True) * rng.uniform(0.7, 1.3, (n, 1))
    P[:, 10] = rng.normal(-0.5, 0.5, n)
    P[:, 11:14] = rng.normal(0.0, 0.5, (n, 3))
    P[:, 14:] = rng.normal(0.0, 0.1, (n, 45))
    return P


def two_cams(W=32, H=24):
    return [cam_at((0.3, -3.5, 1.2), W, H), cam_at((-2.5, 2.0, -1.5), W, H)]


# ----------------------------------------------------------------------------- SH basis
def _scipy_real_sh(l, m, theta, phi):
    if m == 0:
        return ss.sph_harm_y(l, 0, theta, phi).real
    if m > 0:
        return math.sqrt(2) * (-1) ** m * ss.sph_harm_y(l, m, theta, phi).real
    return math.sqrt(2) * (-1) ** m * ss.sph_harm_y(l, -m, theta, phi).imag


def test_sh_basis_matches_scipy_up_to_fixed_sign():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    ours = sh.basis(d[:, 0], d[:, 1], d[:, 2])
    for k, (l, m) in enumerate(sh.LM):
        ref = _scipy_real_sh(l, m, theta, phi)
        s = np.sign(ours[k][np.argmax(np.abs(ref))] * ref[np.argmax(np.abs(ref))])
        assert s != 0
        np.testing.assert_allclose(ours[k], s * ref, atol=1e-12, err_msg=f"k={k} (l={l}, m={m})")


def test_sh_basis_orthonormal_on_sphere():
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly.
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    w = np.repeat(wg[:, None], nphi, axis=1) * (2 * np.pi / nphi)
    st = np.sqrt(1 - ct ** 2)
    Y = np.stack([np.broadcast_to(y, ct.shape) for y in sh.basis(st * np.cos(ph), st * np.sin(ph), ct)])
    G = np.einsum("kab,lab,ab->kl", Y, Y, w)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree0_colour_is_view_independent():
    p = gaussian((0.0, 0.0, 0.0), dc=(0.4, -0.3, 0.9))
    for cam in two_cams():
        pr = projection.project(p[None, :], cam)
        expect = np.maximum(0.0, 0.5 / math.sqrt(math.pi) * np.array([0.4, -0.3, 0.9]) + 0.5)
        np.testing.assert_allclose(pr.y[0, 6:9], expect, rtol=0, atol=1e-14)


# ----------------------------------------------------------------------------- projection
def test_projection_isotropic_gaussian_on_axis():
    z0, ls = 3.0, -2.0
    cam = synth.Camera(np.eye(3), np.zeros(3), 50.0, 60.0, 16.0, 12.0, 32, 24)
    q = np.array([0.3, -0.5, 0.7, 0.4])
    p = gaussian((0.0, 0.0, z0), log_scale=ls, quat=q)
    pr = projection.project(p[None, :], cam)
    s = math.exp(ls)
    a = (50.0 * s / z0) ** 2 + cv.DILATION
    c = (60.0 * s / z0) ** 2 + cv.DILATION
    np.testing.assert_allclose(pr.y[0, 0:2], [16.0, 12.0], atol=1e-12)
    np.testing.assert_allclose(pr.y[0, 2:5], [1 / a, 0.0, 1 / c], rtol=1e-12, atol=1e-15)
    assert pr.radius[0] == math.ceil(3 * math.sqrt(max(a, c)))


def test_projection_off_axis_mean_is_pinhole():
    cam = synth.Camera(np.eye(3), np.array([0.1, -0.2, 0.5]), 40.0, 45.0, 20.0, 10.0, 40, 20)
    p = gaussian((0.5, 0.3, 2.0))
    pr = projection.project(p[None, :], cam)
    tc = np.array([0.6, 0.1, 2.5])
    np.testing.assert_allclose(pr.y[0, 0:2], [40 * tc[0] / tc[2] + 20, 45 * tc[1] / tc[2] + 10], atol=1e-12)


def test_projection_culls_splats_whose_float32_covariance_chain_overflows():
    """The renderer computes a splat's covariance chain in float32; a splat is
    drawn only if that chain stays within the float32 range. For an isotropic
    Gaussian on the optical axis Sigma2 = a I with a = (f s / z)^2 + 0.3 (closed
    form), so the determinant's product a * c = a^2 leaves the range at
    a = sqrt(FLT_MAX): kept at 0.9 sqrt(FLT_MAX), culled at 1.1 sqrt(FLT_MAX).
    A log-scale whose 3D covariance exp(2 s) alone exceeds FLT_MAX is culled
    too, and ordinary log-scales (about -3.5) are 20 orders of magnitude away."""
    f32max = float(np.finfo(np.float32).max)
    z0, f = 3.0, 50.0
    cam = synth.Camera(np.eye(3), np.zeros(3), f, f, 16.0, 12.0, 32, 24)

    def log_scale_for(a):
        return math.log(math.sqrt(a - cv.DILATION) * z0 / f)

    q = np.array([0.3, -0.5, 0.7, 0.4])
    P = np.stack([gaussian((0.0, 0.0, z0), log_scale=log_scale_for(0.9 * math.sqrt(f32max)), quat=q),
                  gaussian((0.0, 0.0, z0), log_scale=log_scale_for(1.1 * math.sqrt(f32max)), quat=q),
                  gaussian((0.0, 0.0, z0), log_scale=0.5 * math.log(f32max) + 0.5, quat=q),
                  gaussian((0.0, 0.0, z0), log_scale=-3.5, quat=q)])
    pr = projection.project(P, cam, want_jac=False)
    assert pr.visible.tolist() == [True, False, False, True]
    a = (f * math.exp(P[0, 3]) / z0) ** 2 + cv.DILATION
    np.testing.assert_allclose(pr.y[0, 2:5] * a, [1.0, 0.0, 1.0], rtol=0, atol=1e-9)


# ----------------------------------------------------------------------------- compositing
def test_two_splat_closed_form_compositing():
    """c = a1 c1 + (1 - a1) a2 c2 for two splats along one pixel's ray (Eq. alpha-blending)."""
    cam = synth.Camera(np.eye(3), np.zeros(3), 30.0, 30.0, 16.0, 16.0, 32, 32)
    P = np.stack([gaussian((0.0, 0.0, 2.0), -1.0, logit=0.3, dc=(0.5, 0.1, -0.4)),
                  gaussian((0.05, -0.02, 3.0), -0.8, logit=-0.2, dc=(-0.2, 0.6, 0.3))])
    pr = projection.project(P, cam)
    ras = raster.rasterize(pr, cam)
    for (px, py) in [(16, 16), (14, 17), (18, 13)]:
        cols, alphas = [], []
        for s in range(2):
            mx, my, A, B, C, o = pr.y[s, :6]
            dx, dy = px + 0.5 - mx, py + 0.5 - my
            G = math.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
            alphas.append(min(0.99, o * G))
            cols.append(pr.y[s, 6:9])
        a1, a2 = alphas
        expect = a1 * cols[0] + (1 - a1) * a2 * cols[1]
        np.testing.assert_allclose(ras.image[py, px], expect, atol=1e-14)


def test_front_to_back_order_and_termination():
    """An opaque splat in front hides everything behind it once T < 1e-4."""
    cam = synth.Camera(np.eye(3), np.zeros(3), 30.0, 30.0, 16.0, 16.0, 32, 32)
    front = gaussian((0.0, 0.0, 2.0), 0.5, logit=12.0, dc=(1.0, 1.0, 1.0))
    back = gaussian((0.0, 0.0, 4.0), 0.5, logit=12.0, dc=(-1.0, 0.0, 1.0))
    for order in ([front, back], [back, front]):
        pr = projection.project(np.stack(order), cam)
        ras = raster.rasterize(pr, cam)
        c_front = pr.y[list(pr.idx).index(0 if order[0] is front else 1), 6:9]
        c_back = pr.y[list(pr.idx).index(1 if order[0] is front else 0), 6:9]
        # alpha = 0.99 at the centre (clamped): c = 0.99 cf + 0.01 * 0.99 cb, then T = 1e-4 stops
        np.testing.assert_allclose(ras.image[16, 16], 0.99 * c_front + 0.0099 * c_back, atol=1e-12)


# ----------------------------------------------------------------------------- derivatives
def _render_flat(P, cams, smooth):
    return J.render(P, cams, smooth)


@pytest.mark.parametrize("seed", [3, 11])
def test_jacobian_matches_central_differences_smooth_mode(seed):
    P = small_scene(5, seed)
    cams = two_cams()
    lin = J.linearise(P, cams, smooth=True)
    Jx = J.explicit_J(lin, J.n_residuals(cams), P.shape[0]).toarray()
    for col in range(P.size):
        g, k = divmod(col, 59)
        h = 1e-6 * max(1.0, abs(P[g, k]))
        Pp, Pm = P.copy(), P.copy()
        Pp[g, k] += h
        Pm[g, k] -= h
        fd = (_render_flat(Pp, cams, True) - _render_flat(Pm, cams, True)) / (2 * h)
        scale = max(np.linalg.norm(fd), np.linalg.norm(Jx[:, col]), 1e-3)
        assert np.linalg.norm(fd - Jx[:, col]) / scale < 1e-6, (g, k)


def _decisions(P, cams):
    out = []
    for cam in cams:
        pr = projection.project(P, cam)
        ras = raster.rasterize(pr, cam)
        out.append((pr.idx.tobytes(), ras.rec_pix.tobytes(), pr.idx[ras.rec_splat].tobytes(),
                    ras.rec_clamped.tobytes(), (pr.raw_rgb >= 0).tobytes()))
    return out


def test_jacobian_matches_central_differences_default_mode():
    """Default mode: FD on every parameter whose +-h perturbation changes no decision."""
    P = small_scene(6, 5, log_scale=-1.6)
    P[0, 10] = 8.0   # one wide, nearly opaque Gaussian so that the alpha clamp is exercised
    P[0, 3:6] = -0.3
    cams = two_cams(40, 24)
    lin = J.linearise(P, cams)
    Jx = J.explicit_J(lin, J.n_residuals(cams), P.shape[0]).toarray()
    assert any(vl.ras.rec_clamped.any() for vl in lin)
    base = _decisions(P, cams)
    checked = 0
    for col in range(P.size):
        g, k = divmod(col, 59)
        h = 1e-6 * max(1.0, abs(P[g, k]))
        Pp, Pm = P.copy(), P.copy()
        Pp[g, k] += h
        Pm[g, k] -= h
        if _decisions(Pp, cams) != base or _decisions(Pm, cams) != base:
            continue
        fd = (J.render(Pp, cams) - J.render(Pm, cams)) / (2 * h)
        # floor of 1e-2: below it, central-difference rounding noise (~1e-9) dominates
        scale = max(np.linalg.norm(fd), np.linalg.norm(Jx[:, col]), 1e-2)
        assert np.linalg.norm(fd - Jx[:, col]) / scale < 1e-6, (g, k)
        checked += 1
    assert checked > 0.9 * P.size


def test_adjoint_identity_tiny_workload():
    wl = synth.WORKLOADS["tiny"]
    P = synth.make_gaussians(wl).astype(np.float64)
    cams = synth.make_cameras(wl)[:3]
    lin = J.linearise(P, cams)
    n_res = J.n_residuals(cams)
    rng = np.random.default_rng(1)
    p = rng.standard_normal(P.shape)
    u = rng.standard_normal(n_res)
    lhs = np.dot(J.apply_J(lin, p, n_res), u)
    rhs = np.sum(p * J.apply_JT(lin, u, P.shape[0]))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_matrix_free_products_equal_explicit_jacobian():
    P = small_scene(8, 21)
    cams = two_cams()
    lin = J.linearise(P, cams)
    n_res = J.n_residuals(cams)
    Jx = J.explicit_J(lin, n_res, P.shape[0])
    rng = np.random.default_rng(2)
    p = rng.standard_normal(P.shape)
    u = rng.standard_normal(n_res)
    np.testing.assert_allclose(J.apply_J(lin, p, n_res), Jx @ p.ravel(), atol=1e-12)
    np.testing.assert_allclose(J.apply_JT(lin, u, P.shape[0]).ravel(), Jx.T @ u, atol=1e-12)


def test_dense_JTJ_symmetric_psd_and_diag():
    """Dense J^T J for a few dozen Gaussians: symmetric, PSD, diagonal = diag(J^T J)."""
    P = small_scene(30, 7, log_scale=-1.8, spread=0.8)
    cams = two_cams(48, 40)
    lin = J.linearise(P, cams)
    Jx = J.explicit_J(lin, J.n_residuals(cams), P.shape[0]).toarray()
    A = Jx.T @ Jx
    assert A.shape == (30 * 59, 30 * 59)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= -1e-10 * ev.max()
    np.testing.assert_allclose(J.jacobi_diag(lin, P.shape[0]).ravel(), np.diag(A), rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------- PCG
def _tiny_system(n_gauss=3, seed=4, W=40, H=32):
    P = small_scene(n_gauss, seed, log_scale=-1.2, spread=0.4)
    cams = [cam_at((0.3, -3.0, 1.0), W, H), cam_at((-2.0, 2.0, -1.0), W, H), cam_at((2.5, 1.0, 2.0), W, H)]
    targets = np.concatenate([im.ravel() for im in synth.smooth_images(9, cams)]).astype(np.float64)
    return P, cams, targets


def test_pcg_equals_dense_cholesky_solve():
    P, cams, tg = _tiny_system()
    sys_ = solver.build_subset(P, cams, tg)
    lam = 1e-3
    x, st = solver.solve_subset(sys_, lam, n_iters=600)
    Jx = J.explicit_J(sys_.lin, J.n_residuals(cams), P.shape[0]).toarray()
    obs = sys_.M.ravel() > 0.0
    A = (Jx.T @ Jx + lam * np.diag(solver.clamp_diag(sys_.M.ravel())))[np.ix_(obs, obs)]
    L = np.linalg.cholesky(A)
    ref = np.zeros(P.size)
    ref[obs] = np.linalg.solve(L.T, np.linalg.solve(L, sys_.b.ravel()[obs]))
    assert not st.breakdown
    assert np.linalg.norm(x.ravel() - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.all(x.ravel()[~obs] == 0.0)


def test_pcg_energy_norm_error_decreases():
    P, cams, tg = _tiny_system(seed=6)
    sys_ = solver.build_subset(P, cams, tg)
    lam = 1e-2
    Jx = J.explicit_J(sys_.lin, J.n_residuals(cams), P.shape[0]).toarray()
    A = Jx.T @ Jx + lam * np.diag(solver.clamp_diag(sys_.M.ravel()))
    xs = np.linalg.lstsq(A, sys_.b.ravel(), rcond=None)[0]
    errs = []
    for n in range(0, 12):
        x, _ = solver.solve_subset(sys_, lam, n_iters=n)
        e = x.ravel() - xs
        errs.append(e @ A @ e)
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.5 * errs[0]


def test_pcg_first_iteration_by_hand():
    """One iteration of Algorithm 1 written out on a 2x2 SPD system."""
    A0 = np.array([[4.0, 1.0], [1.0, 3.0]])
    M = np.diag(A0).copy()          # inside the clamp range, so clamping changes nothing
    b = np.array([1.0, 2.0])
    lam = 0.5
    x, _ = solver.pcg(lambda v: A0 @ v, b, M, lam, n_iters=1)
    Ad = A0 + lam * np.diag(M)
    x0 = b / M
    r0 = b - Ad @ x0
    z0 = r0 / M
    alpha = (r0 @ z0) / (z0 @ Ad @ z0)
    np.testing.assert_allclose(x, x0 + alpha * z0, rtol=1e-15)
    x2, _ = solver.pcg(lambda v: A0 @ v, b, M, lam, n_iters=2)
    np.testing.assert_allclose(x2, np.linalg.solve(Ad, b), rtol=1e-12)


# ----------------------------------------------------------------------------- weighted mean
def test_diag_clamp_bounds_the_jacobi_step():
    """A barely observed parameter (diag 1e-17) no longer gets x0 = b / diag ~ 1e7."""
    M = np.array([1e-17, 2.0, 0.0])
    b = np.array([1e-10, 1.0, 0.0])
    x, _ = solver.pcg(lambda v: M * v, b, M, 1e-3, n_iters=0)
    np.testing.assert_allclose(x, [1e-4, 0.5, 0.0])
    np.testing.assert_allclose(solver.clamp_diag(np.array([1e-9, 5.0, 1e40])), [1e-6, 5.0, 1e32])


def test_combine_single_subset_is_identity():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((7, 59))
    m = rng.uniform(0.1, 2.0, (7, 59))
    m[0, 0] = 0.0
    out = solver.combine([d], [m])
    expect = d.copy()
    expect[0, 0] = 0.0
    np.testing.assert_allclose(out, expect, rtol=1e-15)
    np.testing.assert_allclose(solver.combine([d, d], [m, m]), expect, rtol=1e-15)


def test_combine_is_exact_for_diagonal_subset_systems():
    """Sec. B: with diagonal J_i^T J_i the weighted mean equals the joint solution."""
    rng = np.random.default_rng(1)
    m1, m2, m3 = (rng.uniform(0.1, 3.0, 50) for _ in range(3))
    c1, c2, c3 = (rng.standard_normal(50) for _ in range(3))
    deltas = [c1 / m1, c2 / m2, c3 / m3]
    joint = (c1 + c2 + c3) / (m1 + m2 + m3)
    np.testing.assert_allclose(solver.combine(deltas, [m1, m2, m3]), joint, rtol=1e-13)


# ----------------------------------------------------------------------------- LM
def test_lambda_update_matches_worked_values():
    with open(os.path.join(HERE, "golden", "lambda_update.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        rho = c["rho"]
        factor = (1 - (2 * rho - 1) ** 3) if rho > 1e-5 else 2.0
        assert abs(factor - c["factor"]) < 1e-15


def test_lm_accepted_steps_decrease_cost():
    wl = synth.small_workload("lmtest", 77, 60, 4, 40, 32, cam_radius=3.0, log_scale_mean=-2.2)
    P = synth.make_gaussians(wl).astype(np.float64)
    cams = synth.make_cameras(wl)
    tgt_params = synth.perturbed_copy(wl, synth.make_gaussians(wl)).astype(np.float64)
    tg = J.render(tgt_params, cams)
    lam = 1e-3
    n_acc = 0
    for step in range(3):
        res = solver.lm_step(P, [cams], [tg], lam)
        if res.accepted:
            n_acc += 1
            assert res.cost_new < res.cost
            assert res.rho > 1e-5
        else:
            np.testing.assert_array_equal(res.params, P)
        P, lam = res.params, res.lam
    assert n_acc >= 1


def test_lm_gain_ratio_tends_to_one():
    """rho -> 1 as gamma -> 0: the Gauss-Newton model is first-order exact (smooth mode)."""
    P, cams, tg = _tiny_system(seed=8)
    sys_ = solver.build_subset(P, cams, tg, smooth=True)
    d, _ = solver.solve_subset(sys_, 1e-3, 8)
    n_res = sys_.F.shape[0]
    Jd = J.apply_J(sys_.lin, d, n_res)
    rhos = []
    for gamma in (1e-2, 1e-3, 1e-4):
        F1 = J.render(P + gamma * d, cams, smooth=True) - tg
        pred = sys_.cost - np.sum((gamma * Jd + sys_.F) ** 2)
        rhos.append((sys_.cost - F1 @ F1) / pred)
    assert abs(rhos[-1] - 1) < 1e-3
    assert abs(rhos[-1] - 1) < abs(rhos[0] - 1)


# ----------------------------------------------------------------------------- planted mistakes
def _fd_pin_fails(monkeypatch_fn):
    """Run a reduced smooth-mode FD pin with a mistake planted in the oracle; True if it fails."""
    P = small_scene(3, 13)
    cams = two_cams(24, 20)
    with monkeypatch_fn():
        lin = J.linearise(P, cams, smooth=True)
        Jx = J.explicit_J(lin, J.n_residuals(cams), P.shape[0]).toarray()
    worst = 0.0
    for col in range(P.size):
        g, k = divmod(col, 59)
        h = 1e-6 * max(1.0, abs(P[g, k]))
        Pp, Pm = P.copy(), P.copy()
        Pp[g, k] += h
        Pm[g, k] -= h
        fd = (J.render(Pp, cams, True) - J.render(Pm, cams, True)) / (2 * h)
        scale = max(np.linalg.norm(fd), np.linalg.norm(Jx[:, col]), 1e-3)
        worst = max(worst, np.linalg.norm(fd - Jx[:, col]) / scale)
    return worst > 1e-6


def _patched(module, name, replacement):
    import contextlib

    @contextlib.contextmanager
    def cm():
        orig = getattr(module, name)
        setattr(module, name, replacement(orig))
        try:
            yield
        finally:
            setattr(module, name, orig)
    return cm


def _drop_behind_term(orig):
    def f(proj, ras):
        keep = ras.rec_dcda
        ras.rec_dcda = ras.rec_T[:, None] * proj.y[ras.rec_splat, 6:9]   # T c_s only
        try:
            return orig(proj, ras)
        finally:
            ras.rec_dcda = keep
    return f


def _flip_conic_cross_sign(orig):
    def f(proj, ras):
        a = orig(proj, ras)
        a[:, :, 3] = -a[:, :, 3]
        return a
    return f


def _swap_mean_axes(orig):
    def f(proj, ras):
        a = orig(proj, ras)
        a[:, :, [0, 1]] = a[:, :, [1, 0]]
        return a
    return f


@pytest.mark.parametrize("mistake", [_drop_behind_term, _flip_conic_cross_sign, _swap_mean_axes])
def test_planted_mistakes_are_caught(mistake):
    assert _fd_pin_fails(_patched(J, "dc_dy", mistake))


# ----------------------------------------------------------------------------- learned preconditioner MLP
def _mlp_case(seed=0, n=4):
    """A random network off its Jacobi start and a random SPD system over n Gaussians."""
    from oracle import mlp
    rng = np.random.default_rng(seed)
    net = mlp.init_mlp(seed)
    net.W3 = rng.standard_normal(net.W3.shape) * 0.1
    net.b3 = net.b3 + rng.standard_normal(net.b3.shape) * 0.1
    phi = rng.standard_normal((n, 64))
    m = n * 59
    B = rng.standard_normal((2 * m, m)) * np.exp(rng.normal(0.0, 1.0, m))
    A = B.T @ B / (2 * m) + 0.05 * np.eye(m)
    M = np.diag(A).reshape(n, 59).copy()
    b = rng.standard_normal((n, 59))
    apply_A = lambda v: (A @ v.ravel()).reshape(v.shape)
    return mlp, net, phi, M, b, apply_A, A


def test_mlp_features_layout_on_closed_form_values():
    """phi = [log M (59), log-scale (3), sigmoid(opacity logit) (1), log(1 + entries) (1)]
    for parameter rows whose other columns hold noise that must not leak in."""
    from oracle import mlp
    rng = np.random.default_rng(5)
    P = rng.normal(size=(2, 59))
    P[:, 3:6] = [[-3.0, -2.5, -4.0], [0.5, 0.0, -1.0]]
    P[:, 10] = [math.log(3.0), 0.0]                       # opacities 3/4 and 1/2
    M = np.exp(np.tile(np.linspace(-5.0, 5.0, 59), (2, 1)))
    M[1, 7] = 0.0                                          # a parameter no entry touches
    entries = np.array([math.e ** 2 - 1.0, 0.0])
    phi = mlp.features(M, P, entries)
    assert phi.shape == (2, 64)
    assert np.allclose(phi[0, :59], np.linspace(-5.0, 5.0, 59), atol=1e-9)
    assert phi[1, 7] == pytest.approx(math.log(1e-12)) and np.isfinite(phi).all()
    assert np.array_equal(phi[:, 59:62], P[:, 3:6])
    assert phi[:, 62] == pytest.approx([0.75, 0.5])
    assert phi[:, 63] == pytest.approx([2.0, 0.0])


def test_mlp_standardizer_is_the_population_moments_with_a_floor():
    from oracle import mlp
    phi = np.array([[1.0, 4.0], [2.0, 4.0], [3.0, 4.0]])
    mu, sd = mlp.standardizer(phi)
    assert mu == pytest.approx([2.0, 4.0])
    assert sd == pytest.approx([math.sqrt(2.0 / 3.0), 1e-6])   # 1/n, not 1/(n - 1); a constant column floored


def test_mlp_activations_closed_forms():
    from oracle import mlp
    assert abs(mlp.softplus(0.0) - math.log(2.0)) < 1e-15
    assert abs(mlp.softplus(mlp.B3_INIT) - 1.0) < 1e-15
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu_grad(0.0) - 0.5) < 1e-15
    x = np.array([-3.0, -0.5, 0.7, 2.5])
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in x]))
    np.testing.assert_allclose(mlp.gelu(x), x * phi, rtol=1e-15)


def test_mlp_starts_at_the_jacobi_preconditioner():
    from oracle import mlp
    net = mlp.init_mlp(3)
    rng = np.random.default_rng(1)
    M = np.exp(rng.normal(-3, 3, (25, 59)))
    D = mlp.precond_diag(net, rng.standard_normal((25, 64)), M)
    np.testing.assert_allclose(D, solver.jacobi_inverse(M), rtol=1e-14)


def test_unrolled_pcg_reaches_the_exact_solution_in_n_steps():
    # conjugate gradients terminate in at most n steps in exact arithmetic
    from oracle import mlp
    rng = np.random.default_rng(4)
    n = 14
    B = rng.standard_normal((30, n))
    A = B.T @ B + 0.5 * np.eye(n)
    b = rng.standard_normal(n)
    d = np.exp(rng.normal(0.0, 0.5, n)) / np.diag(A)
    x, tp = mlp.unrolled_pcg(lambda v: A @ v, b, d, n)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(tp.r[n], b - A @ x, atol=1e-9)


def test_unrolled_pcg_matches_algorithm_1_with_the_same_diagonal():
    from oracle import mlp
    rng = np.random.default_rng(6)
    n, lam = 40, 0.3
    J_ = rng.standard_normal((70, n)) * np.exp(rng.normal(0.0, 1.0, n))
    JTJ = J_.T @ J_
    Mraw = np.diag(JTJ).copy()
    b = rng.standard_normal(n)
    d = np.exp(rng.normal(0.0, 0.3, n)) / solver.clamp_diag(Mraw)
    x1, _ = solver.pcg(lambda v: JTJ @ v, b, Mraw, lam, n_iters=6, Minv=d)
    x2, _ = mlp.unrolled_pcg(lambda v: JTJ @ v + lam * solver.clamp_diag(Mraw) * v, b, d, 6)
    np.testing.assert_allclose(x2, x1, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("K", [1, 3, 8])
def test_unrolled_pcg_adjoint_matches_central_differences(K):
    from oracle import mlp
    rng = np.random.default_rng(K)
    n = 30
    B = rng.standard_normal((60, n)) * np.exp(rng.standard_normal(n))
    A = B.T @ B + 0.1 * np.eye(n)
    b = rng.standard_normal(n)
    d = np.exp(rng.standard_normal(n)) / np.diag(A)
    L, g = mlp.unrolled_loss_and_grad(lambda v: A @ v, b, d, K)
    _, tp = mlp.unrolled_pcg(lambda v: A @ v, b, d, K)
    assert abs(L - 0.5 * math.log(np.dot(tp.r[K], tp.r[K]) / np.dot(b, b))) < 1e-14
    for k in range(n):
        h = 1e-6 * d[k]
        e = np.zeros(n)
        e[k] = h
        fd = (mlp.unrolled_loss_and_grad(lambda v: A @ v, b, d + e, K)[0]
              - mlp.unrolled_loss_and_grad(lambda v: A @ v, b, d - e, K)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * np.abs(g).max(), (k, fd, g[k])


def test_bf16_rounding_of_the_network_weights():
    """Round to nearest even on the top 16 bits of the float32 (bfloat16: 8-bit
    exponent, 7 mantissa bits): exact halfway cases go to the even mantissa;
    random values agree with torch's bfloat16 conversion; and the network with
    rounded weights is the exact network evaluated at those weights."""
    from oracle import mlp
    torch = pytest.importorskip("torch")
    one = 1.0
    cases = [(one, one), (one + 2.0 ** -8, one), (one + 3 * 2.0 ** -8, one + 2.0 ** -6),
             (one + 2.0 ** -8 + 2.0 ** -20, one + 2.0 ** -7), (-2.5, -2.5), (0.0, 0.0),
             (3.0e38, float(torch.tensor(3.0e38).to(torch.bfloat16).float()))]
    for x, want in cases:
        assert mlp.bf16_round(np.array([x]))[0] == want, x
    x = np.random.default_rng(1).standard_normal(5000) * np.exp(np.random.default_rng(2).normal(0, 8, 5000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)
    _, net, phi, M, _, _, _ = _mlp_case(0, 20)
    rounded = mlp.MLP(mlp.bf16_round(net.W1), net.b1, mlp.bf16_round(net.W2), net.b2, mlp.bf16_round(net.W3),
                      net.b3)
    np.testing.assert_array_equal(mlp.precond_diag(net, phi, M), mlp.precond_diag(rounded, phi, M, bf16=False))
    assert np.abs(mlp.precond_diag(net, phi, M) - mlp.precond_diag(net, phi, M, bf16=False)).max() > 0


def test_mlp_backward_matches_central_differences():
    mlp, net, phi, M, b, _, _ = _mlp_case(0, 40)
    W = np.random.default_rng(9).standard_normal(M.shape)   # f(net) = sum W * D(net)
    g = np.concatenate([x.ravel() for x in mlp.backward(net, phi, M, W, bf16=False)])
    v = net.flat()
    f = lambda w: float(np.sum(W * mlp.precond_diag(mlp.MLP.from_flat(w), phi, M, bf16=False)))
    rng = np.random.default_rng(5)
    for i in rng.choice(v.size, 150, replace=False):
        h = 1e-6 * max(1.0, abs(v[i]))
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (f(vp) - f(vm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_mlp_loss_gradient_matches_central_differences():
    mlp, net, phi, M, b, apply_A, _ = _mlp_case(1, 3)
    L, grads = mlp.loss_and_grad(net, phi, M, apply_A, b, 5, bf16=False)
    g = np.concatenate([x.ravel() for x in grads])
    v = net.flat()
    rng = np.random.default_rng(7)
    for i in rng.choice(v.size, 60, replace=False):
        h = 1e-6 * max(1.0, abs(v[i]))
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (mlp.loss_and_grad(mlp.MLP.from_flat(vp), phi, M, apply_A, b, 5, bf16=False)[0]
              - mlp.loss_and_grad(mlp.MLP.from_flat(vm), phi, M, apply_A, b, 5, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1e-3, np.abs(g).max()), i


def test_adam_first_step_moves_each_weight_by_the_learning_rate():
    # after one step m_hat = g and v_hat = g^2, so every weight moves by lr * g / (|g| + eps)
    from oracle import mlp
    net = mlp.init_mlp(2)
    rng = np.random.default_rng(3)
    grads = [rng.standard_normal(p.shape) for p in net.params()]
    before = net.flat()
    mlp.Adam(lr=0.01, eps=0.0).step(net, grads)
    np.testing.assert_allclose(net.flat() - before, -0.01 * np.sign(np.concatenate([g.ravel() for g in grads])),
                               rtol=1e-12)


def test_mlp_training_lowers_the_unrolled_residual():
    mlp, net, phi, M, b, apply_A, _ = _mlp_case(2, 3)
    net = mlp.init_mlp(2)
    opt = mlp.Adam(lr=3e-3)
    L0 = mlp.loss_and_grad(net, phi, M, apply_A, b, 6)[0]
    for _ in range(60):
        L, g = mlp.loss_and_grad(net, phi, M, apply_A, b, 6)
        opt.step(net, g)
    assert L < L0 - 0.1


# ----------------------------------------------------------------------------- line search (Eq. line-search)
def _ragged_lm(ls_steps):
    from common import ragged_case
    wl, P, cams, tgt = ragged_case()
    return P.astype(np.float64), cams, tgt.astype(np.float64), solver.lm_step(
        P.astype(np.float64), [cams], [tgt.astype(np.float64)], 1e-3, n_iters=8, ls_steps=ls_steps)


def test_line_search_views_are_the_first_30_percent_in_subset_order():
    assert solver.line_search_views([[0, 1, 2], [3, 4, 5, 6, 7]], 0.3) == [3, 0]
    assert solver.line_search_views([[0], [1, 2, 3], [4, 5, 6, 7, 8], [9, 10, 11]], 0.3) == [1, 3, 0, 0]
    assert solver.line_search_views([[0, 1]], 0.3) == [1]


def test_line_search_with_one_candidate_is_the_full_step():
    import warnings
    warnings.filterwarnings("ignore")
    P, cams, tgt, r1 = _ragged_lm(1)
    r0 = solver.lm_step(P, [cams], [tgt], 1e-3, n_iters=8, ls_steps=0)
    assert r1.gamma == 1.0 and r0.gamma == 1.0
    assert r1.cost_new == r0.cost_new and r1.pred == r0.pred and r1.accepted == r0.accepted


def test_line_search_on_a_doubled_step_halves_gamma():
    # x + 2 Delta 2^-k = x + Delta 2^-(k-1) exactly: the costs shift by one candidate
    import warnings
    warnings.filterwarnings("ignore")
    P, cams, tgt, r = _ragged_lm(8)
    assert r.gamma == 0.5 and len(r.ls_costs) == 3          # 2172 > 1597 < 2007: stops at the rise
    g2, costs2 = solver.line_search(P, 2.0 * r.delta, [cams], [tgt], 8, 0.3)
    assert g2 == r.gamma / 2
    assert costs2[1:] == r.ls_costs
    assert costs2[0] > costs2[1]


def test_line_search_step_is_accepted_and_lowers_the_cost():
    import warnings
    warnings.filterwarnings("ignore")
    P, cams, tgt, r = _ragged_lm(8)
    assert r.accepted and r.cost_new < r.cost
    np.testing.assert_allclose(r.params, P + r.gamma * r.delta)
    # the predicted cost uses gamma Delta: between the full-step prediction and the current cost
    full = solver.lm_step(P, [cams], [tgt], 1e-3, n_iters=8, ls_steps=0)
    assert r.pred != full.pred


# ----------------------------------------------------------------------------- sampled tiles of large scenes
def _records(vl, pixels=None):
    order = np.lexsort((vl.gauss, vl.ras.rec_pix))
    pix, gs, a = vl.ras.rec_pix[order], vl.gauss[order], vl.a[order]
    if pixels is not None:
        keep = np.isin(pix, pixels)
        pix, gs, a = pix[keep], gs[keep], a[keep]
    return pix, gs, a


def test_linearising_selected_tiles_matches_the_whole_view():
    from common import ragged_case
    wl, P, cams, tgt = ragged_case()
    cam = cams[1]
    full = J.linearise_view(P.astype(np.float64), cam)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    every = [(x, y) for y in range(ty) for x in range(tx)]
    part = J.linearise_view_tiles(P, cam, every)
    for u, v in zip(_records(full), _records(part)):
        np.testing.assert_array_equal(u, v) if u.dtype != np.float64 else np.testing.assert_allclose(u, v, rtol=1e-12)
    np.testing.assert_array_equal(full.ras.image, part.ras.image)
    # a few tiles: exactly the whole view's records on their pixels, black elsewhere
    some = [(0, 0), (tx - 1, ty - 1), (1, 2)]
    sub = J.linearise_view_tiles(P, cam, some)
    pixels = np.concatenate([((np.arange(y * 16, min(cam.height, y * 16 + 16))[:, None] * cam.width)
                              + np.arange(x * 16, min(cam.width, x * 16 + 16))[None, :]).ravel() for x, y in some])
    for u, v in zip(_records(full, pixels), _records(sub)):
        np.testing.assert_array_equal(u, v) if u.dtype != np.float64 else np.testing.assert_allclose(u, v, rtol=1e-12)
    img = full.ras.image.reshape(-1, 3)
    np.testing.assert_array_equal(sub.ras.image.reshape(-1, 3)[pixels], img[pixels])
    others = np.setdiff1d(np.arange(cam.width * cam.height), pixels)
    assert not sub.ras.image.reshape(-1, 3)[others].any()
