"""Edge cases of the CUDA path (GPU only): an empty scene, a single Gaussian,
views of 1x1 and 17x3 pixels, a cache of more than 64 views, and invalid
arguments.

The empty scene has every Gaussian behind the camera: no splat, no tile key,
no cache entry. Everything must still run and give the defined results: a
black image, zero J p, J^T u and diag, b = 0 (so PCG reports a breakdown on
p^T g = 0 without producing non-finite values), and a rejected LM step.
"""
import ctypes

import numpy as np
import pytest

import synth
from common import N_PARAMS, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12892_gb300 import build
    build.build()
    import paper_2409_12892_gb300 as g
    return g


def _case(n, W, H, seed=41, behind=False, log_scale_mean=-2.0):
    wl = synth.small_workload("edge", seed, n, 1, W, H, cam_radius=4.0, log_scale_mean=log_scale_mean)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    if behind:
        R = np.asarray(cams[0].R, np.float64)
        campos = -R.T @ np.asarray(cams[0].t, np.float64)
        P = P.copy()
        P[:, 0:3] = (1.5 * campos)[None, :] + 0.1 * synth.random_vector(seed, (n, 3))
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(seed, cams)]).astype(np.float32)
    return P, cams, tgt


def test_empty_scene_runs_and_gives_the_defined_results(lib):
    P, cams, tgt = _case(200, 40, 24, behind=True)
    N = P.shape[0]
    ctx = lib.Context(n_iters=4, break_rel2=0.0)
    tg = torch.from_numpy(tgt).cuda().view(-1, 3)
    cache = ctx.build_cache(lib.to_soa(P), N, cams, tg)
    info = cache.info()
    assert info.entries == 0 and info.segments == 0 and info.splats == 0
    np.testing.assert_array_equal(cache.F.cpu().numpy().ravel(), -tgt)          # black image
    assert abs(cache.cost - float(np.dot(tgt.astype(np.float64), tgt))) <= 1e-6 * cache.cost
    assert not cache.b.any()
    p = torch.from_numpy(synth.random_vector(1, (N_PARAMS, cache.ld)).astype(np.float32)).cuda()
    assert not ctx.apply_J(cache, p).any()
    assert not ctx.apply_JT(cache, tg).any()
    diag = ctx.jacobi_diag(cache)
    assert not diag.any()
    x, st, status = ctx.pcg_solve(cache, cache.b, diag, 1e-3)
    assert status == 1 and st.breakdown == 1 and st.bb == 0.0
    assert torch.isfinite(x).all() and not x.any()
    params = lib.to_soa(P)
    before = params.clone()
    state, stats = ctx.lm_step(params, N, cams, tg, [[0]], 1e-3)
    assert not stats.accepted and abs(state.lambda_ - 2e-3) < 1e-9
    assert torch.equal(params, before)
    cache.free()


@pytest.mark.parametrize("n,W,H", [(1, 40, 24), (300, 1, 1), (300, 17, 3), (300, 16, 16)])
def test_small_cases_match_the_oracle(lib, n, W, H):
    from oracle import jacobian as J
    P, cams, tgt = _case(n, W, H, log_scale_mean=-1.0 if n == 1 else -2.0)
    N = P.shape[0]
    lin = J.linearise(P.astype(np.float64), cams)
    mask = np.concatenate([(vl.ras.margin >= 1e-4) & ~vl.ras.flip for vl in lin])
    n_res = J.n_residuals(cams)
    ctx = lib.Context()
    cache = ctx.build_cache(lib.to_soa(P), N, cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    img = cache.F.cpu().numpy() + tgt.reshape(-1, 3)
    ref = np.concatenate([vl.ras.image.reshape(-1, 3) for vl in lin])
    assert np.abs(img[mask] - ref[mask]).max(initial=0.0) <= 1e-5
    if n == 1:
        assert cache.info().entries > 0
    p = synth.random_vector(2, (N, N_PARAMS))
    u = ctx.apply_J(cache, lib.to_soa(p)).cpu().numpy()
    u_ref = J.apply_J(lin, p.astype(np.float64), n_res).reshape(-1, 3)
    if np.linalg.norm(u_ref[mask]) > 0:
        assert rel_l2(u[mask], u_ref[mask]) < 1e-4
    uu = np.where(np.repeat(mask, 3).reshape(-1, 3), synth.random_vector(3, (n_res // 3, 3)), 0.0).astype(np.float32)
    g = lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(uu).cuda()), N)
    g_ref = J.apply_JT(lin, uu.astype(np.float64).ravel(), N)
    if np.linalg.norm(g_ref) > 0:
        assert rel_l2(g, g_ref) < 1e-4
    d = lib.from_soa(ctx.jacobi_diag(cache), N)
    d_ref = J.jacobi_diag(lin, N)
    if np.linalg.norm(d_ref) > 0 and mask.all():
        assert rel_l2(d, d_ref) < 1e-4
    cache.free()


def test_more_than_64_views_match_the_oracle(lib):
    """A cache of 70 views has no 64-bit view masks, so the per-Gaussian kernels
    (tangent, adjoint, diagonal) walk each Gaussian's views themselves instead of
    dealing the (Gaussian, view) pairs of a warp to its lanes."""
    from oracle import jacobian as J
    wl = synth.small_workload("manyviews", 43, 200, 70, 32, 24, cam_radius=4.0, log_scale_mean=-3.2)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(43, cams)]).astype(np.float32)
    N = P.shape[0]
    lin = J.linearise(P.astype(np.float64), cams)
    mask = np.concatenate([(vl.ras.margin >= 1e-4) & ~vl.ras.flip for vl in lin])
    n_res = J.n_residuals(cams)
    ctx = lib.Context()
    cache = ctx.build_cache(lib.to_soa(P), N, cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    assert cache.info().views == 70 and cache.info().entries > 0
    p = synth.random_vector(2, (N, N_PARAMS))
    u = ctx.apply_J(cache, lib.to_soa(p)).cpu().numpy()
    u_ref = J.apply_J(lin, p.astype(np.float64), n_res).reshape(-1, 3)
    assert rel_l2(u[mask], u_ref[mask]) < 1e-4
    uu = np.where(np.repeat(mask, 3).reshape(-1, 3), synth.random_vector(3, (n_res // 3, 3)), 0.0).astype(np.float32)
    g = lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(uu).cuda()), N)
    assert rel_l2(g, J.apply_JT(lin, uu.astype(np.float64).ravel(), N)) < 1e-4
    # the diagonal of every Gaussian none of whose records sits at a pixel with a
    # near-threshold blending decision (the diagonal sums over all pixels)
    flagged = np.zeros(N, bool)
    for vl in lin:
        bad = ~mask[vl.pix_off // 3 + vl.ras.rec_pix]
        flagged[vl.gauss[bad]] = True
    assert (~flagged).sum() > N // 2
    d = lib.from_soa(ctx.jacobi_diag(cache), N)
    d_ref = J.jacobi_diag(lin, N)
    assert rel_l2(d[~flagged], d_ref[~flagged]) < 1e-4
    cache.free()


def test_invalid_arguments_are_rejected(lib):
    P, cams, tgt = _case(10, 16, 16)
    ctx = lib.Context()
    L = ctx.lib
    params = lib.to_soa(P)
    ca = lib.make_cameras(cams)
    h = ctypes.c_void_p()
    tg = torch.from_numpy(tgt).cuda().view(-1, 3)
    b = torch.zeros((N_PARAMS, params.shape[1]), device="cuda")
    cost = ctypes.c_double()
    args = lambda N, ld, V: (ctx.h, ctypes.c_void_p(params.data_ptr()), N, ld, ca, V, ctypes.c_void_p(tg.data_ptr()),
                             ctypes.byref(h), None, ctypes.c_void_p(b.data_ptr()), ctypes.byref(cost))
    assert L.gslm_build_cache(*args(0, params.shape[1], 1)) == -1                 # no Gaussians
    assert L.gslm_build_cache(*args(10, 6, 1)) == -1                              # ld not a multiple of 4
    assert L.gslm_build_cache(*args(10, 8, 1)) == -1                              # ld < N
    assert L.gslm_build_cache(*args(10, params.shape[1], 0)) == -1                # no views
    assert b"V <= 0" in L.gslm_last_error(ctx.h)
    assert L.gslm_apply_J(ctx.h, None, None, None) == -1
    assert L.gslm_pcg_solve(ctx.h, None, None, None, None, ctypes.c_float(1e-3), None, None) == -1
    opt = lib.gslm.Options()
    L.gslm_default_options(ctypes.byref(opt))
    opt.cache_fmt = 7
    assert L.gslm_set_options(ctx.h, ctypes.byref(opt)) == -1
    # a valid call after the rejected ones still works
    cache = ctx.build_cache(params, P.shape[0], cams, tg)
    assert cache.info().views == 1
    # vectors of the PCG solve must start on a 16-byte boundary (the kernels move float4s)
    ld = params.shape[1]
    shifted = torch.zeros(N_PARAMS * ld + 1, device="cuda")[1:]
    diag = ctx.jacobi_diag(cache)
    x = torch.zeros_like(diag)
    P_ = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.gslm_pcg_solve(ctx.h, ctypes.c_void_p(cache.handle), P_(shifted), P_(diag), None, ctypes.c_float(1e-3),
                            P_(x), None) == -1
    assert b"16-byte" in L.gslm_last_error(ctx.h)
    assert L.gslm_pcg_solve(ctx.h, ctypes.c_void_p(cache.handle), P_(cache.b), P_(diag), None, ctypes.c_float(1e-3),
                            P_(x), None) == 0
    cache.free()
