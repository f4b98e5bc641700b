"""The thin cache (GSLM_CACHE_THIN) against the FP64 oracle and the FP32 cache (GPU only).

A thin cache stores no (pixel, splat) entries: J p, J^T u and diag(J^T J)
blend the tile's segments again (J^T u and the diagonal window by window from
per-pixel checkpoints every 32 segments). They are the same products, so they
are held to the plain FP32 path's bounds against the oracle (J p, J^T u,
diag: 1e-4 relative L2; PCG x: 1e-3 after a well-posed iteration count), and
to float32 summation-order agreement with the FP32 entry cache.
"""
import numpy as np
import pytest

import synth
from common import (N_PARAMS, PCG_SPREAD_MAX, PCG_TOL, pcg_noise_spread, pixel_mask, ragged_case, rel_l2,
                    tiny_case)

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


CASES = {"tiny": tiny_case, "ragged": ragged_case}


@pytest.fixture(scope="module", params=["tiny", "ragged"])
def case(request):
    from oracle import jacobian as J
    wl, P, cams, tgt = CASES[request.param]()
    lin = J.linearise(P.astype(np.float64), cams)
    return request.param, P, cams, tgt, lin


def _caches(lib, P, cams, tgt, **kw):
    out = {}
    for fmt in ("fp32", "thin"):
        ctx = lib.Context(cache_fmt=fmt, **kw)
        out[fmt] = (ctx, ctx.build_cache(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3)))
    return out


def test_thin_cache_products_match_the_oracle(lib, case):
    from oracle import jacobian as J
    name, P, cams, tgt, lin = case
    N = P.shape[0]
    cs = _caches(lib, P, cams, tgt)
    ctx, cache = cs["thin"]
    _, full = cs["fp32"]
    ti, fi = cache.info(), full.info()
    assert ti.segments == fi.segments and ti.entries == fi.entries and ti.cache_fmt == 3
    assert torch.equal(cache.F, full.F)
    assert rel_l2(lib.from_soa(cache.b, N), lib.from_soa(full.b, N)) < 1e-5
    n_res = J.n_residuals(cams)
    mask = np.repeat(pixel_mask(lin), 3)
    for seed in (1, 2):
        p = synth.random_vector(seed, (N, N_PARAMS))
        u = np.where(mask, synth.random_vector(seed + 10, n_res), 0.0).astype(np.float32)
        Jp = ctx.apply_J(cache, lib.to_soa(p)).cpu().numpy().ravel()
        JTu = lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(u).cuda().view(-1, 3)), N)
        assert rel_l2(Jp[mask], J.apply_J(lin, p.astype(np.float64), n_res)[mask]) < 1e-4
        assert rel_l2(JTu, J.apply_JT(lin, u.astype(np.float64), N)) < 1e-4
        Jp_f = cs["fp32"][0].apply_J(full, lib.to_soa(p)).cpu().numpy().ravel()
        JTu_f = lib.from_soa(cs["fp32"][0].apply_JT(full, torch.from_numpy(u).cuda().view(-1, 3)), N)
        assert rel_l2(Jp, Jp_f) < 2e-5 and rel_l2(JTu, JTu_f) < 2e-5
    d = lib.from_soa(ctx.jacobi_diag(cache), N)
    d_ref = J.jacobi_diag(lin, N)
    assert rel_l2(d, d_ref) < 1e-4
    for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 59)]:
        assert rel_l2(d[:, lo:hi], d_ref[:, lo:hi]) < 1e-3, (lo, hi)
    assert rel_l2(d, lib.from_soa(cs["fp32"][0].jacobi_diag(full), N)) < 2e-5
    for c, k in cs.values():
        k.free()
        c.close()


def test_thin_pcg_matches_the_oracle(lib):
    from oracle import solver
    wl, P, cams, tgt = tiny_case()
    sys_ = solver.build_subset(P.astype(np.float64), cams, tgt.astype(np.float64))
    lam, its = 1e-3, 3
    x_ref, _ = solver.solve_subset(sys_, lam, n_iters=its, break_rel2=0.0)
    assert pcg_noise_spread(sys_, lam, its, x_ref) <= PCG_SPREAD_MAX
    ctx = lib.Context(cache_fmt="thin", n_iters=its, break_rel2=0.0)
    cache = ctx.build_cache(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    diag = ctx.jacobi_diag(cache)
    x, st, status = ctx.pcg_solve(cache, cache.b, diag, lam)
    assert status == 0 and st.iters == its
    assert rel_l2(lib.from_soa(x, P.shape[0]), x_ref) < PCG_TOL
    # the batched entry point solves thin caches one after another, with the same arithmetic
    xs, stats, _ = ctx.pcg_solve_batch([cache, cache], [cache.b, cache.b], [diag, diag], lam)
    for xb, sb in zip(xs, stats):
        assert sb.iters == its and rel_l2(lib.from_soa(xb, P.shape[0]), x_ref) < PCG_TOL
    cache.free()
    ctx.close()


def test_thin_lm_step_over_several_subsets_matches_the_oracle(lib):
    import warnings
    from oracle import jacobian as J, solver
    warnings.filterwarnings("ignore")
    wl = synth.small_workload("multi", 606, 600, 16, 64, 64, cam_radius=4.0, subset_sizes=[4, 4, 4, 4])
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    tgt = J.render(synth.perturbed_copy(wl, P).astype(np.float64), cams)
    tgt = (tgt + synth.pixel_noise(wl, tgt.size)).astype(np.float32)
    subsets = synth.subset_views(wl, 0)
    offs = np.concatenate([[0], np.cumsum([c.width * c.height * 3 for c in cams])])
    sc = [[cams[v] for v in s] for s in subsets]
    st = [np.concatenate([tgt[offs[v]:offs[v + 1]] for v in s]).astype(np.float64) for s in subsets]
    res = solver.lm_step(P.astype(np.float64), sc, st, 1e-3, n_iters=8, break_rel2=0.01, ls_steps=8)
    ctx = lib.Context(cache_fmt="thin", n_iters=8, break_rel2=0.01, line_search=8, batch=True)
    params = lib.to_soa(P)
    state, stats = ctx.lm_step(params, P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3), subsets, 1e-3)
    assert stats.gamma == res.gamma
    assert abs(stats.cost - res.cost) <= 1e-5 * res.cost
    assert abs(stats.predicted - res.pred) <= 1e-3 * res.cost
    assert abs(stats.cost_new - res.cost_new) <= 1e-3 * res.cost
    assert bool(stats.accepted) == res.accepted
    assert stats.pcg_iters == sum(s.iters for s in res.pcg)
    if res.accepted:
        assert rel_l2(lib.from_soa(params, P.shape[0]) - P, res.gamma * res.delta) < 1e-3
    ctx.close()


def test_thin_weighted_products_match_the_fp32_cache(lib):
    """The L1 + SSIM objective's weights enter the thin products as they enter the entry cache's."""
    wl, P, cams, tgt = ragged_case()
    N = P.shape[0]
    cs = _caches(lib, P, cams, tgt, objective="l1ssim")
    (cf, full), (ct, thin) = cs["fp32"], cs["thin"]
    p = lib.to_soa(synth.random_vector(7, (N, N_PARAMS)))
    assert rel_l2(ct.apply_J(thin, p).cpu().numpy(), cf.apply_J(full, p).cpu().numpy()) < 2e-5
    assert rel_l2(lib.from_soa(ct.jacobi_diag(thin), N), lib.from_soa(cf.jacobi_diag(full), N)) < 2e-5
    assert rel_l2(lib.from_soa(thin.b, N), lib.from_soa(full.b, N)) < 2e-5
    for c, k in cs.values():
        k.free()
        c.close()


def test_thin_cache_of_an_empty_scene_gives_zeros(lib):
    wl = synth.small_workload("edge", 41, 200, 1, 40, 24, cam_radius=4.0, log_scale_mean=-2.0)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    R = np.asarray(cams[0].R, np.float64)
    campos = -R.T @ np.asarray(cams[0].t, np.float64)
    P = P.copy()
    P[:, 0:3] = (1.5 * campos)[None, :] + 0.1 * synth.random_vector(41, (P.shape[0], 3))
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(41, cams)]).astype(np.float32)
    ctx = lib.Context(cache_fmt="thin")
    tg = torch.from_numpy(tgt).cuda().view(-1, 3)
    cache = ctx.build_cache(lib.to_soa(P), P.shape[0], cams, tg)
    assert cache.info().segments == 0 and not cache.b.any()
    p = torch.from_numpy(synth.random_vector(1, (N_PARAMS, cache.ld)).astype(np.float32)).cuda()
    assert not ctx.apply_J(cache, p).any()
    assert not ctx.apply_JT(cache, tg).any()
    assert not ctx.jacobi_diag(cache).any()
    cache.free()
    ctx.close()


def test_thin_cache_takes_less_memory_when_segments_are_long(lib):
    """Checkpoints cost 16 B per pixel per 32 segments; entries 17 B (FP32) per
    (pixel, splat): with segments of many pixels the thin cache is smaller."""
    wl = synth.small_workload("long", 77, 3000, 4, 256, 192, cam_radius=3.5, log_scale_mean=-2.2)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(77, cams)]).astype(np.float32)
    cs = _caches(lib, P, cams, tgt)
    fi, ti = cs["fp32"][1].info(), cs["thin"][1].info()
    print(f"entries {fi.entries}, segments {fi.segments}, FP32 cache {fi.bytes / 1e6:.1f} MB, "
          f"thin cache {ti.bytes / 1e6:.1f} MB")
    assert fi.entries / fi.segments > 30
    assert ti.bytes < 0.6 * fi.bytes
    for c, k in cs.values():
        k.free()
        c.close()
