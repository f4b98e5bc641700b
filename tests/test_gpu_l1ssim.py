"""The L1 + SSIM objective (Eq. gn-loss, Sec. C) on the CUDA path vs the FP64
oracle (GPU only).

What is compared: the cache's e = sum (dr/dc) r and weights w = sum (dr/dc)^2,
the energy, b = -J^T F, the weighted J p, J^T J p, diag(J^T J), a PCG solve
and one LM step.

Tolerance. A pixel whose blending decision is within float32 reach of its
threshold (the mask of the L2 tests) changes SSIM over its 11 x 11
neighbourhood, so pixel-level comparisons exclude every pixel whose window
holds such a pixel. Elsewhere the rendered colours agree to 1e-5 absolute, and
SSIM is a quotient whose derivative carries 1/(1 - SSIM) and 1/(var_x + var_y +
C2) factors: an input error of 1e-5 becomes a relative error of up to a few
1e-4 in dSSIM/dc and so in e and w. The float32 window statistics add
cancellation of the same order (E[x^2] - mu^2 of a smooth patch). The weighted
quantities are therefore held to 1e-3 relative L2 (J^T u and J p themselves
keep their 1e-4 bound: the weighted J p is compared against the GPU's own
weights times the oracle's unweighted J p), PCG x to 2e-3, the energy to 1e-5.
Whole-image quantities that cannot leave those pixels out (diag(J^T J), b)
are held to 2e-3 (3e-3 per parameter block of the diagonal).
"""
import numpy as np
import pytest
from scipy import ndimage

import synth
from common import N_PARAMS, pixel_mask, ragged_case, rel_l2, tiny_case

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
    from oracle import residual as R
    from oracle import solver
    wl, P, cams, tgt = CASES[request.param]()
    P64 = P.astype(np.float64)
    sys_ = solver.build_subset(P64, cams, tgt.astype(np.float64), objective=R.Objective())
    good = []
    for vl, c in zip(sys_.lin, cams):
        bad = ~((vl.ras.margin >= 1e-4) & ~vl.ras.flip).reshape(c.height, c.width)
        good.append(~ndimage.binary_dilation(bad, structure=np.ones((11, 11), bool)).ravel())
    good = np.repeat(np.concatenate(good), 3)
    return request.param, P, cams, tgt, sys_, good


def _ctx(lib, **kw):
    return lib.Context(objective="l1ssim", **kw)


def test_l1ssim_residuals_weights_energy_and_b(lib, case):
    from oracle import jacobian as J
    name, P, cams, tgt, sys_, good = case
    assert good.mean() > 0.8
    ctx = _ctx(lib)
    cache = ctx.build_cache(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    e = cache.F.cpu().numpy().ravel().astype(np.float64)
    w = cache.weights().cpu().numpy().ravel().astype(np.float64)
    err_e, err_w = rel_l2(e[good], sys_.F[good]), rel_l2(w[good], sys_.W[good])
    print(f"{name}: e {err_e:.2e}, w {err_w:.2e}, energy {cache.cost:.6e} vs {sys_.cost:.6e}")
    assert err_e < 1e-3 and err_w < 1e-3
    assert abs(cache.cost - sys_.cost) <= 1e-5 * sys_.cost
    # b = -J^T e with e zeroed outside the compared pixels on both sides
    em = np.where(good, sys_.F, 0.0)
    b_ref = -J.apply_JT(sys_.lin, em, P.shape[0])
    b_gpu = -lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(em.astype(np.float32)).cuda().view(-1, 3)),
                          P.shape[0])
    assert rel_l2(b_gpu, b_ref) < 1e-4
    b_all = lib.from_soa(cache.b, P.shape[0])
    assert rel_l2(b_all, sys_.b) < 2e-3
    cache.free()


def test_l1ssim_weighted_products_and_diag(lib, case):
    from oracle import jacobian as J
    from oracle import solver
    name, P, cams, tgt, sys_, good = case
    ctx = _ctx(lib)
    cache = ctx.build_cache(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    w = cache.weights().cpu().numpy().ravel().astype(np.float64)
    n_res = J.n_residuals(cams)
    p = synth.random_vector(3, (P.shape[0], N_PARAMS))
    u_ref = J.apply_J(sys_.lin, p.astype(np.float64), n_res)
    u = ctx.apply_J(cache, lib.to_soa(p)).cpu().numpy().ravel()
    # the weighted J p: J's own error against the GPU's weights, then the weights' error
    assert rel_l2(u[good], (w * u_ref)[good]) < 1e-4
    assert rel_l2(u[good], (sys_.W * u_ref)[good]) < 1e-3
    # J^T J p over the compared pixels: J^T of the GPU's weighted J p against the oracle's
    um = np.where(good, u, 0.0).astype(np.float32)
    g = lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(um).cuda().view(-1, 3)), P.shape[0])
    g_ref = J.apply_JT(sys_.lin, np.where(good, sys_.W * u_ref, 0.0), P.shape[0])
    err_g = rel_l2(g, g_ref)
    # the whole diagonal: it cannot leave out the pixels near a flipped decision,
    # whose weights move with the flip (held to twice the weights' bound)
    d = lib.from_soa(ctx.jacobi_diag(cache), P.shape[0])
    err_d = rel_l2(d, sys_.M)
    blocks = [rel_l2(d[:, lo:hi], sys_.M[:, lo:hi]) for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 59)]]
    print(f"{name}: J^T J p {err_g:.2e}, diag {err_d:.2e}, blocks {max(blocks):.2e}")
    assert err_g < 1e-3 and err_d < 2e-3 and max(blocks) < 3e-3
    cache.free()


def test_l1ssim_render_energy(lib, case):
    from oracle import residual as R
    name, P, cams, tgt, sys_, good = case
    ctx = _ctx(lib)
    img, cost = ctx.render(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    assert abs(cost - sys_.cost) <= 1e-5 * sys_.cost
    # the L2 context renders the same image and reports ||c - C||^2
    _, c2 = lib.Context().render(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    ref2 = float(np.sum((img.cpu().numpy().ravel().astype(np.float64) - tgt) ** 2))
    assert abs(c2 - ref2) <= 1e-5 * ref2
    assert abs(ctx.opt.lambda_l1 - R.Objective().lambda1) < 1e-7 and abs(ctx.opt.lambda_ssim - R.Objective().lambda2) < 1e-7


def test_l1ssim_pcg_matches_oracle(lib, case):
    from oracle import solver
    name, P, cams, tgt, sys_, good = case
    ctx = _ctx(lib, n_iters=4, break_rel2=0.0)
    cache = ctx.build_cache(lib.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    diag = ctx.jacobi_diag(cache)
    lam = 1e-2
    x, st, status = ctx.pcg_solve(cache, cache.b, diag, lam)
    x_ref, st_ref = solver.solve_subset(sys_, lam, 4)
    err = rel_l2(lib.from_soa(x, P.shape[0]), x_ref)
    print(f"{name}: PCG x {err:.2e}")
    assert st.iters == 4 and err < 2e-3
    cache.free()


def test_l1ssim_lm_step_matches_oracle(lib):
    from oracle import residual as R
    from oracle import solver
    wl, P, cams, tgt = tiny_case()
    subsets = [[0, 1, 2, 3], [4, 5, 6, 7]]
    offs = np.concatenate([[0], np.cumsum([c.width * c.height * 3 for c in cams])])
    tg = [np.concatenate([tgt[offs[v]:offs[v + 1]] for v in s]).astype(np.float64) for s in subsets]
    # with the line search (Eq. line-search): the full step of weak damping lands where
    # the trial render is discontinuous in Delta, the chosen gamma does not
    res = solver.lm_step(P.astype(np.float64), [[cams[v] for v in s] for s in subsets], tg, 1e-1, n_iters=8,
                         objective=R.Objective(), ls_steps=8)
    ctx = _ctx(lib, n_iters=8, break_rel2=0.0, line_search=8)
    params = lib.to_soa(P)
    state, stats = ctx.lm_step(params, P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3), subsets, 1e-1)
    print(f"l1ssim LM step: gamma {stats.gamma}/{res.gamma} cost {stats.cost:.6e}/{res.cost:.6e} "
          f"pred {stats.predicted:.6e}/{res.pred:.6e} new {stats.cost_new:.6e}/{res.cost_new:.6e} "
          f"accepted {stats.accepted}/{res.accepted}")
    assert stats.gamma == res.gamma
    assert abs(stats.cost - res.cost) <= 1e-5 * res.cost
    assert abs(stats.predicted - res.pred) <= 1e-3 * res.cost
    assert abs(stats.cost_new - res.cost_new) <= 1e-3 * res.cost
    assert bool(stats.accepted) == res.accepted
    if res.accepted:
        assert res.cost_new < res.cost
        assert rel_l2(lib.from_soa(params, P.shape[0]) - P, res.gamma * res.delta) < 1e-3
