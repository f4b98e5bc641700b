"""The 1.5M-Gaussian workload at full size (GPU only), in the configuration the
benchmark times: one LM step's first subset (25 views at 1264x832), FP32 and
BF16 caches, autotuned kernels, and the batched solve from CUDA graphs.

The oracle cannot linearise the whole scene, so it is compared on sampled
outputs it computes exactly: a few 16x16 tiles of two views, blended from every
splat that reaches them (`jacobian.linearise_view_tiles`). Pixels of those tiles
and J p there are compared directly; J^T u is compared for a u supported on
those tiles, where only their entries contribute. On the whole cache, two
properties that hold at any size are checked: the adjoint identity
<J p, u> = <p, J^T u>, and diag(J^T J)_k = ||J e_k||^2 for sampled columns.
"""
import numpy as np
import pytest

import synth
from common import rel_l2

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


@pytest.fixture(scope="module")
def scene():
    wl = synth.WORKLOADS["paper"]
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    subsets = synth.subset_views(wl, 0)
    return wl, P, cams, subsets


def _view_offsets(cams, views):
    offs = [0]
    for v in views:
        offs.append(offs[-1] + cams[v].width * cams[v].height)
    return offs


def _sampled(P, cams, views):
    """Oracle linearisation of 3 tiles in each of 2 of the subset's views, with the
    residual offsets of the subset, and the sampled pixel indices (subset order)."""
    from oracle import jacobian as J
    offs = _view_offsets(cams, views)
    lins, pix, masks = [], [], []
    for k in (0, 12):
        cam = cams[views[k]]
        tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
        tiles = [(tx // 2, ty // 2), (tx // 3, ty // 2), (2 * tx // 3, ty // 3)]
        vl = J.linearise_view_tiles(P, cam, tiles, pix_off=3 * offs[k])
        lins.append(vl)
        for x, y in tiles:
            yy, xx = np.meshgrid(np.arange(y * 16, min(cam.height, y * 16 + 16)),
                                 np.arange(x * 16, min(cam.width, x * 16 + 16)), indexing="ij")
            local = (yy * cam.width + xx).ravel()
            pix.append(offs[k] + local)
            masks.append((vl.ras.margin[local] >= 1e-4) & ~vl.ras.flip[local])
    return lins, np.concatenate(pix), np.concatenate(masks), offs


@pytest.fixture(scope="module")
def sampled(scene):
    wl, P, cams, subsets = scene
    return _sampled(P.astype(np.float64), cams, subsets[0])


@pytest.mark.parametrize("fmt,tol", [("fp32", 1e-4), ("bf16", 2e-2)])
def test_fullsize_render_J_and_JT_on_sampled_tiles(lib, scene, sampled, fmt, tol):
    from oracle import jacobian as J
    wl, P, cams, subsets = scene
    lins, pix, mask, offs = sampled
    views = subsets[0]
    sc = [cams[v] for v in views]
    N = P.shape[0]
    n_pix = offs[-1]
    ctx = lib.Context(cache_fmt=fmt)
    params = lib.to_soa(P)
    zeros = torch.zeros((n_pix, 3), dtype=torch.float32, device="cuda")
    cache = ctx.build_cache(params, N, sc, zeros)         # F = image (targets are zero)
    assert cache.info().entries > 1e9
    img = cache.F.cpu().numpy()
    ref_img = np.zeros((n_pix, 3))
    for vl in lins:
        o = vl.pix_off // 3
        ref_img[o:o + vl.ras.image.shape[0] * vl.ras.image.shape[1]] += vl.ras.image.reshape(-1, 3)
    sel = pix[mask]
    assert mask.mean() > 0.8 and sel.size > 1000      # dense tiles: ~10% of pixels near a decision
    assert np.abs(img[sel] - ref_img[sel]).max() <= 1e-5
    # J p on the sampled pixels
    p = synth.random_vector(7, (N, 59))
    u = ctx.apply_J(cache, lib.to_soa(p)).cpu().numpy()
    u_ref = J.apply_J(lins, p.astype(np.float64), 3 * n_pix).reshape(-1, 3)
    assert rel_l2(u[sel], u_ref[sel]) < tol
    # J^T u for u supported on the sampled pixels
    uu = np.zeros((n_pix, 3), np.float32)
    uu[sel] = synth.random_vector(8, (sel.size, 3))
    g = lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(uu).cuda()), N)
    g_ref = J.apply_JT(lins, uu.astype(np.float64).ravel(), N)
    assert np.abs(g_ref).sum() > 0
    assert rel_l2(g, g_ref) < tol
    cache.free()
    ctx.close()


@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_fullsize_adjoint_identity_and_diag_columns(lib, scene, fmt):
    wl, P, cams, subsets = scene
    views = subsets[0]
    sc = [cams[v] for v in views]
    N = P.shape[0]
    n_pix = sum(c.width * c.height for c in sc)
    ctx = lib.Context(cache_fmt=fmt)
    cache = ctx.build_cache(lib.to_soa(P), N, sc, torch.zeros((n_pix, 3), device="cuda"))
    p = torch.from_numpy(synth.random_vector(11, (59, cache.ld)).astype(np.float32)).cuda()
    u = torch.from_numpy(synth.random_vector(12, (n_pix, 3)).astype(np.float32)).cuda()
    Jp = ctx.apply_J(cache, p).double()
    JTu = ctx.apply_JT(cache, u).double()
    lhs = float((Jp * u.double()).sum())
    rhs = float((p.double()[:, :N] * JTu[:, :N]).sum())
    scale = float(torch.linalg.norm(Jp)) * float(torch.linalg.norm(u.double()))
    assert abs(lhs - rhs) <= 1e-5 * scale
    # diag(J^T J)_k = ||J e_k||^2 for sampled columns with entries
    diag = ctx.jacobi_diag(cache).cpu().numpy()
    rng = np.random.default_rng(13)
    cand = np.argwhere(diag[:, :N] > 1e-3)
    for k, gi in cand[rng.choice(cand.shape[0], 6, replace=False)]:
        e = torch.zeros((59, cache.ld), dtype=torch.float32, device="cuda")
        e[k, gi] = 1.0
        col = ctx.apply_J(cache, e).double()
        assert abs(float((col * col).sum()) - float(diag[k, gi])) <= 1e-3 * float(diag[k, gi]), (k, gi)
    cache.free()
    ctx.close()


def test_fullsize_batched_solve_matches_one_solve_per_subset(lib, scene):
    wl, P, cams, subsets = scene
    N = P.shape[0]
    ctx = lib.Context(cache_fmt="bf16", n_iters=4, break_rel2=0.0)
    params = lib.to_soa(P)
    caches, diags = [], []
    for vs in subsets[:2]:
        sc = [cams[v] for v in vs]
        n_pix = sum(c.width * c.height for c in sc)
        tgt = torch.full((n_pix, 3), 0.25, device="cuda")
        c = ctx.build_cache(params, N, sc, tgt)
        caches.append(c)
        diags.append(ctx.jacobi_diag(c))
    lam = 1.0
    ref = [ctx.pcg_solve(c, c.b, d, lam)[0].clone() for c, d in zip(caches, diags)]
    for rep in range(2):        # autotuned direct run, then the CUDA graph
        xs, stats, status = ctx.pcg_solve_batch(caches, [c.b for c in caches], diags, lam)
        assert status == 0 and all(s.iters == 4 for s in stats)
        errs = [rel_l2(x.cpu().numpy()[:, :N], r.cpu().numpy()[:, :N]) for x, r in zip(xs, ref)]
        print(f"full size, batched vs per-subset solve (call {rep}): {max(errs):.2e}")
        assert max(errs) < 1e-3
    for c in caches:
        c.free()
    ctx.close()
