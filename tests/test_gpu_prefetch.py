"""The tile kernels with L2 prefetch (forced variants 9 and 10) on scenes with
long and with many segments (GPU only).

Variants 9 and 10 have one lane of each group ask L2 for the entries of the
segment 16 or 32 places ahead of the one it takes (and the staging threads
for the first ones of every 256-segment stage). A prefetch changes no value,
but its ranges are widened to 16-byte boundaries and may reach 15 bytes past
the cache's last entry, and it is issued at stage boundaries and for the last
segments of a tile. Here J p, J^T u and the batched solve run on a scene with
long segments and on one with hundreds of short segments per tile (several
stages per tile), against the same kernels without prefetch (variant 3),
which the variant tests hold to the FP64 oracle; they agree to float32
summation order.
"""
import numpy as np
import pytest

import synth
from common import N_PARAMS, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PREFETCHING = (9, 10)
PLAIN = 3


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12892_gb300 import build
    build.build()
    import paper_2409_12892_gb300 as g
    return g


def _scene(kind):
    if kind == "long":   # large splats: long segments
        wl = synth.small_workload("pf-long", 77, 3000, 4, 256, 192, cam_radius=3.5, log_scale_mean=-2.2)
    else:                # many small splats: hundreds of short segments per tile
        wl = synth.small_workload("pf-short", 78, 20000, 2, 96, 64, cam_radius=4.0, log_scale_mean=-3.5)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(wl.seed, cams)]).astype(np.float32)
    return P, cams, tgt


@pytest.fixture(scope="module", params=["long", "short"])
def scene(request):
    return (request.param,) + _scene(request.param)


def _products(lib, fmt, variant, P, cams, tgt):
    N = P.shape[0]
    ctx = lib.Context(cache_fmt=fmt, apply_variant=variant, autotune=False)
    cache = ctx.build_cache(lib.to_soa(P), N, cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    info = cache.info()
    p = lib.to_soa(synth.random_vector(5, (N, N_PARAMS)))
    n_res = sum(c.width * c.height * 3 for c in cams)
    u = torch.from_numpy(synth.random_vector(6, n_res).astype(np.float32)).cuda().view(-1, 3)
    Jp = ctx.apply_J(cache, p).cpu().numpy().ravel()
    JTu = lib.from_soa(ctx.apply_JT(cache, u), N)
    b = lib.from_soa(cache.b, N)
    cache.free()
    ctx.close()
    return info, Jp, JTu, b


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16s"])
def test_prefetching_products_match_the_plain_kernels(lib, scene, fmt):
    kind, P, cams, tgt = scene
    info, Jp0, JTu0, b0 = _products(lib, fmt, PLAIN, P, cams, tgt)
    n_tiles = sum(-(-c.width // 16) * -(-c.height // 16) for c in cams)
    if kind == "long":
        assert info.entries / info.segments > 48   # long segments
    else:
        assert info.segments / n_tiles > 256       # several stages per tile
    assert np.abs(JTu0).max() > 0 and np.abs(Jp0).max() > 0
    for v in PREFETCHING:
        info_v, Jp, JTu, b = _products(lib, fmt, v, P, cams, tgt)
        assert info_v.entries == info.entries and info_v.segments == info.segments
        assert np.isfinite(Jp).all() and np.isfinite(JTu).all()
        assert rel_l2(Jp, Jp0) < 1e-5, (v, fmt)
        assert rel_l2(JTu, JTu0) < 1e-5, (v, fmt)
        assert rel_l2(b, b0) < 1e-5, (v, fmt)


def test_prefetching_batched_solve_matches_the_plain_one(lib):
    """Persistent kernels with prefetch (several tiles per CTA) in a two-subset solve."""
    P, cams, tgt = _scene("long")
    N = P.shape[0]
    offs = np.concatenate([[0], np.cumsum([c.width * c.height * 3 for c in cams])])
    halves = [(cams[:2], tgt[:offs[2]]), (cams[2:], tgt[offs[2]:])]
    xs = {}
    for v in (PLAIN,) + PREFETCHING:
        ctx = lib.Context(cache_fmt="bf16", n_iters=2, break_rel2=0.0, apply_variant=v, autotune=False,
                          batch_ctas=2)
        caches = [ctx.build_cache(lib.to_soa(P), N, c, torch.from_numpy(t).cuda().view(-1, 3)) for c, t in halves]
        diags = [ctx.jacobi_diag(c) for c in caches]
        x, stats, status = ctx.pcg_solve_batch(caches, [c.b for c in caches], diags, 1e-2)
        assert status == 0 and all(s.iters == 2 for s in stats)
        xs[v] = [lib.from_soa(xi, N) for xi in x]
        for c in caches:
            c.free()
        ctx.close()
    for v in PREFETCHING:
        for a, b in zip(xs[v], xs[PLAIN]):
            assert np.isfinite(a).all()
            assert rel_l2(a, b) < 1e-4, v
