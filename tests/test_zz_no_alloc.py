"""gslm_apply_JT_noalloc, the allocation-free J^T u, against gslm_apply_JT (GPU only).

The variant exists for callers that may not allocate device memory while they
run (memory reserved up front by another allocator, or a thread that may not
call cudaMalloc); its partial sums live in a fixed array inside the library that
every call shares. This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from common import ragged_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_SEGMENTS = 1 << 19
GSLM_E_INVALID = -1


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12892_gb300 import build
    build.build()
    import paper_2409_12892_gb300 as mod
    lib = mod.load_library()
    lib.gslm_apply_JT_noalloc.restype = ctypes.c_int32
    lib.gslm_apply_JT_noalloc.argtypes = [ctypes.c_void_p] * 4
    return mod


def _noalloc(g, ctx, cache, u, out):
    return ctx.lib.gslm_apply_JT_noalloc(ctx.h, ctypes.c_void_p(cache.handle), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()))


def _ragged(g, ctx):
    wl, P, cams, tgt = ragged_case()
    cache = ctx.build_cache(g.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    n_res = sum(c.width * c.height * 3 for c in cams)
    us = [torch.from_numpy(synth.random_vector(s, n_res)).cuda().view(-1, 3) for s in (31, 32)]
    return P, cache, us


def test_noalloc_apply_JT_matches_apply_JT_on_two_calls_in_a_row(g):
    ctx = g.Context()
    P, cache, us = _ragged(g, ctx)
    assert cache.info().segments <= MAX_SEGMENTS
    refs = [ctx.apply_JT(cache, u).clone() for u in us]
    for u, ref in zip(us, refs):      # second call reuses the array the first call filled
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(g, ctx, cache, u, out) == 0
        torch.cuda.synchronize()
        a, b = g.from_soa(out, P.shape[0]), g.from_soa(ref, P.shape[0])
        assert np.isfinite(a).all()
        assert rel_l2(a, b) < 1e-4
    cache.free()
    ctx.close()


def test_noalloc_apply_JT_allocates_no_device_memory(g):
    """After a first call (which may load kernel code), a call changes neither
    the library pool's bytes in use or held nor the device's free memory."""
    ctx = g.Context()
    P, cache, us = _ragged(g, ctx)
    out = torch.zeros((59, cache.ld), dtype=torch.float32, device="cuda")
    assert _noalloc(g, ctx, cache, us[0], out) == 0
    torch.cuda.synchronize()
    pool0, free0 = ctx.memory_usage(), torch.cuda.mem_get_info()[0]
    assert _noalloc(g, ctx, cache, us[1], out) == 0
    torch.cuda.synchronize()
    pool1, free1 = ctx.memory_usage(), torch.cuda.mem_get_info()[0]
    assert pool1["used"] == pool0["used"] and pool1["reserved"] == pool0["reserved"]
    assert free1 == free0
    ref = ctx.apply_JT(cache, us[1])
    torch.cuda.synchronize()
    assert rel_l2(g.from_soa(out, P.shape[0]), g.from_soa(ref, P.shape[0])) < 1e-4
    cache.free()
    ctx.close()


@pytest.mark.parametrize("variant", [1, 2, 6, 8, 9, 10])
def test_noalloc_apply_JT_runs_the_forced_variant(g, variant):
    ctx = g.Context(autotune=False, apply_variant=variant)
    P, cache, us = _ragged(g, ctx)
    ref = ctx.apply_JT(cache, us[0]).clone()
    out = torch.full_like(ref, float("nan"))
    assert _noalloc(g, ctx, cache, us[0], out) == 0
    torch.cuda.synchronize()
    assert rel_l2(g.from_soa(out, P.shape[0]), g.from_soa(ref, P.shape[0])) < 1e-4
    cache.free()
    ctx.close()


def test_noalloc_apply_JT_on_a_thin_cache(g):
    ctx = g.Context(cache_fmt="thin")
    P, cache, us = _ragged(g, ctx)
    ref = ctx.apply_JT(cache, us[0]).clone()
    out = torch.full_like(ref, float("nan"))
    assert _noalloc(g, ctx, cache, us[0], out) == 0
    torch.cuda.synchronize()
    assert rel_l2(g.from_soa(out, P.shape[0]), g.from_soa(ref, P.shape[0])) < 1e-4
    cache.free()
    ctx.close()


def test_noalloc_apply_JT_on_a_cache_without_segments_gives_zeros(g):
    """Every Gaussian behind the only camera: no segment, so J^T u = 0."""
    wl = synth.small_workload("edge", 41, 200, 1, 40, 24, cam_radius=4.0, log_scale_mean=-2.0)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    R = np.asarray(cams[0].R, np.float64)
    campos = -R.T @ np.asarray(cams[0].t, np.float64)
    P = P.copy()
    P[:, 0:3] = (1.5 * campos)[None, :] + 0.1 * synth.random_vector(41, (P.shape[0], 3))
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(41, cams)]).astype(np.float32)
    ctx = g.Context()
    tg = torch.from_numpy(tgt).cuda().view(-1, 3)
    cache = ctx.build_cache(g.to_soa(P), P.shape[0], cams, tg)
    assert cache.info().segments == 0
    out = torch.full((59, cache.ld), float("nan"), dtype=torch.float32, device="cuda")
    assert _noalloc(g, ctx, cache, tg, out) == 0
    torch.cuda.synchronize()
    assert not g.from_soa(out, P.shape[0]).any()
    cache.free()
    ctx.close()


def test_noalloc_apply_JT_rejects_caches_beyond_its_maximum(g):
    wl = synth.WORKLOADS["medium"]
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)[:8]
    tgt = np.concatenate([im.ravel() for im in synth.smooth_images(5, cams)]).astype(np.float32)
    ctx = g.Context()
    cache = ctx.build_cache(g.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    assert cache.info().segments > MAX_SEGMENTS
    u = torch.zeros((g.n_pixels(cams), 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((59, cache.ld), dtype=torch.float32, device="cuda")
    assert _noalloc(g, ctx, cache, u, out) == GSLM_E_INVALID
    assert b"524288" in ctx.lib.gslm_last_error(ctx.h)
    cache.free()
    ctx.close()
