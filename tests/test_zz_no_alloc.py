"""gslm_apply_JT_noalloc, the allocation-free J^T u, against gslm_apply_JT (GPU only).

The variant exists for callers that may not allocate device memory while they
run; its partial sums live in a fixed array inside the library that every call
shares. This file is collected last so that a run stopping at the first failure
has already run every other test.
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


def test_noalloc_apply_JT_matches_apply_JT_on_two_calls_in_a_row(g):
    wl, P, cams, tgt = ragged_case()
    ctx = g.Context()
    cache = ctx.build_cache(g.to_soa(P), P.shape[0], cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    assert cache.info().segments <= MAX_SEGMENTS
    n_res = sum(c.width * c.height * 3 for c in cams)
    us = [torch.from_numpy(synth.random_vector(s, n_res)).cuda().view(-1, 3) for s in (31, 32)]
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
