"""Every tile-kernel variant the autotuner may pick, against the FP64 oracle (GPU only).

The autotuner keeps whichever variant runs fastest on the caller's cache, so
each one must compute the same products: J p and J^T u of every variant (lane
groups of 8, 16 or 32, 2 to 4 entries in flight per lane, shared atomics or
per-warp private tiles) are held to the bound of their cache format (FP32 1e-4,
BF16 2e-2, FP16 with scale 5e-3), and a batched solve (persistent kernels) with
each variant forced is held to the PCG bound (`common.pcg_bound`) against the
oracle's Algorithm 1.
"""
import numpy as np
import pytest

import synth
from common import N_PARAMS, pcg_bound, pixel_mask, ragged_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_VARIANTS = 8


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12892_gb300 import build
    build.build()
    import paper_2409_12892_gb300 as g
    return g


@pytest.fixture(scope="module")
def case():
    from oracle import jacobian as J
    wl, P, cams, tgt = ragged_case()
    lin = J.linearise(P.astype(np.float64), cams)
    return P, cams, tgt, lin


def test_the_library_offers_the_variants_tested(lib):
    ctx = lib.Context(apply_variant=N_VARIANTS)        # the last valid forced variant
    ctx.close()
    with pytest.raises(Exception):
        lib.Context(apply_variant=N_VARIANTS + 1)


@pytest.mark.parametrize("variant", range(1, N_VARIANTS + 1))
@pytest.mark.parametrize("fmt,tol", [("fp32", 1e-4), ("bf16", 2e-2), ("fp16s", 5e-3)])
def test_every_variant_matches_the_oracle(lib, case, variant, fmt, tol):
    from oracle import jacobian as J
    P, cams, tgt, lin = case
    N = P.shape[0]
    n_res = J.n_residuals(cams)
    mask = np.repeat(pixel_mask(lin), 3)
    ctx = lib.Context(cache_fmt=fmt, apply_variant=variant, autotune=False)
    cache = ctx.build_cache(lib.to_soa(P), N, cams, torch.from_numpy(tgt).cuda().view(-1, 3))
    p = synth.random_vector(31, (N, N_PARAMS))
    u = np.where(mask, synth.random_vector(32, n_res), 0.0).astype(np.float32)
    Jp = ctx.apply_J(cache, lib.to_soa(p)).cpu().numpy().ravel()
    JTu = lib.from_soa(ctx.apply_JT(cache, torch.from_numpy(u).cuda().view(-1, 3)), N)
    assert rel_l2(Jp[mask], J.apply_J(lin, p.astype(np.float64), n_res)[mask]) < tol
    assert rel_l2(JTu, J.apply_JT(lin, u.astype(np.float64), N)) < tol
    cache.free()
    ctx.close()


@pytest.mark.parametrize("variant", range(1, N_VARIANTS + 1))
def test_every_variant_in_the_batched_solve(lib, case, variant):
    from oracle import solver
    P, cams, tgt, lin = case
    N = P.shape[0]
    halves = [cams[: len(cams) // 2], cams[len(cams) // 2:]]
    offs = np.concatenate([[0], np.cumsum([c.width * c.height * 3 for c in cams])])
    k = len(cams) // 2
    tg = [tgt[:offs[k]], tgt[offs[k]:]]
    lam = 1e-2
    ctx = lib.Context(n_iters=4, break_rel2=0.0, apply_variant=variant, autotune=False)
    caches = [ctx.build_cache(lib.to_soa(P), N, c, torch.from_numpy(t).cuda().view(-1, 3)) for c, t in zip(halves, tg)]
    diags = [ctx.jacobi_diag(c) for c in caches]
    xs, stats, status = ctx.pcg_solve_batch(caches, [c.b for c in caches], diags, lam)
    assert all(s.iters == 4 for s in stats)
    for c, t, x in zip(halves, tg, xs):
        sys_ = solver.build_subset(P.astype(np.float64), c, t.astype(np.float64))
        x_ref, _ = solver.solve_subset(sys_, lam, 4)
        assert rel_l2(lib.from_soa(x, N), x_ref) < pcg_bound(sys_, lam, 4, x_ref, seeds=(0,)), variant
    for c in caches:
        c.free()
    ctx.close()
