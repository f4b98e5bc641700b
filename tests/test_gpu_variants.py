"""Every tile-kernel variant the autotuner may pick, against the FP64 oracle (GPU only).

The autotuner keeps whichever variant runs fastest on the caller's cache, so
each one must compute the same products: J p and J^T u of every variant (lane
groups of 8, 16 or 32, 2 to 4 entries in flight per lane, shared atomics or
per-warp private tiles of three planes or of float4, with or without L2
prefetch of the segments ahead) are held to the bound of their cache format (FP32 1e-4,
BF16 2e-2, FP16 with scale 5e-3), and a batched solve (persistent kernels) with
each variant forced is held to the PCG tolerance of 1e-3 against the oracle's
Algorithm 1 after 2 iterations (where float32 rounding moves x by at most
5e-4: `common.pcg_noise_spread`).
"""
import numpy as np
import pytest

import synth
from common import N_PARAMS, PCG_SPREAD_MAX, PCG_TOL, pcg_noise_spread, pixel_mask, ragged_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_VARIANTS = 10


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


PCG_LAMBDA, PCG_ITERS = 1e-2, 2


@pytest.fixture(scope="module")
def halves(case):
    """The two halves of the ragged case's views, each with the oracle's PCG
    solution after PCG_ITERS iterations (checked to be a well-posed comparison)."""
    from oracle import solver
    P, cams, tgt, lin = case
    offs = np.concatenate([[0], np.cumsum([c.width * c.height * 3 for c in cams])])
    k = len(cams) // 2
    out = []
    for c, t in ((cams[:k], tgt[:offs[k]]), (cams[k:], tgt[offs[k]:])):
        sys_ = solver.build_subset(P.astype(np.float64), c, t.astype(np.float64))
        x_ref, _ = solver.solve_subset(sys_, PCG_LAMBDA, PCG_ITERS)
        spread = pcg_noise_spread(sys_, PCG_LAMBDA, PCG_ITERS, x_ref, seeds=(0,))
        assert spread <= PCG_SPREAD_MAX, spread
        out.append((c, t, x_ref))
    return out


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
def test_every_variant_in_the_batched_solve(lib, case, halves, variant):
    P, cams, tgt, lin = case
    N = P.shape[0]
    ctx = lib.Context(n_iters=PCG_ITERS, break_rel2=0.0, apply_variant=variant, autotune=False)
    caches = [ctx.build_cache(lib.to_soa(P), N, c, torch.from_numpy(t).cuda().view(-1, 3)) for c, t, _ in halves]
    diags = [ctx.jacobi_diag(c) for c in caches]
    xs, stats, status = ctx.pcg_solve_batch(caches, [c.b for c in caches], diags, PCG_LAMBDA)
    assert all(s.iters == PCG_ITERS for s in stats)
    for (_, _, x_ref), x in zip(halves, xs):
        assert rel_l2(lib.from_soa(x, N), x_ref) < PCG_TOL, variant
    for c in caches:
        c.free()
    ctx.close()
