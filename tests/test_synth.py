"""The seeded input generators (no GPU): every case the parity tests and the
bench run is drawn from `synth`, so the draws must repeat exactly, the named
workloads must have the sizes they are named for, and the cameras must look
at the scene.
"""
import math

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def paper():
    wl = synth.WORKLOADS["paper"]
    return wl, synth.make_gaussians(wl), synth.make_cameras(wl)


def test_draws_repeat_and_seeds_separate_them():
    wl = synth.WORKLOADS["tiny"]
    a, b = synth.make_gaussians(wl), synth.make_gaussians(wl)
    assert a.dtype == np.float32 and a.shape == (1000, synth.N_PARAMS)
    assert np.array_equal(a, b)
    other = synth.small_workload("other", wl.seed + 1, 1000, 8, 64, 64)
    assert not np.array_equal(a, synth.make_gaussians(other))
    assert np.array_equal(synth.perturbed_copy(wl, a), synth.perturbed_copy(wl, a))
    assert not np.array_equal(synth.perturbed_copy(wl, a), a)
    assert np.array_equal(synth.random_vector(3, (5, 7)), synth.random_vector(3, (5, 7)))
    assert not np.array_equal(synth.random_vector(3, (5, 7)), synth.random_vector(4, (5, 7)))
    c1, c2 = synth.make_cameras(wl), synth.make_cameras(wl)
    assert all(np.array_equal(x.R, y.R) and np.array_equal(x.t, y.t) for x, y in zip(c1, c2))


def test_paper_workload_sizes(paper):
    wl, P, cams = paper
    assert P.shape == (1_500_000, synth.N_PARAMS) and P.dtype == np.float32 and np.isfinite(P).all()
    assert len(cams) == 200 and {(c.width, c.height) for c in cams} == {(1264, 832)}
    assert wl.subset_sizes == [25, 25, 25, 25] and wl.pcg_iters == 8 and wl.lambda0 == 1e-3
    lab = synth.cluster_labels(wl)
    assert lab.shape == (1_500_000,) and set(np.unique(lab)) == set(range(20))


def test_uneven_workload_sizes():
    wl = synth.WORKLOADS["uneven"]
    cams = synth.make_cameras(wl)
    assert wl.n_gaussians == 3_000_000 and len(cams) == 300
    assert sum(wl.subset_sizes) == 277 and len(wl.subset_sizes) == 8
    # resolutions cycle over the cameras
    assert [(c.width, c.height) for c in cams[:5]] == [(960, 540), (1280, 720), (1264, 832), (1600, 1066), (960, 540)]


@pytest.mark.parametrize("name", ["paper", "uneven", "tiny"])
def test_subsets_are_disjoint_seeded_and_sized(name):
    wl = synth.WORKLOADS[name]
    s0, s0b, s1 = synth.subset_views(wl, 0), synth.subset_views(wl, 0), synth.subset_views(wl, 1)
    assert s0 == s0b
    assert [len(s) for s in s0] == wl.subset_sizes
    flat = [v for s in s0 for v in s]
    assert len(set(flat)) == len(flat) and all(0 <= v < wl.n_cameras for v in flat)
    assert all(s == sorted(s) for s in s0)
    if len(wl.subset_sizes) > 1:
        assert s0 != s1                      # each LM step draws its own subsets


def test_cameras_look_at_the_scene_with_a_60_degree_field_of_view(paper):
    wl, P, cams = paper
    for c in cams:
        # the origin lies in front of the camera, on its optical axis
        o = c.R.astype(np.float64) @ np.zeros(3) + c.t.astype(np.float64)
        assert o[2] > 0 and abs(o[0]) < 1e-4 * o[2] and abs(o[1]) < 1e-4 * o[2]
        assert np.allclose(c.R.astype(np.float64) @ c.R.T.astype(np.float64), np.eye(3), atol=1e-5)
        assert float(c.fx) == pytest.approx((c.width / 2) / math.tan(math.radians(30.0)), rel=1e-6)
        assert (float(c.cx), float(c.cy)) == (c.width / 2, c.height / 2)
        # jittered radius: within a few percent of the workload's radius
        assert float(np.linalg.norm(c.t)) == pytest.approx(wl.cam_radius, rel=0.1)


def test_the_paper_crop_is_the_cluster_core(paper):
    wl, P, cams = paper
    idx = synth.crop_2k(wl, P)
    lab = synth.cluster_labels(wl)
    assert idx.shape == (2000,) and np.all(np.diff(idx) > 0) and np.all(lab[idx] == 0)
    members = np.nonzero(lab == 0)[0]
    c = P[members, 0:3].astype(np.float64).mean(axis=0)
    d = np.linalg.norm(P[:, 0:3].astype(np.float64) - c, axis=1)
    rest = np.setdiff1d(members, idx)
    assert d[idx].max() <= d[rest].min()     # the 2,000 nearest the cluster's mean
