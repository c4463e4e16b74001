"""Pins of the oracle's SART (Eq. 7) by properties that any correct SART has."""
import dataclasses
import math

import numpy as np
import pytest

import bruteforce as bf
from paper_2005_11976_gb300 import synth


def osetup(orc, scan):
    return orc.Setup(**scan.fields())


def one_ray_scan(n_proj=7):
    # a single detector pixel per view: every subset is one ray
    s = synth.Scan(3, 5, 4, 6.0, 8.0, 40.0, 100.0, 1, 1, 1.0, 1.0,
                   synth.full_circle(n_proj) + 0.05, off_u=1.3, off_v=0.7)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.2, 0.1, 0.4, 0.3, -0.2, 0.1
    return s


def test_single_voxel_by_hand(orc):
    # N = (1,1,1): t_j = L_j = chord of ray j, so one subset of one ray gives
    # x1 = x0 + lam * (p - t x0) / t
    s = synth.Scan(1, 1, 1, 5.0, 4.0, 50.0, 100.0, 1, 1, 1.0, 1.0, np.array([0.3]))
    S, D = bf.rays(s)
    t = bf.cylinder_chord(s, S[0, 0, 0], D[0, 0, 0])
    x0, p, lam = 0.02, 0.7, 0.6
    x = orc.sart(osetup(orc, s), np.array([p]), x0=np.array([x0]), n_iter=1, lam=lam)
    assert math.isclose(x.item(), x0 + lam * (p - t * x0) / t, rel_tol=1e-14)


@pytest.mark.parametrize("lam", [1.0, 0.5])
def test_one_ray_subset_moves_residual_by_lambda(orc, lam):
    # a subset of one ray: Eq. 7 adds lam * r / L to every voxel the ray crosses, so that
    # ray's residual is multiplied by exactly (1 - lam)
    s = one_ray_scan()
    rng = np.random.default_rng(4)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.1, 1.0, size=s.sino_shape)
    o = osetup(orc, s)
    x = orc.sart(o, p, x0=x0, n_iter=1, lam=lam)
    last = s.n_proj - 1
    # residual of the last ray before its update equals the residual after all earlier
    # subsets; recompute it by running one iteration over the first n_proj-1 views only
    s_head = dataclasses.replace(s, angles=s.angles[:-1])
    x_head = orc.sart(osetup(orc, s_head), p[:-1], x0=x0, n_iter=1, lam=lam)
    before = p[last, 0, 0] - orc.project(o, x_head, last, 1)[0, 0, 0]
    after = p[last, 0, 0] - orc.project(o, x, last, 1)[0, 0, 0]
    assert abs(before) > 1e-3
    assert abs(after - (1.0 - lam) * before) <= 1e-13 * abs(before) + 1e-15


def test_fixed_point_on_consistent_data(orc):
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p = orc.project(o, x_true)
    x = orc.sart(o, p, x0=x_true, n_iter=2, lam=0.5)
    assert np.abs(x - x_true).max() <= 1e-14 * np.abs(x_true).max() * 10


def test_residual_decreases_on_consistent_tiny_data(orc):
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p = orc.project(o, x_true)
    res = []
    x = np.zeros(s.vol_shape)
    for _ in range(5):
        x = orc.sart(o, p, x0=x, n_iter=2, lam=0.5)
        res.append(np.linalg.norm(orc.project(o, x) - p))
    assert all(b < a for a, b in zip(res, res[1:]))
    assert res[-1] < 0.1 * np.linalg.norm(p)


def test_converges_to_truth_on_determined_case(orc):
    # theta-independent (N_theta = 1) object fully inside an untruncated detector: the
    # consistent system has a unique solution, which SART must reach
    s = synth.Scan(3, 1, 5, 5.0, 6.0, 40.0, 120.0, 24, 24, 1.0, 1.0, synth.full_circle(6))
    s.beta, s.tx = 0.15, 0.3
    rng = np.random.default_rng(9)
    x_true = rng.uniform(0.01, 0.05, size=s.vol_shape)
    o = osetup(orc, s)
    p = orc.project(o, x_true)
    x = orc.sart(o, p, n_iter=300, lam=1.0)
    assert np.abs(x - x_true).max() <= 1e-8


def test_resume_equals_one_run(orc):
    s = synth.tiny_scan()
    rng = synth.rng_for("tiny")
    p = synth.random_sinogram(s, rng)
    o = osetup(orc, s)
    x10 = orc.sart(o, p, n_iter=4, lam=0.5)
    x5 = orc.sart(o, p, n_iter=2, lam=0.5)
    x55 = orc.sart(o, p, x0=x5, n_iter=2, lam=0.5)
    np.testing.assert_allclose(x55, x10, rtol=0, atol=1e-15)


def test_weights(orc):
    s = synth.tiny_scan()
    rng = synth.rng_for("tiny")
    p = synth.random_sinogram(s, rng)
    x0 = synth.random_volume(s, rng)
    o = osetup(orc, s)
    plain = orc.sart(o, p, x0=x0, n_iter=1, lam=0.5)
    # a constant map is normalised to one (weight_mode 1)
    same = orc.sart(o, p, x0=x0, w=np.full(s.vol_shape, 3.0), n_iter=1, lam=0.5)
    np.testing.assert_allclose(same, plain, rtol=0, atol=1e-15)
    # zero weight freezes a region; raw mode with w = 1/2 equals lam/2
    w = np.ones(s.vol_shape)
    w[:, :, :5] = 0.0
    frozen = orc.sart(o, p, x0=x0, w=w, n_iter=1, lam=0.5)
    np.testing.assert_array_equal(frozen[:, :, :5], x0[:, :, :5])
    half_raw = orc.sart(o, p, x0=x0, w=np.full(s.vol_shape, 0.5), n_iter=1, lam=0.5,
                        weight_mode=0)
    half_lam = orc.sart(o, p, x0=x0, n_iter=1, lam=0.25)
    np.testing.assert_allclose(half_raw, half_lam, rtol=0, atol=1e-15)


def test_clamp_nonneg(orc):
    s = synth.tiny_scan()
    rng = synth.rng_for("tiny")
    p = -synth.random_sinogram(s, rng)         # negative data drives x below zero
    o = osetup(orc, s)
    x = orc.sart(o, p, n_iter=1, lam=0.5, clamp_nonneg=True)
    assert x.min() >= 0.0
    assert orc.sart(o, p, n_iter=1, lam=0.5).min() < 0.0


def test_voxels_no_ray_touches_stay(orc):
    # a detector that only sees the lower half of the grid leaves the top slabs unchanged
    s = synth.Scan(4, 8, 4, 5.0, 8.0, 40.0, 100.0, 12, 3, 1.5, 0.5, synth.full_circle(5),
                   off_v=-5.0)
    rng = np.random.default_rng(1)
    x0 = rng.uniform(0, 1, size=s.vol_shape)
    o = osetup(orc, s)
    x = orc.sart(o, rng.uniform(0, 1, size=s.sino_shape), x0=x0, n_iter=1, lam=0.5)
    np.testing.assert_array_equal(x[3], x0[3])
    assert np.abs(x[0] - x0[0]).max() > 0
