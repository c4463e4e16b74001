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


# ---------------------------------------------------------------- ordered subsets (Eq. 7)
# "j in OS" of Eq. 7: one update per subset of consecutive projections, with the residual
# sum and the column sum both taken over every ray of the subset.  The last subset holds
# the remaining n_proj mod subset_size views.

def one_voxel_scan(n_proj, det=1):
    s = synth.Scan(1, 1, 1, 5.0, 4.0, 50.0, 100.0, det, det, 1.3, 1.1,
                   synth.full_circle(n_proj) + 0.21, off_u=0.4, off_v=-0.3)
    s.beta, s.tx, s.tz = 0.05, 0.6, -0.2
    return s


@pytest.mark.parametrize("n_proj,subset,det", [(5, 2, 1), (5, 5, 1), (7, 3, 3), (6, 4, 2)])
def test_one_voxel_ordered_subsets_by_hand(orc, n_proj, subset, det):
    # N = (1,1,1): every ray's only entry is its chord t_j = L_j, so the update of a subset
    # OS is x <- x + lam * sum_{j in OS} (p_j - t_j x) / sum_{j in OS} t_j (rays with
    # t_j = 0 add nothing to either sum).  Written out subset by subset, ragged tail
    # included, from chords of the brute-force foot-of-perpendicular construction.
    s = one_voxel_scan(n_proj, det)
    S, D = bf.rays(s)
    t = np.array([[bf.cylinder_chord(s, S[p, v, u], D[p, v, u]) for v in range(det) for u in range(det)]
                  for p in range(n_proj)])
    assert (t > 0).sum() >= n_proj
    rng = np.random.default_rng(n_proj * 10 + subset)
    p = rng.uniform(0.05, 0.4, size=(n_proj, det * det))
    x0, lam = 0.013, 0.7
    x = x0
    for _ in range(2):
        for a in range(0, n_proj, subset):
            rows = slice(a, min(a + subset, n_proj))
            tt, pp = t[rows].ravel(), p[rows].ravel()
            hit = tt > 0
            x = x + lam * (pp[hit] - tt[hit] * x).sum() / tt[hit].sum()
    got = orc.sart(osetup(orc, s), p.reshape(s.sino_shape), x0=np.array([[[x0]]]), n_iter=2,
                   subset_size=subset, lam=lam)
    assert math.isclose(got.item(), x, rel_tol=1e-13)


def test_ordered_subsets_on_bruteforce_matrix(orc):
    # Eq. 7 over subsets of 3 consecutive views (7 views: subsets of 3, 3 and 1), weighted,
    # on the dense matrix of the independent brute-force clip of every (ray, voxel) pair
    s = synth.Scan(2, 5, 3, 6.0, 8.0, 40.0, 100.0, 5, 4, 2.0, 2.5, synth.full_circle(7) + 0.1)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.3, 0.12, 0.5, 0.4, -0.3, 0.2
    A = bf.dense_matrix(s)
    rng = np.random.default_rng(33)
    x0 = rng.uniform(0.0, 0.05, size=s.n_vox)
    w = rng.choice([1.0, 4.0], size=s.n_vox)
    p = rng.uniform(0.0, 0.5, size=A.shape[0])
    npix, lam, ss = s.det_w * s.det_h, 0.5, 3
    L = A.sum(axis=1)
    what = w / w.max()
    x = x0.copy()
    for _ in range(2):
        for a in range(0, s.n_proj, ss):
            rows = slice(a * npix, min(a + ss, s.n_proj) * npix)
            As = A[rows]
            r = np.where(L[rows] > 0, (p[rows] - As @ x) / np.where(L[rows] > 0, L[rows], 1.0), 0.0)
            num, den = As.T @ r, As.T @ np.ones(As.shape[0])
            upd = den > 0
            x[upd] += lam * what[upd] * num[upd] / den[upd]
    got = orc.sart(osetup(orc, s), p.reshape(s.sino_shape), x0=x0.reshape(s.vol_shape),
                   w=w.reshape(s.vol_shape), n_iter=2, subset_size=ss, lam=lam)
    np.testing.assert_allclose(got.reshape(-1), x, rtol=0, atol=1e-13)


def test_fixed_point_with_subsets(orc):
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p = orc.project(o, x_true)
    x = orc.sart(o, p, x0=x_true, n_iter=2, subset_size=3, lam=0.5)
    assert np.abs(x - x_true).max() <= 1e-14 * np.abs(x_true).max() * 10


def test_resume_with_subsets(orc):
    s = synth.tiny_scan()
    p = synth.random_sinogram(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    x4 = orc.sart(o, p, n_iter=4, subset_size=3, lam=0.5)
    x2 = orc.sart(o, p, n_iter=2, subset_size=3, lam=0.5)
    x22 = orc.sart(o, p, x0=x2, n_iter=2, subset_size=3, lam=0.5)
    np.testing.assert_allclose(x22, x4, rtol=0, atol=1e-15)
    # a subset of every view is one simultaneous step, whatever the order of the views
    perm = np.random.default_rng(2).permutation(s.n_proj)
    sp = dataclasses.replace(s, angles=s.angles[perm])
    a = orc.sart(o, p, n_iter=1, subset_size=s.n_proj, lam=0.5)
    b = orc.sart(osetup(orc, sp), p[perm], n_iter=1, subset_size=s.n_proj, lam=0.5)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-14 * np.abs(a).max())


# ------------------------------------------------------- grazing rays and voxels (Eq. 7)

GRAZE_R = 5.0
GRAZE_EPS = math.ldexp(GRAZE_R, -16)


def graze_scan(chord):
    """One pixel, one view, a one-voxel grid of radius 5 mm: the ray's offset on the
    detector bisected (on the brute-force chord) until its chord in the grid is ``chord``."""
    def scan_at(off):
        return synth.Scan(1, 1, 1, GRAZE_R, 4.0, 50.0, 100.0, 1, 1, 1.0, 1.0, np.array([0.0]), off_u=off)

    def chord_at(off):
        s = scan_at(off)
        S, D = bf.rays(s)
        return bf.cylinder_chord(s, S[0, 0, 0], D[0, 0, 0])

    lo, hi = 0.0, 20.0            # chord(lo) = 2R, chord(hi) = 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if chord_at(mid) > chord:
            lo = mid
        else:
            hi = mid
    s = scan_at(lo)
    return s, chord_at(lo)


@pytest.mark.parametrize("ratio", [0.5, 4.0])
def test_grazing_ray_and_voxel_floor(orc, ratio):
    # Eq. 7 with its row and column sums floored at eps = 2^-16 R: a chord t >= eps moves
    # the voxel by lam (p - t x0) / t as usual; a grazing chord t < eps by
    # lam (t / eps)^2 (p - t x0) / t
    s, t = graze_scan(ratio * GRAZE_EPS)
    assert abs(t - ratio * GRAZE_EPS) <= 1e-3 * ratio * GRAZE_EPS
    x0, p, lam = 0.02, 3e-5, 0.6
    x = orc.sart(osetup(orc, s), np.array([p]), x0=np.array([x0]), n_iter=1, lam=lam).item()
    share = min(t / GRAZE_EPS, 1.0) ** 2
    # a grazing chord is ill-conditioned in FP64 too (R^2 - d^2 cancels): 1e-3
    assert math.isclose(x - x0, lam * share * (p - t * x0) / t, rel_tol=1e-3)
