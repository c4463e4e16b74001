"""Pose estimation (Sec. 2.1, Eq. 3-4) and azimuthal phase (Eq. 5) on the GPU against the
FP64 oracle: corner pixels bit-exact, the tracked points, poses and band moments to
rounding, gamma to the FP32 projector's rounding."""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, synth
import gpu_util as gu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11976_gb300 import build
    build.build()
    return cylct.load()


@pytest.fixture(scope="module")
def op(orc):
    from oracle import pose
    return pose


def rounded(a, code):
    """Values of ``a`` as stored in ``code`` (rounded on the host), as float64."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(gu.torch_dtype(code))
    return t.float().numpy().astype(np.float64)


def cylinder_scan(pose, n_proj=24, det_w=96, det_h=120, pitch=0.8, angles=None):
    s = synth.Scan(4, 8, 4, 8.0, 32.0, 200.0, 800.0, det_w, det_h, pitch, pitch,
                   synth.full_circle(n_proj) + 0.1 if angles is None else angles)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
    return s


def noisy_cylinder(orc, s, seed, mu=0.05, sigma=0.004):
    """Line integrals of a uniform cylinder (mu x chord) with seeded Gaussian noise."""
    rng = np.random.default_rng(seed)
    L = mu * orc.row_sums(orc.Setup(**s.fields()))
    return L + sigma * rng.standard_normal(L.shape)


def corners_gpu(s, sino_np, code, prm):
    import torch
    d = gu.to_dev(sino_np, code)
    cs = torch.empty((s.n_proj, 4, 2), dtype=torch.int32, device="cuda")
    cnt = torch.empty(s.n_proj, dtype=torch.int64, device="cuda")
    cylct.cyl_axis_corners(s, d, code, prm, cs, cnt)
    torch.cuda.synchronize()
    return cs.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("code", [cylct.CYL_F32, cylct.CYL_F16, cylct.CYL_BF16])
@pytest.mark.parametrize("k,roi,det_w", [(0, (0, 0, 0, 0), 96), (2, (0, 0, 0, 0), 96),
                                         (3, (10, 83, 7, 110), 96), (1, (0, 0, 0, 0), 93)])
def test_corners_bit_exact(lib, orc, op, code, k, roi, det_w):
    s = cylinder_scan((0.7, 0.04, 0.0, 1.5, -2.0, 0.8), det_w=det_w)
    sino = rounded(noisy_cylinder(orc, s, 11), code)
    sino[5] = 0.0                                   # a projection without a segment
    prm = cylct.pose_params(0.05, k, roi)
    cs, cnt = corners_gpu(s, sino, code, prm)
    want, wcnt, _, _, _ = op.axis_tracks(sino, 0.05, k, roi)
    np.testing.assert_array_equal(cs, want)
    np.testing.assert_array_equal(cnt, wcnt)
    assert (cs[5] == -1).all()


def test_track_point_matches_oracle(lib, orc, op):
    import torch
    s = cylinder_scan((0, 0, 0, 0, 0, 0), n_proj=21, angles=synth.limited_arc(21, 200.0))
    views = op.stage_views(orc.Setup(**s.fields()))
    rng = np.random.default_rng(3)
    X = np.array([1.0, -2.0, 11.0])
    obs = np.array([op.project_point(v, X)[0] for v in views]) + 0.3 * rng.standard_normal((21, 2))
    valid = np.ones(21, bool)
    valid[[2, 9]] = False
    tr = obs.copy()
    tr[~valid] = np.nan
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    cylct.cyl_track_point(s, torch.from_numpy(tr).cuda(), 100, out)
    got = out.cpu().numpy()
    Xo, rms, _ = op.track_point(views, obs, valid)
    np.testing.assert_allclose(got[:3], Xo, atol=1e-7)
    assert got[3] == pytest.approx(rms, rel=1e-9)
    # fewer than two observed projections: NaN point, no steps
    tr[:] = np.nan
    tr[4] = obs[4]
    cylct.cyl_track_point(s, torch.from_numpy(tr).cuda(), 100, out)
    got = out.cpu().numpy()
    assert np.isnan(got[:4]).all() and got[4] == 0


def test_estimate_pose_matches_oracle_and_batch(lib, orc, op):
    rng = np.random.default_rng(8)
    scans, sinos, want = [], [], []
    for i in range(3):
        pose = (rng.uniform(-3, 3), math.radians(rng.uniform(0.5, 3.0)), 0.0, *rng.uniform(-3, 3, 3))
        s = cylinder_scan(pose, n_proj=30 + 3 * i)
        sino = noisy_cylinder(orc, s, 20 + i)
        scans.append(s)
        sinos.append(sino)
        want.append(op.estimate_pose(orc.Setup(**s.fields()), sino, 0.05, k=1, gamma=0.3))
    prm = cylct.pose_params(0.05, 1, gamma=0.3)
    dev = [gu.to_dev(x) for x in sinos]
    poses, infos = cylct.cyl_estimate_pose_batch(scans, dev, cylct.CYL_F32, prm)
    for i, s in enumerate(scans):
        pose, info = cylct.cyl_estimate_pose(s, dev[i], cylct.CYL_F32, prm)
        assert pose == poses[i]                     # the batch runs the same arithmetic
        wp, wi = want[i]
        np.testing.assert_allclose(pose[:3], wp[:3], atol=1e-9)
        np.testing.assert_allclose(pose[3:], wp[3:], atol=1e-7)
        np.testing.assert_allclose(info["top"], wi["top"], atol=1e-7)
        np.testing.assert_allclose(info["bottom"], wi["bottom"], atol=1e-7)
        np.testing.assert_allclose(info["rms"], wi["rms"], rtol=1e-9)
        assert info["n_views"] == wi["n_views"] and info["status"] == 0


def test_estimate_pose_without_segments(lib):
    import torch
    s = cylinder_scan((0, 0, 0, 0, 0, 0), n_proj=4)
    sino = torch.zeros((4, s.det_h, s.det_w), device="cuda")
    pose, info = cylct.cyl_estimate_pose(s, sino, cylct.CYL_F32, cylct.pose_params(0.05, gamma=0.2))
    assert info["status"] == 1 and info["n_views"] == 0
    assert pose == (0.0, 0.0, 0.2, 0.0, 0.0, 0.0)


def test_pose_at_table1_size(lib, orc, op, golden_table1):
    """Table 1's detector and arc (with the panel's 0.0748 mm pixels): corners of sampled
    projections bit-exact, the pose to rounding, both from one launch over all 21
    projections."""
    import torch
    s = dataclasses.replace(golden_table1, alpha=0.9, beta=math.radians(1.5), tx=1.2, ty=-0.8, tz=0.4,
                            pitch_u=0.0748, pitch_v=0.0748)
    s.radius, s.height = 8.0, 64.0
    L = 0.08 * orc.row_sums(orc.Setup(**s.fields()))
    sino = rounded(L + 0.003 * np.random.default_rng(1).standard_normal(L.shape), cylct.CYL_F16)
    prm = cylct.pose_params(0.04, 2)
    cs, _ = corners_gpu(s, sino, cylct.CYL_F16, prm)
    for p in (0, 10, 20):
        np.testing.assert_array_equal(cs[p], op.corners(op.segment(sino[p], 0.04, 2)[0]))
    pose, info = cylct.cyl_estimate_pose(s, gu.to_dev(sino, cylct.CYL_F16), cylct.CYL_F16, prm)
    wp, wi = op.estimate_pose(orc.Setup(**s.fields()), sino, 0.04, k=2)
    np.testing.assert_allclose(pose[:2], wp[:2], atol=1e-9)
    np.testing.assert_allclose(pose[3:], wp[3:], atol=1e-7)
    torch.cuda.synchronize()


# ------------------------------------------------------------------ Eq. 5


def insert_part(n_proj=48):
    s = synth.Scan(8, 64, 16, 10.0, 20.0, 100.0, 400.0, 64, 48, 1.6, 1.6, synth.full_circle(n_proj) + 0.05)
    return s


@pytest.mark.parametrize("code", [cylct.CYL_F32, cylct.CYL_BF16])
def test_band_moments_match_oracle(lib, orc, op, code):
    import torch
    s = insert_part()
    s.alpha, s.beta, s.tx, s.ty, s.tz = 0.8, 0.03, 1.0, -0.7, 0.3
    rng = np.random.default_rng(4)
    sino = rounded(rng.uniform(0.0, 1.0, size=s.sino_shape), code)
    pose = (s.alpha, s.beta, 0.0, s.tx, s.ty, s.tz)
    m = torch.empty((s.n_proj, 2), dtype=torch.float64, device="cuda")
    cylct.cyl_band_moments(s, pose, gu.to_dev(sino, code), code, cylct.band(-5.0, 5.0, 12.0), m)
    got = m.cpu().numpy()
    want = op.band_moments(orc.Setup(**s.fields()), pose, sino, -5.0, 5.0, 12.0)
    np.testing.assert_allclose(got[:, 0], want[:, 0], rtol=1e-12)
    # first moments: the same band pixels and exact products, summed in another order
    scale = np.array([np.abs(want[:, 1]).max()] * s.n_proj)
    assert np.all(np.abs(got[:, 1] - want[:, 1]) <= 1e-11 * scale)


@pytest.mark.parametrize("passes", [1, 2])
def test_estimate_gamma_matches_oracle(lib, orc, op, passes):
    rng = np.random.default_rng(5)
    for trial in range(2):
        s = insert_part()
        x = synth.part_phantom(s, np.array([rng.uniform(0, 2 * math.pi)]))
        s.alpha, s.beta = rng.uniform(-3, 3), math.radians(rng.uniform(0.5, 3))
        s.tx, s.ty, s.tz = rng.uniform(-2, 2, 3)
        g_true, g_ref = rng.uniform(-3, 3), rng.uniform(-1, 1)
        sino = orc.project(orc.Setup(**dataclasses.replace(s, gamma=g_true).fields()), x)
        sref = dataclasses.replace(s, gamma=g_ref)
        want, wdiag = op.estimate_gamma(orc.Setup(**sref.fields()), sino, x, -5.0, 5.0, 100.0, passes=passes)
        with cylct.Plan(sref) as plan:
            g, diag = plan.cyl_estimate_gamma(gu.to_dev(sino), cylct.CYL_F32, gu.to_dev(x), cylct.CYL_F32,
                                              cylct.band(-5.0, 5.0, 100.0), passes=passes)
            # the plan is left posed with the estimate: its projection of the template
            # equals the oracle's at that spin
            q = gu.project(plan, x, 0, 2)
        assert abs(op.wrap(g - want)) < 1e-4
        np.testing.assert_allclose(np.array(diag)[[1, 3]], np.array(wdiag)[[1, 3]], rtol=1e-4)
        assert abs(math.degrees(op.wrap(g - g_true))) < 0.6
        q_want = orc.project(orc.Setup(**dataclasses.replace(s, gamma=g).fields()), x, 0, 2)
        assert gu.rel_l2(q, q_want) <= 1e-5
        if passes == 1:
            assert cylct.cyl_gamma_from_phase(wdiag[0], wdiag[2], s.alpha, s.beta, g_ref) == \
                pytest.approx(want, abs=1e-12)
