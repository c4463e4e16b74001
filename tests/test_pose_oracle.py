"""Pins of the pose-estimation and azimuthal-phase oracle (Sec. 2.1, Eq. 3-5) against
facts fixed by geometry and by library routines.

None of these retype the oracle's formulas: corners are checked on shapes whose corners
are known by construction, the dilation against scipy's binary dilation, V_i against the
rays of the C oracle, the Jacobian against finite differences, the Levenberg-Marquardt
fit against exact tracks and against scipy's own Levenberg-Marquardt, the pose against
the rotation of Eq. 1, and Eq. 5 against the stage azimuths of the rotated part's axes.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2005_11976_gb300 import synth


@pytest.fixture(scope="module")
def op(orc):
    from oracle import pose
    return pose


def scan(n_proj=24, det_w=96, det_h=120, pitch=0.8, radius=8.0, height=32.0, pose=(0, 0, 0, 0, 0, 0),
         sod=200.0, sdd=800.0, angles=None):
    s = synth.Scan(4, 8, 4, radius, height, sod, sdd, det_w, det_h, pitch, pitch,
                   synth.full_circle(n_proj) + 0.1 if angles is None else angles)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
    return s


# ------------------------------------------------------------------ segmentation


@pytest.mark.parametrize("k", [0, 1, 3])
def test_dilation_matches_scipy(op, k):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(k)
    img = rng.uniform(0.0, 1.0, size=(40, 56))
    roi = (5, 50, 3, 37)
    got, count = op.segment(img, 0.93, k, roi)
    sub = img[3:37, 5:50] > 0.93
    want = np.zeros_like(got)
    want[3:37, 5:50] = ndi.binary_dilation(sub, structure=np.ones((2 * k + 1, 2 * k + 1), bool)) if k else sub
    assert count == int(sub.sum())
    np.testing.assert_array_equal(got, want)


def polygon_mask(shape, verts):
    """Pixels inside a convex polygon (counter-clockwise integer vertices), by half-plane
    tests at the pixel centres."""
    H, W = shape
    b, a = np.mgrid[0:H, 0:W]
    inside = np.ones(shape, bool)
    for (x0, y0), (x1, y1) in zip(verts, verts[1:] + verts[:1]):
        inside &= (x1 - x0) * (b - y0) - (y1 - y0) * (a - x0) >= 0
    return inside


def test_corners_of_rectangles_and_tilted_quadrilaterals(op):
    m = np.zeros((30, 40), bool)
    m[5:21, 7:19] = True
    np.testing.assert_array_equal(op.corners(m), [[7, 20], [18, 20], [7, 5], [18, 5]])
    # a quadrilateral tilted by less than 45 degrees: each diagonal extreme is a vertex
    bl, br, tr, tl = (10, 4), (22, 7), (17, 40), (5, 37)
    q = polygon_mask((48, 32), [bl, br, tr, tl])
    np.testing.assert_array_equal(op.corners(q), [tl, tr, bl, br])
    # empty mask
    np.testing.assert_array_equal(op.corners(np.zeros((4, 4), bool)), -np.ones((4, 2)))


def test_corner_ties_go_outwards(op):
    # a 45-degree edge: every pixel of the top-right edge has the same a + b; the tie goes
    # to the largest b, the bottom-left tie to the smallest b
    m = np.zeros((20, 20), bool)
    for b in range(3, 15):
        m[b, 2: 2 + (17 - b)] = True           # a + b <= 18 on the right edge
    c = op.corners(m)
    assert tuple(c[1]) == (4, 14)              # top-right: max a + b = 18, then max b
    assert tuple(c[2]) == (2, 3)               # bottom-left: min a + b, then min b


def test_dilation_moves_corners_by_k_and_clips_to_the_window(op):
    img = np.zeros((40, 50))
    img[10:20, 12:30] = 1.0
    cs = op.corners(op.segment(img, 0.5, 3)[0])
    np.testing.assert_array_equal(cs, [[9, 22], [32, 22], [9, 7], [32, 7]])
    roi = (11, 31, 8, 21)                       # clips the dilated square on every side
    cs = op.corners(op.segment(img, 0.5, 3, roi)[0])
    np.testing.assert_array_equal(cs, [[11, 20], [30, 20], [11, 8], [30, 8]])


# ------------------------------------------------------------------ V_i and Eq. 4


@pytest.mark.parametrize("frames", [False, True])
def test_projection_of_points_on_rays(orc, op, frames):
    s = scan(n_proj=5, pose=(0.4, 0.2, -0.3, 1.0, -2.0, 0.5))
    if frames:
        s = dataclasses.replace(s, frames=synth.conveyor_frames(5, 200.0, 800.0, 96, 120, 0.8, 30.0))
    o = orc.Setup(**dataclasses.replace(s, alpha=0, beta=0, gamma=0, tx=0, ty=0, tz=0).fields())
    views = op.stage_views(orc.Setup(**s.fields()))
    rng = np.random.default_rng(2)
    for p in range(s.n_proj):
        for _ in range(5):
            iu, iv = int(rng.integers(0, 96)), int(rng.integers(0, 120))
            S, D = orc.ray(o, p, iu, iv)
            X = S + rng.uniform(0.2, 0.8) * (D - S)
            ab, _, _ = op.project_point(views[p], X)
            np.testing.assert_allclose(ab, [iu, iv], atol=1e-9)


def test_jacobian_matches_finite_differences(orc, op):
    views = op.stage_views(orc.Setup(**scan(n_proj=4).fields()))
    X = np.array([3.0, -2.0, 5.0])
    for v in views:
        _, J = op.project_point_jacobian(v, X)
        h = 1e-5
        Jn = np.column_stack([(op.project_point(v, X + h * e)[0] - op.project_point(v, X - h * e)[0]) / (2 * h)
                              for e in np.eye(3)])
        np.testing.assert_allclose(J, Jn, rtol=1e-7, atol=1e-9)


def tracks_of(op, views, X, noise=0.0, seed=0):
    rng = np.random.default_rng(seed)
    obs = np.array([op.project_point(v, X)[0] for v in views])
    return obs + noise * rng.standard_normal(obs.shape)


def test_lm_recovers_a_point_from_exact_tracks(orc, op):
    views = op.stage_views(orc.Setup(**scan(n_proj=21, angles=synth.limited_arc(21, 200.0)).fields()))
    for X in ([0.5, -1.0, 14.0], [-3.0, 2.5, -12.0]):
        obs = tracks_of(op, views, np.array(X))
        valid = np.ones(len(views), bool)
        valid[3] = False                        # an unobserved projection is skipped
        obs[3] = (1e6, -1e6)
        Xe, rms, it = op.track_point(views, obs, valid)
        np.testing.assert_allclose(Xe, X, atol=1e-8)
        assert rms < 1e-9 and it < 100


def test_lm_agrees_with_scipy_least_squares(orc, op):
    opt = pytest.importorskip("scipy.optimize")
    views = op.stage_views(orc.Setup(**scan(n_proj=36).fields()))
    obs = tracks_of(op, views, np.array([1.0, 2.0, -9.0]), noise=0.4, seed=3)
    valid = np.ones(len(views), bool)
    Xe, rms, _ = op.track_point(views, obs, valid)

    def res(X):
        return np.concatenate([(o - op.project_point(v, X)[0]) * [np.linalg.norm(v[2]), np.linalg.norm(v[3])]
                               for v, o in zip(views, obs)])

    ref = opt.least_squares(res, op.initial_point(views, obs, valid), method="lm", xtol=1e-15, ftol=1e-15)
    np.testing.assert_allclose(Xe, ref.x, atol=1e-7)
    assert rms == pytest.approx(math.sqrt(2.0 * ref.cost / len(views)), rel=1e-9)


def test_pose_from_axis_matches_the_rotation_of_eq1(orc, op):
    rng = np.random.default_rng(4)
    for _ in range(50):
        a, b, g = rng.uniform(-3, 3), rng.uniform(0.01, 1.5), rng.uniform(-3, 3)
        T = rng.uniform(-5, 5, 3)
        O = orc.pose_matrix(a, b, g).T          # object-to-stage rotation
        top, bottom = O @ [0, 0, 7.0] + T, O @ [0, 0, -7.0] + T
        pose = op.pose_from_axis(top, bottom, gamma=0.25)
        Oe = orc.pose_matrix(*pose[:3]).T
        np.testing.assert_allclose(Oe[:, 2], O[:, 2], atol=1e-12)     # same axis
        np.testing.assert_allclose(pose[3:], T, atol=1e-12)
        assert pose[2] == 0.25
        np.testing.assert_allclose(pose[:2], [math.atan2(math.sin(a), math.cos(a)), b], atol=1e-9)


def test_pose_chain_on_a_projected_cylinder(orc, op):
    # uniform cylinder: line integrals = mu x chord through the grid cylinder (row sums)
    rng = np.random.default_rng(7)
    for _ in range(3):
        pose = (rng.uniform(-3, 3), math.radians(rng.uniform(0.5, 3.0)), 0.0, *rng.uniform(-3, 3, 3))
        s = scan(n_proj=36, det_w=128, det_h=160, pose=pose)
        sino = 0.05 * orc.row_sums(orc.Setup(**s.fields()))
        est, info = op.estimate_pose(orc.Setup(**s.fields()), sino, 0.05, k=1)
        O, Oe = orc.pose_matrix(*pose[:3]).T, orc.pose_matrix(*est[:3]).T
        axis_err = math.degrees(math.acos(min(1.0, O[:, 2] @ Oe[:, 2])))
        dc = np.array(est[3:]) - pose[3:]
        lateral = np.linalg.norm(dc - (dc @ O[:, 2]) * O[:, 2])
        assert axis_err < 0.3 and lateral < 0.1 and abs(dc @ O[:, 2]) < 1.5, (axis_err, dc)
        assert info["n_views"] == 36 and max(info["rms"]) < 1.0


# ------------------------------------------------------------------ Eq. 5


def test_eq5_inversion_and_the_printed_form(orc, op):
    rng = np.random.default_rng(1)
    for _ in range(500):
        a, b, g = rng.uniform(-1.5, 1.5), rng.uniform(0.0, 1.4), rng.uniform(-3, 3)
        O = orc.pose_matrix(a, b, g).T
        ex, ez = O[:, 0], O[:, 2]
        psi = math.atan2(ex[1], ex[0])          # stage azimuth of the part's x' axis
        assert abs(op.wrap(op.inplane_angle(psi, a, b) - g)) < 1e-12
        # printed Eq. 5: the phase read in the tilted plane from the direction above the
        # stage x axis
        w = np.array([ez[2], 0.0, -ez[0]])
        w /= np.linalg.norm(w)
        phi = math.atan2(np.cross(w, ex) @ ez, w @ ex)
        assert abs(op.wrap(op.eq5_printed(phi, 0.0, a, b) - g)) < 1e-12
    # a reference phase: the spin difference, whatever the reference spin
    for _ in range(50):
        a, b, g, gr = rng.uniform(-3, 3), rng.uniform(0, 1.2), rng.uniform(-3, 3), rng.uniform(-3, 3)
        psi = lambda gam: math.atan2(*(orc.pose_matrix(a, b, gam).T[:, 0][[1, 0]]))
        ph, ph_ref = math.pi / 2 - psi(g), math.pi / 2 - psi(gr)
        assert abs(op.wrap(op.gamma_from_phase(ph, ph_ref, a, b, gr) - g)) < 1e-12


def test_phase_fit_of_a_shifted_cosine(op):
    ang = np.sort(np.random.default_rng(0).uniform(0, 2 * math.pi, 37))
    g = 2.0 + 0.3 * np.cos(ang - 1.1)
    ph, amp = op.phase(ang, g)
    assert ph == pytest.approx(1.1, abs=1e-12) and amp == pytest.approx(0.3, rel=1e-12)


def test_band_of_an_upright_centred_axis(orc, op):
    # beta = 0, T = 0, detector centred: the axis projects on the middle column (W odd)
    s = scan(n_proj=1, det_w=41, det_h=31, pitch=1.0, angles=np.array([0.3]))
    views = op.stage_views(orc.Setup(**s.fields()))
    c = op.band_constants(views[0], (0, 0, 0, 0, 0, 0), -2.0, 3.0)
    mag = 800.0 / 200.0
    assert c[0] == 20.0 and c[1] == pytest.approx(15.0 - 2.0 * mag, abs=1e-4)
    mask, d = op.band_offsets((31, 41), c, 4.5)
    want = np.zeros((31, 41), bool)
    want[7:28, 16:25] = True                     # v in [-8, 12] mm, |u| <= 4.5 mm
    np.testing.assert_array_equal(mask, want)
    np.testing.assert_array_equal(d[0], np.arange(41) - 20.0)


def test_gamma_of_a_part_with_one_insert(orc, op):
    rng = np.random.default_rng(5)
    for _ in range(3):
        s = synth.Scan(8, 64, 16, 10.0, 20.0, 100.0, 400.0, 64, 48, 1.6, 1.6, synth.full_circle(48) + 0.05)
        x = synth.part_phantom(s, np.array([rng.uniform(0, 2 * math.pi)]))
        s.alpha, s.beta = rng.uniform(-3, 3), math.radians(rng.uniform(0.5, 3))
        s.tx, s.ty, s.tz = rng.uniform(-2, 2, 3)
        g_true, g_ref = rng.uniform(-3, 3), rng.uniform(-1, 1)
        sino = orc.project(orc.Setup(**dataclasses.replace(s, gamma=g_true).fields()), x)
        g, diag = op.estimate_gamma(orc.Setup(**dataclasses.replace(s, gamma=g_ref).fields()), sino, x,
                                    -5.0, 5.0, 100.0)
        assert abs(math.degrees(op.wrap(g - g_true))) < 0.6
        assert diag[1] == pytest.approx(diag[3], rel=0.05)     # same insert, same amplitude


def test_gamma_refinement_on_a_partial_arc(orc, op):
    # Table 1's 200 deg arc (binned panel): the first pass is biased by the harmonics of
    # the two signals; passes that move the reference to the estimate remove the bias
    import dataclasses as dc
    base = dc.replace(synth.table1_scan(grid=(32, 96, 32)), det_w=243, det_h=192, pitch_u=0.5984, pitch_v=0.5984)
    x = synth.pinned_tube(base)
    rng = np.random.default_rng(3)
    e1, e3 = [], []
    for _ in range(3):
        t = (rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(0.5, 3)), rng.uniform(-math.pi, math.pi),
             *rng.uniform(-2, 2, 3))
        s = dc.replace(base, alpha=t[0], beta=t[1], gamma=t[2], tx=t[3], ty=t[4], tz=t[5])
        sino = orc.project(orc.Setup(**s.fields()), x)
        ref = orc.Setup(**dc.replace(s, gamma=0.0).fields())
        e1.append(abs(op.wrap(op.estimate_gamma(ref, sino, x, -16.0, 16.0, 12.0, passes=1)[0] - t[2])))
        e3.append(abs(op.wrap(op.estimate_gamma(ref, sino, x, -16.0, 16.0, 12.0, passes=3)[0] - t[2])))
    assert math.degrees(max(e3)) < 0.1 and max(e3) < max(e1)
