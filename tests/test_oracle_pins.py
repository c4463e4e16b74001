"""Pins of the FP64 oracle against facts fixed by the paper and by geometry.

None of these re-derive the oracle's own formulas: the brute-force matrix clips the
line against single voxels (no sorted crossings), chords come from the
foot-of-perpendicular construction (not the quadratic formula), and the invariants are
symmetries of the cylindrical grid of Sec. 2 (Eq. 2).
"""
import dataclasses
import math

import numpy as np
import pytest

import bruteforce as bf
from paper_2005_11976_gb300 import synth


def small_scan(n_h, n_t, n_r, n_proj=5, det=8, pose=(0.3, 0.2, 0.7, 0.4, -0.3, 0.5),
               pitch=1.9, radius=6.0, height=8.0):
    s = synth.Scan(n_h, n_t, n_r, radius, height, 40.0, 100.0, det, det, pitch, pitch,
                   synth.full_circle(n_proj) + 0.1)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
    return s


def osetup(orc, scan):
    return orc.Setup(**scan.fields())


def oracle_matrix(orc, scan):
    o = osetup(orc, scan)
    rows = []
    for p in range(scan.n_proj):
        for iv in range(scan.det_h):
            for iu in range(scan.det_w):
                S, D = orc.ray(o, p, iu, iv)
                idx, ln = orc.ray_row(o, S, D)
                r = np.zeros(scan.n_vox)
                np.add.at(r, idx, ln)
                rows.append(r)
    return np.array(rows)


# ------------------------------------------------------------------ ray geometry

def test_pose_matrix_is_zxz(orc):
    a, b, g = 0.3, -0.7, 1.9
    R = orc.pose_matrix(a, b, g)
    O = bf.rot_z(a) @ bf.rot_x(b) @ bf.rot_z(g)      # intrinsic zxz orientation
    np.testing.assert_allclose(R, O.T, atol=1e-15)
    # gamma is the spin about the object's own axis: it only rotates x', y'
    Rg = orc.pose_matrix(a, b, g + 0.5)
    np.testing.assert_allclose(Rg, bf.rot_z(-0.5) @ R, atol=1e-15)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    # zxz: the z' axis of the object is tilted by beta from z
    assert math.isclose(R[2, 2], math.cos(b), abs_tol=1e-15)


def test_ray_endpoints_match_conventions(orc):
    scan = small_scan(2, 3, 2)
    o = osetup(orc, scan)
    S, D = bf.rays(scan)
    for p in range(scan.n_proj):
        for iv in (0, 3, 7):
            for iu in (0, 5, 7):
                So, Do = orc.ray(o, p, iu, iv)
                np.testing.assert_allclose(So, S[p, iv, iu], atol=1e-12)
                np.testing.assert_allclose(Do, D[p, iv, iu], atol=1e-12)
    # untilted object, first view: the central ray runs along +x through the origin
    s0 = synth.Scan(2, 3, 2, 5.0, 5.0, 40.0, 100.0, 3, 3, 1.0, 1.0, np.array([0.0]))
    So, Do = orc.ray(osetup(orc, s0), 0, 1, 1)
    np.testing.assert_allclose(So, [-40.0, 0.0, 0.0])
    np.testing.assert_allclose(Do, [60.0, 0.0, 0.0])


# ------------------------------------------------------- brute-force dense matrix

@pytest.mark.parametrize("grid", [(2, 1, 2), (3, 2, 3), (2, 3, 4), (4, 8, 3), (3, 5, 2)])
def test_traversal_equals_bruteforce(orc, grid):
    scan = small_scan(*grid, n_proj=4)
    A_bf = bf.dense_matrix(scan)
    A_or = oracle_matrix(orc, scan)
    assert A_bf.shape == A_or.shape
    assert np.count_nonzero(A_bf) > 0.2 * A_bf.size / max(grid)  # rays really hit the grid
    np.testing.assert_allclose(A_or, A_bf, rtol=0, atol=1e-12 * np.abs(A_bf).max())


def test_single_voxel_by_hand(orc):
    # one voxel = the whole grid cylinder; central ray of an untilted scan crosses a
    # diameter: t = 2R
    s = synth.Scan(1, 1, 1, 5.0, 4.0, 50.0, 100.0, 1, 1, 1.0, 1.0, np.array([0.0]))
    o = osetup(orc, s)
    S, D = orc.ray(o, 0, 0, 0)
    idx, ln = orc.ray_row(o, S, D)
    assert list(idx) == [0]
    assert math.isclose(ln[0], 10.0, rel_tol=1e-14)
    # two shells: outer R/2, inner a full diameter R (the axis is no boundary), outer R/2
    s2 = dataclasses.replace(s, n_r=2)
    idx, ln = orc.ray_row(osetup(orc, s2), S, D)
    assert list(idx) == [1, 0, 1]
    np.testing.assert_allclose(ln, [2.5, 5.0, 2.5], rtol=1e-14)
    # four wedges, ray from (-50, 0, 0) to (50, 3, 0): it crosses the theta = pi/2 wedge
    # boundary (the y axis) at t = 1/2, so wedge 1 then wedge 0, split at t = 1/2 of a
    # chord centred on the foot of the perpendicular from the axis
    s4 = dataclasses.replace(s, n_theta=4, off_u=3.0)
    S4, D4 = orc.ray(osetup(orc, s4), 0, 0, 0)
    np.testing.assert_allclose(D4, [50.0, 3.0, 0.0])
    idx, ln = orc.ray_row(osetup(orc, s4), S4, D4)
    assert list(idx) == [1, 0]
    a = 100.0 ** 2 + 3.0 ** 2
    tc = 5000.0 / a
    dist2 = (-50.0 + 100.0 * tc) ** 2 + (3.0 * tc) ** 2
    hw = math.sqrt((25.0 - dist2) / a)
    dn = math.sqrt(a)
    np.testing.assert_allclose(ln, [(0.5 - (tc - hw)) * dn, ((tc + hw) - 0.5) * dn], rtol=1e-13)


# ----------------------------------------------------------- closed-form chords

def scan_grid_rays(scan, step=1, window=None):
    S, D = bf.rays(scan)
    us = range(0, scan.det_w, step)
    vs = range(0, scan.det_h, step)
    if window is not None:
        cu, cv, hu, hv = window
        us = range(cu - hu, cu + hu + 1, step)
        vs = range(cv - hv, cv + hv + 1, step)
    for p in range(0, scan.n_proj, max(1, scan.n_proj // 4)):
        for iv in vs:
            for iu in us:
                yield p, iu, iv, S[p, iv, iu], D[p, iv, iu]


@pytest.mark.parametrize("which", ["tiny", "medium_tilted", "table1"])
def test_row_sums_equal_cylinder_chord(orc, which, golden_table1):
    window = None
    if which == "tiny":
        scan, step = synth.tiny_scan(), 1
    elif which == "medium_tilted":
        scan = synth.medium_scan(synth.rng_for("medium"), n_proj=8)
        step = 9
    else:
        # Table 1 geometry: the part's shadow is ~25 x 100 pixels around the centre
        scan, step = golden_table1, 3
        window = (scan.det_w // 2, scan.det_h // 2, 16, 66)
    o = osetup(orc, scan)
    L = orc.row_sums(o)
    n = 0
    for p, iu, iv, S, D in scan_grid_rays(scan, step, window):
        ref = bf.cylinder_chord(scan, S, D)
        # 1e-12 relative to the grid's size: near tangency the chord's condition number
        # grows like R / chord, so the scale is max(chord, R)
        assert abs(L[p, iv, iu] - ref) <= 1e-12 * max(ref, scan.radius), (p, iu, iv)
        n += ref > 0
    assert n > 10


def test_uniform_cylinder_projection(orc):
    scan = synth.medium_scan(synth.rng_for("medium"), n_proj=3, grid=(16, 48, 16), det=64,
                             pitch=3.2)
    o = osetup(orc, scan)
    q = orc.project(o, np.full(scan.vol_shape, 0.03))
    S, D = bf.rays(scan)
    for p in range(scan.n_proj):
        for iv in range(0, 64, 7):
            for iu in range(0, 64, 5):
                ref = 0.03 * bf.cylinder_chord(scan, S[p, iv, iu], D[p, iv, iu])
                assert abs(q[p, iv, iu] - ref) <= 1e-13, (p, iu, iv)


def test_annulus_and_slab_closed_forms(orc):
    # shell-aligned annulus x slab-aligned band: chord(r_b) - chord(r_a), each clipped in h
    scan = small_scan(8, 12, 10, n_proj=3, det=16, pitch=1.0, radius=5.0, height=6.0)
    x = np.zeros(scan.vol_shape)
    ia, ib, ha, hb = 3, 7, 2, 6          # r in [1.5, 3.5], h in [-1.5, 1.5]
    x[ha:hb, :, ia:ib] = 0.7
    q = orc.project(osetup(orc, scan), x)
    dr, dh = scan.radius / scan.n_r, scan.height / scan.n_h
    r_a, r_b = ia * dr, ib * dr
    h_a, h_b = -scan.height / 2 + ha * dh, -scan.height / 2 + hb * dh
    S, D = bf.rays(scan)
    worst = 0.0
    for p in range(scan.n_proj):
        for iv in range(16):
            for iu in range(16):
                ref = 0.7 * (bf.cylinder_chord(scan, S[p, iv, iu], D[p, iv, iu], r_b, h_a, h_b)
                             - bf.cylinder_chord(scan, S[p, iv, iu], D[p, iv, iu], r_a, h_a, h_b))
                worst = max(worst, abs(q[p, iv, iu] - ref))
    assert worst <= 1e-12


def test_axial_plane_annulus_textbook(orc):
    # ray in the plane z = 0 of an untilted object, distance d from the axis: the chord
    # through the annulus r_a..r_b is 2 (sqrt(r_b^2 - d^2) - sqrt(r_a^2 - d^2))
    s = synth.Scan(1, 7, 10, 10.0, 4.0, 50.0, 150.0, 41, 1, 0.9, 1.0, np.array([0.0]))
    o = osetup(orc, s)
    x = np.zeros(s.vol_shape)
    x[:, :, 4:8] = 1.0                       # r in [4, 8]
    q = orc.project(o, x)[0, 0]
    for iu in range(41):
        u = (iu - 20) * 0.9
        dist = abs(u) * 50.0 / math.hypot(150.0, u)   # distance of the ray from the axis
        ref = 0.0
        if dist < 8.0:
            ref = 2 * math.sqrt(64.0 - dist * dist)
            if dist < 4.0:
                ref -= 2 * math.sqrt(16.0 - dist * dist)
        assert abs(q[iu] - ref) <= 1e-12, iu


def test_sector_phantom(orc):
    # one wedge-aligned sector (all r, all h, theta in wedge k): the line clipped by the
    # disk and by two half-planes, computed here without the grid
    scan = small_scan(3, 6, 4, n_proj=4, det=12, pitch=1.3)
    k = 2
    x = np.zeros(scan.vol_shape)
    x[:, k, :] = 1.0
    q = orc.project(osetup(orc, scan), x)
    S, D = bf.rays(scan)
    for p in range(scan.n_proj):
        for iv in range(12):
            for iu in range(12):
                s0, d0 = S[p, iv, iu], D[p, iv, iu] - S[p, iv, iu]
                c = bf._cap((0.0, 1.0), bf.disk_interval(s0, d0, scan.radius))
                c = bf._cap(c, bf.slab_interval(s0, d0, -scan.height / 2, scan.height / 2))
                c = bf._cap(c, bf.wedge_interval(s0, d0, k, scan.n_theta))
                ref = 0.0 if c is None else (c[1] - c[0]) * np.linalg.norm(d0)
                assert abs(q[p, iv, iu] - ref) <= 1e-12


# ---------------------------------------------------------------- invariants

def test_theta_independent_volume_ignores_n_theta_and_gamma(orc):
    base = small_scan(5, 1, 6, n_proj=4, det=12, pitch=1.3)
    radial = np.linspace(0.01, 0.06, base.n_r)
    ref = None
    for n_t in (1, 2, 3, 64):
        for gamma in (0.0, 1.234):
            s = dataclasses.replace(base, n_theta=n_t, gamma=gamma)
            x = np.broadcast_to(radial, s.vol_shape)
            q = orc.project(osetup(orc, s), x)
            if ref is None:
                ref = q
            np.testing.assert_allclose(q, ref, rtol=0, atol=1e-12)


def test_h_refinement_invariance(orc):
    base = small_scan(2, 6, 4, n_proj=3, det=10, pitch=1.4)
    rng = np.random.default_rng(3)
    xt = rng.uniform(0, 1, size=(base.n_theta, base.n_r))
    ref = None
    for n_h in (1, 2, 8):
        s = dataclasses.replace(base, n_h=n_h)
        q = orc.project(osetup(orc, s), np.broadcast_to(xt, s.vol_shape))
        if ref is None:
            ref = q
        np.testing.assert_allclose(q, ref, rtol=0, atol=1e-12)


def test_gamma_by_one_wedge_rolls_theta(orc):
    # rotating the grid about its own axis by one wedge (gamma += 2 pi / N_theta) is the
    # same as rolling the volume by one wedge index
    s = small_scan(3, 7, 4, n_proj=3, det=10, pitch=1.4, pose=(0.0, 0.0, 0.3, 0.2, 0.1, 0.0))
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, size=s.vol_shape)
    q0 = orc.project(osetup(orc, s), x)
    s1 = dataclasses.replace(s, gamma=s.gamma + 2 * math.pi / s.n_theta)
    q1 = orc.project(osetup(orc, s1), np.roll(x, 1, axis=1))
    q2 = orc.project(osetup(orc, s1), np.roll(x, -1, axis=1))
    # exactly one of the two directions is the symmetry
    e1, e2 = np.abs(q1 - q0).max(), np.abs(q2 - q0).max()
    assert min(e1, e2) <= 1e-12 and max(e1, e2) > 1e-3


def test_adjoint_identity(orc):
    scan = small_scan(6, 20, 7, n_proj=6, det=14, pitch=1.1)
    o = osetup(orc, scan)
    rng = np.random.default_rng(11)
    for _ in range(3):
        x = rng.standard_normal(scan.vol_shape)
        y = rng.standard_normal(scan.sino_shape)
        lhs = float(np.sum(orc.project(o, x) * y))
        rhs = float(np.sum(x * orc.backproject(o, y)))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10, (lhs, rhs)


def test_backproject_equals_bruteforce_transpose(orc):
    scan = small_scan(3, 5, 3, n_proj=3, det=8)
    A = bf.dense_matrix(scan)
    rng = np.random.default_rng(2)
    y = rng.standard_normal(A.shape[0])
    bp = orc.backproject(osetup(orc, scan), y).reshape(-1)
    np.testing.assert_allclose(bp, A.T @ y, rtol=0, atol=1e-12 * np.abs(A.T @ y).max())


@pytest.mark.parametrize("grid", [(3, 6, 3), (2, 2, 4)])
def test_row_segment_count_matches_bruteforce(orc, grid):
    # segments per ray = pieces of the line inside voxels (a voxel of an annulus can be
    # entered twice when the ray dips into the shell below and comes back)
    scan = small_scan(*grid, n_proj=3, det=8)
    P = bf.dense_matrix(scan, pieces=True)
    nnz = orc.row_nnz(osetup(orc, scan)).reshape(-1)
    np.testing.assert_array_equal(nnz, P.sum(axis=1).astype(np.int64))


# ------------------------------------------------------------------ log transform

def test_log_transform_closed_form(orc):
    I0 = 1.0e4
    p_true = np.array([0.0, 0.5, 2.0, 7.0])
    I = I0 * np.exp(-p_true)
    np.testing.assert_allclose(orc.log_transform(I, I0), p_true, atol=1e-12)
    # counts below one are clamped to one count
    assert math.isclose(orc.log_transform(np.array([0.0]), I0)[0], math.log(I0))


# ------------------------------------------------------ general trajectories (frames)

def test_frames_of_a_circular_scan_reproduce_it(orc):
    # the frames of a circular scan (its stage turns applied to source and detector) must
    # give the circular scan's rays and projections exactly
    scan = small_scan(3, 8, 3, n_proj=5)
    fscan = dataclasses.replace(scan, frames=synth.frames_from_circular(scan))
    o, of = osetup(orc, scan), osetup(orc, fscan)
    for p in range(scan.n_proj):
        for iu, iv in ((0, 0), (3, 5), (7, 7)):
            a, b = orc.ray(o, p, iu, iv), orc.ray(of, p, iu, iv)
            np.testing.assert_allclose(b[0], a[0], atol=1e-12)
            np.testing.assert_allclose(b[1], a[1], atol=1e-12)
    x = np.random.default_rng(4).uniform(0.0, 0.05, size=scan.vol_shape)
    np.testing.assert_allclose(orc.project(of, x), orc.project(o, x), rtol=0, atol=1e-12)


def conveyor_scan(n_proj=6, det=12, grid=(3, 8, 4)):
    s = synth.Scan(*grid, 5.0, 6.0, 40.0, 100.0, det, det, 1.5, 1.5, np.zeros(n_proj))
    s.frames = synth.conveyor_frames(n_proj, 40.0, 100.0, det, det, 1.5, 30.0)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.3, 0.12, 0.8, 0.4, -0.2, 0.3
    return s


def test_conveyor_trajectory_rays_chords_and_bruteforce(orc):
    scan = conveyor_scan()
    o = osetup(orc, scan)
    S, D = bf.rays(scan)
    for p in range(scan.n_proj):
        for iu, iv in ((0, 0), (5, 6), (11, 11)):
            So, Do = orc.ray(o, p, iu, iv)
            np.testing.assert_allclose(So, S[p, iv, iu], atol=1e-12)
            np.testing.assert_allclose(Do, D[p, iv, iu], atol=1e-12)
    L = orc.row_sums(o)
    hit = 0
    for p in range(scan.n_proj):
        for iv in range(scan.det_h):
            for iu in range(scan.det_w):
                ref = bf.cylinder_chord(scan, S[p, iv, iu], D[p, iv, iu])
                assert abs(L[p, iv, iu] - ref) <= 1e-12 * max(ref, scan.radius)
                hit += ref > 0
    assert hit > 50
    A_bf = bf.dense_matrix(scan)
    A_or = oracle_matrix(orc, scan)
    np.testing.assert_allclose(A_or, A_bf, rtol=0, atol=1e-12 * np.abs(A_bf).max())
