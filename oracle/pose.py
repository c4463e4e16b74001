"""FP64 oracle of the projection-based pose estimation (Sec. 2.1) and the azimuthal
phase (Sec. 2.1, Eq. 5).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
baseline may call it; the product path never does.  It shares no code with the CUDA
path: views come from the C oracle's ray geometry, every step is written out as its
plain definition with numpy, in the paper's order.

* Axis tracking (Sec. 2.1, "Axis tracking"): threshold the line integrals, dilate the
  mask with a square structuring element, take the four corner pixels of the dilated
  mask, and pair them: the centre of the two top corners and the centre of the two
  bottom corners lie on the projected symmetry axis.
* Point tracking (Sec. 2.1, Eq. 3-4): the 3-D point whose projections V_i best match a
  track (u, v)_i, found by Levenberg-Marquardt with analytic derivatives of V_i.
* Pose from two axis points: the axis direction and centre fix five degrees of freedom
  of Eq. 1; the internal rotation gamma stays free.
* Azimuthal phase (Eq. 5): the grey values of a band along the projected axis, as a
  function of the projection angle: the first-harmonic phase of their centroid's
  offset across the axis, and the tilt-corrected conversion of the phase to gamma.

Conventions (the same as the reconstruction's): the object-to-stage rotation is the
intrinsic zxz rotation O = R_z(alpha) R_x(beta) R_z(gamma), a stage point is
X = O X' + T, and the object axis is the z' axis.  Detector coordinates (a, b) are pixel
indices: a along u (the detector's pixel step du), b along v (dv); pixel (0, 0) has its
centre at D0.

Corner keys.  "Corner pixel" is read as the pixel of the dilated mask that is extreme
along a diagonal of the detector: top-right maximises a + b, top-left -a + b,
bottom-left -a - b, bottom-right a - b.  Ties go to the pixel farthest from the middle
row in the corner's direction (largest b for the top corners, smallest for the bottom).
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as _orc

# top-left, top-right, bottom-left, bottom-right: (sign of a, sign of b) of the key
CORNERS = ((-1, 1), (1, 1), (-1, -1), (1, -1))


# ------------------------------------------------------------------ views (Eq. 3)
def stage_views(s: _orc.Setup):
    """Per projection: source S, pixel (0, 0) centre D0 and pixel steps du, dv in stage
    coordinates, read from the oracle's rays of the scan with the identity pose."""
    import dataclasses
    s0 = dataclasses.replace(s, alpha=0.0, beta=0.0, gamma=0.0, tx=0.0, ty=0.0, tz=0.0)
    out = []
    for p in range(s0.n_proj):
        S, D0 = _orc.ray(s0, p, 0, 0)
        _, D1 = _orc.ray(s0, p, 1, 0)
        _, D2 = _orc.ray(s0, p, 0, 1)
        out.append((S, D0, D1 - D0, D2 - D0))
    return out


def project_point(view, X):
    """V_i(X) (Eq. 3): pixel coordinates (a, b) where the line from the source through X
    meets the detector plane, from D0 + a du + b dv = S + t (X - S)."""
    S, D0, du, dv = view
    M = np.column_stack([du, dv, -(np.asarray(X, float) - S)])
    a, b, t = np.linalg.solve(M, S - D0)
    return np.array([a, b]), t, M


def project_point_jacobian(view, X):
    """V_i(X) and its analytic derivative: differentiating M(X) (a, b, t) = S - D0 gives
    d(a, b, t)/dX = t M^-1, of which the first two rows belong to (a, b)."""
    ab, t, M = project_point(view, X)
    return ab, (t * np.linalg.inv(M))[:2]


# ------------------------------------------------------------------ axis tracking
def window(roi, det_w: int, det_h: int):
    """Detector window [u0, u1) x [v0, v1); all zeros selects the whole detector."""
    if roi is None or all(int(x) == 0 for x in roi):
        return 0, det_w, 0, det_h
    return tuple(int(x) for x in roi)


def segment(p_view, threshold: float, k: int, roi=None):
    """Threshold (p > threshold) and dilation by the (2k+1)^2 square, both inside the
    window; pixels outside the window are background.  Returns (dilated mask, number of
    thresholded pixels)."""
    H, W = p_view.shape
    u0, u1, v0, v1 = window(roi, W, H)
    m = np.zeros((H, W), bool)
    m[v0:v1, u0:u1] = np.asarray(p_view, np.float64)[v0:v1, u0:u1] > threshold
    d = np.zeros_like(m)
    for dv in range(-k, k + 1):
        for du in range(-k, k + 1):
            # d[v + dv, u + du] |= m[v, u] for target pixels inside the window
            ts_v = slice(max(v0, v0 + dv), min(v1, v1 + dv))
            ts_u = slice(max(u0, u0 + du), min(u1, u1 + du))
            ss_v = slice(ts_v.start - dv, ts_v.stop - dv)
            ss_u = slice(ts_u.start - du, ts_u.stop - du)
            if ts_v.start < ts_v.stop and ts_u.start < ts_u.stop:
                d[ts_v, ts_u] |= m[ss_v, ss_u]
    return d, int(m.sum())


def corners(mask):
    """The four corner pixels (a, b) of a mask in the order TL, TR, BL, BR; (-1, -1) each
    when the mask is empty."""
    bs, as_ = np.nonzero(mask)
    if as_.size == 0:
        return -np.ones((4, 2), np.int64)
    out = np.zeros((4, 2), np.int64)
    for c, (sa, sb) in enumerate(CORNERS):
        key = sa * as_ + sb * bs
        tie = bs if sb > 0 else -bs
        best = np.lexsort((tie, key))[-1]      # primary key, then the tie-break
        out[c] = (as_[best], bs[best])
    return out


def axis_tracks(sino, threshold: float, k: int, roi=None):
    """Corners of every projection and the pairwise centres: (corners (n, 4, 2), counts
    (n,), top (n, 2), bottom (n, 2), valid (n,))."""
    n = sino.shape[0]
    cs = np.zeros((n, 4, 2), np.int64)
    counts = np.zeros(n, np.int64)
    for p in range(n):
        mask, counts[p] = segment(sino[p], threshold, k, roi)
        cs[p] = corners(mask)
    valid = cs[:, 0, 0] >= 0
    top = 0.5 * (cs[:, 0] + cs[:, 1]).astype(np.float64)
    bottom = 0.5 * (cs[:, 2] + cs[:, 3]).astype(np.float64)
    return cs, counts, top, bottom, valid


# ------------------------------------------------------------------ point tracking
def _residuals(views, obs, valid, X):
    rows, jac = [], []
    for view, o, ok in zip(views, obs, valid):
        if not ok:
            continue
        ab, J = project_point_jacobian(view, X)
        su, sv = np.linalg.norm(view[2]), np.linalg.norm(view[3])
        rows.append([(o[0] - ab[0]) * su, (o[1] - ab[1]) * sv])
        jac.append(J * np.array([[su], [sv]]))
    return np.concatenate(rows), np.concatenate(jac)


def initial_point(views, obs, valid):
    """Start of the iteration: on the ray of the first observed projection, at the
    distance of the stage origin from that projection's source."""
    i = int(np.flatnonzero(valid)[0])
    S, D0, du, dv = views[i]
    P = D0 + obs[i][0] * du + obs[i][1] * dv
    return S + np.linalg.norm(S) * (P - S) / np.linalg.norm(P - S)


def track_point(views, obs, valid, max_iter: int = 100):
    """Eq. 4 by Levenberg-Marquardt: minimise the squared detector distances (mm)
    between the track and V_i(X).  Damping mu starts at 1e-3, falls tenfold after an
    accepted step (not below 1e-15) and rises tenfold after a rejected one; the
    iteration stops after a step (accepted or not) shorter than 1e-10 (1 + |X|), when mu
    exceeds 1e15, or after max_iter steps.  Returns (X, rms distance in mm, steps taken)."""
    valid = np.asarray(valid, bool)
    X = initial_point(views, obs, valid)
    mu = 1e-3
    r, J = _residuals(views, obs, valid, X)
    cost = float(r @ r)
    it = 0
    while it < max_iter:
        it += 1
        A = J.T @ J
        g = J.T @ r
        try:
            step = np.linalg.solve(A + mu * np.diag(np.diag(A)), g)
        except np.linalg.LinAlgError:
            mu *= 10.0
            if mu > 1e15:
                break
            continue
        Xn = X + step
        rn, Jn = _residuals(views, obs, valid, Xn)
        cn = float(rn @ rn)
        small = np.linalg.norm(step) <= 1e-10 * (1.0 + np.linalg.norm(Xn if cn < cost else X))
        if cn < cost:
            X, r, J, cost = Xn, rn, Jn, cn
            mu = max(mu / 10.0, 1e-15)
        else:
            mu *= 10.0
        if small or mu > 1e15:
            break
    return X, math.sqrt(cost / int(valid.sum())), it


def pose_from_axis(top, bottom, gamma: float = 0.0):
    """Pose (alpha, beta, gamma, tx, ty, tz) whose z' axis runs from ``bottom`` to ``top``
    and whose origin is their midpoint: O e_z = (sin a sin b, -cos a sin b, cos b)."""
    top = np.asarray(top, float)
    bottom = np.asarray(bottom, float)
    ax = (top - bottom) / np.linalg.norm(top - bottom)
    beta = math.acos(max(-1.0, min(1.0, ax[2])))
    alpha = math.atan2(ax[0], -ax[1]) if math.hypot(ax[0], ax[1]) > 1e-15 else 0.0
    c = 0.5 * (top + bottom)
    return (alpha, beta, gamma, c[0], c[1], c[2])


def estimate_pose(s: _orc.Setup, sino, threshold: float, k: int = 0, roi=None,
                  max_iter: int = 100, gamma: float = 0.0):
    """The whole chain of Sec. 2.1: tracks of the two axis points, Eq. 4 for each, and
    the pose.  Returns (pose, dict of the intermediate results)."""
    cs, counts, top, bottom, valid = axis_tracks(sino, threshold, k, roi)
    views = stage_views(s)
    Xt, rt, it_t = track_point(views, top, valid, max_iter)
    Xb, rb, it_b = track_point(views, bottom, valid, max_iter)
    return pose_from_axis(Xt, Xb, gamma), dict(
        corners=cs, counts=counts, top=Xt, bottom=Xb, rms=(rt, rb), iters=(it_t, it_b),
        n_views=int(valid.sum()))


# ------------------------------------------------------------------ azimuthal phase
def axis_point(pose, h: float):
    """Stage coordinates of the object point (0, 0, h): X = O X' + T."""
    R = _orc.pose_matrix(pose[0], pose[1], pose[2])       # object-from-stage, = O^T
    return R.T @ np.array([0.0, 0.0, h]) + np.array(pose[3:6], float)


def band_constants(view, pose, h_lo: float, h_hi: float):
    """FP32 constants of the band test of one projection: the projected axis point A of
    height h_lo, and the coefficients that turn a pixel offset from A into the
    perpendicular distance d (mm on the detector, positive towards +u) and the fraction s
    of the way to the projected point of height h_hi."""
    A, _, _ = project_point(view, axis_point(pose, h_lo))
    B, _, _ = project_point(view, axis_point(pose, h_hi))
    su, sv = np.linalg.norm(view[2]), np.linalg.norm(view[3])
    Lu, Lv = (B[0] - A[0]) * su, (B[1] - A[1]) * sv
    L2 = Lu * Lu + Lv * Lv
    L = math.sqrt(L2)
    f = np.float32
    return (f(A[0]), f(A[1]), f(su * Lv / L), f(-sv * Lu / L), f(su * Lu / L2), f(sv * Lv / L2))


def band_offsets(shape, consts, half_width: float):
    """Band beside the projected axis, 0 <= s <= 1 and |d| <= half_width, and the signed
    distance d of every pixel, both evaluated in FP32 as d = (a - A_u) c_du +
    (b - A_v) c_dv and s = (a - A_u) c_su + (b - A_v) c_sv: (mask, d)."""
    H, W = shape
    Au, Av, cdu, cdv, csu, csv = consts
    f = np.float32
    fa = (np.arange(W, dtype=f) - Au)[None, :]
    fb = (np.arange(H, dtype=f) - Av)[:, None]
    d = fa * cdu + fb * cdv
    s = fa * csu + fb * csv
    hw = f(half_width)
    return (s >= f(0)) & (s <= f(1)) & (d >= -hw) & (d <= hw), d


def band_moments(s: _orc.Setup, pose, sino, h_lo: float, h_hi: float, half_width: float):
    """Per projection, the grey-value sum of the band and its first moment across the
    projected axis, (sum p, sum p d): (n, 2)."""
    views = stage_views(s)
    m = np.zeros((len(views), 2))
    for p, view in enumerate(views):
        mask, d = band_offsets(sino[p].shape, band_constants(view, pose, h_lo, h_hi), half_width)
        img = np.asarray(sino[p], np.float64)
        m[p] = (float(img[mask].sum()), float((img[mask] * d[mask].astype(np.float64)).sum()))
    return m


def band_signal(s: _orc.Setup, pose, sino, h_lo: float, h_hi: float, half_width: float):
    """Grey-value centroid of the band, as a signed distance (mm) from the projected
    axis, per projection (0 where the band holds no grey value).  An axisymmetric part
    has its centroid on the axis in every projection; material off the axis pulls the
    centroid to its side, in a sine of the projection angle."""
    m = band_moments(s, pose, sino, h_lo, h_hi, half_width)
    return np.where(m[:, 0] != 0.0, m[:, 1] / np.where(m[:, 0] != 0.0, m[:, 0], 1.0), 0.0)


def phase(angles, g):
    """First-harmonic phase phi_P and amplitude of g over the projection angles: the
    least-squares fit g ~ c0 + c1 cos(phi) + c2 sin(phi), phi_P = atan2(c2, c1)."""
    angles = np.asarray(angles, float)
    M = np.column_stack([np.ones_like(angles), np.cos(angles), np.sin(angles)])
    c = np.linalg.lstsq(M, np.asarray(g, float), rcond=None)[0]
    return math.atan2(c[2], c[1]), math.hypot(c[1], c[2])


def inplane_angle(psi: float, alpha: float, beta: float) -> float:
    """Angle from the line of nodes, inside the object's tilted x'y' plane, of the
    direction whose stage azimuth is psi: the exact inverse of
    psi = alpha + atan2(cos(beta) sin(e), cos(e))."""
    return math.atan2(math.sin(psi - alpha), math.cos(beta) * math.cos(psi - alpha))


def wrap(x: float) -> float:
    return math.atan2(math.sin(x), math.cos(x))


def gamma_from_phase(phi_p: float, phi_p_ref: float, alpha: float, beta: float,
                     gamma_ref: float = 0.0, phi_g: float = 0.5 * math.pi) -> float:
    """Eq. 5 with the tilt correction applied exactly.  The centroid moves furthest to
    the +u side for material at lab azimuth phi_g = 90 deg, so material at stage azimuth
    psi peaks at phi_P = phi_g - psi.  The reference is the same measurement on
    projections of a template whose spin is gamma_ref; the part's spin differs from it by
    the difference of the two in-plane angles."""
    e = inplane_angle(phi_g - phi_p, alpha, beta)
    e_ref = inplane_angle(phi_g - phi_p_ref, alpha, beta)
    return wrap(gamma_ref + e - e_ref)


def azimuthal_mean(x):
    """The axisymmetric part of a volume: its mean over theta in every (h, r) cell."""
    x = np.asarray(x, np.float64)
    return np.broadcast_to(x.mean(axis=1, keepdims=True), x.shape).copy()


def estimate_gamma(s: _orc.Setup, sino, tmpl, h_lo: float, h_hi: float, half_width: float,
                   passes: int = 1):
    """Spin of the scanned part relative to a template.  ``s`` carries the part's alpha,
    beta and T and the template's starting spin as gamma.  The template and its azimuthal
    mean are projected at that pose; the centroid signal of the mean (the geometric part,
    present in all three) is subtracted from those of the scan and the template before
    their phases are taken.  Every further pass projects the template at the current
    estimate and repeats.  Returns (gamma, (phi_P, amplitude, phi_P_ref, reference
    amplitude) of the last pass)."""
    import dataclasses
    pose = (s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz)
    q_mean = _orc.project(s, azimuthal_mean(tmpl))
    c_scan = band_signal(s, pose, sino, h_lo, h_hi, half_width)
    c_mean = band_signal(s, pose, q_mean, h_lo, h_hi, half_width)
    ph, amp = phase(s.angles, c_scan - c_mean)
    gamma, diag = s.gamma, None
    for _ in range(passes):
        sr = dataclasses.replace(s, gamma=gamma)
        c_tmpl = band_signal(sr, pose, _orc.project(sr, tmpl), h_lo, h_hi, half_width)
        ph_ref, amp_ref = phase(s.angles, c_tmpl - c_mean)
        gamma = gamma_from_phase(ph, ph_ref, s.alpha, s.beta, gamma)
        diag = (ph, amp, ph_ref, amp_ref)
    return gamma, diag


def eq5_printed(phi_p: float, phi_g: float, alpha: float, beta: float) -> float:
    """Eq. 5 as printed: gamma = phi_P - phi_G - arctan(tan(alpha) / cos(beta))."""
    return phi_p - phi_g - math.atan(math.tan(alpha) / math.cos(beta))
