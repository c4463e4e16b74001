"""Brute-force dense system matrix and closed-form chords (FP64, numpy).

An independent check of the oracle's traversal: instead of sorting crossings along a ray,
every (ray, voxel) entry is computed by clipping the line against that one voxel, an
annular sector [rho_i, rho_i+1] x [theta_k, theta_k+1] x [h_l, h_l+1] (the voxel of the
cylindrical grid of Sec. 2, Eq. 2), as an intersection of parameter intervals:

* the slab is one interval;
* the annulus is the disk of radius rho_i+1 minus the disk of radius rho_i, each disk
  cut out of the line with the foot-of-perpendicular construction (closest approach
  point and Pythagoras), giving up to two intervals;
* the wedge is the intersection of two half-planes for N_theta >= 3, one half-plane for
  N_theta = 2 and the whole plane for N_theta = 1.

The entry t_jl (Sec. 2.2, definition below Eq. 6) is the total length of the result.
Ray geometry (source and pixel positions) is restated here from the stated conventions
without calling the oracle.
"""
from __future__ import annotations

import math

import numpy as np


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rays(scan):
    """(S, D) arrays of shape (n_proj, H, W, 3): source and pixel centre, object frame."""
    # orientation Rz(alpha) Rx(beta) Rz(gamma); scanner -> object uses its transpose
    R = (rot_z(scan.alpha) @ rot_x(scan.beta) @ rot_z(scan.gamma)).T
    T = np.array([scan.tx, scan.ty, scan.tz])
    iu = np.arange(scan.det_w)
    iv = np.arange(scan.det_h)
    u = (iu - (scan.det_w - 1) / 2.0) * scan.pitch_u + scan.off_u
    v = (iv - (scan.det_h - 1) / 2.0) * scan.pitch_v + scan.off_v
    pix = np.zeros((scan.det_h, scan.det_w, 3))
    pix[..., 0] = scan.sdd - scan.sod
    pix[..., 1] = u[None, :]
    pix[..., 2] = v[:, None]
    src = np.array([-scan.sod, 0.0, 0.0])
    frames = getattr(scan, "frames", None)
    n = len(frames) if frames is not None else len(scan.angles)
    S = np.zeros((n, scan.det_h, scan.det_w, 3))
    D = np.zeros_like(S)
    if frames is not None:
        # general trajectory: each projection's own source and detector, in stage
        # coordinates (no stage turn)
        for p in range(n):
            f = np.asarray(frames[p], dtype=np.float64)
            pts = f[3:6][None, None, :] + iu[None, :, None] * f[6:9] + iv[:, None, None] * f[9:12]
            S[p] = R @ (f[0:3] - T)
            D[p] = (pts - T) @ R.T
        return S, D
    for p, phi in enumerate(scan.angles):
        # lab -> stage (rotate by -phi) -> object: X' = R (X - T)
        S[p] = R @ (rot_z(-phi) @ src - T)
        D[p] = (pix @ rot_z(-phi).T - T) @ R.T
    return S, D


def disk_interval(o, d, rho):
    """Parameter interval of the line o + t d (2-D part) inside the disk r <= rho, by the
    foot of the perpendicular; None if the line misses it."""
    a = d[0] * d[0] + d[1] * d[1]
    if a == 0.0:
        return (-np.inf, np.inf) if o[0] ** 2 + o[1] ** 2 <= rho * rho else None
    t0 = -(o[0] * d[0] + o[1] * d[1]) / a
    fx, fy = o[0] + t0 * d[0], o[1] + t0 * d[1]
    h2 = rho * rho - (fx * fx + fy * fy)
    if h2 <= 0.0:
        return None
    half = math.sqrt(h2 / a)
    return (t0 - half, t0 + half)


def slab_interval(o, d, h_a, h_b):
    if d[2] == 0.0:
        return (-np.inf, np.inf) if h_a <= o[2] <= h_b else None
    t1, t2 = (h_a - o[2]) / d[2], (h_b - o[2]) / d[2]
    return (min(t1, t2), max(t1, t2))


def halfplane_interval(o, d, nx, ny):
    """{t : n . P(t) >= 0} as an interval."""
    f0 = nx * o[0] + ny * o[1]
    f1 = nx * d[0] + ny * d[1]
    if f1 == 0.0:
        return (-np.inf, np.inf) if f0 >= 0.0 else None
    t = -f0 / f1
    return (t, np.inf) if f1 > 0.0 else (-np.inf, t)


def _cap(a, b):
    if a is None or b is None:
        return None
    lo, hi = max(a[0], b[0]), min(a[1], b[1])
    return (lo, hi) if hi > lo else None


def annulus_intervals(o, d, rho_a, rho_b):
    outer = disk_interval(o, d, rho_b)
    if outer is None:
        return []
    inner = disk_interval(o, d, rho_a) if rho_a > 0.0 else None
    if inner is None:
        return [outer]
    out = []
    left = _cap(outer, (-np.inf, inner[0]))
    right = _cap(outer, (inner[1], np.inf))
    if left:
        out.append(left)
    if right:
        out.append(right)
    return out


def wedge_interval(o, d, k, n_theta):
    if n_theta == 1:
        return (-np.inf, np.inf)
    th0 = 2.0 * math.pi * k / n_theta
    th1 = 2.0 * math.pi * (k + 1) / n_theta
    if n_theta == 2:
        # wedge 0 is y >= 0 side of the x axis, wedge 1 the other side
        s = 1.0 if k == 0 else -1.0
        return halfplane_interval(o, d, 0.0, s)
    a = halfplane_interval(o, d, -math.sin(th0), math.cos(th0))   # left of theta_k
    b = halfplane_interval(o, d, math.sin(th1), -math.cos(th1))   # right of theta_k+1
    return _cap(a, b)


def dense_row(scan, S, D, pieces=False):
    """Dense row of the system matrix (length n_vox) for the segment S -> D; with
    ``pieces`` the number of disjoint pieces of the line inside each voxel instead."""
    d = D - S
    dn = float(np.linalg.norm(d))
    row = np.zeros((scan.n_h, scan.n_theta, scan.n_r))
    dr = scan.radius / scan.n_r
    dh = scan.height / scan.n_h
    seg = (0.0, 1.0)
    for ih in range(scan.n_h):
        hi = _cap(seg, slab_interval(S, d, -scan.height / 2 + ih * dh,
                                     -scan.height / 2 + (ih + 1) * dh))
        if hi is None:
            continue
        for it in range(scan.n_theta):
            ti = _cap(hi, wedge_interval(S, d, it, scan.n_theta))
            if ti is None:
                continue
            for ir in range(scan.n_r):
                tot = 0.0
                cnt = 0
                for piece in annulus_intervals(S, d, ir * dr, (ir + 1) * dr):
                    c = _cap(ti, piece)
                    if c:
                        tot += c[1] - c[0]
                        cnt += 1
                row[ih, it, ir] = cnt if pieces else tot * dn
    return row.reshape(-1)


def dense_matrix(scan, pieces=False):
    S, D = rays(scan)
    rows = [dense_row(scan, S[p, v, u], D[p, v, u], pieces)
            for p in range(len(scan.angles)) for v in range(scan.det_h)
            for u in range(scan.det_w)]
    return np.array(rows)


def cylinder_chord(scan, S, D, rho=None, h_a=None, h_b=None):
    """Length of the segment S -> D inside {r <= rho, h_a <= h <= h_b} (defaults: the grid
    cylinder), by the foot-of-perpendicular construction."""
    rho = scan.radius if rho is None else rho
    h_a = -scan.height / 2 if h_a is None else h_a
    h_b = scan.height / 2 if h_b is None else h_b
    d = D - S
    c = _cap((0.0, 1.0), disk_interval(S, d, rho))
    c = _cap(c, slab_interval(S, d, h_a, h_b))
    return 0.0 if c is None else (c[1] - c[0]) * float(np.linalg.norm(d))
