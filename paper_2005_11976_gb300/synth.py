"""Seeded synthetic inputs: scan descriptions, phantoms, weight maps, noise.

This module is shared by the tests, the benchmark and the oracle checks.  It holds no
reconstruction arithmetic (no rays, no intersection lengths, no SART): only the
description of each workload and the voxel values of the phantoms placed on the
cylindrical grid.

Workloads mirror the parts the paper inspects (Sec. 2.4 and 3.3: axisymmetric
industrial parts with metal inserts, some with a component missing).  Sizes follow
the five workloads the library is benchmarked on:

* ``tiny``      grid (16, 64, 16), R 10 mm, H 20 mm; SOD 100, SDD 400; 32 views over
                360 deg; 32x32 detector at 1.6 mm; mu = 0.02/mm cylinder with two
                full-height r = 2 mm holes at r = 5 mm, seeded azimuths.
* ``medium``    grid (128, 512, 128), R 25, H 50; SOD 200, SDD 800; 180 views;
                256x256 detector at 0.8 mm; five concentric shells plus eight r = 2 mm
                inserts at r = 15 mm (one removed); seeded pose |T| <= 2 mm, beta <= 1 deg.
* ``precision`` grid (256, 1024, 256); 360 views; 512x512 detector at 0.4 mm.
* ``batched``   64 scans on the medium grid, N_p in {60, 90, 120, 180}, T in +-5 mm,
                beta in +-3 deg.
* ``serving``   Poisson arrivals of mixed part types (64,256,64) / (128,512,128) /
                (256,1024,256) with detectors 128^2 / 256^2 / 512^2.

Seeds: numpy PCG64, base seed 20051197 + workload index; per-scan seed = base + scan id.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20051197
WORKLOAD_INDEX = {"tiny": 0, "medium": 1, "precision": 2, "batched": 3, "serving": 4, "pose": 5,
                  "table1": 6, "phase": 7}


@dataclasses.dataclass
class Scan:
    """One scan: cylindrical grid, circular cone-beam geometry and object pose.

    Lengths in mm, angles in radians.  ``angles`` are the stage angles phi_p.
    """
    n_h: int
    n_theta: int
    n_r: int
    radius: float
    height: float
    sod: float
    sdd: float
    det_w: int
    det_h: int
    pitch_u: float
    pitch_v: float
    angles: np.ndarray
    off_u: float = 0.0
    off_v: float = 0.0
    alpha: float = 0.0
    beta: float = 0.0
    gamma: float = 0.0
    tx: float = 0.0
    ty: float = 0.0
    tz: float = 0.0
    frames: np.ndarray | None = None   # (n_proj, 12) general trajectory, or None (circular)

    @property
    def n_proj(self) -> int:
        return int(len(self.frames)) if self.frames is not None else int(len(self.angles))

    @property
    def vol_shape(self):
        return (self.n_h, self.n_theta, self.n_r)

    @property
    def sino_shape(self):
        return (self.n_proj, self.det_h, self.det_w)

    @property
    def n_vox(self) -> int:
        return self.n_h * self.n_theta * self.n_r

    @property
    def n_rays(self) -> int:
        return self.n_proj * self.det_h * self.det_w

    def fields(self) -> dict:
        return dataclasses.asdict(self)


def rng_for(workload: str, scan_id: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + WORKLOAD_INDEX[workload] + scan_id))


def full_circle(n_proj: int) -> np.ndarray:
    """Equally spaced stage angles over 360 degrees."""
    return 2.0 * math.pi * np.arange(n_proj) / n_proj


def limited_arc(n_proj: int, last_angle_deg: float) -> np.ndarray:
    """n_proj angles from 0 to the last scan angle inclusive (the Table 1 style of scan)."""
    return np.deg2rad(last_angle_deg) * np.arange(n_proj) / max(n_proj - 1, 1)


def frames_from_circular(scan: Scan, stage_y_mm: float = 0.0) -> np.ndarray:
    """The (n_proj, 12) frames (source, pixel (0, 0) centre, pixel steps du, dv, in stage
    coordinates) of a circular scan: the stage turn of each projection applied to the
    fixed source and detector.  ``stage_y_mm`` moves the turning stage sideways (along
    the detector's u) off the line from the source to the detector centre."""
    out = np.zeros((scan.n_proj, 12))
    u0 = -0.5 * (scan.det_w - 1) * scan.pitch_u + scan.off_u
    v0 = -0.5 * (scan.det_h - 1) * scan.pitch_v + scan.off_v
    y = stage_y_mm
    for p, phi in enumerate(scan.angles):
        c, s_ = math.cos(phi), math.sin(phi)
        rot = lambda v: (c * v[0] + s_ * v[1], -s_ * v[0] + c * v[1], v[2])
        out[p, 0:3] = rot((-scan.sod, -y, 0.0))
        out[p, 3:6] = rot((scan.sdd - scan.sod, u0 - y, v0))
        out[p, 6:9] = rot((0.0, scan.pitch_u, 0.0))
        out[p, 9:12] = rot((0.0, 0.0, scan.pitch_v))
    return out


# Table 1 (circular cone-beam scans of medical devices) and Sec. 3.2.  The detector is
# the named 1944 x 1536 panel with 0.0748 mm pixels (the printed 0.748 mm would make it
# 1.45 m wide at 791 mm from the source).  The part (KN-S) is 64 mm high with an 8 mm
# radius; the five scans of each part put the stage's axis on these detector columns.
TABLE1 = dict(sod=679.0, sdd=791.0, n_proj=21, last_angle_deg=200.0, det_w=1944, det_h=1536,
              pixel_mm=0.0748, height_mm=64.0, radius_mm=8.0)
TABLE1_STAGE_COLUMNS = (185.2, 574.5, 963.9, 1353.25, 1742.6)


def table1_scan(grid=(1, 1, 8)) -> Scan:
    """Table 1's acquisition, on a coarse grid over the part (for synthesising its
    projections from a radial profile)."""
    t = TABLE1
    return Scan(grid[0], grid[1], grid[2], t["radius_mm"], t["height_mm"], t["sod"], t["sdd"],
                t["det_w"], t["det_h"], t["pixel_mm"], t["pixel_mm"],
                limited_arc(t["n_proj"], t["last_angle_deg"]))


def stage_shift_mm(column_px: float) -> float:
    """Sideways stage position that puts the stage axis's shadow on a detector column."""
    t = TABLE1
    return (column_px - 0.5 * (t["det_w"] - 1)) * t["pixel_mm"] * t["sod"] / t["sdd"]


def conveyor_frames(n_proj: int, sod: float, sdd: float, det_w: int, det_h: int, pitch: float,
                    travel: float) -> np.ndarray:
    """A part carried along +y on a belt through a fixed cone beam: in the part's stage
    frame the source and the detector move along -y, over `travel` mm centred on the axis."""
    out = np.zeros((n_proj, 12))
    u0 = -0.5 * (det_w - 1) * pitch
    v0 = -0.5 * (det_h - 1) * pitch
    for p, y in enumerate(np.linspace(-0.5 * travel, 0.5 * travel, n_proj)):
        out[p, 0:3] = (-sod, -y, 0.0)
        out[p, 3:6] = (sdd - sod, u0 - y, v0)
        out[p, 6:9] = (0.0, pitch, 0.0)
        out[p, 9:12] = (0.0, 0.0, pitch)
    return out


# --------------------------------------------------------------------------- scans

def tiny_scan() -> Scan:
    return Scan(16, 64, 16, 10.0, 20.0, 100.0, 400.0, 32, 32, 1.6, 1.6, full_circle(32))


def medium_scan(pose_seed_rng: np.random.Generator | None = None, n_proj: int = 180,
                grid=(128, 512, 128), det: int = 256, pitch: float = 0.8,
                pose=None) -> Scan:
    n_h, n_t, n_r = grid
    s = Scan(n_h, n_t, n_r, 25.0, 50.0, 200.0, 800.0, det, det, pitch, pitch,
             full_circle(n_proj))
    if pose is not None:
        s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
    elif pose_seed_rng is not None:
        s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = seeded_pose(pose_seed_rng, 2.0, 1.0)
    return s


def precision_scan(rng: np.random.Generator | None = None) -> Scan:
    return medium_scan(rng, n_proj=360, grid=(256, 1024, 256), det=512, pitch=0.4)


def seeded_pose(rng: np.random.Generator, t_max_mm: float, tilt_max_deg: float):
    """(alpha, beta, gamma, tx, ty, tz): |T| <= t_max, |beta| <= tilt_max."""
    while True:
        t = rng.uniform(-t_max_mm, t_max_mm, size=3)
        if np.linalg.norm(t) <= t_max_mm:
            break
    alpha = rng.uniform(0.0, 2.0 * math.pi)
    beta = math.radians(rng.uniform(-tilt_max_deg, tilt_max_deg))
    gamma = rng.uniform(0.0, 2.0 * math.pi)
    return (alpha, beta, gamma, float(t[0]), float(t[1]), float(t[2]))


def batched_scans(n_scans: int = 64, base: str = "batched"):
    """Scans of one part type: N_p ~ U{60,90,120,180}, T ~ U[-5,5]^3 mm, beta ~ U[-3,3] deg."""
    out = []
    for i in range(n_scans):
        rng = rng_for(base, i)
        n_proj = int(rng.choice([60, 90, 120, 180]))
        t = rng.uniform(-5.0, 5.0, size=3)
        pose = (rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(-3.0, 3.0)),
                rng.uniform(0, 2 * math.pi), float(t[0]), float(t[1]), float(t[2]))
        out.append(medium_scan(n_proj=n_proj, pose=pose))
    return out


SERVING_PART_TYPES = {
    "small": dict(grid=(64, 256, 64), det=128),
    "medium": dict(grid=(128, 512, 128), det=256),
    "large": dict(grid=(256, 1024, 256), det=512),
}


def serving_stream(rate_per_s: float = 20.0, duration_s: float = 60.0, seed_offset: int = 0,
                   part_types=("small", "medium", "large"), n_proj_choices=(60, 90, 120, 180, 240, 360)):
    """Poisson arrival stream: list of (arrival_s, part_type, Scan, removed_insert or -1)."""
    rng = rng_for("serving", seed_offset)
    t = 0.0
    out = []
    k = 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s:
            break
        pt = part_types[int(rng.integers(len(part_types)))]
        cfg = SERVING_PART_TYPES[pt]
        n_proj = int(rng.choice(list(n_proj_choices)))
        pose = seeded_pose(rng, 2.0, 1.0)
        scan = medium_scan(n_proj=n_proj, grid=cfg["grid"], det=cfg["det"],
                           pitch=204.8 / cfg["det"], pose=pose)
        removed = int(rng.integers(8)) if rng.uniform() < 0.1 else -1
        out.append((t, pt, scan, removed))
        k += 1
    return out


# ------------------------------------------------------------------------- phantoms

def _annulus_fraction(scan: Scan, r_a: float, r_b: float) -> np.ndarray:
    """Area fraction of each radial bin covered by r_a <= r <= r_b (exact)."""
    dr = scan.radius / scan.n_r
    lo = np.arange(scan.n_r) * dr
    hi = lo + dr
    a = np.clip(np.maximum(lo, r_a), None, None)
    b = np.minimum(hi, r_b)
    cov = np.where(b > a, b * b - a * a, 0.0)
    return cov / (hi * hi - lo * lo)


def _disk_fraction(scan: Scan, cx: float, cy: float, rad: float, ss: int = 8) -> np.ndarray:
    """(n_theta, n_r) area fraction of each (theta, r) cell inside a disk, by ss x ss
    samples uniform in (r^2, theta) per cell (equal-area sampling)."""
    n_t, n_r = scan.n_theta, scan.n_r
    dr = scan.radius / n_r
    dth = 2.0 * math.pi / n_t
    frac = np.zeros((n_t, n_r))
    dc = math.hypot(cx, cy)
    r_lo = max(dc - rad, 0.0)
    r_hi = dc + rad
    ir0 = max(int(r_lo / dr) - 1, 0)
    ir1 = min(int(r_hi / dr) + 2, n_r)
    off = (np.arange(ss) + 0.5) / ss
    for ir in range(ir0, ir1):
        r2 = ((ir * dr) ** 2 + off * (((ir + 1) * dr) ** 2 - (ir * dr) ** 2))
        rs = np.sqrt(r2)
        if dc - rad > 1e-12 + (ir + 1) * dr or dc + rad < ir * dr - 1e-12:
            continue
        if dc > rad:
            half = math.asin(min(rad / max(dc, 1e-12), 1.0))
            phi = math.atan2(cy, cx) % (2 * math.pi)
            it = np.arange(int(math.floor((phi - half) / dth)) - 1,
                           int(math.floor((phi + half) / dth)) + 2) % n_t
            it = np.unique(it)
        else:
            it = np.arange(n_t)
        th = (it[:, None] + off[None, :]) * dth          # (cells, ss)
        x = rs[None, None, :] * np.cos(th)[:, :, None]
        y = rs[None, None, :] * np.sin(th)[:, :, None]
        inside = (x - cx) ** 2 + (y - cy) ** 2 <= rad * rad
        frac[it, ir] = inside.mean(axis=(1, 2))
    return frac


def _slab_fraction(scan: Scan, h_a: float, h_b: float) -> np.ndarray:
    dh = scan.height / scan.n_h
    lo = -0.5 * scan.height + np.arange(scan.n_h) * dh
    hi = lo + dh
    return np.clip(np.minimum(hi, h_b) - np.maximum(lo, h_a), 0.0, None) / dh


def tiny_phantom(scan: Scan, rng: np.random.Generator) -> np.ndarray:
    """mu = 0.02/mm over the whole grid cylinder with two full-height r = 2 mm holes
    centred at r = 5 mm, at seeded azimuths."""
    x = np.full(scan.vol_shape, 0.02)
    for _ in range(2):
        phi = rng.uniform(0.0, 2.0 * math.pi)
        f = _disk_fraction(scan, 5.0 * math.cos(phi), 5.0 * math.sin(phi), 2.0)
        x *= (1.0 - f)[None, :, :]
    return x


def insert_azimuths(rng: np.random.Generator, n: int = 8) -> np.ndarray:
    """Seeded insert azimuths: evenly spread with a jitter, so inserts never overlap."""
    base = 2.0 * math.pi * np.arange(n) / n
    return base + rng.uniform(-0.25, 0.25, size=n) * (2.0 * math.pi / n)


def part_phantom(scan: Scan, azimuths: np.ndarray, removed: int = -1,
                 insert_mu: float = 0.10) -> np.ndarray:
    """Five equal concentric shells, mu 0.05 .. 0.01/mm inner to outer, plus r = 2 mm
    inserts (mu 0.10/mm) centred at 0.6 R over h in [-H/4, H/4]; insert ``removed``
    (if >= 0) is left out (the missing component)."""
    R = scan.radius
    radial = np.zeros(scan.n_r)
    mus = [0.05, 0.04, 0.03, 0.02, 0.01]
    for k, mu in enumerate(mus):
        radial += mu * _annulus_fraction(scan, k * R / 5.0, (k + 1) * R / 5.0)
    x = np.broadcast_to(radial, scan.vol_shape).copy()
    hf = _slab_fraction(scan, -0.25 * scan.height, 0.25 * scan.height)
    rc = 0.6 * R
    rad = 0.08 * R
    for k, phi in enumerate(azimuths):
        if k == removed:
            continue
        f = _disk_fraction(scan, rc * math.cos(phi), rc * math.sin(phi), rad)
        # the insert replaces the shell material it occupies
        x += hf[:, None, None] * f[None, :, :] * (insert_mu - radial[None, None, :])
    return x


# --------------------------------------------------------- analytic line integrals

PART_SHELL_MU = (0.05, 0.04, 0.03, 0.02, 0.01)


def _object_rays(scan: Scan, p: int):
    """Source (3,) and pixel centres (H*W, 3) of projection p in the part's frame:
    X' = R (X - T), R = (Rz(alpha) Rx(beta) Rz(gamma))^T, from the scan's stage frames."""
    f = (scan.frames if scan.frames is not None else frames_from_circular(scan))[p]
    ca, sa = math.cos(scan.alpha), math.sin(scan.alpha)
    cb, sb = math.cos(scan.beta), math.sin(scan.beta)
    cg, sg = math.cos(scan.gamma), math.sin(scan.gamma)
    rz = lambda c, s_: np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    rx = np.array([[1.0, 0.0, 0.0], [0.0, cb, -sb], [0.0, sb, cb]])
    R = (rz(ca, sa) @ rx @ rz(cg, sg)).T
    T = np.array([scan.tx, scan.ty, scan.tz])
    iu, iv = np.meshgrid(np.arange(scan.det_w), np.arange(scan.det_h))
    pts = f[3:6] + iu.reshape(-1, 1) * f[6:9] + iv.reshape(-1, 1) * f[9:12]
    return R @ (f[0:3] - T), (pts - T) @ R.T


def _cap(lo1, hi1, lo2, hi2):
    return np.maximum(lo1, lo2), np.minimum(hi1, hi2)


def _disk_span(S, d, cx, cy, rad):
    """Parameter interval [lo, hi] of the lines S + t d (t along each row of d) inside the
    infinite cylinder of radius rad about the z' axis through (cx, cy); empty: lo >= hi."""
    ox, oy = S[0] - cx, S[1] - cy
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = ox * d[:, 0] + oy * d[:, 1]
    c = ox * ox + oy * oy - rad * rad
    disc = b * b - a * c
    ok = (disc > 0.0) & (a > 0.0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    aa = np.where(ok, a, 1.0)
    lo = np.where(ok, (-b - sq) / aa, np.inf)
    hi = np.where(ok, (-b + sq) / aa, -np.inf)
    inside = (a == 0.0) & (c <= 0.0)          # parallel to the axis, inside the disk
    return np.where(inside, -np.inf, lo), np.where(inside, np.inf, hi)


def _slab_span(S, d, h_a, h_b):
    dz = d[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        t1, t2 = (h_a - S[2]) / dz, (h_b - S[2]) / dz
    par = dz == 0.0
    inside = (S[2] >= h_a) & (S[2] <= h_b)
    lo = np.where(par, -np.inf if inside else np.inf, np.minimum(t1, t2))
    hi = np.where(par, np.inf if inside else -np.inf, np.maximum(t1, t2))
    return lo, hi


def part_line_integrals(scan: Scan, azimuths: np.ndarray, removed: int = -1, insert_mu: float = 0.10):
    """Line integrals through the continuous part of part_phantom() (five equal shells over
    the full height, r = 0.08 R inserts centred at 0.6 R over h in [-H/4, H/4] replacing the
    shell material they occupy; insert ``removed`` left out) for every ray of the scan, in
    the sinogram's layout [N_p][H][W]: the measured data of the part, not a projection of
    its voxelisation.  Each shape is a clipped cylinder, so each line integral is a sum of
    chord lengths times attenuations."""
    R, H = scan.radius, scan.height
    out = np.zeros(scan.sino_shape)
    rs = [k * R / 5.0 for k in range(6)]
    for p in range(scan.n_proj):
        S, D = _object_rays(scan, p)
        d = D - S
        norm = np.linalg.norm(d, axis=1)
        s_lo, s_hi = _cap(*_slab_span(S, d, -0.5 * H, 0.5 * H), 0.0, 1.0)
        i_lo, i_hi = _cap(*_slab_span(S, d, -0.25 * H, 0.25 * H), 0.0, 1.0)
        # chord of each shell disk within the grid's height
        disk = []
        for r_ in rs:
            lo, hi = _cap(*_disk_span(S, d, 0.0, 0.0, r_), s_lo, s_hi) if r_ > 0 else (np.zeros(len(d)), np.zeros(len(d)))
            disk.append((lo, hi))
        val = np.zeros(len(d))
        for k, mu in enumerate(PART_SHELL_MU):
            val += mu * (np.clip(disk[k + 1][1] - disk[k + 1][0], 0.0, None)
                         - np.clip(disk[k][1] - disk[k][0], 0.0, None))
        for i, phi in enumerate(azimuths):
            if i == removed:
                continue
            lo, hi = _cap(*_disk_span(S, d, 0.6 * R * math.cos(phi), 0.6 * R * math.sin(phi), 0.08 * R), i_lo, i_hi)
            # split the insert's chord by the shells it crosses: each part replaces its shell
            inner = np.zeros(len(d))              # its chord inside the previous shell disk
            for k, mu in enumerate(PART_SHELL_MU):
                a_lo, a_hi = _cap(lo, hi, *disk[k + 1])
                upto = np.clip(a_hi - a_lo, 0.0, None)
                val += (insert_mu - mu) * (upto - inner)
                inner = upto
        out[p] = (val * norm).reshape(scan.det_h, scan.det_w)
    return out


def pinned_tube(scan: Scan, r_in: float = 3.0, pin_r: float = 0.8, pin_c: float = 5.5,
                pin_az: float = 0.0, pin_h=(-16.0, 16.0), mu_wall: float = 0.05,
                mu_pin: float = 0.3) -> np.ndarray:
    """A tube (wall r_in .. R) with one metal pin off the axis: radius pin_r, centred at
    radius pin_c and azimuth pin_az, over heights pin_h.  The pin gives the part an
    azimuthal phase (Sec. 2.1)."""
    wall = mu_wall * _annulus_fraction(scan, r_in, scan.radius)
    x = np.broadcast_to(wall, scan.vol_shape).copy()
    f = _disk_fraction(scan, pin_c * math.cos(pin_az), pin_c * math.sin(pin_az), pin_r)
    hf = _slab_fraction(scan, pin_h[0], pin_h[1])
    x += hf[:, None, None] * f[None, :, :] * (mu_pin - wall[None, None, :])
    return x


def roi_weights(scan: Scan, r_a: float = 12.0, r_b: float = 18.0, inside: float = 4.0,
                scale_to_radius: bool = True) -> np.ndarray:
    """Weight map on the grid: ``inside`` for voxel centres in the annulus r_a..r_b, 1
    elsewhere (radii given for R = 25 mm and scaled with the grid radius)."""
    dr = scan.radius / scan.n_r
    rc = (np.arange(scan.n_r) + 0.5) * dr
    s = scan.radius / 25.0 if scale_to_radius else 1.0
    wr = np.where((rc >= r_a * s) & (rc <= r_b * s), inside, 1.0)
    return np.broadcast_to(wr, scan.vol_shape).copy()


def random_volume(scan: Scan, rng: np.random.Generator, lo=0.0, hi=0.05) -> np.ndarray:
    return rng.uniform(lo, hi, size=scan.vol_shape)


def random_sinogram(scan: Scan, rng: np.random.Generator, lo=0.0, hi=2.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=scan.sino_shape)


def poisson_counts(p_clean: np.ndarray, i0: float, rng: np.random.Generator) -> np.ndarray:
    """Detector counts for line integrals p_clean: I ~ Poisson(I0 exp(-p))."""
    return rng.poisson(i0 * np.exp(-np.asarray(p_clean, dtype=np.float64))).astype(np.float64)
