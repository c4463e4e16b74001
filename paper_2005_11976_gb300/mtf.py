"""Directional MTF of the cylindrical reconstruction on line phantoms (Sec. 2.3, Eq. 8).

Azimuthal lines (a Siemens-star pattern in every slice) and radial lines (concentric
circles) are modelled by a cosine of the line frequency n_l (the number of lines over the
full circle, or over the radius), sampled on a fine simulation grid, projected, and
reconstructed by SART on the reconstruction grid.  In the central slice (away from
cone-beam artefacts) the modulation of Eq. 8,

    m = (mu_max - mu_min) / (mu_max + mu_min),

is measured at every radius for the azimuthal MTF (MTF_theta: extremes over theta in one
radial bin), and over windows of one line period in r for the radial MTF (MTF_r: extremes
over the window, windows stepped by their width).

This module holds the phantoms and the measurement (host side, numpy); the projections
and reconstructions go through the library (cylct.Plan).
"""
from __future__ import annotations

import math

import numpy as np


def line_phantom(kind: str, n_l: int, shape, mu0: float = 0.02) -> np.ndarray:
    """Cosine line phantom on an (N_h, N_theta, N_r) grid, sampled at voxel centres:
    kind 'theta': mu0 (1 + cos(n_l theta)) / 2 (n_l lines around the circle);
    kind 'r':     mu0 (1 + cos(2 pi n_l r / R)) / 2 (n_l lines over the radius)."""
    n_h, n_t, n_r = shape
    if kind == "theta":
        th = 2.0 * math.pi * (np.arange(n_t) + 0.5) / n_t
        prof = 0.5 * mu0 * (1.0 + np.cos(n_l * th))
        return np.broadcast_to(prof[None, :, None], shape).copy()
    if kind == "r":
        rr = (np.arange(n_r) + 0.5) / n_r
        prof = 0.5 * mu0 * (1.0 + np.cos(2.0 * math.pi * n_l * rr))
        return np.broadcast_to(prof[None, None, :], shape).copy()
    raise ValueError("kind must be 'theta' or 'r'")


def modulation(mu_max, mu_min):
    """Eq. 8 (0 where mu_max + mu_min is not positive)."""
    mu_max = np.asarray(mu_max, dtype=np.float64)
    mu_min = np.asarray(mu_min, dtype=np.float64)
    den = mu_max + mu_min
    return np.where(den > 0.0, (mu_max - mu_min) / np.where(den > 0.0, den, 1.0), 0.0)


def central_slice(x: np.ndarray) -> np.ndarray:
    """The slice at the grid's mid height (the mean of the two middle slabs for an even
    N_h), shape (N_theta, N_r)."""
    n_h = x.shape[0]
    if n_h % 2:
        return x[n_h // 2]
    return 0.5 * (x[n_h // 2 - 1] + x[n_h // 2])


def mtf_theta(x: np.ndarray) -> np.ndarray:
    """Azimuthal MTF at every radial bin of the central slice."""
    s = central_slice(x)
    return modulation(s.max(axis=0), s.min(axis=0))


def mtf_r(x: np.ndarray, n_l: int):
    """Radial MTF over windows of one line period (N_r / n_l bins, at least 1), stepped by
    their width: (window centre radii as fractions of R, modulation per window)."""
    s = central_slice(x)
    n_r = s.shape[1]
    width = max(1, int(round(n_r / n_l)))
    centres, m = [], []
    for a in range(0, n_r - width + 1, width):
        win = s[:, a:a + width]
        centres.append((a + 0.5 * width) / n_r)
        m.append(float(modulation(win.max(), win.min())))
    return np.array(centres), np.array(m)


def frequencies(n_r: int):
    """Line frequencies 1, 2, 4, ... up to N_r / 2 (the paper doubles up to 128 = S_r / 2)."""
    out, f = [], 1
    while f <= n_r // 2:
        out.append(f)
        f *= 2
    return out


def summarise(values: np.ndarray, radii: np.ndarray, bands=((0.0, 0.25), (0.25, 0.5), (0.5, 0.75), (0.75, 1.0))):
    """Mean of a radially resolved MTF over radial bands (fractions of R)."""
    out = {}
    for lo, hi in bands:
        sel = (radii >= lo) & (radii < hi)
        out[f"{lo:.2f}-{hi:.2f}"] = float(values[sel].mean()) if sel.any() else None
    return out
