"""The MTF measurement (Sec. 2.3, Eq. 8) on arrays whose modulation is known in closed form."""
import math

import numpy as np
import pytest

from paper_2005_11976_gb300 import mtf


def test_modulation_of_a_cosine():
    # a + b cos(.) sampled densely: max a + b, min a - b, so Eq. 8 gives b / a
    t = np.linspace(0.0, 2.0 * math.pi, 10001)
    a, b = 0.03, 0.012
    v = a + b * np.cos(t)
    assert mtf.modulation(v.max(), v.min()) == pytest.approx(b / a, rel=1e-9)
    assert mtf.modulation(1.0, 1.0) == 0.0
    assert mtf.modulation(0.0, 0.0) == 0.0
    assert mtf.modulation(2.0, 0.0) == 1.0


@pytest.mark.parametrize("n_l", [1, 4, 16, 64])
def test_phantoms_have_the_sampled_modulation(n_l):
    # voxel-centre samples of (1 + cos(.)) / 2 with k = n / n_l samples per period sit
    # half a sample away from both extremes: modulation cos(pi n_l / n)
    shape = (4, 1024, 256)
    xt = mtf.line_phantom("theta", n_l, shape)
    np.testing.assert_allclose(mtf.mtf_theta(xt), math.cos(math.pi * n_l / 1024), rtol=1e-12)
    xr = mtf.line_phantom("r", n_l, shape)
    c, mr = mtf.mtf_r(xr, n_l)
    assert len(c) == n_l
    np.testing.assert_allclose(mr, math.cos(math.pi * n_l / 256), rtol=1e-12)
    # a theta phantom has no radial modulation and vice versa
    assert mtf.mtf_theta(xr).max() == pytest.approx(0.0, abs=1e-12)


def test_blur_lowers_modulation():
    shape = (2, 512, 64)
    x = mtf.line_phantom("theta", 32, shape)
    # a three-tap circular blur along theta: modulation falls by the filter's response
    # at the line frequency, (1 + 2 cos(2 pi 32 / 512)) / 3
    xb = (x + np.roll(x, 1, axis=1) + np.roll(x, -1, axis=1)) / 3.0
    resp = (1.0 + 2.0 * math.cos(2.0 * math.pi * 32 / 512)) / 3.0
    np.testing.assert_allclose(mtf.mtf_theta(xb), resp * math.cos(math.pi * 32 / 512), rtol=1e-12)


def test_central_slice_and_frequencies():
    x = np.arange(4 * 3 * 2, dtype=float).reshape(4, 3, 2)
    np.testing.assert_allclose(mtf.central_slice(x), 0.5 * (x[1] + x[2]))
    np.testing.assert_allclose(mtf.central_slice(x[:3]), x[1])
    assert mtf.frequencies(256) == [1, 2, 4, 8, 16, 32, 64, 128]
    s = mtf.summarise(np.array([1.0, 0.5, 0.25, 0.1]), np.array([0.1, 0.3, 0.6, 0.9]))
    assert s["0.00-0.25"] == 1.0 and s["0.75-1.00"] == 0.1
