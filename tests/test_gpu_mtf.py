"""The MTF experiment's pipeline (line phantom, projection, SART, Eq. 8) against the oracle."""
import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, mtf, synth
import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11976_gb300 import build
    build.build()
    return cylct.load()


def osetup(orc, s):
    return orc.Setup(**s.fields())


@pytest.mark.parametrize("kind,n_l", [("theta", 4), ("theta", 8), ("r", 2), ("r", 4)])
def test_line_phantom_mtf_matches_oracle(lib, orc, kind, n_l):
    # a fine simulation grid, a coarser reconstruction grid: the data come from the
    # oracle's projection of the fine phantom, both sides reconstruct them, and the
    # measured modulation agrees
    fine = synth.Scan(4, 96, 16, 5.0, 2.0, 60.0, 200.0, 48, 16, 0.5, 0.5, synth.full_circle(24))
    rec = synth.Scan(4, 32, 16, 5.0, 2.0, 60.0, 200.0, 48, 16, 0.5, 0.5, synth.full_circle(24))
    p = orc.project(osetup(orc, fine), mtf.line_phantom(kind, n_l, fine.vol_shape))
    ref = orc.sart(osetup(orc, rec), p, n_iter=3, lam=0.5, clamp_nonneg=True)
    with cylct.Plan(rec) as plan:
        got = gu.sart(plan, p, n_iter=3, lam=0.5, clamp_nonneg=True)
    assert gu.rel_l2(got, ref) <= 1e-5
    if kind == "theta":
        np.testing.assert_allclose(mtf.mtf_theta(got), mtf.mtf_theta(ref), atol=1e-4)
    else:
        np.testing.assert_allclose(mtf.mtf_r(got, n_l)[1], mtf.mtf_r(ref, n_l)[1], atol=1e-4)
