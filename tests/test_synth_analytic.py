"""The analytic data of the part phantom (line integrals of the continuous shapes) against
the oracle's projection of its voxelisation: exact for the shells, which the grid resolves
exactly, and converging with the grid for the inserts, which it samples."""
import dataclasses

import numpy as np

from paper_2005_11976_gb300 import synth


def scan(grid, det=16, n_proj=3):
    s = synth.medium_scan(n_proj=n_proj, grid=grid, det=det, pitch=204.8 / det,
                          pose=(0.4, 0.02, 1.1, 0.8, -0.5, 0.3))
    return s


def test_shells_equal_the_projection_of_their_exact_voxelisation(orc):
    # N_r a multiple of 5: every shell boundary is a grid shell, so part_phantom's shells are
    # exact (area fractions 0 or 1) and A x is their exact line integral
    s = scan((6, 8, 20))
    x = synth.part_phantom(s, np.array([]))
    ref = orc.project(orc.Setup(**s.fields()), x)
    got = synth.part_line_integrals(s, np.array([]))
    assert np.abs(got).max() > 0.5
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)


def test_inserts_converge_to_the_projection_of_a_fine_voxelisation(orc):
    az = synth.insert_azimuths(np.random.default_rng(3))
    errs = []
    for grid in ((8, 64, 20), (16, 256, 80)):
        s = scan(grid, det=24, n_proj=2)
        got = synth.part_line_integrals(s, az, removed=2)
        ref = orc.project(orc.Setup(**s.fields()), synth.part_phantom(s, az, removed=2))
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # boundary voxels are sampled: first order in the voxel size (2.1e-2 -> 4.1e-3 here)
    assert errs[1] < 0.3 * errs[0] and errs[1] < 6e-3, errs
    # the removed insert changes exactly the rays that cross its cylinder
    s = scan((8, 64, 20), det=24, n_proj=2)
    diff = synth.part_line_integrals(s, az) - synth.part_line_integrals(s, az, removed=2)
    assert (diff > 0).any() and (diff >= 0).all()
