import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.load()
    return oracle


@pytest.fixture(scope="session")
def golden_table1():
    """Scan built from the paper's Table 1 geometry and the Sec. 3.3 grid."""
    import json
    from paper_2005_11976_gb300 import synth
    with open(os.path.join(ROOT, "tests", "golden", "table1_geometry.json")) as f:
        g = json.load(f)
    return synth.Scan(g["grid_n_h"], g["grid_n_theta"], g["grid_n_r"], g["sample_radius_mm"],
                      g["sample_height_mm"], g["sod_mm"], g["sdd_mm"], g["det_w"], g["det_h"],
                      g["pixel_mm"], g["pixel_mm"], synth.limited_arc(g["n_proj"], g["last_angle_deg"]))
