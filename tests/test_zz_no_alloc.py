"""cyl_project_noalloc: the allocation-free forward projection gives what cyl_project gives.

Some callers cannot allocate device memory while they run (a framework that owns the
device memory through its own allocator, an in-line loop that cannot stall on an
allocation); cyl_project_noalloc keeps its accumulator in a fixed static device array
instead.  This file is collected last, so a stop at its first failure has run every
other test already; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5   # the FP32 projector tolerance used by the parity tests


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11976_gb300 import build
    build.build()
    return cylct.load()


def scan():
    s = synth.Scan(24, 96, 20, 10.0, 20.0, 100.0, 400.0, 77, 45, 1.2, 1.2,
                   synth.full_circle(7) + 0.3)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.4, 0.2, 1.1, 0.7, -0.4, 0.3
    return s


def rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_cyl_project_twice(lib):
    import torch
    s = scan()
    rng = np.random.default_rng(17)
    with cylct.Plan(s) as plan:
        for call, (p0, np_) in enumerate([(0, 7), (2, 3)]):      # two calls in a row
            x = torch.from_numpy(rng.uniform(0.0, 0.05, size=s.vol_shape).astype(np.float32)).cuda()
            ref = torch.empty((np_, s.det_h, s.det_w), device="cuda")
            got = torch.full_like(ref, -1.0)
            plan.cyl_project(x, cylct.CYL_F32, p0, np_, ref, cylct.CYL_F32)
            rc = lib.cyl_project_noalloc(plan.h, x.data_ptr(), cylct.CYL_F32, p0, np_,
                                         got.data_ptr(), cylct.CYL_F32, None)
            assert rc == cylct.CYL_OK, lib.cyl_last_error_detail()
            torch.cuda.synchronize()
            assert rel(got, ref) <= TOL_FP32, call
        # 16-bit output through the same array
        ref16 = torch.empty((7, s.det_h, s.det_w), dtype=torch.float16, device="cuda")
        got16 = torch.empty_like(ref16)
        plan.cyl_project(x, cylct.CYL_F32, 0, 7, ref16, cylct.CYL_F16)
        plan.cyl_project_noalloc(x, cylct.CYL_F32, 0, 7, got16, cylct.CYL_F16)
        torch.cuda.synchronize()
        assert rel(got16, ref16) <= 1e-3


def test_noalloc_rejects_oversize(lib):
    import torch
    s = synth.Scan(4, 16, 4, 10.0, 20.0, 100.0, 400.0, 1024, 1024, 0.2, 0.2, synth.full_circle(5))
    with cylct.Plan(s) as plan:
        x = torch.zeros(s.vol_shape, device="cuda")
        out = torch.zeros(1, device="cuda")
        rc = lib.cyl_project_noalloc(plan.h, x.data_ptr(), cylct.CYL_F32, 0, 5, out.data_ptr(),
                                     cylct.CYL_F32, None)
        assert rc == cylct.CYL_EINVAL
        assert b"allocation-free" in lib.cyl_last_error_detail()
