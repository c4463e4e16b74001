"""cyl_project_noalloc: the allocation-free forward projection gives what cyl_project gives.

Some callers cannot allocate device memory while they run (a framework that owns the
device memory through its own allocator, an in-line loop that cannot stall on an
allocation); cyl_project_noalloc keeps its accumulator in a fixed static device array
instead.  This file is collected last, so a stop at its first failure has run every
other test already; it also passes on its own in a fresh process.
"""
import ctypes
import dataclasses

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


def test_noalloc_compact_plan_twice(lib):
    """A part that sits mostly off the detector gives a compact plan, whose projector writes
    only the rays that meet the grid: the shared array must be cleared between calls, or
    the second, smaller call would return the first call's sums on the other rays."""
    import torch
    base = synth.Scan(5, 16, 6, 6.0, 10.0, 60.0, 240.0, 28, 24, 1.6, 1.6, synth.full_circle(7) + 0.2)
    dense = dataclasses.replace(base, alpha=0.2, beta=0.1, gamma=0.3)
    off = dataclasses.replace(base, alpha=0.2, beta=0.1, gamma=0.3, tx=14.0, ty=7.0)
    with cylct.Plan(dense) as pd:
        dense_bytes = pd.sizes()[3]
    rng = np.random.default_rng(23)
    with cylct.Plan(off) as plan:
        assert plan.sizes()[3] < dense_bytes          # the plan is compact
        for call, (p0, np_) in enumerate([(0, 7), (2, 3), (4, 2)]):
            x = torch.from_numpy(rng.uniform(0.0, 0.05, size=off.vol_shape).astype(np.float32)).cuda()
            ref = torch.empty((np_, off.det_h, off.det_w), device="cuda")
            got = torch.full_like(ref, -1.0)
            plan.cyl_project(x, cylct.CYL_F32, p0, np_, ref, cylct.CYL_F32)
            rc = lib.cyl_project_noalloc(plan.h, x.data_ptr(), cylct.CYL_F32, p0, np_,
                                         got.data_ptr(), cylct.CYL_F32, None)
            assert rc == cylct.CYL_OK, lib.cyl_last_error_detail()
            torch.cuda.synchronize()
            assert (ref == 0).any()                        # rays that miss the grid
            if call == 0:
                assert (ref > 0).any()                     # and rays that meet it
            assert torch.equal(got == 0, ref == 0), call
            if (ref > 0).any():
                assert rel(got, ref) <= TOL_FP32, call
            else:       # views that miss the part: nothing of an earlier call may be left
                assert torch.equal(got, ref), call


def test_noalloc_first_call_allocates_nothing(lib):
    """On a fresh plan, before any cyl_project: a 16-bit output (for which cyl_project
    would allocate FP32 scratch) leaves the plan's device footprint and the device's free
    memory as they were."""
    import torch
    s = scan()
    x = torch.from_numpy(np.random.default_rng(5).uniform(0.0, 0.05, size=s.vol_shape)
                         .astype(np.float32)).cuda()
    got16 = torch.empty((7, s.det_h, s.det_w), dtype=torch.bfloat16, device="cuda")
    # the driver loads a kernel's code on its first launch: load them with another plan
    with cylct.Plan(s) as warm:
        warm.cyl_project_noalloc(x, cylct.CYL_F32, 0, 7, got16, cylct.CYL_BF16)
        torch.cuda.synchronize()
    with cylct.Plan(s) as plan:
        torch.cuda.synchronize()
        before_plan = plan.sizes()[3]
        before_free = torch.cuda.mem_get_info()[0]
        plan.cyl_project_noalloc(x, cylct.CYL_F32, 0, 7, got16, cylct.CYL_BF16)
        torch.cuda.synchronize()
        assert plan.sizes()[3] == before_plan
        assert torch.cuda.mem_get_info()[0] == before_free
        ref16 = torch.empty_like(got16)
        plan.cyl_project(x, cylct.CYL_F32, 0, 7, ref16, cylct.CYL_BF16)
        torch.cuda.synchronize()
        assert plan.sizes()[3] > before_plan          # cyl_project took its scratch
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
