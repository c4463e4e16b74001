"""Stored segment records (cyl_plan_set_records): SART subsets that replay each pose's
pieces instead of walking the rays, back-projecting either by gathering per voxel from
the records' transpose (form 1) or by replaying the records again into a numerator
(form 2), against the FP64 oracle and against the walking subsets.

The records round each piece's length to 20 mantissa bits (relative error <= 2^-21),
so the FP32 bound of 1e-5 relative L2 per iterate still holds with margin; the walking
and replaying forms agree to a few 1e-7.
"""
import dataclasses

import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, synth
import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11976_gb300 import build
    build.build()
    return cylct.load()


def osetup(orc, scan):
    return orc.Setup(**scan.fields())


def tilted_scan(n_proj=8, det_w=77, det_h=45):
    # 77 x 45 detector: 109 tasks of 32 pixels per view, the last one ragged (9 pixels)
    s = synth.Scan(24, 96, 20, 10.0, 20.0, 100.0, 400.0, det_w, det_h, 1.2, 1.2,
                   synth.full_circle(n_proj) + 0.3)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.4, 0.2, 1.1, 0.7, -0.4, 0.3
    return s


def test_records_report_and_release(lib):
    s = tilted_scan(n_proj=3)
    with cylct.Plan(s) as plan:
        assert plan.cyl_plan_records_full() == (False, 0, False, 0)
        base = plan.sizes()[3]
        segs = int(gu.count_segments(plan).sum())
        for form in (2, 1):
            plan.cyl_plan_set_records(form)
            ready, nbytes, gather, gbytes = plan.cyl_plan_records_full()
            assert ready and nbytes > 0 and nbytes % 128 == 0
            # about 4 bytes per piece: at least the exact piece count, padded to whole rows
            assert 4 * segs <= nbytes <= 4 * 32 * segs
            assert gather == (form == 1)
            if gather:
                # 8 bytes per piece (zero-length pieces included) and 4 per voxel and view
                assert 8 * segs + 4 * (s.n_vox + 1) * s.n_proj <= gbytes
                assert gbytes <= 8 * 2 * segs + 4 * (s.n_vox + 1) * s.n_proj
            assert plan.sizes()[3] >= base + nbytes + gbytes
        plan.cyl_plan_set_records(0)
        assert plan.cyl_plan_records_full() == (False, 0, False, 0)
        assert plan.sizes()[3] == base
        with pytest.raises(cylct.CylError):
            plan.cyl_plan_set_records(3)
        with pytest.raises(cylct.CylError):
            plan.cyl_plan_set_records(1, runs=3)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("runs", [0, 1, 4, 32])
@pytest.mark.parametrize("kw", [dict(subset_size=1, clamp_nonneg=False, weight_mode=1),
                                dict(subset_size=3, clamp_nonneg=True, weight_mode=1),
                                dict(subset_size=2, clamp_nonneg=False, weight_mode=0, lam=0.2)])
def test_records_sart_matches_oracle_and_walk(lib, orc, kw, runs, form):
    # form 1: back-projection gathered per voxel from the records' transpose; form 2:
    # replayed into a numerator with the pose's column sums
    s = tilted_scan()
    rng = np.random.default_rng(21)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    w = synth.roi_weights(s, 4.0, 7.0, 4.0, scale_to_radius=False)
    kw = dict(kw)
    lam = kw.pop("lam", 0.5)
    ref = orc.sart(osetup(orc, s), p, x0=x0, w=w, n_iter=2, lam=lam, **kw)
    with cylct.Plan(s) as plan:
        walk = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=lam, **kw)
        plan.cyl_plan_set_records(form, runs=runs)
        assert plan.cyl_plan_records_full()[0] and plan.cyl_plan_records_full()[2] == (form == 1)
        got = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=lam, **kw)
        eager = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=lam, use_graph=False, **kw)
    assert gu.rel_l2(got, ref) <= TOL_FP32
    assert gu.rel_l2(got, walk) <= 2e-6
    assert gu.rel_l2(eager, got) <= 1e-6


@pytest.mark.parametrize("form", [1, 2])
def test_records_follow_the_pose(lib, orc, form):
    # a new pose rebuilds the records (and their transpose): the result equals a fresh
    # plan's at that pose
    s = tilted_scan(n_proj=5)
    s2 = dataclasses.replace(s, alpha=1.3, beta=-0.1, gamma=0.2, tx=-0.5, ty=0.9, tz=-0.2)
    rng = np.random.default_rng(5)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    ref = orc.sart(osetup(orc, s2), p, x0=x0, n_iter=2, lam=0.5)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(form)
        gu.sart(plan, p, x0=x0, n_iter=1, lam=0.5)        # captures a sweep at the first pose
        plan.cyl_plan_set_pose((s2.alpha, s2.beta, s2.gamma, s2.tx, s2.ty, s2.tz))
        assert plan.cyl_plan_records()[0]
        got = gu.sart(plan, p, x0=x0, n_iter=2, lam=0.5)
    assert gu.rel_l2(got, ref) <= TOL_FP32


def test_records_tiny_per_iterate(lib, orc):
    # the tiny workload (consistent data, zero start, lambda 0.5): every iterate of ten
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p = orc.project(o, x_true)
    x_o = np.zeros(s.vol_shape)
    x_g = np.zeros(s.vol_shape)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(1)
        for it in range(10):
            x_o = orc.sart(o, p, x0=x_o, n_iter=1, lam=0.5)
            x_g = gu.sart(plan, p, x0=x_g, n_iter=1, lam=0.5)
            assert gu.rel_l2(x_g, x_o) <= TOL_FP32, it


@pytest.mark.parametrize("x_dt", [cylct.CYL_F16, cylct.CYL_BF16])
def test_records_16bit_storage(lib, orc, x_dt):
    # sinogram and volume stored in 16 bits; the oracle gets the same rounded inputs
    s = tilted_scan(n_proj=6)
    rng = np.random.default_rng(31)
    x0 = gu.stored(rng.uniform(0.0, 0.05, size=s.vol_shape), x_dt)
    p = gu.stored(rng.uniform(0.0, 1.0, size=s.sino_shape), x_dt)
    ref = orc.sart(osetup(orc, s), p, x0=x0, n_iter=3, lam=0.5)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(1)
        got = gu.sart(plan, p, x0=x0, n_iter=3, lam=0.5, x_dt=x_dt, sino_dt=x_dt)
    assert gu.rel_l2(got, ref) <= 2e-3


def test_records_compact_plan_walks(lib, orc):
    # a small part on a wide detector makes a compact plan, which keeps no records and
    # walks its listed rays; the result is the oracle's
    s = dataclasses.replace(synth.Scan(5, 16, 6, 6.0, 10.0, 60.0, 240.0, 28, 24, 1.6, 1.6,
                                       synth.full_circle(7) + 0.2), alpha=0.2, beta=0.1, gamma=0.3,
                            tx=14.0, ty=7.0)
    rng = np.random.default_rng(12)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(1)
        assert plan.cyl_plan_records() == (False, 0)
        got = gu.sart(plan, p, x0=x0, n_iter=2, lam=0.5)
    assert gu.rel_l2(got, orc.sart(osetup(orc, s), p, x0=x0, n_iter=2, lam=0.5)) <= TOL_FP32


@pytest.mark.parametrize("form", [1, 2])
def test_records_medium_two_sweeps_per_iterate(lib, orc, form):
    # the medium workload at full size on 8 of its 180 views (as the walking test of the
    # same name): both sweeps against the FP64 oracle fed the FP32 values the GPU holds
    full = synth.medium_scan(synth.rng_for("medium"))
    s = dataclasses.replace(full, angles=full.angles[::23][:8])
    az = synth.insert_azimuths(synth.rng_for("medium"))
    x0 = gu.stored(synth.part_phantom(s, az), cylct.CYL_F32)
    o = osetup(orc, s)
    p_clean = orc.project(o, synth.part_phantom(s, az, removed=5))
    p = gu.stored(orc.log_transform(synth.poisson_counts(p_clean, 1.0e4, np.random.default_rng(8)), 1.0e4),
                  cylct.CYL_F32)
    w = synth.roi_weights(s)
    ref1 = orc.sart(o, p, x0=x0, w=w, n_iter=1, lam=0.5)
    ref2 = orc.sart(o, p, x0=ref1, w=w, n_iter=1, lam=0.5)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(form)
        assert plan.cyl_plan_records_full()[0] and plan.cyl_plan_records_full()[2] == (form == 1)
        got1 = gu.sart(plan, p, x0=x0, w=w, n_iter=1, lam=0.5)
        got2 = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=0.5)
    assert gu.rel_l2(got1, ref1) <= TOL_FP32
    assert gu.rel_l2(got2, ref2) <= TOL_FP32
    assert gu.rel_l2(got1 - x0, ref1 - x0) <= TOL_FP32 * 5
    assert gu.rel_l2(got2 - ref1, ref2 - ref1) <= TOL_FP32 * 10


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("x_dt", [cylct.CYL_F16, cylct.CYL_BF16])
@pytest.mark.parametrize("strict", [False, True])
def test_records_tiny_16bit_storage(lib, orc, x_dt, strict, form):
    # as the walking test of 16-bit storage: the oracle gets the same 16-bit sinogram; the
    # strict mode (16-bit iterate rounded after every subset) against its looser bounds
    from test_gpu_parity import STRICT_BOUND, TOL_16
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p16 = gu.to_np(gu.to_dev(orc.project(o, x_true), x_dt))
    ref = orc.sart(o, p16, n_iter=10, lam=0.5)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(form)
        got = gu.sart(plan, p16, n_iter=10, lam=0.5, x_dt=x_dt, sino_dt=x_dt, strict_16bit=strict)
    err = gu.rel_l2(got, ref)
    assert err <= (STRICT_BOUND[x_dt] if strict else TOL_16), err


@pytest.mark.parametrize("form", [1, 2])
def test_records_column_sums_follow_subset_size(lib, orc, form):
    # the pose's column sums are kept per subset size: solves with subsets of 1, then 3,
    # then 1 view again each match the oracle
    s = tilted_scan(n_proj=7)
    rng = np.random.default_rng(44)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    o = osetup(orc, s)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_records(form)
        for ss in (1, 3, 1):
            got = gu.sart(plan, p, x0=x0, n_iter=2, lam=0.5, subset_size=ss)
            assert gu.rel_l2(got, orc.sart(o, p, x0=x0, n_iter=2, lam=0.5, subset_size=ss)) <= TOL_FP32, ss
