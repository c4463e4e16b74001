"""GPU path vs the FP64 oracle, element by element, on seeded inputs.

Tolerances: the FP32 path must match the oracle to <= 1e-5 relative L2 per projection
and per SART iterate; the 16-bit storage path to <= 2e-3 relative L2 of the
reconstruction.  Row sums are FP64 chords rounded to FP32 (<= 1e-6 relative).
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, synth
import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_16 = 2e-3


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


def tilted_scan(n_h=24, n_t=96, n_r=20, n_proj=7, det_w=77, det_h=45):
    # ragged detector (77 x 45 is no multiple of the 32 x 4 ray tile), tilted pose
    s = synth.Scan(n_h, n_t, n_r, 10.0, 20.0, 100.0, 400.0, det_w, det_h, 1.2, 1.2,
                   synth.full_circle(n_proj) + 0.3)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.4, 0.2, 1.1, 0.7, -0.4, 0.3
    return s


def per_projection_rel(a, b):
    return max(gu.rel_l2(a[k], b[k]) for k in range(a.shape[0]))


# ------------------------------------------------------------- projector

@pytest.mark.parametrize("case", ["tiny", "tilted", "ntheta1", "ntheta2", "ntheta3"])
def test_project_matches_oracle(lib, orc, case):
    rng = np.random.default_rng(101)
    if case == "tiny":
        s = synth.tiny_scan()
        x = synth.tiny_phantom(s, synth.rng_for("tiny"))
    else:
        s = tilted_scan()
        if case.startswith("ntheta"):
            s = dataclasses.replace(s, n_theta=int(case[-1]))
        x = rng.uniform(0.0, 0.05, size=s.vol_shape)
    ref = orc.project(osetup(orc, s), x)
    with cylct.Plan(s) as plan:
        got = gu.project(plan, x)
    assert per_projection_rel(got, ref) <= TOL_FP32


def test_set_pose_equals_fresh_plan(lib):
    s = tilted_scan(n_proj=3)
    s2 = dataclasses.replace(s, alpha=1.3, beta=-0.1, gamma=0.2, tx=-0.5, ty=0.9, tz=-0.2)
    x = np.random.default_rng(8).uniform(0, 0.05, size=s.vol_shape)
    with cylct.Plan(s2) as fresh:
        ref = gu.project(fresh, x)
    with cylct.Plan(s) as plan:
        gu.project(plan, x)
        plan.cyl_plan_set_pose((s2.alpha, s2.beta, s2.gamma, s2.tx, s2.ty, s2.tz))
        got = gu.project(plan, x)
    # same rays and tiles; only the order of the per-tile atomic sums may differ
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7)


def test_row_sums_match_oracle(lib, orc):
    s = tilted_scan()
    ref = orc.row_sums(osetup(orc, s))
    with cylct.Plan(s) as plan:
        got = gu.row_sums(plan)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6)


def test_backproject_and_colsums_match_oracle(lib, orc):
    s = tilted_scan()
    rng = np.random.default_rng(7)
    y = rng.uniform(0.0, 1.0, size=s.sino_shape)
    o = osetup(orc, s)
    ref = orc.backproject(o, y)
    ref1 = orc.backproject(o, np.ones(s.sino_shape))
    with cylct.Plan(s) as plan:
        got, cs = gu.backproject(plan, y, colsum=True)
        # sub-range of projections
        got_sub = gu.backproject(plan, y[2:5], p0=2, np_=3)
        # signed data: A^T y sums terms of both signs, so the error is measured against
        # the size of the terms, A^T |y|
        ys = rng.uniform(-1.0, 1.0, size=s.sino_shape)
        got_s = gu.backproject(plan, ys)
    assert gu.rel_l2(got, ref) <= TOL_FP32
    assert gu.rel_l2(cs, ref1) <= TOL_FP32
    assert gu.rel_l2(got_sub, orc.backproject(o, y[2:5], 2, 3)) <= TOL_FP32
    ref_s = orc.backproject(o, ys)
    scale = np.linalg.norm(orc.backproject(o, np.abs(ys)))
    assert np.linalg.norm(got_s - ref_s) / scale <= TOL_FP32


def test_adjoint_identity_on_gpu(lib):
    s = tilted_scan()
    rng = np.random.default_rng(3)
    x = rng.standard_normal(s.vol_shape)
    y = rng.standard_normal(s.sino_shape)
    with cylct.Plan(s) as plan:
        ax = gu.project(plan, x)
        aty = gu.backproject(plan, y)
    lhs = float(np.sum(ax * y))
    rhs = float(np.sum(x * aty))
    scale = float(np.sqrt(np.sum(ax * ax) * np.sum(y * y)))
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_segment_counts_match_oracle(lib, orc):
    s = tilted_scan()
    ref = orc.row_nnz(osetup(orc, s)).reshape(s.n_proj, -1).sum(axis=1)
    with cylct.Plan(s) as plan:
        got = gu.count_segments(plan)
    # coincident crossings can leave a sliver piece at a tile boundary: <= 2e-3 extra
    assert np.all(np.abs(got - ref) <= 4 + 2e-3 * ref), (got, ref)


def test_axis_parallel_ray(lib, orc):
    # alpha = beta = pi/2 turns the part's axis onto the beam: the central ray runs along
    # the z' axis (no shell or wedge crossings); use a theta-independent volume
    s = synth.Scan(8, 16, 6, 5.0, 10.0, 50.0, 150.0, 9, 9, 0.7, 0.7, np.array([0.0, 0.2]))
    s.alpha, s.beta = math.pi / 2, math.pi / 2
    radial = np.linspace(0.01, 0.06, s.n_r)
    slabs = np.linspace(1.0, 2.0, s.n_h)
    x = slabs[:, None, None] * radial[None, None, :] * np.ones(s.vol_shape)
    ref = orc.project(osetup(orc, s), x)
    with cylct.Plan(s) as plan:
        got = gu.project(plan, x)
    assert per_projection_rel(got, ref) <= TOL_FP32
    # the central ray of view 0 sees the whole height in shell 0
    assert math.isclose(got[0, 4, 4], float(np.sum(x[:, 0, 0]) * s.height / s.n_h), rel_tol=1e-5)


def test_rays_that_miss_give_zero(lib):
    s = dataclasses.replace(tilted_scan(n_proj=2), off_u=500.0)
    with cylct.Plan(s) as plan:
        got = gu.project(plan, np.ones(s.vol_shape))
        L = gu.row_sums(plan)
        res = gu.sart(plan, np.ones(s.sino_shape), n_iter=1, x0=np.full(s.vol_shape, 0.5))
    assert np.all(got == 0) and np.all(L == 0)
    np.testing.assert_array_equal(res, np.full(s.vol_shape, 0.5, dtype=np.float32))


def test_small_part_on_a_wide_detector(lib, orc):
    """A part that covers a small fraction of the detector (the in-line set-up of
    Table 1): the projector and back-projector walk only the rays of positive chord; the
    projection is zero elsewhere and every result equals the oracle's."""
    import torch
    s = synth.Scan(6, 16, 5, 3.0, 6.0, 100.0, 400.0, 41, 37, 1.6, 1.6, synth.full_circle(5) + 0.2)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = 0.3, 0.1, 0.5, 1.5, -2.0, 0.4
    rng = np.random.default_rng(12)
    x = rng.uniform(0.0, 0.05, size=s.vol_shape)
    o = osetup(orc, s)
    want = orc.project(o, x)
    L = orc.row_sums(o)
    assert 0.02 < (L > 0).mean() < 0.3                    # most rays miss the grid
    with cylct.Plan(s) as plan:
        got = gu.project(plan, x)
        out = torch.full(s.sino_shape, 7.0, device="cuda")
        plan.cyl_project_noalloc(gu.to_dev(x), cylct.CYL_F32, 0, s.n_proj, out, cylct.CYL_F32)
        got_na = gu.to_np(out)
        y = rng.uniform(0.0, 1.0, size=s.sino_shape)
        bp = gu.backproject(plan, y)
        p = want + 0.01 * rng.standard_normal(want.shape)
        xs = gu.sart(plan, p, x0=x, n_iter=2, lam=0.5)
        L_gpu = gu.row_sums(plan)
        segs = gu.count_segments(plan)
    np.testing.assert_allclose(L_gpu, L, rtol=1e-6, atol=1e-6)
    ref = orc.row_nnz(o).reshape(s.n_proj, -1).sum(axis=1)
    assert np.all(np.abs(segs - ref) <= 4 + 2e-3 * ref), (segs, ref)
    assert np.all(got[L == 0] == 0) and np.all(got_na[L == 0] == 0)
    assert per_projection_rel(got, want) <= TOL_FP32 and per_projection_rel(got_na, want) <= TOL_FP32
    assert gu.rel_l2(bp, orc.backproject(o, y)) <= TOL_FP32
    assert gu.rel_l2(xs, orc.sart(o, p, x0=x, n_iter=2, lam=0.5)) <= TOL_FP32


def test_sart_update_fallbacks(lib, orc):
    """The FP32 update takes 16-byte vectors when the voxel count is a multiple of 4 and
    the arrays are aligned; an odd grid and a misaligned output take the scalar path.
    Both give the oracle's iterate."""
    import torch
    s = synth.Scan(5, 9, 7, 6.0, 8.0, 60.0, 200.0, 23, 19, 1.3, 1.3, synth.full_circle(4) + 0.1)
    s.alpha, s.beta, s.tx = 0.3, 0.15, 0.4
    assert (s.n_h * s.n_theta * s.n_r) % 4 != 0
    rng = np.random.default_rng(31)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    want = orc.sart(osetup(orc, s), p, x0=x0, n_iter=2, lam=0.5)
    with cylct.Plan(s) as plan:
        assert gu.rel_l2(gu.sart(plan, p, x0=x0, n_iter=2, lam=0.5), want) <= TOL_FP32
    s2 = dataclasses.replace(s, n_r=8)                      # 360 voxels: the vector path ...
    want2 = orc.sart(osetup(orc, s2), p, x0=np.zeros(s2.vol_shape), n_iter=2, lam=0.5)
    with cylct.Plan(s2) as plan:
        buf = torch.zeros(s2.n_vox + 1, device="cuda")
        out = buf[1:].view(s2.vol_shape)                     # ... unless the output is misaligned
        plan.cyl_sart_solve(gu.to_dev(p), cylct.CYL_F32, None, None,
                            cylct.sart_params(n_iter=2, lam=0.5), out, cylct.CYL_F32)
        assert gu.rel_l2(gu.to_np(out), want2) <= TOL_FP32
        assert gu.rel_l2(gu.sart(plan, p, n_iter=2, lam=0.5), want2) <= TOL_FP32


def test_dense_and_compact_plans_through_all_poses(lib, orc):
    """A plan is dense (records for every ray) or compact (each pose lists the rays that
    meet the grid and keeps records for those only), decided by its first pose.  Both
    kinds re-posed through poses where the grid fills the detector and where the part sits
    mostly off it give the oracle's projections and SART iterates (captured sweeps
    included), and the compact plan holds far less."""
    s = synth.Scan(5, 16, 6, 6.0, 10.0, 60.0, 240.0, 28, 24, 1.6, 1.6, synth.full_circle(3) + 0.2)
    # the third pose spins the second about the part's axis (a compact plan keeps its list)
    poses = [(0.2, 0.1, 0.3, 0.0, 0.0, 0.0), (0.2, 0.1, 0.3, 14.0, 7.0, 0.0), (0.2, 0.1, 1.7, 14.0, 7.0, 0.0),
             (0.2, 0.1, 0.3, 0.5, -0.5, 0.0), (0.2, 0.1, 0.3, -14.0, 7.0, 1.0)]
    rng = np.random.default_rng(41)
    x = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)

    def posed(pose):
        return dataclasses.replace(s, alpha=pose[0], beta=pose[1], gamma=pose[2], tx=pose[3], ty=pose[4], tz=pose[5])

    sizes = []
    for first in (0, 1):                         # dense first pose, then mostly-off first pose
        with cylct.Plan(posed(poses[first])) as plan:
            sizes.append(plan.sizes()[3])
            for pose in poses[first:] + poses[:first]:
                plan.cyl_plan_set_pose(pose)
                o = osetup(orc, posed(pose))
                want = orc.project(o, x)
                got = gu.project(plan, x)
                assert np.all(got[want == 0] == 0)
                assert np.abs(got - want).max() <= TOL_FP32 * max(np.abs(want).max(), 1.0)
                np.testing.assert_allclose(gu.row_sums(plan), orc.row_sums(o), rtol=1e-6, atol=1e-6)
                xs = gu.sart(plan, p, x0=x, n_iter=2, lam=0.5)
                assert gu.rel_l2(xs, orc.sart(o, p, x0=x, n_iter=2, lam=0.5)) <= TOL_FP32
    assert sizes[1] < sizes[0]


def test_empty_projection_range(lib):
    import torch
    s = tilted_scan(n_proj=2)
    with cylct.Plan(s) as plan:
        out = torch.full((1,), 7.0, device="cuda")
        plan.cyl_project(torch.zeros(s.vol_shape, device="cuda"), cylct.CYL_F32, 1, 0, out,
                         cylct.CYL_F32)
        torch.cuda.synchronize()
        assert out.item() == 7.0
        with pytest.raises(cylct.CylError):
            plan.cyl_project(torch.zeros(s.vol_shape, device="cuda"), cylct.CYL_F32, 1, 2, out,
                             cylct.CYL_F32)


@pytest.mark.parametrize("vol_dt", [cylct.CYL_F16, cylct.CYL_BF16])
def test_project_16bit_storage(lib, orc, vol_dt):
    s = tilted_scan()
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 0.05, size=s.vol_shape)
    import torch
    xr = gu.to_np(gu.to_dev(x, vol_dt))         # the stored 16-bit volume
    ref = orc.project(osetup(orc, s), xr)
    with cylct.Plan(s) as plan:
        got = gu.project(plan, x, vol_dt=vol_dt, out_dt=cylct.CYL_F32)
    assert per_projection_rel(got, ref) <= TOL_FP32


def test_log_transform(lib, orc):
    import torch
    rng = np.random.default_rng(9)
    counts = rng.poisson(1e4 * np.exp(-rng.uniform(0, 4, size=1000))).astype(np.float64)
    counts[:5] = 0.0
    ref = orc.log_transform(counts, 1e4)
    c = gu.to_dev(counts)
    out = torch.empty_like(c)
    cylct.cyl_log_transform(c, cylct.CYL_F32, 1e4, out, cylct.CYL_F32, counts.size)
    np.testing.assert_allclose(gu.to_np(out), ref, rtol=0, atol=2e-6)


# ------------------------------------------------------------------ SART

def test_sart_tiny_per_iterate(lib, orc):
    # tiny workload: consistent data, zero start, 10 iterations, lambda 0.5
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p = orc.project(o, x_true)
    x_o = np.zeros(s.vol_shape)
    x_g = np.zeros(s.vol_shape)
    with cylct.Plan(s) as plan:
        for it in range(10):
            x_o = orc.sart(o, p, x0=x_o, n_iter=1, lam=0.5)
            x_g = gu.sart(plan, p, x0=x_g, n_iter=1, lam=0.5)
            assert gu.rel_l2(x_g, x_o) <= TOL_FP32, it
        # ten sweeps in one call (one captured graph replayed) give the same iterate
        x_10 = gu.sart(plan, p, n_iter=10, lam=0.5)
    assert gu.rel_l2(x_10, x_o) <= TOL_FP32


def test_sart_weighted_warm_started_subsets(lib, orc):
    s = tilted_scan(n_proj=8)
    rng = np.random.default_rng(21)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    w = synth.roi_weights(s, 4.0, 7.0, 4.0, scale_to_radius=False)
    o = osetup(orc, s)
    for kw in (dict(subset_size=1, clamp_nonneg=False, weight_mode=1),
               dict(subset_size=3, clamp_nonneg=True, weight_mode=1),
               dict(subset_size=2, clamp_nonneg=False, weight_mode=0, lam=0.2)):
        lam = kw.pop("lam", 0.5)
        ref = orc.sart(o, p, x0=x0, w=w, n_iter=2, lam=lam, **kw)
        with cylct.Plan(s) as plan:
            got = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=lam, **kw)
            eager = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=lam, use_graph=False, **kw)
        assert gu.rel_l2(got, ref) <= TOL_FP32, kw
        assert gu.rel_l2(eager, got) <= 1e-6


@pytest.mark.parametrize("w_dt", [cylct.CYL_F32, cylct.CYL_F16, cylct.CYL_BF16, cylct.CYL_U8])
def test_sart_weight_map_dtypes(lib, orc, w_dt):
    """Weight maps of every element type (Sec. 2.2 weighted back-projection): the oracle
    gets the values as stored.  A U8 class map holds the weights 1 and 4 exactly; the
    16-bit maps hold non-integer weights rounded on the host.  Each through the vector
    update (voxel count a multiple of 4, aligned arrays), the scalar update (the weight
    map one element off its alignment) and the host-staged form."""
    import torch
    s = tilted_scan(n_proj=6)
    assert s.n_vox % 4 == 0
    rng = np.random.default_rng(23)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape)
    if w_dt == cylct.CYL_U8:
        w = synth.roi_weights(s, 4.0, 7.0, 4.0, scale_to_radius=False)
    else:
        w = gu.stored(rng.uniform(0.5, 3.0, size=s.vol_shape), w_dt)
    o = osetup(orc, s)
    first = None
    for mode in (1, 0):
        lam = 0.5 if mode else 0.15
        ref = orc.sart(o, p, x0=x0, w=w, n_iter=2, lam=lam, weight_mode=mode)
        with cylct.Plan(s) as plan:
            vec = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=lam, weight_mode=mode, w_dt=w_dt)
            wd = gu.to_dev(w, w_dt).ravel()
            buf = torch.zeros(s.n_vox + 1, dtype=wd.dtype, device="cuda")
            buf[1:] = wd
            out = torch.empty(s.vol_shape, device="cuda")
            prm = cylct.sart_params(n_iter=2, lam=lam, weight_mode=mode, weight_dtype=w_dt)
            plan.cyl_sart_solve(gu.to_dev(p), cylct.CYL_F32, gu.to_dev(x0), buf[1:], prm, out, cylct.CYL_F32)
            scalar = gu.to_np(out)
            host = np.zeros(s.vol_shape, dtype=np.float32)
            plan.cyl_sart_solve(np.ascontiguousarray(p, dtype=np.float32), cylct.CYL_F32,
                                np.ascontiguousarray(x0, dtype=np.float32), wd.view(torch.uint8).cpu().numpy(),
                                prm, host, cylct.CYL_F32)
        for got in (vec, scalar, host):
            assert gu.rel_l2(got, ref) <= TOL_FP32, (mode, w_dt)
        first = vec if first is None else first
    # an FP32 map of the same values gives the same iterate (up to the order of the
    # back-projector's atomic sums)
    with cylct.Plan(s) as plan:
        f32 = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=0.5)
    assert gu.rel_l2(first, f32) <= 1e-6


def test_sart_host_buffers_equal_device_buffers(lib):
    import torch
    s = tilted_scan(n_proj=4)
    rng = np.random.default_rng(2)
    p = rng.uniform(0.0, 1.0, size=s.sino_shape).astype(np.float32)
    x0 = rng.uniform(0.0, 0.05, size=s.vol_shape).astype(np.float32)
    with cylct.Plan(s) as plan:
        dev = gu.sart(plan, p, x0=x0, n_iter=2)
        out = np.zeros(s.vol_shape, dtype=np.float32)
        plan.cyl_sart_solve(p, cylct.CYL_F32, x0, None, cylct.sart_params(n_iter=2), out,
                            cylct.CYL_F32)
        pinned = torch.from_numpy(p).pin_memory()
        out2 = torch.zeros(s.vol_shape).pin_memory()
        plan.cyl_sart_solve(pinned, cylct.CYL_F32, x0, None, cylct.sart_params(n_iter=2), out2,
                            cylct.CYL_F32)
    assert gu.rel_l2(out, dev) <= 1e-6
    assert gu.rel_l2(out2.numpy(), dev) <= 1e-6


# Strict mode rounds the iterate to 16 bits after every subset, so increments below half
# an ulp are lost (BF16 keeps 8 significant bits): it is reported against looser bounds.
STRICT_BOUND = {cylct.CYL_F16: 5e-3, cylct.CYL_BF16: 3e-2}


@pytest.mark.parametrize("x_dt", [cylct.CYL_F16, cylct.CYL_BF16])
@pytest.mark.parametrize("strict", [False, True])
def test_sart_16bit_storage(lib, orc, x_dt, strict):
    # the oracle gets the same 16-bit sinogram as the GPU, so the error measures the
    # 16-bit storage of the volume, not the rounding of the data
    s = synth.tiny_scan()
    x_true = synth.tiny_phantom(s, synth.rng_for("tiny"))
    o = osetup(orc, s)
    p16 = gu.to_np(gu.to_dev(orc.project(o, x_true), x_dt))
    ref = orc.sart(o, p16, n_iter=10, lam=0.5)
    with cylct.Plan(s) as plan:
        got = gu.sart(plan, p16, n_iter=10, lam=0.5, x_dt=x_dt, sino_dt=x_dt, strict_16bit=strict)
    err = gu.rel_l2(got, ref)
    assert err <= (STRICT_BOUND[x_dt] if strict else TOL_16), err


@pytest.mark.parametrize("pieces", [1, 2, 4, 8, 16])
def test_pieces_per_ray_do_not_change_results(lib, orc, pieces):
    # cutting each ray into P pieces walked by different threads changes only the
    # summation order: projections and back-projections stay within the FP32 bound, per
    # voxel against the size of its terms
    s = tilted_scan()
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 0.05, size=s.vol_shape)
    y = rng.standard_normal(s.sino_shape)
    o = osetup(orc, s)
    ref_q, ref_b = orc.project(o, x), orc.backproject(o, y)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_pieces(pieces, pieces)
        assert plan.cyl_plan_get_pieces() == (pieces, pieces)
        got_q = gu.project(plan, x)
        got_b = gu.backproject(plan, y)
        plan.cyl_plan_set_pieces(0, 0)
        assert plan.cyl_plan_get_pieces() == (8, 2)
    assert per_projection_rel(got_q, ref_q) <= TOL_FP32
    abs_ref = orc.backproject(o, np.abs(y))
    assert np.max(np.abs(got_b - ref_b)) <= TOL_FP32 * np.max(abs_ref)


def test_tune_and_piece_settings(lib):
    s = tilted_scan()
    with cylct.Plan(s) as plan:
        plan.cyl_plan_tune()
        fp, bp = plan.cyl_plan_get_pieces()
        assert fp in (1, 2, 4, 8, 16) and bp in (1, 2, 4, 8, 16)
        with pytest.raises(cylct.CylError) as e:
            plan.cyl_plan_set_pieces(3, 3)
        assert e.value.code == cylct.CYL_EINVAL
        assert plan.cyl_plan_get_pieces() == (fp, bp)


# ------------------------------------------------- medium workload, sampled

def test_medium_single_view_projection_and_subset(lib, orc):
    # full medium grid (128, 512, 128) and 256^2 detector in the bench's launch
    # configuration; one view so the oracle finishes in seconds
    full = synth.medium_scan(synth.rng_for("medium"))
    s = dataclasses.replace(full, angles=full.angles[37:38])
    az = synth.insert_azimuths(synth.rng_for("medium"))
    x = synth.part_phantom(s, az)
    o = osetup(orc, s)
    ref_q = orc.project(o, x)
    with cylct.Plan(s) as plan:
        got_q = gu.project(plan, x)
        assert gu.rel_l2(got_q, ref_q) <= TOL_FP32
        # one SART subset (one view) from the defect-free warm start toward data with an
        # insert removed
        p = orc.project(o, synth.part_phantom(s, az, removed=3))
        w = synth.roi_weights(s)
        got = gu.sart(plan, p, x0=x, w=w, n_iter=1, lam=0.5)
    ref = orc.sart(o, p, x0=x, w=w, n_iter=1, lam=0.5)
    assert gu.rel_l2(got - x, ref - x) <= TOL_FP32 * 10
    assert gu.rel_l2(got, ref) <= TOL_FP32


@pytest.mark.parametrize("fused", [True, False])
def test_medium_two_sweeps_per_iterate(lib, orc, fused):
    # the medium workload at full size (grid (128, 512, 128), 256^2 detector, its pose,
    # warm start, ROI weights and Poisson data) on 8 of its 180 views, so that the oracle
    # finishes in seconds: both sweeps and both increments against the FP64 oracle
    full = synth.medium_scan(synth.rng_for("medium"))
    s = dataclasses.replace(full, angles=full.angles[::23][:8])
    az = synth.insert_azimuths(synth.rng_for("medium"))
    x0 = gu.stored(synth.part_phantom(s, az), cylct.CYL_F32)      # the values the GPU holds
    o = osetup(orc, s)
    p_clean = orc.project(o, synth.part_phantom(s, az, removed=5))
    p = gu.stored(orc.log_transform(synth.poisson_counts(p_clean, 1.0e4, np.random.default_rng(8)), 1.0e4),
                  cylct.CYL_F32)
    w = synth.roi_weights(s)
    ref1 = orc.sart(o, p, x0=x0, w=w, n_iter=1, lam=0.5)
    ref2 = orc.sart(o, p, x0=ref1, w=w, n_iter=1, lam=0.5)
    with cylct.Plan(s) as plan:
        plan.cyl_plan_set_fused(fused)
        got1 = gu.sart(plan, p, x0=x0, w=w, n_iter=1, lam=0.5)
        got2 = gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=0.5)
    assert gu.rel_l2(got1, ref1) <= TOL_FP32
    assert gu.rel_l2(got2, ref2) <= TOL_FP32
    # Each sweep changes x by a few per cent of it; the FP32 iterate and the FP32 crossing
    # positions round at 1e-7 of x, so the increments themselves hold to a few 1e-5
    # (2.1e-5 measured for the first sweep, 7.5e-7 for the iterate).
    assert gu.rel_l2(got1 - x0, ref1 - x0) <= TOL_FP32 * 5
    assert gu.rel_l2(got2 - ref1, ref2 - ref1) <= TOL_FP32 * 10


def test_fused_and_two_launch_subsets_agree(lib, orc):
    # one launch per subset (walk once, replay the recorded segments) and two launches
    # (walk twice) give the same iterates to rounding, with subsets of 3 views, a compact
    # plan included
    rng = np.random.default_rng(12)
    for s in (tilted_scan(),
              dataclasses.replace(synth.Scan(5, 16, 6, 6.0, 10.0, 60.0, 240.0, 28, 24, 1.6, 1.6,
                                             synth.full_circle(7) + 0.2), alpha=0.2, beta=0.1,
                                  gamma=0.3, tx=14.0, ty=7.0)):
        x0 = rng.uniform(0.0, 0.05, size=s.vol_shape)
        p = rng.uniform(0.0, 1.0, size=s.sino_shape)
        with cylct.Plan(s) as plan:
            a = gu.sart(plan, p, x0=x0, n_iter=2, lam=0.5, subset_size=3)
            plan.cyl_plan_set_fused(False)
            b = gu.sart(plan, p, x0=x0, n_iter=2, lam=0.5, subset_size=3)
        assert gu.rel_l2(a, b) <= 1e-6
        ref = orc.sart(osetup(orc, s), p, x0=x0, n_iter=2, lam=0.5, subset_size=3)
        assert gu.rel_l2(a, ref) <= TOL_FP32


@pytest.mark.parametrize("vol_dt", [cylct.CYL_F16, cylct.CYL_BF16])
def test_precision_size_single_view_projection(lib, orc, vol_dt):
    # full precision-variant grid (256, 1024, 256) and 512^2 detector, volume stored in
    # 16 bits; one view so the oracle finishes in seconds.  The oracle projects the same
    # rounded volume, so the bound is the FP32 one.
    import torch
    full = synth.precision_scan(synth.rng_for("precision"))
    s = dataclasses.replace(full, angles=full.angles[101:102])
    az = synth.insert_azimuths(synth.rng_for("precision"))
    x = synth.part_phantom(s, az)
    tdt = torch.float16 if vol_dt == cylct.CYL_F16 else torch.bfloat16
    x16 = torch.from_numpy(x.astype(np.float32)).to(tdt)
    ref = orc.project(osetup(orc, s), x16.float().numpy().astype(np.float64))
    with cylct.Plan(s) as plan:
        out = torch.empty(s.sino_shape, dtype=torch.float32, device="cuda")
        plan.cyl_project(x16.cuda(), vol_dt, 0, 1, out, cylct.CYL_F32)
        got = gu.to_np(out)
    assert gu.rel_l2(got, ref) <= TOL_FP32


def test_general_trajectory_frames(lib, orc):
    # frames of a circular scan give the circular plan's projections; a conveyor-belt
    # trajectory matches the oracle (projection and SART)
    s = tilted_scan()
    fs = dataclasses.replace(s, frames=synth.frames_from_circular(s))
    rng = np.random.default_rng(21)
    x = rng.uniform(0.0, 0.05, size=s.vol_shape)
    with cylct.Plan(s) as a, cylct.Plan(fs) as b:
        assert gu.rel_l2(gu.project(b, x), gu.project(a, x)) <= 1e-6
    c = synth.Scan(20, 64, 16, 10.0, 20.0, 100.0, 400.0, 48, 40, 1.6, 1.6, np.zeros(24))
    c.frames = synth.conveyor_frames(24, 100.0, 400.0, 48, 40, 1.6, 120.0)
    c.alpha, c.beta, c.gamma, c.tx, c.ty, c.tz = 0.5, 0.1, 1.3, 0.6, -0.3, 0.2
    o = osetup(orc, c)
    xc = rng.uniform(0.0, 0.05, size=c.vol_shape)
    ref_q = orc.project(o, xc)
    with cylct.Plan(c) as plan:
        assert per_projection_rel(gu.project(plan, xc), ref_q) <= TOL_FP32
        got = gu.sart(plan, ref_q, n_iter=2, lam=0.5)
    assert gu.rel_l2(got, orc.sart(o, ref_q, n_iter=2, lam=0.5)) <= TOL_FP32



@pytest.mark.parametrize("ratio", [0.5, 4.0])
def test_grazing_ray_and_voxel_floor_on_gpu(lib, orc, ratio):
    # a ray that grazes the one-voxel grid over eps / 2 or 4 eps (eps = 2^-16 R, the floor
    # of Eq. 7's row and column sums): the update equals the oracle's
    from test_oracle_sart import GRAZE_EPS, graze_scan
    s, t = graze_scan(ratio * GRAZE_EPS)
    x0, p = np.array([[[0.02]]]), np.array([[[3e-5]]])
    ref = orc.sart(osetup(orc, s), p, x0=x0, n_iter=1, lam=0.6)
    with cylct.Plan(s) as plan:
        for fused in (True, False):
            plan.cyl_plan_set_fused(fused)
            got = gu.sart(plan, p, x0=x0, n_iter=1, lam=0.6)
            assert abs(got.item() - ref.item()) <= 2e-3 * abs(ref.item() - 0.02)


@pytest.mark.parametrize("size", ["medium", "precision"])
def test_column_sums_at_full_size(lib, orc, size):
    # The normalisation sums of Eq. 7 at full size: den_m = sum_j t_jm over one view,
    # accumulated in FP32 by the walking back-projector, against the FP64 oracle's A^T 1.
    # A voxel receives about two pieces per view, so the FP32 additions round at ~1e-7;
    # the error is that of the pieces' FP32 end positions.  Written out for the record (-s)
    # for whole rays (1 piece per ray) and rays cut into 16 pieces.
    full = (synth.medium_scan(synth.rng_for("medium")) if size == "medium"
            else synth.precision_scan(synth.rng_for("precision")))
    s = dataclasses.replace(full, angles=full.angles[37:38])
    o = osetup(orc, s)
    ref = orc.backproject(o, np.ones(s.sino_shape))
    eps = s.radius * 2.0 ** -16                       # the floor of the sums
    hit = ref >= eps
    dr = s.radius / s.n_r
    with cylct.Plan(s) as plan:
        for pieces in (1, 16):
            plan.cyl_plan_set_pieces(8, pieces)
            _, cs = gu.backproject(plan, np.ones(s.sino_shape), colsum=True)
            err = np.abs(cs - ref)
            worst = np.unravel_index(int(np.argmax(err)), s.vol_shape)
            rel = err[hit] / ref[hit]
            print(f"\ncolumn sums {size}, {pieces} pieces per ray: rel L2 {gu.rel_l2(cs, ref):.2e}, "
                  f"max abs {err.max():.2e} mm at (ih, itheta, ir) {tuple(int(v) for v in worst)} "
                  f"(den {ref[worst]:.3e}), max rel over sums >= eps {rel.max():.2e}, "
                  f"sums on opposite sides of eps {int(np.sum((cs >= eps) != hit))}")
            assert gu.rel_l2(cs, ref) <= 2 * TOL_FP32
            assert err.max() <= 0.01 * dr
