"""Batched SART: every scan of a batch equals its own single-scan solve and the oracle."""
import dataclasses

import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, synth
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


def scans():
    base = synth.Scan(12, 48, 10, 10.0, 20.0, 100.0, 400.0, 45, 29, 1.6, 1.6, synth.full_circle(5))
    out = []
    for i, (n_proj, pose) in enumerate([(5, (0.3, 0.05, 0.2, 0.4, -0.2, 0.1)),
                                         (7, (1.1, -0.04, 2.0, -0.6, 0.3, -0.2)),
                                         (4, (2.0, 0.02, 0.7, 0.1, 0.5, 0.3))]):
        s = dataclasses.replace(base, angles=synth.full_circle(n_proj) + 0.1 * i)
        s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
        out.append(s)
    return out


def inputs(s, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, 1.0, size=s.sino_shape), rng.uniform(0.0, 0.05, size=s.vol_shape),
            synth.roi_weights(s, 4.0, 7.0, 4.0, scale_to_radius=False))


@pytest.mark.parametrize("subset,w_dt", [(1, cylct.CYL_F32), (2, cylct.CYL_F32), (1, cylct.CYL_U8)])
def test_batch_equals_single_and_oracle(lib, orc, subset, w_dt):
    import torch
    ss = scans()
    plans = [cylct.Plan(s) for s in ss]
    data = [inputs(s, 10 + i) for i, s in enumerate(ss)]
    sinos = [gu.to_dev(d[0]) for d in data]
    x0s = [gu.to_dev(d[1]) for d in data]
    ws = [gu.to_dev(d[2], w_dt) for d in data]
    outs = [torch.empty(s.vol_shape, device="cuda") for s in ss]
    prm = cylct.sart_params(n_iter=2, subset_size=subset, lam=0.5, weight_dtype=w_dt)
    cylct.cyl_sart_solve_batch(plans, sinos, cylct.CYL_F32, x0s, ws, prm, outs, cylct.CYL_F32)
    got = [gu.to_np(o) for o in outs]
    for i, s in enumerate(ss):
        single = gu.sart(plans[i], data[i][0], x0=data[i][1], w=data[i][2], n_iter=2,
                         subset_size=subset, lam=0.5, w_dt=w_dt)
        assert gu.rel_l2(got[i], single) <= 1e-6, i
        ref = orc.sart(orc.Setup(**s.fields()), data[i][0], x0=data[i][1], w=data[i][2],
                       n_iter=2, subset_size=subset, lam=0.5)
        assert gu.rel_l2(got[i], ref) <= 1e-5, i
    for p in plans:
        p.close()


def test_batch_16bit_and_eager(lib, orc):
    # batched with BF16 storage: against each scan's own solve, and against the FP64 oracle
    # fed the same BF16 sinogram (the reduced-precision bound, 2e-3)
    import torch
    ss = scans()
    plans = [cylct.Plan(s) for s in ss]
    data = [inputs(s, 20 + i) for i, s in enumerate(ss)]
    sinos = [gu.to_dev(d[0], cylct.CYL_BF16) for d in data]
    outs = [torch.empty(s.vol_shape, dtype=torch.bfloat16, device="cuda") for s in ss]
    prm = cylct.sart_params(n_iter=2, lam=0.5, use_graph=False)
    cylct.cyl_sart_solve_batch(plans, sinos, cylct.CYL_BF16, None, None, prm, outs, cylct.CYL_BF16)
    for i, s in enumerate(ss):
        p16 = gu.stored(data[i][0], cylct.CYL_BF16)
        got = gu.to_np(outs[i])
        single = gu.sart(plans[i], p16, n_iter=2, lam=0.5, x_dt=cylct.CYL_BF16, sino_dt=cylct.CYL_BF16)
        assert gu.rel_l2(got, single) <= 1e-2 / 4, i   # a few BF16 ulps
        ref = orc.sart(orc.Setup(**s.fields()), p16, n_iter=2, lam=0.5)
        assert gu.rel_l2(got, ref) <= 2e-3, i
    for p in plans:
        p.close()


def test_batch_rejects_host_arrays(lib):
    ss = scans()[:1]
    plan = cylct.Plan(ss[0])
    sino = np.zeros(ss[0].sino_shape, dtype=np.float32)
    out = np.zeros(ss[0].vol_shape, dtype=np.float32)
    with pytest.raises(cylct.CylError) as e:
        cylct.cyl_sart_solve_batch([plan], [sino], cylct.CYL_F32, None, None,
                                   cylct.sart_params(n_iter=1), [out], cylct.CYL_F32)
    assert e.value.code == cylct.CYL_EINVAL
    plan.close()


scans_ = scans


def test_batch_autotuner_keeps_results(lib, orc):
    # the tuner touches only scratch: a batch tuned before solving gives the same volumes
    scans = scans_()[:2]
    rng = np.random.default_rng(9)
    ps = [orc.project(orc.Setup(**s.fields()), rng.uniform(0.0, 0.05, size=s.vol_shape)) for s in scans]
    plans = [cylct.Plan(s) for s in scans]
    try:
        sinos = [gu.to_dev(p) for p in ps]
        outs = [gu.to_dev(np.full(s.vol_shape, 7.0)) for s in scans]
        prm = cylct.sart_params(n_iter=2, lam=0.5)
        cylct.cyl_sart_tune_batch(plans, sinos, cylct.CYL_F32, None, None, prm, outs, cylct.CYL_F32)
        assert all(np.all(gu.to_np(o) == 7.0) for o in outs)      # outputs untouched
        fp, bp = plans[0].cyl_plan_get_pieces()
        assert fp in (1, 2, 4, 8, 16) and bp in (1, 2, 4, 8, 16)
        cylct.cyl_sart_solve_batch(plans, sinos, cylct.CYL_F32, None, None, prm, outs, cylct.CYL_F32)
        for s, p, o in zip(scans, ps, outs):
            assert gu.rel_l2(gu.to_np(o), orc.sart(orc.Setup(**s.fields()), p, n_iter=2, lam=0.5)) <= 1e-5
    finally:
        for p in plans:
            p.close()



def test_batch_with_listed_and_dense_scans(lib, orc):
    """Scans whose rays mostly miss their grid take their tasks from their ray lists
    inside the batched rounds, next to a dense scan; every result equals its own solve
    and the oracle."""
    small = synth.Scan(6, 16, 5, 3.0, 6.0, 100.0, 400.0, 41, 37, 1.6, 1.6, synth.full_circle(5) + 0.2)
    ss = []
    for i, pose in enumerate([(0.3, 0.1, 0.5, 1.5, -2.0, 0.4), (1.2, 0.05, -0.7, -1.0, 1.0, -0.3)]):
        s = dataclasses.replace(small, angles=synth.full_circle(5 + i) + 0.2)
        s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
        ss.append(s)
    ss.append(scans()[0])                                   # a dense scan of another part
    rng = np.random.default_rng(17)
    data = [(rng.uniform(0.0, 1.0, size=s.sino_shape), rng.uniform(0.0, 0.05, size=s.vol_shape)) for s in ss]
    plans = [cylct.Plan(s) for s in ss]
    try:
        import torch
        outs = [torch.empty(s.vol_shape, device="cuda") for s in ss]
        prm = cylct.sart_params(n_iter=2, lam=0.5)
        cylct.cyl_sart_solve_batch(plans, [gu.to_dev(d[0]) for d in data], cylct.CYL_F32,
                                   [gu.to_dev(d[1]) for d in data], None, prm, outs, cylct.CYL_F32)
        for i, s in enumerate(ss):
            got = gu.to_np(outs[i])
            single = gu.sart(plans[i], data[i][0], x0=data[i][1], n_iter=2, lam=0.5)
            assert gu.rel_l2(got, single) <= 1e-6, i
            ref = orc.sart(orc.Setup(**s.fields()), data[i][0], x0=data[i][1], n_iter=2, lam=0.5)
            assert gu.rel_l2(got, ref) <= 1e-5, i
    finally:
        for p in plans:
            p.close()
