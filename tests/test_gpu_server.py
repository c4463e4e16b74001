"""Serving with continuous batching: each result equals the same scan solved alone."""
import dataclasses
import time

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


PART_A = synth.Scan(12, 48, 10, 10.0, 20.0, 100.0, 400.0, 45, 29, 1.6, 1.6, synth.full_circle(1))
PART_B = synth.Scan(8, 32, 12, 8.0, 16.0, 90.0, 360.0, 37, 33, 1.5, 1.5, synth.full_circle(1))


def request_scan(part_scan, n_proj, pose, offset):
    s = dataclasses.replace(part_scan, angles=synth.full_circle(n_proj) + offset)
    s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = pose
    return s


def stream(n, seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        part = i % 2
        base = (PART_A, PART_B)[part]
        pose = (rng.uniform(0, 6.28), rng.uniform(-0.05, 0.05), rng.uniform(0, 6.28),
                *rng.uniform(-0.5, 0.5, size=3))
        s = request_scan(base, int(rng.choice([3, 4, 6])), pose, 0.05 * (i % 3))
        reqs.append((part, s, rng.uniform(0.0, 1.0, size=s.sino_shape)))
    return reqs


def start(budget=8 << 30, storage=cylct.CYL_F32, weight_dtype=cylct.CYL_F32, **kw):
    srv = cylct.Server(budget, n_iter=2, lam=0.5, storage=storage, weight_dtype=weight_dtype, **kw)
    parts = []
    for base in (PART_A, PART_B):
        x0 = np.random.default_rng(1).uniform(0.0, 0.05, size=base.vol_shape)
        w = synth.roi_weights(base, 3.0, 6.0, 4.0, scale_to_radius=False)
        parts.append((srv.cyl_server_add_part(base, gu.to_dev(x0, storage), gu.to_dev(w, weight_dtype)), x0, w))
    return srv, parts


def alone(s, p, x0, w, storage=cylct.CYL_F32, w_dt=cylct.CYL_F32):
    with cylct.Plan(s) as plan:
        return gu.sart(plan, p, x0=x0, w=w, n_iter=2, lam=0.5, x_dt=storage, sino_dt=storage, w_dt=w_dt)


@pytest.mark.parametrize("w_dt", [cylct.CYL_F32, cylct.CYL_U8])
def test_served_results_equal_solo(lib, orc, w_dt):
    import torch
    srv, parts = start(weight_dtype=w_dt)
    reqs = stream(8)
    outs, tickets = [], []
    for k, (part, s, p) in enumerate(reqs):
        if k % 2:   # host buffers
            sino = np.ascontiguousarray(p, dtype=np.float32)
            out = np.zeros(s.vol_shape, dtype=np.float32)
        else:       # device buffers
            sino = gu.to_dev(p)
            out = torch.zeros(s.vol_shape, device="cuda")
        outs.append(out)
        tickets.append(srv.cyl_submit(parts[part][0], (s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz),
                                      s.angles, sino, out))
        time.sleep(0.002 * (k % 3))     # arrivals while earlier scans run
    for t in tickets:
        rc, res = srv.cyl_wait(t, 120000)
        assert rc == cylct.CYL_OK and res.done_ns >= res.admit_ns >= res.submit_ns > 0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["rounds"] > 0
    for k, (part, s, p) in enumerate(reqs):
        got = outs[k] if isinstance(outs[k], np.ndarray) else gu.to_np(outs[k])
        solo = alone(s, p, parts[part][1], parts[part][2], w_dt=w_dt)
        assert gu.rel_l2(got, solo) <= 1e-6, k
    # and one of them against the oracle
    part, s, p = reqs[0]
    ref = orc.sart(orc.Setup(**s.fields()), p, x0=parts[part][1], w=parts[part][2], n_iter=2, lam=0.5)
    assert gu.rel_l2(gu.to_np(outs[0]), ref) <= 1e-5
    srv.close()


def test_budget_serialises_but_completes(lib):
    import torch
    budget = 1 << 20                         # the parts plus one or two scans at a time
    srv, parts = start(budget=budget)
    reqs = stream(4, seed=9)
    outs = [torch.zeros(s.vol_shape, device="cuda") for _, s, _ in reqs]
    tickets = [srv.cyl_submit(parts[part][0], (s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz), s.angles,
                              gu.to_dev(p), outs[k]) for k, (part, s, p) in enumerate(reqs)]
    for t in tickets:
        assert srv.cyl_wait(t, 120000)[0] == cylct.CYL_OK
    for k, (part, s, p) in enumerate(reqs):
        assert gu.rel_l2(gu.to_np(outs[k]), alone(s, p, parts[part][1], parts[part][2])) <= 1e-6
    assert srv.stats()["hbm_in_use"] <= budget
    srv.close()


def test_errors(lib):
    srv, parts = start(budget=4 << 20)
    big = request_scan(PART_A, 2000, (0, 0, 0, 0, 0, 0), 0.0)
    with pytest.raises(cylct.CylError) as e:
        srv.cyl_submit(parts[0][0], (0, 0, 0, 0, 0, 0), big.angles, np.zeros(1, np.float32),
                       np.zeros(1, np.float32))
    assert e.value.code == cylct.CYL_EADMIT
    assert srv.cyl_poll(12345)[0] == cylct.CYL_ENOTFOUND
    with pytest.raises(cylct.CylError):
        srv.cyl_submit(7, (0, 0, 0, 0, 0, 0), [0.0], np.zeros(1, np.float32), np.zeros(1, np.float32))
    srv.close()


def test_bf16_storage(lib, orc):
    # served with BF16 storage: against the scan solved alone, and against the FP64 oracle
    # fed the same BF16 sinogram and warm start (the reduced-precision bound, 2e-3)
    import torch
    srv, parts = start(storage=cylct.CYL_BF16)
    reqs = stream(4, seed=5)
    outs = [torch.zeros(s.vol_shape, dtype=torch.bfloat16, device="cuda") for _, s, _ in reqs]
    sinos = [gu.to_dev(p, cylct.CYL_BF16) for _, _, p in reqs]
    tickets = [srv.cyl_submit(parts[part][0], (s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz), s.angles,
                              sinos[k], outs[k]) for k, (part, s, p) in enumerate(reqs)]
    for t in tickets:
        assert srv.cyl_wait(t, 120000)[0] == cylct.CYL_OK
    for k, (part, s, p) in enumerate(reqs):
        x0 = gu.stored(parts[part][1], cylct.CYL_BF16)
        p16 = gu.stored(p, cylct.CYL_BF16)
        got = gu.to_np(outs[k])
        solo = alone(s, p16, x0, parts[part][2], cylct.CYL_BF16)
        assert gu.rel_l2(got, solo) <= 2.5e-3, k
        ref = orc.sart(orc.Setup(**s.fields()), p16, x0=x0, w=parts[part][2], n_iter=2, lam=0.5)
        assert gu.rel_l2(got, ref) <= 2e-3, k
    srv.close()


def test_zero_sweeps_return_the_warm_start(lib):
    srv = cylct.Server(8 << 30, n_iter=0, lam=0.5)
    x0 = np.random.default_rng(2).uniform(0.0, 0.05, size=PART_A.vol_shape)
    pid = srv.cyl_server_add_part(PART_A, gu.to_dev(x0), None)
    s = request_scan(PART_A, 3, (0.1, 0.02, 0.3, 0.1, 0.0, -0.1), 0.0)
    out = np.zeros(s.vol_shape, np.float32)
    t = srv.cyl_submit(pid, (s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz), s.angles,
                       np.ones(s.sino_shape, np.float32), out)
    assert srv.cyl_wait(t, 60000)[0] == cylct.CYL_OK
    assert np.array_equal(out, x0.astype(np.float32))
    srv.close()



def test_served_small_parts_on_a_wide_detector(lib):
    """Parts that cover a small fraction of the detector are served by compact plans (their
    rounds walk the listed rays only), mixed with a dense part type; each result equals
    the same scan solved alone."""
    import torch
    small = synth.Scan(6, 16, 5, 3.0, 6.0, 100.0, 400.0, 41, 37, 1.6, 1.6, synth.full_circle(1))
    srv = cylct.Server(8 << 30, n_iter=2, lam=0.5)
    try:
        rng = np.random.default_rng(8)
        bases = (small, PART_A)
        parts = []
        for base in bases:
            x0 = rng.uniform(0.0, 0.05, size=base.vol_shape)
            parts.append((srv.cyl_server_add_part(base, gu.to_dev(x0)), x0))
        jobs = []
        for k in range(6):
            part = k % 2
            pose = (rng.uniform(0, 6.28), rng.uniform(-0.05, 0.05), rng.uniform(0, 6.28),
                    *rng.uniform(-1.5, 1.5, size=3))
            s = request_scan(bases[part], int(rng.choice([3, 5])), pose, 0.1 * k)
            p = rng.uniform(0.0, 1.0, size=s.sino_shape)
            out = torch.zeros(s.vol_shape, device="cuda")
            t = srv.cyl_submit(parts[part][0], pose, s.angles, gu.to_dev(p), out)
            jobs.append((t, part, s, p, out))
        for t, part, s, p, out in jobs:
            rc, _ = srv.cyl_wait(t, 120000)
            assert rc == cylct.CYL_OK
            want = alone(s, p, parts[part][1], None)
            assert gu.rel_l2(gu.to_np(out), want) <= 1e-5
    finally:
        srv.close()
