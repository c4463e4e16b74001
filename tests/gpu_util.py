"""Helpers of the GPU parity tests: run the library's entry points on numpy inputs."""
from __future__ import annotations

import numpy as np

from paper_2005_11976_gb300 import cylct

TORCH_DT = {}


def torch_dtype(code):
    import torch
    return {cylct.CYL_F32: torch.float32, cylct.CYL_F16: torch.float16,
            cylct.CYL_BF16: torch.bfloat16, cylct.CYL_U8: torch.uint8}[code]


def to_dev(a, code=cylct.CYL_F32):
    """``a`` on the device in ``code`` (U8: a class map of integer values 0..255)."""
    import torch
    if code == cylct.CYL_U8:
        v = np.asarray(a)
        assert np.all(v == np.rint(v)) and v.min() >= 0 and v.max() <= 255
        return torch.from_numpy(np.ascontiguousarray(v, dtype=np.uint8)).to("cuda")
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(
        "cuda").to(torch_dtype(code)).contiguous()


def stored(a, code):
    """The values of ``a`` as ``code`` holds them (rounded on the host), as float64."""
    import torch
    if code == cylct.CYL_U8:
        return np.asarray(a, dtype=np.uint8).astype(np.float64)
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch_dtype(code))
    return t.float().numpy().astype(np.float64)


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.float().cpu().numpy().astype(np.float64)


def project(plan, x, p0=0, np_=None, vol_dt=cylct.CYL_F32, out_dt=cylct.CYL_F32):
    import torch
    s = plan.scan
    np_ = s.n_proj - p0 if np_ is None else np_
    xd = to_dev(x, vol_dt)
    out = torch.empty((np_, s.det_h, s.det_w), dtype=torch_dtype(out_dt), device="cuda")
    plan.cyl_project(xd, vol_dt, p0, np_, out, out_dt)
    return to_np(out)


def backproject(plan, y, p0=0, np_=None, colsum=False, y_dt=cylct.CYL_F32):
    import torch
    s = plan.scan
    np_ = s.n_proj - p0 if np_ is None else np_
    yd = to_dev(y, y_dt)
    out = torch.empty(s.vol_shape, dtype=torch.float32, device="cuda")
    cs = torch.empty(s.vol_shape, dtype=torch.float32, device="cuda") if colsum else None
    plan.cyl_backproject(yd, y_dt, p0, np_, out, cs)
    return (to_np(out), to_np(cs)) if colsum else to_np(out)


def row_sums(plan, p0=0, np_=None):
    import torch
    s = plan.scan
    np_ = s.n_proj - p0 if np_ is None else np_
    L = torch.empty((np_, s.det_h, s.det_w), dtype=torch.float32, device="cuda")
    plan.cyl_row_sums(p0, np_, L)
    return to_np(L)


def count_segments(plan, p0=0, np_=None):
    import torch
    s = plan.scan
    np_ = s.n_proj - p0 if np_ is None else np_
    c = torch.zeros(np_, dtype=torch.int64, device="cuda")
    plan.cyl_count_segments(p0, np_, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def sart(plan, p, x0=None, w=None, n_iter=1, x_dt=cylct.CYL_F32, sino_dt=cylct.CYL_F32,
         w_dt=cylct.CYL_F32, **kw):
    import torch
    s = plan.scan
    pd = to_dev(p, sino_dt)
    x0d = to_dev(x0, x_dt) if x0 is not None else None
    wd = to_dev(w, w_dt) if w is not None else None
    out = torch.empty(s.vol_shape, dtype=torch_dtype(x_dt), device="cuda")
    prm = cylct.sart_params(n_iter=n_iter, weight_dtype=w_dt, **kw)
    plan.cyl_sart_solve(pd, sino_dt, x0d, wd, prm, out, x_dt)
    return to_np(out)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
