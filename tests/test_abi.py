"""The C-ABI library builds, loads and exports every entry point of include/cylct.h, and
its host-side validation answers without a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2005_11976_gb300 import cylct, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_11976_gb300 import build
    build.build()
    return cylct.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cylct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cyl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cyl_plan_create", "cyl_plan_destroy", "cyl_project", "cyl_backproject",
                     "cyl_sart_solve", "cyl_log_transform", "cyl_row_sums"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", cylct.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (cyl_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # the binding marshals every entry point
    assert not [n for n in declared_functions() if n not in cylct.SIGNATURES]


def test_build_targets_sm_103a_only():
    from paper_2005_11976_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.gpu
def test_kernels_run_as_sm_103_binaries(lib):
    # the runtime's view of the loaded kernel image: compiled for compute capability 10.3
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    v = cylct._I32()
    assert lib.cyl_binary_version(0, ctypes.byref(v)) == cylct.CYL_OK, lib.cyl_last_error_detail()
    assert v.value == 103
    assert lib.cyl_binary_version(0, None) == cylct.CYL_EINVAL


def test_host_validation_without_gpu(lib):
    assert lib.cyl_strerror(cylct.CYL_EINVAL) == b"CYL_EINVAL"
    assert lib.cyl_version().startswith(b"cylct")
    scan = synth.tiny_scan()
    grid, geom, pose, ang = cylct.structs_from_scan(scan)
    h = ctypes.c_void_p()
    bad = cylct.cyl_grid(0, 4, 4, 1.0, 1.0)
    assert lib.cyl_plan_create(ctypes.byref(bad), ctypes.byref(geom), ctypes.byref(pose), 0,
                               ctypes.byref(h)) == cylct.CYL_EINVAL
    assert b"grid" in lib.cyl_last_error_detail()
    g2 = cylct.cyl_geom(400.0, 100.0, geom.n_proj, geom.det_w, geom.det_h, 1.0, 1.0, 0.0, 0.0,
                        geom.angles_rad)
    assert lib.cyl_plan_create(ctypes.byref(grid), ctypes.byref(g2), ctypes.byref(pose), 0,
                               ctypes.byref(h)) == cylct.CYL_EINVAL
    # general trajectories: a zero pixel step, a source inside the grid, a NaN
    fr = synth.frames_from_circular(scan)
    for k, v in ((6, 0.0), (0, 0.5), (4, float("nan"))):
        bad_f = fr.copy()
        if k == 6:
            bad_f[2, 6:9] = 0.0
        elif k == 0:
            bad_f[1, 0:3] = (0.5, 0.0, 0.0)
        else:
            bad_f[3, 4] = v
        gf = cylct.cyl_geom(0.0, 0.0, geom.n_proj, geom.det_w, geom.det_h, 0.0, 0.0, 0.0, 0.0,
                            None, np.ascontiguousarray(bad_f).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert lib.cyl_plan_create(ctypes.byref(grid), ctypes.byref(gf), ctypes.byref(pose), 0,
                                   ctypes.byref(h)) == cylct.CYL_EINVAL
    assert b"frame" in lib.cyl_last_error_detail()
    p2 = cylct.cyl_pose(float("nan"), 0, 0, 0, 0, 0)
    assert lib.cyl_plan_create(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(p2), 0,
                               ctypes.byref(h)) == cylct.CYL_EINVAL
    assert lib.cyl_plan_create(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(pose), 0,
                               None) == cylct.CYL_EINVAL
    # zero-length work and bad arguments are answered on the host
    assert lib.cyl_log_transform(None, 0, 1e4, None, 0, 0, None) == cylct.CYL_OK
    assert lib.cyl_log_transform(None, 7, 1e4, None, 0, 10, None) == cylct.CYL_EINVAL
    assert lib.cyl_log_transform(1, 0, -1.0, 2, 0, 10, None) == cylct.CYL_EINVAL
    # U8 is a weight-map type only: never a sinogram or volume type
    assert lib.cyl_log_transform(1, cylct.CYL_U8, 1e4, 2, 0, 10, None) == cylct.CYL_EINVAL
    assert lib.cyl_log_transform(1, 0, 1e4, 2, cylct.CYL_U8, 10, None) == cylct.CYL_EINVAL
    assert cylct.dtype_code("torch.uint8") == cylct.CYL_U8
    prm = cylct.sart_params(weight_dtype=cylct.CYL_U8)
    assert prm.weight_dtype == cylct.CYL_U8 and cylct.sart_params().weight_dtype == cylct.CYL_F32
    assert lib.cyl_sart_solve(None, None, 0, None, None, None, None, 0, None) == cylct.CYL_EINVAL
    assert lib.cyl_plan_destroy(None) == cylct.CYL_OK


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError):
        saved = cylct._lib
        cylct._lib = None
        try:
            cylct.load(str(tmp_path / "missing.so"))
        finally:
            cylct._lib = saved


def test_server_config_validation_without_gpu(lib):
    bad = [dict(hbm_budget_bytes=0), dict(max_active=0), dict(max_active=5000), dict(n_iter=-1),
           dict(subset_size=0), dict(weight_mode=3), dict(storage=9), dict(rounds_ahead=99),
           dict(storage=cylct.CYL_U8), dict(weight_dtype=4), dict(weight_dtype=-1)]
    for b in bad:
        cfg = dict(device=0, hbm_budget_bytes=1 << 30, max_active=8, n_iter=2, subset_size=1,
                   lambda_=0.5, weight_mode=1, clamp_nonneg=0, storage=0, rounds_ahead=4)
        cfg.update(b)
        c = cylct.cyl_server_cfg(**cfg)
        h = ctypes.c_void_p()
        assert lib.cyl_server_create(ctypes.byref(c), ctypes.byref(h)) == cylct.CYL_EINVAL, b
    # every weight-map type passes the configuration check (what follows needs a device)
    for wt in (cylct.CYL_F32, cylct.CYL_F16, cylct.CYL_BF16, cylct.CYL_U8):
        c = cylct.cyl_server_cfg(device=0, hbm_budget_bytes=1 << 30, max_active=8, n_iter=2, subset_size=1,
                                 lambda_=0.5, weight_mode=1, clamp_nonneg=0, storage=0, rounds_ahead=4,
                                 weight_dtype=wt)
        h = ctypes.c_void_p()
        rc = lib.cyl_server_create(ctypes.byref(c), ctypes.byref(h))
        assert rc != cylct.CYL_EINVAL, wt
        if rc == cylct.CYL_OK:
            lib.cyl_server_destroy(h)
    assert lib.cyl_server_destroy(None) == cylct.CYL_OK
    assert lib.cyl_poll(None, 1, None) == cylct.CYL_EINVAL
    assert lib.cyl_sart_solve_batch(-1, None, None, 0, None, None, None, None, 0, None) == cylct.CYL_EINVAL


def test_pose_calls_validate_on_the_host(lib, orc):
    from oracle import pose as op
    scan = synth.tiny_scan()
    grid, geom, pose, keep = cylct.structs_from_scan(scan)
    info = cylct.cyl_pose_info()
    out = cylct.cyl_pose()
    bad = [cylct.pose_params(float("nan")), cylct.pose_params(0.1, -1),
           cylct.pose_params(0.1, 0, (5, 5, 0, 10)), cylct.pose_params(0.1, 0, (0, 40, 0, 10)),
           cylct.pose_params(0.1, gamma=float("inf"))]
    for prm in bad:
        assert lib.cyl_estimate_pose(ctypes.byref(geom), 1, 0, ctypes.byref(prm), ctypes.byref(out),
                                     ctypes.byref(info), None) == cylct.CYL_EINVAL
    prm = cylct.pose_params(0.1)
    assert lib.cyl_estimate_pose(ctypes.byref(geom), None, 0, ctypes.byref(prm), ctypes.byref(out),
                                 None, None) == cylct.CYL_EINVAL
    assert lib.cyl_estimate_pose(ctypes.byref(geom), 1, 9, ctypes.byref(prm), ctypes.byref(out),
                                 None, None) == cylct.CYL_EINVAL
    wide = cylct.cyl_geom(100.0, 400.0, geom.n_proj, cylct.CYL_MAX_DET_SIDE + 1, 2, 1.0, 1.0, 0.0, 0.0,
                          geom.angles_rad)
    assert lib.cyl_axis_corners(ctypes.byref(wide), 1, 0, ctypes.byref(prm), 1, None, None) == cylct.CYL_EINVAL
    assert lib.cyl_estimate_pose_batch(-1, None, None, 0, None, None, None, None) == cylct.CYL_EINVAL
    assert lib.cyl_estimate_pose_batch(0, None, None, 0, None, None, None, None) == cylct.CYL_OK
    cp = cylct.cyl_pose(0, 0, 0, 0, 0, 0)
    for b in (cylct.band(1.0, 1.0, 2.0), cylct.band(-1.0, 1.0, 0.0), cylct.band(float("nan"), 1.0, 1.0)):
        assert lib.cyl_band_moments(ctypes.byref(geom), ctypes.byref(cp), 1, 0, ctypes.byref(b), 1,
                                    None) == cylct.CYL_EINVAL
    assert lib.cyl_estimate_gamma(None, None, 0, None, 0, None, 1, None, None, None) == cylct.CYL_EINVAL
    # Eq. 5 is host arithmetic: the library and the oracle agree
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.uniform(-3, 3, 5)
        a[3] = abs(a[3]) % 1.4
        assert cylct.cyl_gamma_from_phase(*a) == pytest.approx(op.gamma_from_phase(*a), abs=1e-14)
    g = ctypes.c_double()
    assert lib.cyl_gamma_from_phase(float("nan"), 0, 0, 0, 0, ctypes.byref(g)) == cylct.CYL_EINVAL


def test_struct_layout_matches_header(tmp_path):
    """Every struct of the boundary has the same size and field offsets in the header (as
    a C compiler lays it out) and in the binding."""
    structs = {name: getattr(cylct, name) for name in (
        "cyl_grid", "cyl_geom", "cyl_pose", "cyl_sart_params", "cyl_server_cfg", "cyl_request",
        "cyl_result", "cyl_server_stats", "cyl_pose_params", "cyl_pose_info", "cyl_band")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "cylct.h")}"',
             "int main(void) {"]
    for name, st in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            c = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {c}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for name, st in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)
