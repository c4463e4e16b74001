"""Thin ctypes binding of libcylct.so (C ABI in include/cylct.h).

Argument marshalling only: every step of the reconstruction runs in the library's CUDA
kernels.  Arrays are passed as raw pointers; torch tensors are accepted for convenience
(their ``data_ptr()``), numpy arrays for the host-memory forms of ``cyl_sart_solve``.
The library must have been built (``python -m paper_2005_11976_gb300.build``); there is
no fallback path, and :func:`load` raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcylct.so")

CYL_OK = 0
CYL_EINVAL = -1
CYL_ENOMEM = -2
CYL_EDEVICE = -3
CYL_EADMIT = -4
CYL_ETIMEOUT = -5
CYL_ENOTFOUND = -6
CYL_EPENDING = -7
CYL_ECANCELLED = -8

CYL_F32, CYL_F16, CYL_BF16, CYL_U8 = 0, 1, 2, 3   # CYL_U8: weight maps only
CYL_MAX_BATCH = 4096
CYL_MAX_DET_SIDE = 262143
KIND_FORWARD, KIND_BACK, KIND_UPDATE = 0, 1, 2


class CylError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__(f"{where} failed: {code} ({detail})")
        self.code = code


class cyl_grid(ctypes.Structure):
    _fields_ = [("n_h", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("n_r", ctypes.c_int32),
                ("radius_mm", ctypes.c_double), ("height_mm", ctypes.c_double)]


class cyl_geom(ctypes.Structure):
    _fields_ = [("sod_mm", ctypes.c_double), ("sdd_mm", ctypes.c_double),
                ("n_proj", ctypes.c_int32), ("det_w", ctypes.c_int32), ("det_h", ctypes.c_int32),
                ("pitch_u_mm", ctypes.c_double), ("pitch_v_mm", ctypes.c_double),
                ("off_u_mm", ctypes.c_double), ("off_v_mm", ctypes.c_double),
                ("angles_rad", ctypes.POINTER(ctypes.c_double)),
                ("frames_mm", ctypes.POINTER(ctypes.c_double))]


class cyl_pose(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("tx", ctypes.c_double), ("ty", ctypes.c_double), ("tz", ctypes.c_double)]


class cyl_sart_params(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int32), ("subset_size", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("clamp_nonneg", ctypes.c_int32),
                ("weight_mode", ctypes.c_int32), ("strict_16bit", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("weight_dtype", ctypes.c_int32)]


class cyl_server_cfg(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("max_active", ctypes.c_int32), ("n_iter", ctypes.c_int32),
                ("subset_size", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("weight_mode", ctypes.c_int32), ("clamp_nonneg", ctypes.c_int32),
                ("storage", ctypes.c_int), ("rounds_ahead", ctypes.c_int32),
                ("weight_dtype", ctypes.c_int32)]


class cyl_request(ctypes.Structure):
    _fields_ = [("part", ctypes.c_int32), ("pose", cyl_pose), ("n_proj", ctypes.c_int32),
                ("angles_rad", ctypes.POINTER(ctypes.c_double)), ("sino", ctypes.c_void_p),
                ("x_out", ctypes.c_void_p)]


class cyl_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("submit_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class cyl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("active", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("hbm_in_use", ctypes.c_int64)]


class cyl_pose_params(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("dilate_px", ctypes.c_int32),
                ("roi", ctypes.c_int32 * 4), ("max_iter", ctypes.c_int32),
                ("gamma", ctypes.c_double)]


class cyl_pose_info(ctypes.Structure):
    _fields_ = [("top_mm", ctypes.c_double * 3), ("bottom_mm", ctypes.c_double * 3),
                ("rms_mm", ctypes.c_double * 2), ("iters", ctypes.c_int32 * 2),
                ("n_views", ctypes.c_int32), ("status", ctypes.c_int32)]


class cyl_band(ctypes.Structure):
    _fields_ = [("h_lo_mm", ctypes.c_double), ("h_hi_mm", ctypes.c_double),
                ("half_width_mm", ctypes.c_double)]


_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double

# name -> (restype, argtypes); the exported C ABI
SIGNATURES = {
    "cyl_last_error_detail": (ctypes.c_char_p, []),
    "cyl_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cyl_version": (ctypes.c_char_p, []),
    "cyl_plan_create": (ctypes.c_int, [ctypes.POINTER(cyl_grid), ctypes.POINTER(cyl_geom),
                                       ctypes.POINTER(cyl_pose), ctypes.c_int, ctypes.POINTER(_VP)]),
    "cyl_plan_destroy": (ctypes.c_int, [_VP]),
    "cyl_plan_set_pose": (ctypes.c_int, [_VP, ctypes.POINTER(cyl_pose), _VP]),
    "cyl_log_transform": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, _VP, ctypes.c_int,
                                         _I64, _VP]),
    "cyl_row_sums": (ctypes.c_int, [_VP, _I32, _I32, _VP, _VP]),
    "cyl_project": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _I32, _I32, _VP, ctypes.c_int, _VP]),
    "cyl_plan_set_fused": (ctypes.c_int, [_VP, _I32]),
    "cyl_plan_set_sart_pieces": (ctypes.c_int, [_VP, _I32]),
    "cyl_plan_set_records": (ctypes.c_int, [_VP, _I32, _I32, _VP]),
    "cyl_plan_records": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                                        ctypes.POINTER(_I64)]),
    "cyl_binary_version": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_I32)]),
    "cyl_project_noalloc": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _I32, _I32, _VP, ctypes.c_int, _VP]),
    "cyl_backproject": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _I32, _I32, _VP, _VP, _VP]),
    "cyl_sart_solve": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP,
                                      ctypes.POINTER(cyl_sart_params), _VP, ctypes.c_int, _VP]),
    "cyl_count_segments": (ctypes.c_int, [_VP, _I32, _I32, _VP, _VP]),
    "cyl_sart_solve_batch": (ctypes.c_int, [_I32, _VP, _VP, ctypes.c_int, _VP, _VP,
                                            ctypes.POINTER(cyl_sart_params), _VP, ctypes.c_int, _VP]),
    "cyl_sart_tune_batch": (ctypes.c_int, [_I32, _VP, _VP, ctypes.c_int, _VP, _VP,
                                           ctypes.POINTER(cyl_sart_params), _VP, ctypes.c_int, _VP]),
    "cyl_server_create": (ctypes.c_int, [ctypes.POINTER(cyl_server_cfg), ctypes.POINTER(_VP)]),
    "cyl_server_add_part": (ctypes.c_int, [_VP, ctypes.POINTER(cyl_grid), ctypes.POINTER(cyl_geom),
                                           _VP, _VP, ctypes.POINTER(_I32)]),
    "cyl_submit": (ctypes.c_int, [_VP, ctypes.POINTER(cyl_request), ctypes.POINTER(ctypes.c_uint64)]),
    "cyl_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(cyl_result)]),
    "cyl_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, _I64, ctypes.POINTER(cyl_result)]),
    "cyl_server_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(cyl_server_stats)]),
    "cyl_server_destroy": (ctypes.c_int, [_VP]),
    "cyl_plan_tune": (ctypes.c_int, [_VP, _VP]),
    "cyl_plan_get_pieces": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "cyl_plan_set_pieces": (ctypes.c_int, [_VP, _I32, _I32]),
    "cyl_plan_set_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "cyl_plan_kernel_time": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(_I64)]),
    "cyl_plan_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "cyl_axis_corners": (ctypes.c_int, [ctypes.POINTER(cyl_geom), _VP, ctypes.c_int,
                                        ctypes.POINTER(cyl_pose_params), _VP, _VP, _VP]),
    "cyl_track_point": (ctypes.c_int, [ctypes.POINTER(cyl_geom), _VP, _I32, _VP, _VP]),
    "cyl_estimate_pose": (ctypes.c_int, [ctypes.POINTER(cyl_geom), _VP, ctypes.c_int,
                                         ctypes.POINTER(cyl_pose_params), ctypes.POINTER(cyl_pose),
                                         ctypes.POINTER(cyl_pose_info), _VP]),
    "cyl_estimate_pose_batch": (ctypes.c_int, [_I32, ctypes.POINTER(cyl_geom), _VP, ctypes.c_int,
                                               ctypes.POINTER(cyl_pose_params), ctypes.POINTER(cyl_pose),
                                               ctypes.POINTER(cyl_pose_info), _VP]),
    "cyl_band_moments": (ctypes.c_int, [ctypes.POINTER(cyl_geom), ctypes.POINTER(cyl_pose), _VP,
                                        ctypes.c_int, ctypes.POINTER(cyl_band), _VP, _VP]),
    "cyl_gamma_from_phase": (ctypes.c_int, [_D, _D, _D, _D, _D, ctypes.POINTER(_D)]),
    "cyl_pose_set_timing": (ctypes.c_int, [ctypes.c_int]),
    "cyl_pose_kernel_time": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "cyl_estimate_gamma": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, ctypes.c_int,
                                          ctypes.POINTER(cyl_band), _I32, ctypes.POINTER(_D), _VP, _VP]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libcylct.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libcylct.so not built ({p}); run "
                                   "python -m paper_2005_11976_gb300.build")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc, where):
    if rc != CYL_OK:
        lib = load()
        raise CylError(rc, where, lib.cyl_last_error_detail().decode())
    return rc


def ptr(a):
    """Raw address of a torch tensor, numpy array, int or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    raise TypeError(type(a))


def stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(t) -> int:
    name = str(t)
    if "bfloat16" in name:
        return CYL_BF16
    if "float16" in name or name.endswith("half"):
        return CYL_F16
    if "float32" in name:
        return CYL_F32
    if "uint8" in name:
        return CYL_U8
    raise TypeError(f"unsupported dtype {t}")


def structs_from_scan(scan):
    """(grid, geom, pose, kept arrays) ctypes structs for a synth.Scan-like object (a
    general trajectory when it carries ``frames``)."""
    frames = getattr(scan, "frames", None)
    D = ctypes.POINTER(ctypes.c_double)
    if frames is not None:
        fr = np.ascontiguousarray(frames, dtype=np.float64).reshape(-1, 12)
        n = fr.shape[0]
        ang = np.zeros(n)
    else:
        fr = None
        ang = np.ascontiguousarray(scan.angles, dtype=np.float64)
        n = len(ang)
    grid = cyl_grid(scan.n_h, scan.n_theta, scan.n_r, scan.radius, scan.height)
    geom = cyl_geom(scan.sod, scan.sdd, n, scan.det_w, scan.det_h, scan.pitch_u,
                    scan.pitch_v, scan.off_u, scan.off_v, ang.ctypes.data_as(D),
                    fr.ctypes.data_as(D) if fr is not None else None)
    pose = cyl_pose(scan.alpha, scan.beta, scan.gamma, scan.tx, scan.ty, scan.tz)
    return grid, geom, pose, (ang, fr)


def sart_params(n_iter=10, subset_size=1, lam=0.5, clamp_nonneg=False, weight_mode=1,
                strict_16bit=False, use_graph=True, weight_dtype=CYL_F32) -> cyl_sart_params:
    return cyl_sart_params(n_iter, subset_size, lam, int(clamp_nonneg), weight_mode,
                           int(strict_16bit), int(use_graph), weight_dtype)


class Plan:
    """Owns one cyl_plan handle; methods map one to one onto the C entry points."""

    def __init__(self, scan, device: int = 0):
        lib = load()
        grid, geom, pose, ang = structs_from_scan(scan)
        h = _VP()
        _check(lib.cyl_plan_create(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(pose),
                                   device, ctypes.byref(h)), "cyl_plan_create")
        self.h = h
        self.scan = scan

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().cyl_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sizes(self):
        nv, npix, npj, nb = _I64(), _I64(), _I32(), _I64()
        _check(load().cyl_plan_sizes(self.h, ctypes.byref(nv), ctypes.byref(npix),
                                     ctypes.byref(npj), ctypes.byref(nb)), "cyl_plan_sizes")
        return nv.value, npix.value, npj.value, nb.value

    def cyl_plan_set_pose(self, pose, stream=None):
        """pose: (alpha, beta, gamma, tx, ty, tz)."""
        c = cyl_pose(*[float(v) for v in pose])
        _check(load().cyl_plan_set_pose(self.h, ctypes.byref(c), stream_ptr(stream)),
               "cyl_plan_set_pose")

    def cyl_row_sums(self, p0, np_, L_out, stream=None):
        _check(load().cyl_row_sums(self.h, p0, np_, ptr(L_out), stream_ptr(stream)), "cyl_row_sums")

    def cyl_project(self, vol, vol_dtype, p0, np_, sino_out, sino_dtype, stream=None):
        _check(load().cyl_project(self.h, ptr(vol), vol_dtype, p0, np_, ptr(sino_out), sino_dtype,
                                  stream_ptr(stream)), "cyl_project")

    def cyl_project_noalloc(self, vol, vol_dtype, p0, np_, sino_out, sino_dtype, stream=None):
        _check(load().cyl_project_noalloc(self.h, ptr(vol), vol_dtype, p0, np_, ptr(sino_out),
                                          sino_dtype, stream_ptr(stream)), "cyl_project_noalloc")

    def cyl_backproject(self, sino, sino_dtype, p0, np_, vol_out, colsum_out=None, stream=None):
        _check(load().cyl_backproject(self.h, ptr(sino), sino_dtype, p0, np_, ptr(vol_out),
                                      ptr(colsum_out), stream_ptr(stream)), "cyl_backproject")

    def cyl_sart_solve(self, sino, sino_dtype, x0, w, params, x_out, x_dtype, stream=None):
        _check(load().cyl_sart_solve(self.h, ptr(sino), sino_dtype, ptr(x0), ptr(w),
                                     ctypes.byref(params), ptr(x_out), x_dtype,
                                     stream_ptr(stream)), "cyl_sart_solve")

    def cyl_count_segments(self, p0, np_, counts_out, stream=None):
        _check(load().cyl_count_segments(self.h, p0, np_, ptr(counts_out), stream_ptr(stream)),
               "cyl_count_segments")

    def cyl_plan_tune(self, stream=None):
        _check(load().cyl_plan_tune(self.h, stream_ptr(stream)), "cyl_plan_tune")

    def cyl_plan_get_pieces(self):
        a, b = _I32(), _I32()
        _check(load().cyl_plan_get_pieces(self.h, ctypes.byref(a), ctypes.byref(b)), "cyl_plan_get_pieces")
        return a.value, b.value

    def cyl_plan_set_pieces(self, fp: int = 0, bp: int = 0):
        _check(load().cyl_plan_set_pieces(self.h, int(fp), int(bp)), "cyl_plan_set_pieces")

    def cyl_plan_set_fused(self, enable: bool):
        _check(load().cyl_plan_set_fused(self.h, int(bool(enable))), "cyl_plan_set_fused")

    def cyl_plan_set_sart_pieces(self, pieces: int = 0):
        _check(load().cyl_plan_set_sart_pieces(self.h, int(pieces)), "cyl_plan_set_sart_pieces")

    def cyl_plan_set_records(self, enable: int, runs: int = 0, stream=None):
        _check(load().cyl_plan_set_records(self.h, int(enable), int(runs), stream_ptr(stream)),
               "cyl_plan_set_records")

    def cyl_plan_records(self):
        """(ready, bytes) of the plan's stored segment records."""
        return self.cyl_plan_records_full()[:2]

    def cyl_plan_records_full(self):
        """(ready, record bytes, gather form, transpose bytes) of the plan's stored records."""
        r, b, g, gb = _I32(), _I64(), _I32(), _I64()
        _check(load().cyl_plan_records(self.h, ctypes.byref(r), ctypes.byref(b), ctypes.byref(g),
                                       ctypes.byref(gb)), "cyl_plan_records")
        return bool(r.value), b.value, bool(g.value), gb.value

    def cyl_plan_set_timing(self, enable: bool):
        _check(load().cyl_plan_set_timing(self.h, int(enable)), "cyl_plan_set_timing")

    def cyl_estimate_gamma(self, sino, sino_dtype, tmpl, tmpl_dtype, band_, passes=1, stream=None):
        """(gamma, (phi_P, amplitude, phi_P_ref, reference amplitude) of the last pass)."""
        g = ctypes.c_double()
        diag = (ctypes.c_double * 4)()
        _check(load().cyl_estimate_gamma(self.h, ptr(sino), sino_dtype, ptr(tmpl), tmpl_dtype,
                                         ctypes.byref(band_), int(passes), ctypes.byref(g), diag,
                                         stream_ptr(stream)),
               "cyl_estimate_gamma")
        return g.value, tuple(diag)

    def cyl_plan_kernel_time(self, kind: int):
        ms, n = ctypes.c_double(), _I64()
        _check(load().cyl_plan_kernel_time(self.h, kind, ctypes.byref(ms), ctypes.byref(n)),
               "cyl_plan_kernel_time")
        return ms.value, n.value


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))(*[ptr(a) for a in items])
    return arr


def cyl_sart_solve_batch(plans, sinos, sino_dtype, x0s, ws, params, x_outs, x_dtype, stream=None):
    """Batched SART over Plan objects; x0s / ws may be None or lists with None entries."""
    n = len(plans)
    hp = _ptr_array([p.h.value for p in plans])
    hs = _ptr_array(sinos)
    hx0 = _ptr_array(x0s) if x0s is not None else None
    hw = _ptr_array(ws) if ws is not None else None
    ho = _ptr_array(x_outs)
    _check(load().cyl_sart_solve_batch(n, hp, hs, sino_dtype, hx0, hw, ctypes.byref(params), ho,
                                       x_dtype, stream_ptr(stream)), "cyl_sart_solve_batch")


def cyl_sart_tune_batch(plans, sinos, sino_dtype, x0s, ws, params, x_outs, x_dtype, stream=None):
    """Batch autotuner (same arguments as cyl_sart_solve_batch); the choice lands in plans[0]."""
    n = len(plans)
    hp = _ptr_array([p.h.value for p in plans])
    hs = _ptr_array(sinos)
    hx0 = _ptr_array(x0s) if x0s is not None else None
    hw = _ptr_array(ws) if ws is not None else None
    ho = _ptr_array(x_outs)
    _check(load().cyl_sart_tune_batch(n, hp, hs, sino_dtype, hx0, hw, ctypes.byref(params), ho,
                                      x_dtype, stream_ptr(stream)), "cyl_sart_tune_batch")


def pose_params(threshold, dilate_px=0, roi=(0, 0, 0, 0), max_iter=100, gamma=0.0) -> cyl_pose_params:
    return cyl_pose_params(float(threshold), int(dilate_px), (ctypes.c_int32 * 4)(*roi), int(max_iter),
                           float(gamma))


def band(h_lo_mm, h_hi_mm, half_width_mm) -> cyl_band:
    return cyl_band(float(h_lo_mm), float(h_hi_mm), float(half_width_mm))


def _info_dict(f: cyl_pose_info) -> dict:
    return dict(top=np.array(f.top_mm[:]), bottom=np.array(f.bottom_mm[:]), rms=tuple(f.rms_mm),
                iters=tuple(f.iters), n_views=f.n_views, status=f.status)


def cyl_axis_corners(scan, sino, sino_dtype, params, corners_out, counts_out=None, stream=None):
    """Corner pixels of every projection of ``scan``'s geometry (device outputs)."""
    _, geom, _, keep = structs_from_scan(scan)
    _check(load().cyl_axis_corners(ctypes.byref(geom), ptr(sino), sino_dtype, ctypes.byref(params),
                                   ptr(corners_out), ptr(counts_out), stream_ptr(stream)),
           "cyl_axis_corners")


def cyl_track_point(scan, track, max_iter, out, stream=None):
    _, geom, _, keep = structs_from_scan(scan)
    _check(load().cyl_track_point(ctypes.byref(geom), ptr(track), int(max_iter), ptr(out),
                                  stream_ptr(stream)), "cyl_track_point")


def cyl_estimate_pose(scan, sino, sino_dtype, params, stream=None):
    """(pose tuple (alpha, beta, gamma, tx, ty, tz), info dict)."""
    _, geom, _, keep = structs_from_scan(scan)
    pose, info = cyl_pose(), cyl_pose_info()
    _check(load().cyl_estimate_pose(ctypes.byref(geom), ptr(sino), sino_dtype, ctypes.byref(params),
                                    ctypes.byref(pose), ctypes.byref(info), stream_ptr(stream)),
           "cyl_estimate_pose")
    return (pose.alpha, pose.beta, pose.gamma, pose.tx, pose.ty, pose.tz), _info_dict(info)


def cyl_estimate_pose_batch(scans, sinos, sino_dtype, params, stream=None):
    """Poses and info dicts of many scans; ``params`` is one cyl_pose_params or a list."""
    n = len(scans)
    made = [structs_from_scan(s) for s in scans]
    geoms = (cyl_geom * n)(*[m[1] for m in made])
    prms = params if isinstance(params, (list, tuple)) else [params] * n
    hp = (cyl_pose_params * n)(*prms)
    poses, infos = (cyl_pose * n)(), (cyl_pose_info * n)()
    _check(load().cyl_estimate_pose_batch(n, geoms, _ptr_array(sinos), sino_dtype, hp, poses, infos,
                                          stream_ptr(stream)), "cyl_estimate_pose_batch")
    return ([(p.alpha, p.beta, p.gamma, p.tx, p.ty, p.tz) for p in poses],
            [_info_dict(f) for f in infos])


def cyl_band_moments(scan, pose, sino, sino_dtype, band_, moments_out, stream=None):
    _, geom, _, keep = structs_from_scan(scan)
    cp = cyl_pose(*pose)
    _check(load().cyl_band_moments(ctypes.byref(geom), ctypes.byref(cp), ptr(sino), sino_dtype,
                                   ctypes.byref(band_), ptr(moments_out), stream_ptr(stream)),
           "cyl_band_moments")


def cyl_pose_set_timing(enable: bool):
    _check(load().cyl_pose_set_timing(int(enable)), "cyl_pose_set_timing")


def cyl_pose_kernel_time(kind: int):
    ms, n = ctypes.c_double(), _I64()
    _check(load().cyl_pose_kernel_time(int(kind), ctypes.byref(ms), ctypes.byref(n)), "cyl_pose_kernel_time")
    return ms.value, n.value


def cyl_gamma_from_phase(phi_p, phi_p_ref, alpha, beta, gamma_ref=0.0) -> float:
    g = ctypes.c_double()
    _check(load().cyl_gamma_from_phase(float(phi_p), float(phi_p_ref), float(alpha), float(beta),
                                       float(gamma_ref), ctypes.byref(g)), "cyl_gamma_from_phase")
    return g.value


def cyl_log_transform(counts, in_dtype, i0, p_out, out_dtype, n, stream=None):
    _check(load().cyl_log_transform(ptr(counts), in_dtype, float(i0), ptr(p_out), out_dtype, n,
                                    stream_ptr(stream)), "cyl_log_transform")


class Server:
    """Owns a cyl_server; methods map one to one onto the serving entry points."""

    def __init__(self, hbm_budget_bytes, max_active=64, n_iter=10, subset_size=1, lam=0.5,
                 weight_mode=1, clamp_nonneg=False, storage=CYL_F32, rounds_ahead=4, device=0,
                 weight_dtype=CYL_F32):
        lib = load()
        self.cfg = cyl_server_cfg(device, int(hbm_budget_bytes), max_active, n_iter, subset_size,
                                  lam, weight_mode, int(clamp_nonneg), storage, rounds_ahead, weight_dtype)
        h = _VP()
        _check(lib.cyl_server_create(ctypes.byref(self.cfg), ctypes.byref(h)), "cyl_server_create")
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().cyl_server_destroy(self.h)
            self.h = None
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def cyl_server_add_part(self, scan, x0=None, w=None) -> int:
        grid, geom, pose, ang = structs_from_scan(scan)
        part = _I32()
        _check(load().cyl_server_add_part(self.h, ctypes.byref(grid), ctypes.byref(geom), ptr(x0),
                                          ptr(w), ctypes.byref(part)), "cyl_server_add_part")
        return part.value

    def cyl_submit(self, part, pose, angles, sino, x_out) -> int:
        ang = np.ascontiguousarray(angles, dtype=np.float64)
        req = cyl_request(part, cyl_pose(*[float(v) for v in pose]), len(ang),
                          ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ptr(sino), ptr(x_out))
        t = ctypes.c_uint64()
        _check(load().cyl_submit(self.h, ctypes.byref(req), ctypes.byref(t)), "cyl_submit")
        self._keep[t.value] = (sino, x_out)       # the caller's buffers stay referenced
        return t.value

    def cyl_poll(self, ticket):
        r = cyl_result()
        rc = load().cyl_poll(self.h, ticket, ctypes.byref(r))
        if rc != CYL_EPENDING:
            self._keep.pop(ticket, None)
        return rc, r

    def cyl_wait(self, ticket, timeout_ms=600000):
        r = cyl_result()
        rc = load().cyl_wait(self.h, ticket, int(timeout_ms), ctypes.byref(r))
        if rc not in (CYL_EPENDING, CYL_ETIMEOUT):
            self._keep.pop(ticket, None)
        return rc, r

    def stats(self) -> dict:
        s = cyl_server_stats()
        _check(load().cyl_server_get_stats(self.h, ctypes.byref(s)), "cyl_server_get_stats")
        return {k: getattr(s, k) for k, _ in cyl_server_stats._fields_}
