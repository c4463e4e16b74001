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

CYL_F32, CYL_F16, CYL_BF16 = 0, 1, 2
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
                ("angles_rad", ctypes.POINTER(ctypes.c_double))]


class cyl_pose(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("tx", ctypes.c_double), ("ty", ctypes.c_double), ("tz", ctypes.c_double)]


class cyl_sart_params(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int32), ("subset_size", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("clamp_nonneg", ctypes.c_int32),
                ("weight_mode", ctypes.c_int32), ("strict_16bit", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

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
    "cyl_backproject": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _I32, _I32, _VP, _VP, _VP]),
    "cyl_sart_solve": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP,
                                      ctypes.POINTER(cyl_sart_params), _VP, ctypes.c_int, _VP]),
    "cyl_count_segments": (ctypes.c_int, [_VP, _I32, _I32, _VP, _VP]),
    "cyl_plan_set_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "cyl_plan_kernel_time": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(_I64)]),
    "cyl_plan_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
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
    raise TypeError(f"unsupported dtype {t}")


def structs_from_scan(scan):
    """(grid, geom, pose, angle array) ctypes structs for a synth.Scan-like object."""
    ang = np.ascontiguousarray(scan.angles, dtype=np.float64)
    grid = cyl_grid(scan.n_h, scan.n_theta, scan.n_r, scan.radius, scan.height)
    geom = cyl_geom(scan.sod, scan.sdd, len(ang), scan.det_w, scan.det_h, scan.pitch_u,
                    scan.pitch_v, scan.off_u, scan.off_v,
                    ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    pose = cyl_pose(scan.alpha, scan.beta, scan.gamma, scan.tx, scan.ty, scan.tz)
    return grid, geom, pose, ang


def sart_params(n_iter=10, subset_size=1, lam=0.5, clamp_nonneg=False, weight_mode=1,
                strict_16bit=False, use_graph=True) -> cyl_sart_params:
    return cyl_sart_params(n_iter, subset_size, lam, int(clamp_nonneg), weight_mode,
                           int(strict_16bit), int(use_graph))


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

    def cyl_plan_set_timing(self, enable: bool):
        _check(load().cyl_plan_set_timing(self.h, int(enable)), "cyl_plan_set_timing")

    def cyl_plan_kernel_time(self, kind: int):
        ms, n = ctypes.c_double(), _I64()
        _check(load().cyl_plan_kernel_time(self.h, kind, ctypes.byref(ms), ctypes.byref(n)),
               "cyl_plan_kernel_time")
        return ms.value, n.value


def cyl_log_transform(counts, in_dtype, i0, p_out, out_dtype, n, stream=None):
    _check(load().cyl_log_transform(ptr(counts), in_dtype, float(i0), ptr(p_out), out_dtype, n,
                                    stream_ptr(stream)), "cyl_log_transform")
