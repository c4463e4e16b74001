"""ctypes wrapper of the FP64 C oracle (``cyl_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
baseline may call it; the product path never does.  The C source follows the paper's
definitions directly (Sec. 2 Eq. 1-2 for the pose and cylindrical coordinates, Sec. 2.2
Eq. 6 for the intersection-length model, Eq. 7 for SART); see the header comment of
``cyl_oracle.c``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cyl_oracle.c")
_HDR = os.path.join(_HERE, "cyl_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcyl_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
               "-Wall", "-Wno-unknown-pragmas", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _COrcSetup(ctypes.Structure):
    _fields_ = [
        ("n_h", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_r", ctypes.c_int),
        ("radius", ctypes.c_double), ("height", ctypes.c_double),
        ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
        ("n_proj", ctypes.c_int), ("det_w", ctypes.c_int), ("det_h", ctypes.c_int),
        ("pitch_u", ctypes.c_double), ("pitch_v", ctypes.c_double),
        ("off_u", ctypes.c_double), ("off_v", ctypes.c_double),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
        ("tx", ctypes.c_double), ("ty", ctypes.c_double), ("tz", ctypes.c_double),
        ("frames", ctypes.POINTER(ctypes.c_double)),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_COrcSetup)
            lib.orc_pose_matrix.argtypes = [ctypes.c_double] * 3 + [_D]
            lib.orc_ray.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            lib.orc_clip.argtypes = [P, _D, _D, _D, _D]
            lib.orc_clip.restype = ctypes.c_int
            lib.orc_ray_row.argtypes = [P, _D, _D, _L, _D, ctypes.c_int]
            lib.orc_ray_row.restype = ctypes.c_int
            for name in ("orc_project", "orc_backproject"):
                getattr(lib, name).argtypes = [P, _D, ctypes.c_int, ctypes.c_int, _D]
                getattr(lib, name).restype = ctypes.c_int
            lib.orc_row_sums.argtypes = [P, ctypes.c_int, ctypes.c_int, _D]
            lib.orc_row_sums.restype = ctypes.c_int
            lib.orc_row_nnz.argtypes = [P, ctypes.c_int, ctypes.c_int, _L]
            lib.orc_row_nnz.restype = ctypes.c_int
            lib.orc_sart.argtypes = [P, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, _D]
            lib.orc_sart.restype = ctypes.c_int
            lib.orc_log_transform.argtypes = [_D, ctypes.c_double, ctypes.c_long, _D]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            lib.orc_set_num_threads.restype = None
            _lib = lib
    return _lib


@dataclasses.dataclass
class Setup:
    """Grid, cone-beam geometry and pose of one scan (lengths in mm).  ``frames``, when
    given, is an (n_proj, 12) array of lab-frame source, pixel (0, 0) centre and pixel
    steps du, dv per projection (a general trajectory: the circular fields are unused)."""
    n_h: int
    n_theta: int
    n_r: int
    radius: float
    height: float
    sod: float
    sdd: float
    det_w: int
    det_h: int
    pitch_u: float
    pitch_v: float
    angles: np.ndarray
    off_u: float = 0.0
    off_v: float = 0.0
    alpha: float = 0.0
    beta: float = 0.0
    gamma: float = 0.0
    tx: float = 0.0
    ty: float = 0.0
    tz: float = 0.0
    frames: np.ndarray | None = None

    @property
    def n_proj(self) -> int:
        return int(len(self.frames)) if self.frames is not None else int(len(self.angles))

    @property
    def n_vox(self) -> int:
        return self.n_h * self.n_theta * self.n_r

    @property
    def n_pix(self) -> int:
        return self.det_w * self.det_h

    def _c(self):
        n = self.n_proj
        ang = np.ascontiguousarray(self.angles if self.frames is None else np.zeros(n), dtype=np.float64)
        fr = None if self.frames is None else np.ascontiguousarray(self.frames, dtype=np.float64).reshape(n, 12)
        c = _COrcSetup(
            self.n_h, self.n_theta, self.n_r, self.radius, self.height, self.sod, self.sdd,
            n, self.det_w, self.det_h, self.pitch_u, self.pitch_v, self.off_u,
            self.off_v, ang.ctypes.data_as(_D), self.alpha, self.beta, self.gamma,
            self.tx, self.ty, self.tz, fr.ctypes.data_as(_D) if fr is not None else None)
        return c, (ang, fr)  # keep the arrays alive alongside the struct


def _dptr(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (n >= 1)."""
    load().orc_set_num_threads(int(n))


def pose_matrix(alpha, beta, gamma) -> np.ndarray:
    R = np.zeros(9)
    load().orc_pose_matrix(alpha, beta, gamma, _dptr(R))
    return R.reshape(3, 3)


def ray(s: Setup, p: int, iu: int, iv: int):
    c, keep = s._c()
    S = np.zeros(3)
    D = np.zeros(3)
    load().orc_ray(ctypes.byref(c), p, iu, iv, _dptr(S), _dptr(D))
    return S, D


def clip(s: Setup, o, d):
    c, keep = s._c()
    o = _f64(o)
    d = _f64(d)
    ti = ctypes.c_double()
    to = ctypes.c_double()
    ok = load().orc_clip(ctypes.byref(c), _dptr(o), _dptr(d), ctypes.byref(ti), ctypes.byref(to))
    return (ti.value, to.value) if ok else None


def ray_row(s: Setup, S, D):
    """(voxel indices, lengths in mm) of the segment S -> D."""
    c, keep = s._c()
    cap = 2 * s.n_r + s.n_theta + s.n_h + 8
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap)
    S = _f64(S)
    D = _f64(D)
    n = load().orc_ray_row(ctypes.byref(c), _dptr(S), _dptr(D),
                           idx.ctypes.data_as(_L), _dptr(ln), cap)
    if n < 0:
        raise RuntimeError("orc_ray_row failed")
    return idx[:n].copy(), ln[:n].copy()


def project(s: Setup, x, p0: int = 0, np_: int | None = None) -> np.ndarray:
    np_ = s.n_proj - p0 if np_ is None else np_
    c, keep = s._c()
    x = _f64(x).reshape(-1)
    assert x.size == s.n_vox
    q = np.zeros(np_ * s.n_pix)
    if load().orc_project(ctypes.byref(c), _dptr(x), p0, np_, _dptr(q)):
        raise RuntimeError("orc_project failed")
    return q.reshape(np_, s.det_h, s.det_w)


def backproject(s: Setup, y, p0: int = 0, np_: int | None = None) -> np.ndarray:
    np_ = s.n_proj - p0 if np_ is None else np_
    c, keep = s._c()
    y = _f64(y).reshape(-1)
    assert y.size == np_ * s.n_pix
    out = np.zeros(s.n_vox)
    if load().orc_backproject(ctypes.byref(c), _dptr(y), p0, np_, _dptr(out)):
        raise RuntimeError("orc_backproject failed")
    return out.reshape(s.n_h, s.n_theta, s.n_r)


def row_sums(s: Setup, p0: int = 0, np_: int | None = None) -> np.ndarray:
    np_ = s.n_proj - p0 if np_ is None else np_
    c, keep = s._c()
    L = np.zeros(np_ * s.n_pix)
    if load().orc_row_sums(ctypes.byref(c), p0, np_, _dptr(L)):
        raise RuntimeError("orc_row_sums failed")
    return L.reshape(np_, s.det_h, s.det_w)


def row_nnz(s: Setup, p0: int = 0, np_: int | None = None) -> np.ndarray:
    np_ = s.n_proj - p0 if np_ is None else np_
    c, keep = s._c()
    n = np.zeros(np_ * s.n_pix, dtype=np.int64)
    if load().orc_row_nnz(ctypes.byref(c), p0, np_, n.ctypes.data_as(_L)):
        raise RuntimeError("orc_row_nnz failed")
    return n.reshape(np_, s.det_h, s.det_w)


def sart(s: Setup, p, x0=None, w=None, n_iter: int = 1, subset_size: int = 1,
         lam: float = 0.5, clamp_nonneg: bool = False, weight_mode: int = 1) -> np.ndarray:
    """Eq. 7 SART; returns the final volume [N_h][N_theta][N_r]."""
    c, keep = s._c()
    p = _f64(p).reshape(-1)
    assert p.size == s.n_proj * s.n_pix
    x0k = _f64(x0).reshape(-1) if x0 is not None else None
    x0p = _dptr(x0k) if x0k is not None else None
    wk = _f64(w).reshape(-1) if w is not None else None
    wp = _dptr(wk) if wk is not None else None
    x = np.zeros(s.n_vox)
    rc = load().orc_sart(ctypes.byref(c), _dptr(p), x0p, wp, n_iter, subset_size, lam,
                         int(clamp_nonneg), weight_mode, _dptr(x))
    if rc:
        raise RuntimeError("orc_sart failed")
    return x.reshape(s.n_h, s.n_theta, s.n_r)


def log_transform(I, I0: float) -> np.ndarray:
    I = _f64(I)
    out = np.zeros_like(I)
    load().orc_log_transform(_dptr(I.reshape(-1)), float(I0), I.size, _dptr(out.reshape(-1)))
    return out
