"""O(S) CPU renderer (double precision, OpenMP over rays): the fast route of
the DiffUS forward on the host cores.  Benchmark use only: it times the
recurrence route on the CPU beside the GPU and is never a parity reference
(the tests compare the CUDA path with the oracle's definition route).  It
shares no code with the CUDA library or the oracle."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recurrence.c")
_LIB = os.path.join(_HERE, "_build", "librecurrence.so")
_lock = threading.Lock()
_lib = None


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad_", C.c_int32),
                ("sx", C.c_double), ("sy", C.c_double), ("sz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class _Fan(C.Structure):
    _fields_ = [("n_rays", C.c_int32), ("n_samples", C.c_int32), ("fov", C.c_double),
                ("depth", C.c_double), ("f_mhz", C.c_double), ("alpha", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("mode", C.c_int32), ("speckle", C.c_int32),
                ("Ar", C.c_double), ("pr", C.c_double), ("Ag", C.c_double), ("pg", C.c_double),
                ("Lr", C.c_int32), ("gshift", C.c_int32), ("blur", C.c_int32), ("atten", C.c_int32),
                ("sigma0", C.c_double), ("sigma1", C.c_double)]


def build(force: bool = False) -> str:
    """Compile ``cpu_baseline/_build/librecurrence.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            lib.rc_render.argtypes = [C.c_void_p, C.POINTER(_Grid), dp, C.POINTER(_Fan), C.POINTER(_Params),
                                      C.c_uint32, dp]
            lib.rc_threads.restype = C.c_int
            _lib = lib
    return _lib


def threads() -> int:
    return int(_load().rc_threads())


def render(vol, pose, fan, params, pose_ctr: int = 0):
    """Image [n_rays][S] of one pose by the O(S) recurrence (double)."""
    d = np.ascontiguousarray(vol.data, dtype=np.float32)
    nz, ny, nx = d.shape
    g = _Grid(nx, ny, nz, 0, *(float(v) for v in vol.spacing), *(float(v) for v in vol.origin))
    f = _Fan(int(fan.n_rays), int(fan.n_samples), float(fan.fov), float(fan.depth), float(fan.f_mhz),
             float(fan.alpha))
    p = _Params(int(params.seed) & (2**64 - 1), int(params.mode), int(params.speckle), float(params.Ar),
                float(params.pr), float(params.Ag), float(params.pg), int(params.Lr), int(params.gshift),
                int(params.blur), int(getattr(params, "atten", 0)), float(params.sigma0), float(params.sigma1))
    pz = np.ascontiguousarray(np.asarray(pose, dtype=np.float64))
    img = np.zeros((int(fan.n_rays), int(fan.n_samples)))
    _load().rc_render(d.ctypes.data, C.byref(g), pz.ctypes.data_as(C.POINTER(C.c_double)), C.byref(f),
                      C.byref(p), int(pose_ctr), img.ctypes.data_as(C.POINTER(C.c_double)))
    return img
