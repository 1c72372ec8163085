"""Oracle: plain FP64 CPU statement of the two-component step on the D3Q19
lattice (the paper's own velocity set, Section 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  ``lbm3d_oracle.c`` holds
the step (the same method as ``lbm_oracle.c`` on nineteen velocities in
three dimensions); this module compiles it with gcc and loads it through
ctypes.  The 3-D inputs (the paper's sinusoidal tube) come from the shared
input module, paper_1601_00918_gb300/workloads.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm3d_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle3d.so")


def build(force: bool = False) -> str:
    """Compile lbm3d_oracle.c with gcc (IEEE FP64, no contraction) into _build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32 * 3), ("tau", ctypes.c_double * 2), ("G", ctypes.c_double),
                ("rho_wall", ctypes.c_double * 2), ("g", ctypes.c_double * 3),
                ("eq_order", ctypes.c_int32), ("collision", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp, u8, pp = P(ctypes.c_double), P(ctypes.c_uint8), P(Params3)
        lib.oracle3_check.argtypes = [pp, u8]
        lib.oracle3_feq.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [dp]
        lib.oracle3_init.argtypes = [pp, u8, dp, dp]
        lib.oracle3_step.argtypes = [pp, u8, dp, dp, dp]
        lib.oracle3_run.argtypes = [pp, u8, dp, ctypes.c_int64, dp]
        lib.oracle3_density.argtypes = [pp, u8, dp, dp]
        lib.oracle3_fields.argtypes = [pp, u8, dp, dp, dp]
        lib.oracle3_lattice.argtypes = [P(ctypes.c_int32), dp]
        for name in ("oracle3_check", "oracle3_step", "oracle3_run"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def lattice():
    """(c [19, 3] int, w [19]) of the velocity set the oracle uses."""
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    _load().oracle3_lattice(_ptr(c, ctypes.c_int32), _ptr(w, ctypes.c_double))
    return c.astype(np.int64), w


def feq(rho, ux, uy, uz, order=3):
    out = np.empty(19)
    _load().oracle3_feq(int(order), float(rho), float(ux), float(uy), float(uz), _ptr(out, ctypes.c_double))
    return out


class Problem3:
    """A 3-D grid [nz, ny, nx], its solid mask and the physical parameters
    (as oracle.Problem, with g = (gx, gy, gz) and periodic = (px, py, pz))."""

    def __init__(self, mask, tau=(1.0, 1.0), G=0.0, rho_wall=(0.0, 0.0), g=(0.0, 0.0, 0.0),
                 periodic=(True, True, True), eq_order=3, collision="bgk"):
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.nz, self.ny, self.nx = self.mask.shape
        self.p = Params3(self.nx, self.ny, self.nz, (ctypes.c_int32 * 3)(*[int(v) for v in periodic]),
                         (ctypes.c_double * 2)(*tau), float(G), (ctypes.c_double * 2)(*rho_wall),
                         (ctypes.c_double * 3)(*g), int(eq_order), {"bgk": 0, "regularized": 1}[collision])
        if _load().oracle3_check(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8)) != 0:
            raise ValueError("mask breaks the boundary rule: a non-periodic direction needs solid "
                             "boundary planes")

    def init(self, rho_init):
        r = np.ascontiguousarray(rho_init, dtype=np.float64)
        assert r.shape == (2, self.nz, self.ny, self.nx)
        f = np.zeros((2, 19, self.nz, self.ny, self.nx))
        _load().oracle3_init(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8), _ptr(r, ctypes.c_double),
                             _ptr(f, ctypes.c_double))
        return f

    def step(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        obs = np.zeros(5)
        rc = _load().oracle3_step(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8), _ptr(f, ctypes.c_double),
                                  _ptr(out, ctypes.c_double), _ptr(obs, ctypes.c_double))
        if rc:
            raise RuntimeError(f"oracle3_step failed ({rc})")
        return out, obs

    def run(self, f, nsteps, history=False):
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        hist = np.zeros((max(int(nsteps), 1), 5)) if history else None
        rc = _load().oracle3_run(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8), _ptr(f, ctypes.c_double),
                                 int(nsteps), _ptr(hist, ctypes.c_double) if history else None)
        if rc:
            raise RuntimeError(f"oracle3_run failed ({rc})")
        return (f, hist[:nsteps]) if history else f

    def fields(self, f):
        """(rho [2, nz, ny, nx], u [3, nz, ny, nx]) one pull ahead of f."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        rho = np.empty((2, self.nz, self.ny, self.nx))
        u = np.empty((3, self.nz, self.ny, self.nx))
        _load().oracle3_fields(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8), _ptr(f, ctypes.c_double),
                               _ptr(rho, ctypes.c_double), _ptr(u, ctypes.c_double))
        return rho, u
