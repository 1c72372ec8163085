"""Oracle: plain FP64 CPU statement of the two-component D2Q9 LBM step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1601_00918_gb300``) never imports it and shares no code with it.

``lbm_oracle.c`` holds the time step (Section 2 of the paper: Eqs. basic_LBM_eq,
LBM_BGK, feq, comp_interaction, collision_term, the mixture relaxation time and
the wall potentials); this module loads it through ctypes.  ``analytic.py``
holds the closed forms and fits of Section 3 (Laplace law, layered
Hagen-Poiseuille, contact angle, Bond number, the 2-D critical pressure).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

T0 = 1.0 / 3.0


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c with gcc (IEEE FP64, no fast-math) into _build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OracleParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("tau", ctypes.c_double * 2), ("G", ctypes.c_double),
                ("rho_wall", ctypes.c_double * 2), ("g", ctypes.c_double * 2),
                ("eq_order", ctypes.c_int32), ("collision", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        u8 = P(ctypes.c_uint8)
        i32 = P(ctypes.c_int32)
        pp = P(OracleParams)
        lib.oracle_check.argtypes = [pp, u8]
        lib.oracle_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, dp]
        lib.oracle_init.argtypes = [pp, u8, dp, dp]
        lib.oracle_step.argtypes = [pp, u8, dp, dp, dp]
        lib.oracle_run.argtypes = [pp, u8, dp, ctypes.c_int64, dp]
        lib.oracle_density.argtypes = [pp, u8, dp, dp]
        lib.oracle_accel.argtypes = [pp, u8, dp, dp]
        lib.oracle_fields.argtypes = [pp, u8, dp, dp, dp, dp]
        lib.oracle_step_nodes.argtypes = [pp, u8, dp, ctypes.c_int64, i32, i32, dp]
        for name in ("oracle_check", "oracle_step", "oracle_run"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Problem:
    """A grid, its solid mask and the physical parameters of one run.

    mask: uint8 [ny, nx], 1 = solid.  tau = (tau^o, tau^w); G the interaction
    strength of Eq. comp_interaction (repulsive for G < 0); rho_wall =
    (rho_s^o, rho_s^w); g = body-force acceleration (gx, gy); collision =
    "bgk" (f' = f - f^eq) or "regularized" (Eq. Regualize)."""

    def __init__(self, mask, tau=(1.0, 1.0), G=0.0, rho_wall=(0.0, 0.0), g=(0.0, 0.0),
                 periodic=(True, True), eq_order=3, collision="bgk"):
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8)
        ny, nx = self.mask.shape
        self.nx, self.ny = nx, ny
        self.p = OracleParams(nx, ny, int(periodic[0]), int(periodic[1]),
                              (ctypes.c_double * 2)(*tau), float(G),
                              (ctypes.c_double * 2)(*rho_wall), (ctypes.c_double * 2)(*g),
                              int(eq_order), {"bgk": 0, "regularized": 1}[collision])
        if _load().oracle_check(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8)) != 0:
            raise ValueError("mask breaks the boundary rule: a non-periodic direction needs "
                             "solid nodes on both of its boundary lines")

    # --- state ------------------------------------------------------------
    def init(self, rho_init):
        """Stored state f*_i = w_i rho_init at fluid nodes; rho_init [2, ny, nx]."""
        r = np.ascontiguousarray(rho_init, dtype=np.float64)
        assert r.shape == (2, self.ny, self.nx)
        f = np.zeros((2, 9, self.ny, self.nx))
        _load().oracle_init(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                            _ptr(r, ctypes.c_double), _ptr(f, ctypes.c_double))
        return f

    def step(self, f):
        """One step; returns (f_next, obs[5]) with obs as in oracle_step."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        obs = np.zeros(5)
        rc = _load().oracle_step(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                                 _ptr(f, ctypes.c_double), _ptr(out, ctypes.c_double),
                                 _ptr(obs, ctypes.c_double))
        if rc:
            raise RuntimeError(f"oracle_step failed ({rc})")
        return out, obs

    def run(self, f, nsteps, history=False):
        """nsteps steps; returns f (a new array) and, if history, obs [nsteps, 5]."""
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        hist = np.zeros((max(int(nsteps), 1), 5)) if history else None
        rc = _load().oracle_run(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                                _ptr(f, ctypes.c_double), int(nsteps),
                                _ptr(hist, ctypes.c_double) if history else None)
        if rc:
            raise RuntimeError(f"oracle_run failed ({rc})")
        return (f, hist[:nsteps]) if history else f

    def density(self, f):
        """Density field [2, ny, nx] of the state one pull ahead of f."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        rho = np.empty((2, self.ny, self.nx))
        _load().oracle_density(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                               _ptr(f, ctypes.c_double), _ptr(rho, ctypes.c_double))
        return rho

    def accel(self, rho):
        """F^a/rho^a + g, shape [2 species, 2 components, ny, nx], from rho [2, ny, nx]."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        acc = np.empty((2, 2, self.ny, self.nx))
        _load().oracle_accel(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                             _ptr(rho, ctypes.c_double), _ptr(acc, ctypes.c_double))
        return acc

    def fields(self, f):
        """(rho [2,ny,nx], u [2,ny,nx] = (ux, uy), p [ny,nx]) one pull ahead of f."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        rho = np.empty((2, self.ny, self.nx))
        u = np.empty((2, self.ny, self.nx))
        pr = np.empty((self.ny, self.nx))
        _load().oracle_fields(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                              _ptr(f, ctypes.c_double), _ptr(rho, ctypes.c_double),
                              _ptr(u, ctypes.c_double), _ptr(pr, ctypes.c_double))
        return rho, u, pr

    def step_nodes(self, f, xs, ys):
        """Post-collision populations [k, 2, 9] of one step at nodes (xs[k], ys[k])."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        ys = np.ascontiguousarray(ys, dtype=np.int32)
        out = np.empty((len(xs), 2, 9))
        _load().oracle_step_nodes(ctypes.byref(self.p), _ptr(self.mask, ctypes.c_uint8),
                                  _ptr(f, ctypes.c_double), len(xs),
                                  _ptr(xs, ctypes.c_int32), _ptr(ys, ctypes.c_int32),
                                  _ptr(out, ctypes.c_double))
        return out


def feq(rho, ux, uy, order=3):
    """Eq. feq at one node: 9 equilibrium populations."""
    out = np.empty(9)
    _load().oracle_feq(int(order), float(rho), float(ux), float(uy), _ptr(out, ctypes.c_double))
    return out


# D2Q9 velocity set in the ordering the oracle uses (tests only need it to
# take moments; it is the textbook set c_0..c_8 with weights 4/9, 1/9, 1/36).
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36])
