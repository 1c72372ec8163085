"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

Every call goes to libgb300lbm.so, built in-tree by ``build.py``; there is no
fallback: if the library is missing or no CUDA device is present the calls
raise.  PyTorch is used only as the provider of device memory (the optional
workspace arena) and of the CUDA stream.

The functions keep the C names: ``lbm_create``, ``lbm_step``,
``lbm_observables``, ``lbm_get_fields``, ``lbm_set_body_force``, ``lbm_save``,
``lbm_load``, ``lbm_destroy``, ``lbm_last_error``, ``lbm_workspace_size``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgb300lbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT = 0, -1, -2, -3, -4, -5
LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S, LBM_FP32C = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S, "bf16s": LBM_BF16S, "fp32c": LBM_FP32C}

# symbols declared in include/lbm.h
EXPORTS = ("lbm_workspace_size", "lbm_create", "lbm_step", "lbm_observables", "lbm_get_fields",
           "lbm_set_body_force", "lbm_save", "lbm_load", "lbm_kernel_info", "lbm_destroy",
           "lbm_last_error", "lbm_batch_create", "lbm_batch_step", "lbm_batch_observables",
           "lbm_batch_set_body_force", "lbm_batch_save", "lbm_critical_pressure_batch",
           "lbm_batch_destroy", "lbm_batch_last_error", "lbm_mlp_create", "lbm_mlp_params",
           "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_adam", "lbm_mlp_train", "lbm_mlp_destroy",
           "lbm_mlp_last_error", "lbm_step_noalloc", "lbm_wait_selftest", "lbm_batch_kernel_info",
           "lbm_channel_shape", "lbm_channel_geometry", "lbm_wetting_calibrate", "lbm_surface_tension",
           "lbm_planar_critical_balance", "lbm_planar_critical_balance_hysteresis", "lbm_contact_angle",
           "lbm_slug_area", "lbm_wall_potentials", "lbm_meniscus_angles", "lbm_critical_pressure_channels", "lbm_channel_last_error", "lbm3d_create", "lbm3d_step",
           "lbm3d_observables", "lbm3d_get_fields", "lbm3d_save", "lbm3d_load", "lbm3d_destroy",
           "lbm3d_last_error")


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("tau", ctypes.c_double * 2), ("G", ctypes.c_double),
                ("rho_wall", ctypes.c_double * 2), ("g", ctypes.c_double * 2),
                ("precision", ctypes.c_int32), ("eq_order", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


class Obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2), ("oil_mom_x", ctypes.c_double),
                ("oil_disp_x", ctypes.c_double), ("max_u", ctypes.c_double),
                ("step", ctypes.c_int64), ("nan_flag", ctypes.c_int32),
                ("timeout_flag", ctypes.c_int32)]

    def as_dict(self):
        return {"mass": (self.mass[0], self.mass[1]), "oil_mom_x": self.oil_mom_x,
                "oil_disp_x": self.oil_disp_x, "max_u": self.max_u, "step": self.step,
                "nan_flag": self.nan_flag, "timeout_flag": self.timeout_flag}


class Instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("tau", ctypes.c_double * 2), ("G", ctypes.c_double),
                ("rho_wall", ctypes.c_double * 2), ("g", ctypes.c_double * 2),
                ("mask", ctypes.POINTER(ctypes.c_uint8)), ("rho_init", ctypes.POINTER(ctypes.c_double)),
                ("disp_threshold", ctypes.c_double), ("collision", ctypes.c_int32)]


class BisectOpts(ctypes.Structure):
    _fields_ = [("rel_bracket", ctypes.c_double), ("t_eq", ctypes.c_int64), ("t_obs", ctypes.c_int64),
                ("max_probes", ctypes.c_int32), ("check_bracket", ctypes.c_int32),
                ("timeout_s", ctypes.c_double)]


class CritResult(ctypes.Structure):
    _fields_ = [("g_lo", ctypes.c_double), ("g_hi", ctypes.c_double), ("probes", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32 * 3), ("tau", ctypes.c_double * 2), ("G", ctypes.c_double),
                ("rho_wall", ctypes.c_double * 2), ("g", ctypes.c_double * 3), ("precision", ctypes.c_int32),
                ("eq_order", ctypes.c_int32), ("collision", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p)]


class ChannelSpec(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_int32), ("amp_ratio", ctypes.c_double),
                ("slug_len_over_lambda", ctypes.c_double), ("theta_deg", ctypes.c_double),
                ("visc_ratio", ctypes.c_double), ("n_periods", ctypes.c_int32), ("n_slugs", ctypes.c_int32)]


class ChannelOpts(ctypes.Structure):
    _fields_ = [("rel_bracket", ctypes.c_double), ("t_eq", ctypes.c_int64), ("t_obs", ctypes.c_int64),
                ("max_probes", ctypes.c_int32), ("precision", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("use_surrogate", ctypes.c_int32), ("surrogate", ctypes.c_void_p),
                ("feature_mean", ctypes.c_float * 5), ("feature_std", ctypes.c_float * 5),
                ("k_sigma", ctypes.c_double), ("bracket_lo", ctypes.c_double), ("bracket_hi", ctypes.c_double),
                ("calib_r", ctypes.POINTER(ctypes.c_double)), ("calib_theta", ctypes.POINTER(ctypes.c_double)),
                ("calib_n", ctypes.c_int32), ("sigma", ctypes.c_double), ("rho_bulk", ctypes.c_double),
                ("timeout_s", ctypes.c_double), ("cuda_stream", ctypes.c_void_p)]


class ChannelResult(ctypes.Structure):
    _fields_ = [("g_lo", ctypes.c_double), ("g_hi", ctypes.c_double), ("bo_lo", ctypes.c_double),
                ("bo_hi", ctypes.c_double), ("g_start_lo", ctypes.c_double), ("g_start_hi", ctypes.c_double),
                ("g_analytic", ctypes.c_double), ("rho_wall", ctypes.c_double * 2), ("tau", ctypes.c_double * 2),
                ("sigma", ctypes.c_double), ("rho_bulk", ctypes.c_double), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("probes", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {"g_lo": self.g_lo, "g_hi": self.g_hi, "bo_lo": self.bo_lo, "bo_hi": self.bo_hi,
                "g_start_lo": self.g_start_lo, "g_start_hi": self.g_start_hi, "g_analytic": self.g_analytic,
                "rho_wall": (self.rho_wall[0], self.rho_wall[1]), "tau": (self.tau[0], self.tau[1]),
                "sigma": self.sigma, "rho_bulk": self.rho_bulk, "nx": self.nx, "ny": self.ny,
                "probes": self.probes, "status": self.status}


_lib = None


def library(path: str | None = None) -> ctypes.CDLL:
    """Load libgb300lbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1601_00918_gb300.build.build()")
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    dp = P(ctypes.c_double)
    lib.lbm_workspace_size.argtypes = [P(Params), P(ctypes.c_size_t)]
    lib.lbm_create.argtypes = [P(ctypes.c_uint8), dp, P(Params), P(vp)]
    lib.lbm_step.argtypes = [vp, ctypes.c_int64]
    lib.lbm_observables.argtypes = [vp, P(Obs)]
    lib.lbm_get_fields.argtypes = [vp, dp, dp, dp]
    lib.lbm_set_body_force.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.lbm_save.argtypes = [vp, dp]
    lib.lbm_load.argtypes = [vp, dp]
    lib.lbm_kernel_info.argtypes = [vp, P(ctypes.c_int32)]
    lib.lbm_step_noalloc.argtypes = [vp, vp, vp, vp, P(Params)]
    lib.lbm_step_noalloc.restype = ctypes.c_int
    lib.lbm_wait_selftest.argtypes = [vp, dp]
    lib.lbm_wait_selftest.restype = ctypes.c_int
    lib.lbm_batch_create.argtypes = [P(Instance), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, P(vp)]
    lib.lbm_batch_step.argtypes = [vp, ctypes.c_int64]
    lib.lbm_batch_observables.argtypes = [vp, P(Obs)]
    lib.lbm_batch_set_body_force.argtypes = [vp, dp]
    lib.lbm_batch_save.argtypes = [vp, ctypes.c_int32, dp]
    lib.lbm_batch_kernel_info.argtypes = [vp, P(ctypes.c_int32)]
    lib.lbm_critical_pressure_batch.argtypes = [vp, dp, dp, P(BisectOpts), P(CritResult)]
    lib.lbm_batch_destroy.argtypes = [vp]
    lib.lbm_batch_destroy.restype = None
    lib.lbm_batch_last_error.argtypes = [vp]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    fp = P(ctypes.c_float)
    lib.lbm_mlp_create.argtypes = [fp, ctypes.c_uint64, vp, P(vp)]
    lib.lbm_mlp_params.argtypes = [vp, fp, fp]
    lib.lbm_mlp_forward.argtypes = [vp, fp, ctypes.c_int32, fp]
    lib.lbm_mlp_loss_grad.argtypes = [vp, fp, fp, ctypes.c_int32, fp, fp]
    lib.lbm_mlp_adam.argtypes = [vp, ctypes.c_float]
    lib.lbm_mlp_train.argtypes = [vp, fp, fp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                  ctypes.c_uint64, fp]
    lib.lbm_mlp_destroy.argtypes = [vp]
    lib.lbm_mlp_destroy.restype = None
    lib.lbm_mlp_last_error.argtypes = []
    lib.lbm_mlp_last_error.restype = ctypes.c_char_p
    for name in ("lbm_mlp_create", "lbm_mlp_params", "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_adam",
                 "lbm_mlp_train"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lbm_channel_shape.argtypes = [P(ChannelSpec), P(ctypes.c_int32), P(ctypes.c_int32)]
    lib.lbm_channel_geometry.argtypes = [P(ChannelSpec), P(ctypes.c_uint8), dp]
    lib.lbm_wetting_calibrate.argtypes = [dp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, vp, dp]
    lib.lbm_surface_tension.argtypes = [ctypes.c_int64, ctypes.c_int32, vp, dp, dp]
    lib.lbm_planar_critical_balance.argtypes = [ctypes.c_double] * 6 + [dp]
    lib.lbm_planar_critical_balance_hysteresis.argtypes = [ctypes.c_double] * 7 + [dp]
    lib.lbm_meniscus_angles.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, dp]
    lib.lbm_meniscus_angles.restype = ctypes.c_int
    lib.lbm_slug_area.argtypes = [dp, P(ctypes.c_uint8), ctypes.c_int32, ctypes.c_int32, dp]
    lib.lbm_slug_area.restype = ctypes.c_int
    lib.lbm_contact_angle.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, dp]
    lib.lbm_wall_potentials.argtypes = [dp, dp, ctypes.c_int32, ctypes.c_double, dp]
    lib.lbm_critical_pressure_channels.argtypes = [P(ChannelSpec), ctypes.c_int32, P(ChannelOpts),
                                                   P(ChannelResult)]
    lib.lbm_channel_last_error.argtypes = []
    lib.lbm_channel_last_error.restype = ctypes.c_char_p
    for name in ("lbm_channel_shape", "lbm_channel_geometry", "lbm_wetting_calibrate", "lbm_surface_tension",
                 "lbm_planar_critical_balance", "lbm_planar_critical_balance_hysteresis", "lbm_contact_angle", "lbm_wall_potentials",
                 "lbm_critical_pressure_channels"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lbm3d_create.argtypes = [P(ctypes.c_uint8), dp, P(Params3), P(vp)]
    lib.lbm3d_step.argtypes = [vp, ctypes.c_int64]
    lib.lbm3d_observables.argtypes = [vp, P(Obs)]
    lib.lbm3d_get_fields.argtypes = [vp, dp, dp]
    lib.lbm3d_save.argtypes = [vp, dp]
    lib.lbm3d_load.argtypes = [vp, dp]
    lib.lbm3d_destroy.argtypes = [vp]
    lib.lbm3d_destroy.restype = None
    lib.lbm3d_last_error.argtypes = [vp]
    lib.lbm3d_last_error.restype = ctypes.c_char_p
    for name in ("lbm3d_create", "lbm3d_step", "lbm3d_observables", "lbm3d_get_fields", "lbm3d_save",
                 "lbm3d_load"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lbm_destroy.argtypes = [vp]
    lib.lbm_destroy.restype = None
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = ctypes.c_char_p
    for name in ("lbm_workspace_size", "lbm_create", "lbm_step", "lbm_observables",
                 "lbm_get_fields", "lbm_set_body_force", "lbm_save", "lbm_load", "lbm_kernel_info",
                 "lbm_batch_create", "lbm_batch_step", "lbm_batch_observables",
                 "lbm_batch_set_body_force", "lbm_batch_save", "lbm_critical_pressure_batch",
                 "lbm_batch_kernel_info"):
        getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, handle=None):
    if rc != LBM_OK:
        msg = library().lbm_last_error(handle)
        raise LbmError(rc, (msg or b"").decode())
    return rc


VARIANTS = {"auto": 0, "simple": 1, "staged": 2, "pipelined": 3, "private": 4, "persistent": 5}
COLLISIONS = {"bgk": 0, "regularized": 1}


def make_params(nx, ny, tau=(1.0, 1.0), G=0.0, rho_wall=(0.0, 0.0), g=(0.0, 0.0),
                periodic=(True, True), precision="fp32", eq_order=3, stream=None,
                workspace=None, workspace_bytes=0, variant="auto", collision="bgk") -> Params:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    col = COLLISIONS[collision] if isinstance(collision, str) else int(collision)
    return Params(int(nx), int(ny), int(periodic[0]), int(periodic[1]),
                  (ctypes.c_double * 2)(*tau), float(G), (ctypes.c_double * 2)(*rho_wall),
                  (ctypes.c_double * 2)(*g), prec, int(eq_order), var, col,
                  ctypes.c_void_p(stream) if stream else None,
                  ctypes.c_void_p(workspace) if workspace else None, int(workspace_bytes))


def lbm_workspace_size(params: Params) -> int:
    out = ctypes.c_size_t(0)
    _check(library().lbm_workspace_size(ctypes.byref(params), ctypes.byref(out)))
    return out.value


def lbm_create(mask, rho_init, params: Params) -> int:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    rho = np.ascontiguousarray(rho_init, dtype=np.float64)
    if mask.shape != (params.ny, params.nx) or rho.shape != (2, params.ny, params.nx):
        raise ValueError("mask must be [ny, nx] and rho_init [2, ny, nx]")
    h = ctypes.c_void_p()
    _check(library().lbm_create(mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dptr(rho),
                                ctypes.byref(params), ctypes.byref(h)))
    return h.value


def lbm_step(h, nsteps: int):
    _check(library().lbm_step(h, int(nsteps)), h)


def lbm_observables(h, check=True) -> dict:
    o = Obs()
    rc = library().lbm_observables(h, ctypes.byref(o))
    if check:
        _check(rc, h)
    d = o.as_dict()
    d["status"] = rc
    return d


def lbm_get_fields(h, nx, ny, out=None):
    """(rho [2, ny, nx], u [2, ny, nx], p [ny, nx]) as float64; `out` may
    supply the three arrays (C-contiguous float64, e.g. in pinned memory)."""
    if out is None:
        out = (np.empty((2, ny, nx)), np.empty((2, ny, nx)), np.empty((ny, nx)))
    rho, u, p = out
    for a, shape in ((rho, (2, ny, nx)), (u, (2, ny, nx)), (p, (ny, nx))):
        if a.shape != shape or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"lbm_get_fields: expected a C-contiguous float64 array of shape {shape}")
    _check(library().lbm_get_fields(h, _dptr(rho), _dptr(u), _dptr(p)), h)
    return rho, u, p


def lbm_set_body_force(h, gx, gy=0.0):
    _check(library().lbm_set_body_force(h, float(gx), float(gy)), h)


def lbm_save(h, nx, ny):
    f = np.empty((2, 9, ny, nx))
    _check(library().lbm_save(h, _dptr(f)), h)
    return f


def lbm_load(h, f, nx, ny):
    """Load populations f [2, 9, ny, nx] (the C call reads exactly that many
    values, so the shape is checked here)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.shape != (2, 9, ny, nx):
        raise ValueError(f"lbm_load: expected populations of shape {(2, 9, ny, nx)}, got {f.shape}")
    _check(library().lbm_load(h, _dptr(f)), h)


def lbm_wait_selftest(stream=None):
    """Run the bounded device wait on a barrier nothing completes; returns
    (status, seconds): LBM_ETIMEOUT when the wait gave up as it must."""
    sec = ctypes.c_double(0.0)
    rc = library().lbm_wait_selftest(ctypes.c_void_p(stream) if stream else None, ctypes.byref(sec))
    return rc, sec.value


def lbm_kernel_info(h) -> dict:
    info = (ctypes.c_int32 * 5)()
    _check(library().lbm_kernel_info(h, info), h)
    if info[0] == 1:
        return {"variant": "simple", "rows_per_cta": info[2]}
    if info[0] == 5:
        return {"variant": "persistent", "rows_per_tile": info[2], "ctas": info[3]}
    d = {"variant": {2: "staged", 3: "pipelined", 4: "private"}[info[0]], "depth": info[1], "cols_per_cta": info[2],
         "strips": info[3]}
    if info[0] == 2:
        d["strip_rows"] = "absolute" if info[4] else "per block"
    return d


def lbm_destroy(h):
    if h:
        library().lbm_destroy(h)


def lbm_last_error(h=None) -> str:
    return (library().lbm_last_error(h) or b"").decode()


class Simulation:
    """Owning wrapper: device arena from PyTorch, work on torch's current stream."""

    def __init__(self, mask, rho_init, tau=(1.0, 1.0), G=0.0, rho_wall=(0.0, 0.0),
                 g=(0.0, 0.0), periodic=(True, True), precision="fp32", eq_order=3,
                 device=0, use_torch_arena=True, variant="auto", collision="bgk"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.ny, self.nx = mask.shape
        self.device = torch.device("cuda", device)
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            p = make_params(self.nx, self.ny, tau, G, rho_wall, g, periodic, precision, eq_order,
                            stream=stream, variant=variant, collision=collision)
            self._arena = None
            if use_torch_arena:
                nbytes = lbm_workspace_size(p)
                self._arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
                base = self._arena.data_ptr()
                aligned = (base + 255) // 256 * 256
                p.workspace = ctypes.c_void_p(aligned)
                p.workspace_bytes = nbytes
            self.params = p
            self.h = lbm_create(mask, rho_init, p)

    def step(self, n=1):
        lbm_step(self.h, n)

    def observables(self, check=True):
        return lbm_observables(self.h, check)

    def fields(self):
        return lbm_get_fields(self.h, self.nx, self.ny)

    def kernel_info(self):
        return lbm_kernel_info(self.h)

    def set_body_force(self, gx, gy=0.0):
        lbm_set_body_force(self.h, gx, gy)

    def save(self):
        return lbm_save(self.h, self.nx, self.ny)

    def load(self, f):
        lbm_load(self.h, f, self.nx, self.ny)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# batches and the critical body force
# ----------------------------------------------------------------------------
def _bcheck(rc, b=None):
    if rc != LBM_OK:
        msg = library().lbm_batch_last_error(b)
        raise LbmError(rc, (msg or b"").decode())
    return rc


def _collision_code(c):
    return COLLISIONS[c] if isinstance(c, str) else int(c)


def lbm_batch_create(instances, precision="fp32", eq_order=3, stream=None):
    """instances: list of dicts with mask [ny, nx], rho_init [2, ny, nx], tau, G,
    rho_wall, g, periodic, disp_threshold, collision ("bgk" or "regularized")."""
    keep = []
    arr = (Instance * len(instances))()
    for k, d in enumerate(instances):
        mask = np.ascontiguousarray(d["mask"], dtype=np.uint8)
        rho = np.ascontiguousarray(d["rho_init"], dtype=np.float64)
        ny, nx = mask.shape
        if rho.shape != (2, ny, nx):
            raise ValueError(f"instance {k}: rho_init must have shape {(2, ny, nx)}, got {rho.shape}")
        keep += [mask, rho]
        per = d.get("periodic", (True, False))
        arr[k] = Instance(nx, ny, int(per[0]), int(per[1]), (ctypes.c_double * 2)(*d.get("tau", (1.0, 1.0))),
                          float(d.get("G", 0.0)), (ctypes.c_double * 2)(*d.get("rho_wall", (0.0, 0.0))),
                          (ctypes.c_double * 2)(*d.get("g", (0.0, 0.0))),
                          mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dptr(rho),
                          float(d.get("disp_threshold", 0.0)), _collision_code(d.get("collision", "bgk")))
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    h = ctypes.c_void_p()
    _bcheck(library().lbm_batch_create(arr, len(instances), prec, int(eq_order),
                                       ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
    return h.value


def lbm_batch_step(b, nsteps):
    _bcheck(library().lbm_batch_step(b, int(nsteps)), b)


def lbm_batch_observables(b, n, check=True):
    out = (Obs * n)()
    rc = library().lbm_batch_observables(b, out)
    if check:
        _bcheck(rc, b)
    return [o.as_dict() for o in out]


def _per_instance(values, n, name):
    """values as a C-contiguous float64 array of exactly n entries (the C
    calls read, and write results for, every instance of the batch)."""
    v = np.ascontiguousarray(values, dtype=np.float64).ravel()
    if n is not None and v.shape != (n,):
        raise ValueError(f"{name}: expected {n} values, one per instance, got {v.shape[0]}")
    return v


def lbm_batch_set_body_force(b, gx, n=None):
    gx = _per_instance(gx, n, "lbm_batch_set_body_force")
    _bcheck(library().lbm_batch_set_body_force(b, _dptr(gx)), b)


def lbm_batch_save(b, i, nx, ny):
    f = np.empty((2, 9, ny, nx))
    _bcheck(library().lbm_batch_save(b, int(i), _dptr(f)), b)
    return f


def lbm_batch_kernel_info(b) -> dict:
    info = (ctypes.c_int32 * 3)()
    _bcheck(library().lbm_batch_kernel_info(b, info), b)
    return {"variant": {1: "register-pull", 2: "staged"}[info[0]], "strip_rows": info[1], "ctas_per_step": info[2]}


def lbm_critical_pressure_batch(b, g_lo, g_hi, rel_bracket=0.02, t_eq=1000, t_obs=2000, max_probes=24,
                                check_bracket=True, timeout_s=0.0, check=True, n=None):
    g_lo = _per_instance(g_lo, n, "lbm_critical_pressure_batch")
    g_hi = _per_instance(g_hi, len(g_lo), "lbm_critical_pressure_batch")
    n = len(g_lo)
    out = (CritResult * n)()
    o = BisectOpts(float(rel_bracket), int(t_eq), int(t_obs), int(max_probes), int(bool(check_bracket)),
                   float(timeout_s))
    rc = library().lbm_critical_pressure_batch(b, _dptr(g_lo), _dptr(g_hi), ctypes.byref(o), out)
    if check and rc not in (LBM_OK,):
        _bcheck(rc, b)
    return [{"g_lo": r.g_lo, "g_hi": r.g_hi, "probes": r.probes, "status": r.status} for r in out]


def lbm_batch_destroy(b):
    if b:
        library().lbm_batch_destroy(b)


class Batch:
    """Owning wrapper of a batch; work on torch's current stream."""

    def __init__(self, instances, precision="fp32", eq_order=3, device=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.n = len(instances)
        self.shapes = [np.asarray(d["mask"]).shape for d in instances]
        with torch.cuda.device(device):
            stream = torch.cuda.current_stream().cuda_stream
            self.h = lbm_batch_create(instances, precision, eq_order, stream)

    def step(self, n=1):
        lbm_batch_step(self.h, n)

    def observables(self, check=True):
        return lbm_batch_observables(self.h, self.n, check)

    def set_body_force(self, gx):
        lbm_batch_set_body_force(self.h, gx, self.n)

    def save(self, i):
        ny, nx = self.shapes[i]
        return lbm_batch_save(self.h, i, nx, ny)

    def kernel_info(self):
        return lbm_batch_kernel_info(self.h)

    def critical_pressure(self, g_lo, g_hi, **opts):
        return lbm_critical_pressure_batch(self.h, g_lo, g_hi, n=self.n, **opts)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# surrogate network
# ----------------------------------------------------------------------------
MLP_PARAMS = 34050


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _mcheck(rc):
    if rc != LBM_OK:
        raise LbmError(rc, (library().lbm_mlp_last_error() or b"").decode())


def _mlp_params(p):
    p = np.ascontiguousarray(p, dtype=np.float32).ravel()
    if p.shape != (MLP_PARAMS,):
        raise ValueError(f"surrogate: expected {MLP_PARAMS} parameters, got {p.shape[0]}")
    return p


def _mlp_data(x, y=None):
    """Features x [B, 5] and targets y [B] as the C calls read them."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim != 2 or x.shape[1] != 5 or x.shape[0] < 1:
        raise ValueError(f"surrogate: features must have shape (B, 5), B >= 1, got {x.shape}")
    if y is None:
        return x
    y = np.ascontiguousarray(y, dtype=np.float32).ravel()
    if y.shape != (x.shape[0],):
        raise ValueError(f"surrogate: {x.shape[0]} feature rows but {y.shape[0]} targets")
    return x, y


class Surrogate:
    """The 5 -> 128 -> 128 -> 128 -> 2 network on the device (C ABI lbm_mlp_*)."""

    def __init__(self, params=None, seed=0, stream=None):
        h = ctypes.c_void_p()
        p = None if params is None else _mlp_params(params)
        _mcheck(library().lbm_mlp_create(_fptr(p) if p is not None else None, int(seed),
                                         ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self.h = h.value

    def params(self):
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        _mcheck(library().lbm_mlp_params(self.h, _fptr(out), None))
        return out

    def set_params(self, p):
        p = _mlp_params(p)
        _mcheck(library().lbm_mlp_params(self.h, None, _fptr(p)))

    def forward(self, x):
        x = _mlp_data(x)
        out = np.empty((x.shape[0], 2), dtype=np.float32)
        _mcheck(library().lbm_mlp_forward(self.h, _fptr(x), x.shape[0], _fptr(out)))
        return out

    def loss_grad(self, x, y):
        x, y = _mlp_data(x, y)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        _mcheck(library().lbm_mlp_loss_grad(self.h, _fptr(x), _fptr(y), x.shape[0], _fptr(loss), _fptr(g)))
        return float(loss[0]), g

    def adam(self, lr):
        _mcheck(library().lbm_mlp_adam(self.h, float(lr)))

    def train(self, x, y, epochs, batch=256, lr=1e-3, seed=0):
        x, y = _mlp_data(x, y)
        loss = np.zeros(1, dtype=np.float32)
        _mcheck(library().lbm_mlp_train(self.h, _fptr(x), _fptr(y), x.shape[0], int(epochs), int(batch),
                                        float(lr), int(seed), _fptr(loss)))
        return float(loss[0])

    def close(self):
        if getattr(self, "h", None):
            library().lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# the paper's question from channel descriptions (Sections 3.1, 3.3, 3.4)
# ----------------------------------------------------------------------------
def _ccheck(rc, ok=(LBM_OK,)):
    if rc not in ok:
        raise LbmError(rc, (library().lbm_channel_last_error() or b"").decode())
    return rc


def channel_spec(spec) -> ChannelSpec:
    """C struct of a channel description (any object with lam, amp_ratio,
    slug_len_over_lambda, theta_deg, visc_ratio and optionally n_periods,
    n_slugs)."""
    return ChannelSpec(int(spec.lam), float(spec.amp_ratio), float(spec.slug_len_over_lambda),
                       float(spec.theta_deg), float(spec.visc_ratio), int(getattr(spec, "n_periods", 4)),
                       int(getattr(spec, "n_slugs", 1)))


def lbm_channel_geometry(spec):
    """(mask [ny, nx] uint8, rho_init [2, ny, nx]) of a channel with its slug."""
    cs = channel_spec(spec)
    nx, ny = ctypes.c_int32(), ctypes.c_int32()
    _ccheck(library().lbm_channel_shape(ctypes.byref(cs), ctypes.byref(nx), ctypes.byref(ny)))
    mask = np.empty((ny.value, nx.value), dtype=np.uint8)
    rho = np.empty((2, ny.value, nx.value))
    _ccheck(library().lbm_channel_geometry(ctypes.byref(cs), mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                           _dptr(rho)))
    return mask, rho


def lbm_wetting_calibrate(r_values, steps=20000, precision="fp32", stream=None):
    r = np.ascontiguousarray(r_values, dtype=np.float64).ravel()
    theta = np.empty_like(r)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _ccheck(library().lbm_wetting_calibrate(_dptr(r), len(r), int(steps), prec,
                                            ctypes.c_void_p(stream) if stream else None, _dptr(theta)))
    return theta


def lbm_surface_tension(steps=6000, precision="fp32", stream=None):
    sigma, rho = ctypes.c_double(), ctypes.c_double()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _ccheck(library().lbm_surface_tension(int(steps), prec, ctypes.c_void_p(stream) if stream else None,
                                          ctypes.byref(sigma), ctypes.byref(rho)))
    return sigma.value, rho.value


def lbm_planar_critical_balance(theta_deg, area, h0, amp, lam, x_rest):
    out = ctypes.c_double()
    _ccheck(library().lbm_planar_critical_balance(float(theta_deg), float(area), float(h0), float(amp),
                                                  float(lam), float(x_rest), ctypes.byref(out)))
    return out.value


def lbm_planar_critical_balance_hysteresis(theta_front, theta_rear, area, h0, amp, lam, x_rest):
    out = ctypes.c_double()
    _ccheck(library().lbm_planar_critical_balance_hysteresis(float(theta_front), float(theta_rear), float(area),
                                                             float(h0), float(amp), float(lam), float(x_rest),
                                                             ctypes.byref(out)))
    return out.value


def _densities(rho, name):
    """rho as a C-contiguous float64 [2, ny, nx] array, and (ny, nx): the C
    calls read both species' planes, so the shape is checked here."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.ndim != 3 or rho.shape[0] != 2:
        raise ValueError(f"{name}: densities must have shape (2, ny, nx), got {rho.shape}")
    return rho, rho.shape[1], rho.shape[2]


def lbm_meniscus_angles(rho, h0, amp, lam):
    """{theta_rear, theta_front, x_rear, x_front, r_rear, r_front} of a slug
    in the planar sinusoidal channel (lbm_meniscus_angles)."""
    rho, ny, nx = _densities(rho, "lbm_meniscus_angles")
    out = np.zeros(6)
    _ccheck(library().lbm_meniscus_angles(_dptr(rho), nx, ny, float(h0), float(amp), float(lam), _dptr(out)))
    return dict(zip(("theta_rear", "theta_front", "x_rear", "x_front", "r_rear", "r_front"), out.tolist()))


def lbm_contact_angle(rho, y_lo, y_hi, right=True):
    rho, ny, nx = _densities(rho, "lbm_contact_angle")
    out = ctypes.c_double()
    _ccheck(library().lbm_contact_angle(_dptr(rho), nx, ny, int(y_lo), int(y_hi), int(bool(right)),
                                        ctypes.byref(out)))
    return out.value


def lbm_slug_area(rho, mask):
    """(oil-rich nodes, the paper's bulk + 90 % interface count) of a slug."""
    rho, ny, nx = _densities(rho, "lbm_slug_area")
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    if mask.shape != (ny, nx):
        raise ValueError(f"lbm_slug_area: mask must have shape {(ny, nx)}, got {mask.shape}")
    out = (ctypes.c_double * 2)()
    _ccheck(library().lbm_slug_area(_dptr(rho), mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nx, ny, out))
    return out[0], out[1]


def lbm_wall_potentials(r, theta, theta_deg):
    r = np.ascontiguousarray(r, dtype=np.float64).ravel()
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    if th.shape != r.shape:
        raise ValueError(f"lbm_wall_potentials: {len(r)} potentials but {len(th)} angles")
    out = (ctypes.c_double * 2)()
    _ccheck(library().lbm_wall_potentials(_dptr(r), _dptr(th), len(r), float(theta_deg), out))
    return (out[0], out[1])


def lbm_critical_pressure_channels(specs, precision="fp32", collision="regularized", rel_bracket=0.02,
                                   t_eq=1000, t_obs=2000, max_probes=24, surrogate=None, feature_mean=None,
                                   feature_std=None, k_sigma=2.0, bracket=(0.5, 2.0), table=None, sigma=0.0,
                                   rho_bulk=0.0, timeout_s=0.0, stream=None, check=True):
    """Bisect the critical body force of every channel description inside
    the library; returns a list of result dicts (lbm_channel_result)."""
    n = len(specs)
    arr = (ChannelSpec * n)(*[channel_spec(s) for s in specs])
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o = ChannelOpts()
    o.rel_bracket = float(rel_bracket)
    o.t_eq, o.t_obs, o.max_probes = int(t_eq), int(t_obs), int(max_probes)
    o.precision, o.collision = prec, _collision_code(collision)
    keep = []
    if surrogate is not None:
        o.use_surrogate = 1
        o.surrogate = surrogate.h
        o.feature_mean = (ctypes.c_float * 5)(*[float(v) for v in feature_mean])
        o.feature_std = (ctypes.c_float * 5)(*[float(v) for v in feature_std])
        o.k_sigma = float(k_sigma)
    o.bracket_lo, o.bracket_hi = float(bracket[0]), float(bracket[1])
    if table is not None:
        r = np.ascontiguousarray(table.r, dtype=np.float64)
        th = np.ascontiguousarray(table.theta, dtype=np.float64)
        keep += [r, th]
        o.calib_r, o.calib_theta, o.calib_n = _dptr(r), _dptr(th), len(r)
    o.sigma, o.rho_bulk = float(sigma), float(rho_bulk)
    o.timeout_s = float(timeout_s)
    o.cuda_stream = stream
    out = (ChannelResult * n)()
    rc = library().lbm_critical_pressure_channels(arr, n, ctypes.byref(o), out)
    if check:
        _ccheck(rc, ok=(LBM_OK, LBM_ETIMEOUT))
    return [r.as_dict() for r in out]


# ----------------------------------------------------------------------------
# the D3Q19 step (lbm3d_*)
# ----------------------------------------------------------------------------
def _check3(rc, h=None, ok=(LBM_OK,)):
    if rc not in ok:
        raise LbmError(rc, (library().lbm3d_last_error(h) or b"").decode())
    return rc


class Simulation3:
    """Owning wrapper of an lbm3d handle on torch's current stream.  mask
    [nz, ny, nx] (1 = solid), rho_init [2, nz, ny, nx]."""

    def __init__(self, mask, rho_init, tau=(1.0, 1.0), G=0.0, rho_wall=(0.0, 0.0), g=(0.0, 0.0, 0.0),
                 periodic=(True, True, True), precision="fp64", eq_order=3, collision="bgk", device=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        rho = np.ascontiguousarray(rho_init, dtype=np.float64)
        self.nz, self.ny, self.nx = mask.shape
        if rho.shape != (2,) + mask.shape:
            raise ValueError(f"rho_init must have shape {(2,) + mask.shape}, got {rho.shape}")
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        with torch.cuda.device(device):
            stream = torch.cuda.current_stream().cuda_stream
        p = Params3(self.nx, self.ny, self.nz, (ctypes.c_int32 * 3)(*[int(v) for v in periodic]),
                    (ctypes.c_double * 2)(*tau), float(G), (ctypes.c_double * 2)(*rho_wall),
                    (ctypes.c_double * 3)(*g), prec, int(eq_order), _collision_code(collision),
                    ctypes.c_void_p(stream) if stream else None)
        h = ctypes.c_void_p()
        _check3(library().lbm3d_create(mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dptr(rho),
                                       ctypes.byref(p), ctypes.byref(h)))
        self.h = h.value

    def step(self, n=1):
        _check3(library().lbm3d_step(self.h, int(n)), self.h)

    def observables(self, check=True):
        o = Obs()
        rc = library().lbm3d_observables(self.h, ctypes.byref(o))
        if check:
            _check3(rc, self.h)
        return o.as_dict()

    def fields(self):
        rho = np.empty((2, self.nz, self.ny, self.nx))
        u = np.empty((3, self.nz, self.ny, self.nx))
        _check3(library().lbm3d_get_fields(self.h, _dptr(rho), _dptr(u)), self.h)
        return rho, u

    def save(self):
        f = np.empty((2, 19, self.nz, self.ny, self.nx))
        _check3(library().lbm3d_save(self.h, _dptr(f)), self.h)
        return f

    def load(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (2, 19, self.nz, self.ny, self.nx):
            raise ValueError(f"load: expected populations of shape {(2, 19, self.nz, self.ny, self.nx)}, "
                             f"got {f.shape}")
        _check3(library().lbm3d_load(self.h, _dptr(f)), self.h)

    def close(self):
        if getattr(self, "h", None):
            library().lbm3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
