"""GB300 (sm_103a) coupled thermal lattice Boltzmann step for liquid-vapor
phase change (Wang, Huang & He, arXiv 2205.00686).

Thin Python binding of the C ABI in ``include/lbm.h``: the functions keep the
ABI's names and only marshal arguments; every step of the method runs in the
CUDA library ``liblbm_gb300.so`` built from ``csrc/``.  There is no CPU
fallback: if the library is missing or cannot load, every call raises.

Host arrays are float64 ``[ny][nx]`` fields or ``[q][ny][nx]`` populations,
as numpy arrays or CPU torch tensors (pinned tensors make the copies
asynchronous-capable DMA).  Streams are passed as raw ``cudaStream_t``
handles, e.g. ``torch.cuda.Stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ENONFINITE, LBM_EPSI, LBM_ECUDA, LBM_EIO, LBM_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
LBM_ETOOBIG = -8
LBM_ETIMEOUT = -9
LBM_NOALLOC_MAX_NODES = 33554432
LBM_FP64, LBM_FP32, LBM_FP32_G16 = 0, 1, 2
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp32_g16": LBM_FP32_G16}
LBM_PERIODIC, LBM_WALL, LBM_OPEN = 0, 1, 2
LBM_T_PERIODIC, LBM_T_DIRICHLET, LBM_T_ADIABATIC = 0, 1, 2

# every symbol include/lbm.h declares
ABI_FUNCTIONS = (
    "lbm_default_params", "lbm_state_bytes", "lbm_create", "lbm_init_fields", "lbm_step",
    "lbm_get_rho_u_T", "lbm_diagnostics", "lbm_get_populations", "lbm_set_populations",
    "lbm_step_count", "lbm_sync", "lbm_save", "lbm_load", "lbm_destroy", "lbm_last_error",
    "lbm_set_target",
    "lbm_batch_create", "lbm_batch_attach", "lbm_batch_detach", "lbm_batch_size",
    "lbm_batch_step", "lbm_batch_sync", "lbm_batch_destroy", "lbm_batch_autotune",
    "lbm_batch_errors_async",
    "lbm_batch_get_tile", "lbm_set_tile", "lbm_get_tile",
    "lbm_autotune", "lbm_set_staging", "lbm_get_staging", "lbm_set_wait_probe",
    "lbm_diag_reduce_noalloc", "lbm_reconfigure", "lbm_contact_angle",
    "lbm_regions", "lbm_rows_bytes", "lbm_pack_rows", "lbm_unpack_rows", "lbm_set_partition",
    "lbm_mass_ring",
    # include/lbm3d.h
    "lbm3d_state_bytes", "lbm3d_create", "lbm3d_init_fields", "lbm3d_step", "lbm3d_get_fields",
    "lbm3d_get_populations", "lbm3d_diagnostics", "lbm3d_set_path", "lbm3d_get_path",
    "lbm3d_step_count", "lbm3d_sync",
    "lbm3d_destroy", "lbm3d_last_error",
)


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__("lbm error %d%s" % (code, (": " + msg) if msg else ""))
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "a", "b", "R", "omega", "G", "sigma", "nu", "s0", "s_e", "s_eps", "s_j", "s_q",
        "lambda_", "cv", "w_dot", "vs0", "vs3", "vs4", "gravity", "rho_ref", "T_ref")] + [
        ("frozen_flow", ctypes.c_int), ("frozen_thermal", ctypes.c_int)]


class lbm_bc(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int * 4), ("therm", ctypes.c_int * 4),
                ("T_edge", ctypes.c_double * 4), ("theta_deg", ctypes.c_double),
                ("heater_x0", ctypes.c_int), ("heater_x1", ctypes.c_int),
                ("T_heater", ctypes.c_double)]


class lbm_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "mass", "energy", "liquid_mass", "liquid_area", "liquid_area_smooth",
        "diameter", "diameter_smooth", "max_u")] + [
        ("step", ctypes.c_longlong), ("nonfinite", ctypes.c_int)]


class lbm_contact(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "theta_deg", "xc", "yc", "radius", "base_width", "height")] + [
        ("n_points", ctypes.c_int)]


class lbm3d_bc(ctypes.Structure):
    _fields_ = [("flow_z", ctypes.c_int), ("therm", ctypes.c_int * 2),
                ("T_edge", ctypes.c_double * 2), ("theta_deg", ctypes.c_double)]


class lbm_region(ctypes.Structure):
    _fields_ = [("label", ctypes.c_longlong), ("area", ctypes.c_longlong),
                ("sum_y", ctypes.c_longlong), ("y_min", ctypes.c_int), ("y_max", ctypes.c_int),
                ("touches_w", ctypes.c_int), ("touches_e", ctypes.c_int),
                ("touches_s", ctypes.c_int), ("touches_n", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    """The loaded CUDA library (raises if it is missing or cannot load)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("CUDA library %s is missing; run __graft_entry__.build() or "
                              "python -m paper_2205_00686_gb300._build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, B, D = ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_bc), ctypes.POINTER(lbm_diag)
        sig = {
            "lbm_default_params": ([P], ctypes.c_int),
            "lbm_state_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
            "lbm_create": ([ctypes.c_int, ctypes.c_int, P, B, ctypes.c_int, _vp, _vp,
                            ctypes.c_size_t, ctypes.POINTER(_vp)], ctypes.c_int),
            "lbm_init_fields": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
            "lbm_step": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm_get_rho_u_T": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
            "lbm_diagnostics": ([_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, D],
                                ctypes.c_int),
            "lbm_get_populations": ([_vp, _vp, _vp, _vp], ctypes.c_int),
            "lbm_set_populations": ([_vp, _vp, _vp, _vp, ctypes.c_longlong, ctypes.c_double],
                                    ctypes.c_int),
            "lbm_step_count": ([_vp], ctypes.c_longlong),
            "lbm_set_target": ([_vp, ctypes.c_longlong], ctypes.c_int),
            "lbm_sync": ([_vp], ctypes.c_int),
            "lbm_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
            "lbm_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
            "lbm_destroy": ([_vp], None),
            "lbm_last_error": ([_vp], ctypes.c_char_p),
            "lbm_batch_create": ([_vp, ctypes.POINTER(_vp)], ctypes.c_int),
            "lbm_batch_attach": ([_vp, _vp], ctypes.c_int),
            "lbm_batch_detach": ([_vp, _vp], ctypes.c_int),
            "lbm_batch_size": ([_vp], ctypes.c_int),
            "lbm_batch_step": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm_batch_sync": ([_vp], ctypes.c_int),
            "lbm_batch_errors_async": ([_vp, _vp], ctypes.c_int),
            "lbm_batch_destroy": ([_vp], None),
            "lbm_batch_autotune": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm_batch_get_tile": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "lbm_set_tile": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "lbm_get_tile": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                             ctypes.c_int),
            "lbm_autotune": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm_set_staging": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm_get_staging": ([_vp], ctypes.c_int),
            "lbm_set_wait_probe": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm_diag_reduce_noalloc": ([_vp, _vp, _vp, _vp, ctypes.c_longlong, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, _vp, _vp],
                                        ctypes.c_int),
            "lbm_reconfigure": ([_vp, P, B], ctypes.c_int),
            "lbm_rows_bytes": ([_vp, ctypes.c_int], ctypes.c_size_t),
            "lbm_pack_rows": ([_vp, ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
            "lbm_unpack_rows": ([_vp, ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
            "lbm_set_partition": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong],
                                  ctypes.c_int),
            "lbm_mass_ring": ([_vp, ctypes.POINTER(_vp)], ctypes.c_int),
            "lbm_contact_angle": ([_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(lbm_contact)], ctypes.c_int),
            "lbm_regions": ([_vp, ctypes.c_double, ctypes.c_int, _vp,
                             ctypes.POINTER(lbm_region), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "lbm3d_state_bytes": ([ctypes.c_int] * 4, ctypes.c_size_t),
            "lbm3d_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                              ctypes.POINTER(lbm3d_bc), ctypes.c_int, _vp, ctypes.POINTER(_vp)],
                             ctypes.c_int),
            "lbm3d_init_fields": ([_vp] * 6, ctypes.c_int),
            "lbm3d_step": ([_vp, ctypes.c_int], ctypes.c_int),
            "lbm3d_get_fields": ([_vp] * 6, ctypes.c_int),
            "lbm3d_get_populations": ([_vp] * 4, ctypes.c_int),
            "lbm3d_diagnostics": ([_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, D],
                                  ctypes.c_int),
            "lbm3d_set_path": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "lbm3d_get_path": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                               ctypes.c_int),
            "lbm3d_step_count": ([_vp], ctypes.c_longlong),
            "lbm3d_sync": ([_vp], ctypes.c_int),
            "lbm3d_destroy": ([_vp], None),
            "lbm3d_last_error": ([_vp], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(a):
    """Address of a host float64 array (numpy or CPU torch tensor), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("expected a C-contiguous float64 array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.is_cuda:
            raise TypeError("expected a contiguous float64 CPU tensor")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def make_params(d: dict) -> lbm_params:
    p = lbm_params()
    lib().lbm_default_params(ctypes.byref(p))
    for k, v in d.items():
        name = "lambda_" if k == "lambda" else k
        if any(name == f[0] for f in lbm_params._fields_):
            setattr(p, name, v)
    return p


def make_bc(d: dict) -> lbm_bc:
    b = lbm_bc()
    for e in range(4):
        b.flow[e] = int(d["flow"][e])
        b.therm[e] = int(d["therm"][e])
        b.T_edge[e] = float(d.get("T_edge", (0.0,) * 4)[e])
    b.theta_deg = float(d.get("theta_deg", 90.0))
    b.heater_x0 = int(d.get("heater_x0", 0))
    b.heater_x1 = int(d.get("heater_x1", 0))
    b.T_heater = float(d.get("T_heater", 0.0))
    return b


def _check(rc, ctx=None):
    if rc != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(rc, msg)
    return rc


def lbm_state_bytes(nx: int, ny: int, prec) -> int:
    return int(lib().lbm_state_bytes(nx, ny, PRECISIONS.get(prec, prec)))


class Domain:
    """One simulation context (``lbm_ctx``)."""

    def __init__(self, nx: int, ny: int, params: dict, bc: dict, prec="fp32", stream=None,
                 device_mem=None, device_bytes=0):
        self.nx, self.ny = int(nx), int(ny)
        self.prec = PRECISIONS.get(prec, prec)
        self._p = make_params(params)
        self._b = make_bc(bc)
        h = _vp()
        _check(lib().lbm_create(self.nx, self.ny, ctypes.byref(self._p), ctypes.byref(self._b),
                                self.prec, stream, device_mem, int(device_bytes),
                                ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f(self, a):
        return a if a is None or hasattr(a, "data_ptr") else np.ascontiguousarray(a, np.float64)

    def init_fields(self, rho, ux, uy, T):
        arrs = [self._f(a) for a in (rho, ux, uy, T)]
        _check(lib().lbm_init_fields(self._h, *[_ptr(a) for a in arrs]), self._h)

    def step(self, n: int = 1):
        _check(lib().lbm_step(self._h, int(n)), self._h)

    def sync(self):
        return _check(lib().lbm_sync(self._h), self._h)

    def get_rho_u_T(self, out=None):
        out = out or tuple(np.empty((self.ny, self.nx)) for _ in range(4))
        _check(lib().lbm_get_rho_u_T(self._h, *[_ptr(a) for a in out]), self._h)
        return out

    def diagnostics(self, rho_l, rho_g, sessile=False) -> dict:
        d = lbm_diag()
        _check(lib().lbm_diagnostics(self._h, rho_l, rho_g, int(sessile), ctypes.byref(d)),
               self._h)
        return {k: getattr(d, k) for k, _ in lbm_diag._fields_}

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, self.ny, self.nx))
        P = np.empty((self.ny, self.nx))
        _check(lib().lbm_get_populations(self._h, _ptr(f), _ptr(g), _ptr(P)), self._h)
        return f, g, P

    def set_populations(self, f, g, P, step: int, rho_ave_prev: float):
        f, g, P = (np.ascontiguousarray(a, np.float64) for a in (f, g, P))
        _check(lib().lbm_set_populations(self._h, _ptr(f), _ptr(g), _ptr(P), int(step),
                                         float(rho_ave_prev)), self._h)

    @property
    def step_count(self) -> int:
        return int(lib().lbm_step_count(self._h))

    def save(self, path: str):
        _check(lib().lbm_save(self._h, path.encode()), self._h)

    def load(self, path: str):
        _check(lib().lbm_load(self._h, path.encode()), self._h)

    def set_tile(self, threads: int, rows: int):
        _check(lib().lbm_set_tile(self._h, threads, rows), self._h)

    def tile(self):
        t, r = ctypes.c_int(), ctypes.c_int()
        lib().lbm_get_tile(self._h, ctypes.byref(t), ctypes.byref(r))
        return t.value, r.value

    def autotune(self, steps_per_trial: int = 10):
        _check(lib().lbm_autotune(self._h, steps_per_trial), self._h)
        return self.tile()

    @property
    def staged(self) -> bool:
        """True when the FP32 step brings its rows in by bulk asynchronous
        copies (see lbm_set_staging)."""
        return lib().lbm_get_staging(self._h) == 1

    @staged.setter
    def staged(self, on: bool):
        _check(lib().lbm_set_staging(self._h, 1 if on else 0), self._h)

    def set_wait_probe(self, on: bool):
        """Test hook: staged launches also wait on an mbarrier nothing arms,
        so each CTA's bounded wait runs out and LBM_ETIMEOUT is reported."""
        _check(lib().lbm_set_wait_probe(self._h, 1 if on else 0), self._h)

    @property
    def last_error(self) -> str:
        return lib().lbm_last_error(self._h).decode()

    def set_target(self, target: int):
        """Stop at step count `target` (0: no stop); see lbm_set_target."""
        _check(lib().lbm_set_target(self._h, int(target)), self._h)

    # ---- slabs of one larger domain (lbm_rows_bytes ... lbm_mass_ring) ----
    def rows_bytes(self, n: int) -> int:
        return int(lib().lbm_rows_bytes(self._h, int(n)))

    def pack_rows(self, y0: int, n: int, dev_ptr: int):
        _check(lib().lbm_pack_rows(self._h, int(y0), int(n), ctypes.c_void_p(dev_ptr)), self._h)

    def unpack_rows(self, y0: int, n: int, dev_ptr: int):
        _check(lib().lbm_unpack_rows(self._h, int(y0), int(n), ctypes.c_void_p(dev_ptr)), self._h)

    def set_partition(self, own_y0: int, own_y1: int, global_nodes: int):
        _check(lib().lbm_set_partition(self._h, int(own_y0), int(own_y1), int(global_nodes)),
               self._h)

    def mass_ring(self) -> int:
        """Device address of the three-slot density-sum ring (doubles)."""
        p = _vp()
        _check(lib().lbm_mass_ring(self._h, ctypes.byref(p)), self._h)
        return int(p.value)

    def reconfigure(self, params: dict, bc: dict):
        """New params / boundary values for the following steps (flow boundary
        kinds and w_dot fixed)."""
        self._p = make_params(params)
        self._b = make_bc(bc)
        _check(lib().lbm_reconfigure(self._h, ctypes.byref(self._p), ctypes.byref(self._b)),
               self._h)

    def contact_angle(self, rho_l, rho_g, skip_rows: int = 3) -> dict:
        c = lbm_contact()
        _check(lib().lbm_contact_angle(self._h, rho_l, rho_g, int(skip_rows), ctypes.byref(c)),
               self._h)
        return {k: getattr(c, k) for k, _ in lbm_contact._fields_}

    def regions(self, threshold: float, below: bool = True, labels: bool = False,
                max_regions: int = 4096):
        """Regions of the phase rho < threshold (below) or rho > threshold, as
        a list of dicts sorted by label, plus the label field if asked."""
        lab = np.empty((self.ny, self.nx), dtype=np.int32) if labels else None
        n = ctypes.c_int(0)
        buf = (lbm_region * max(int(max_regions), 1))()
        _check(lib().lbm_regions(self._h, float(threshold), int(bool(below)),
                                 lab.ctypes.data if lab is not None else None, buf,
                                 int(max_regions), ctypes.byref(n)), self._h)
        out = [{k: getattr(buf[i], k) for k, _ in lbm_region._fields_}
               for i in range(min(n.value, int(max_regions)))]
        return (out, lab) if labels else out

    def region_count(self, threshold: float, below: bool = True) -> int:
        n = ctypes.c_int(0)
        _check(lib().lbm_regions(self._h, float(threshold), int(bool(below)), None, None, 0,
                                 ctypes.byref(n)), self._h)
        return n.value


def _check3(rc, ctx):
    if rc != LBM_OK:
        raise LbmError(rc, lib().lbm3d_last_error(ctx).decode() if ctx else "")
    return rc


def lbm3d_state_bytes(nx: int, ny: int, nz: int, prec) -> int:
    return int(lib().lbm3d_state_bytes(nx, ny, nz, PRECISIONS.get(prec, prec)))


class Domain3:
    """One three-dimensional simulation context (``lbm3d_ctx``); host fields
    are float64 arrays [nz][ny][nx]."""

    def __init__(self, nx: int, ny: int, nz: int, params: dict, bc3: dict, prec="fp32",
                 stream=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.prec = PRECISIONS.get(prec, prec)
        self._p = make_params(params)
        b = lbm3d_bc()
        b.flow_z = int(bc3["flow_z"])
        for e in range(2):
            b.therm[e] = int(bc3["therm"][e])
            b.T_edge[e] = float(bc3.get("T_edge", (0.0, 0.0))[e])
        b.theta_deg = float(bc3.get("theta_deg", 90.0))
        self._b = b
        h = _vp()
        _check(lib().lbm3d_create(self.nx, self.ny, self.nz, ctypes.byref(self._p),
                                  ctypes.byref(self._b), self.prec, stream, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self):
        return (self.nz, self.ny, self.nx)

    def init_fields(self, rho, ux, uy, uz, T):
        arrs = [a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, np.float64)
                for a in (rho, ux, uy, uz, T)]
        _check3(lib().lbm3d_init_fields(self._h, *[_ptr(a) for a in arrs]), self._h)

    def step(self, n: int = 1):
        _check3(lib().lbm3d_step(self._h, int(n)), self._h)

    def sync(self):
        return _check3(lib().lbm3d_sync(self._h), self._h)

    def get_fields(self, out=None):
        out = out or tuple(np.empty(self._shape()) for _ in range(5))
        _check3(lib().lbm3d_get_fields(self._h, *[_ptr(a) for a in out]), self._h)
        return out

    def populations(self):
        f = np.empty((19,) + self._shape())
        g = np.empty((7,) + self._shape())
        P = np.empty(self._shape())
        _check3(lib().lbm3d_get_populations(self._h, _ptr(f), _ptr(g), _ptr(P)), self._h)
        return f, g, P

    def diagnostics(self, rho_l, rho_g, sessile=False) -> dict:
        d = lbm_diag()
        _check3(lib().lbm3d_diagnostics(self._h, rho_l, rho_g, int(sessile), ctypes.byref(d)),
                self._h)
        return {k: getattr(d, k) for k, _ in lbm_diag._fields_}

    def set_path(self, fused: bool = True, zseg: int = 0):
        """fused: one kernel per step over z-marching tiles (zseg planes per
        CTA, 0 = automatic); else three kernels per step."""
        _check3(lib().lbm3d_set_path(self._h, int(bool(fused)), int(zseg)), self._h)

    @property
    def path(self):
        f, z = ctypes.c_int(0), ctypes.c_int(0)
        _check3(lib().lbm3d_get_path(self._h, ctypes.byref(f), ctypes.byref(z)), self._h)
        return bool(f.value), int(z.value)

    @property
    def step_count(self) -> int:
        return int(lib().lbm3d_step_count(self._h))


def lbm_diag_reduce_noalloc(rho, ux, uy, T, n, cv, rho_l, rho_g, out7, stream=None) -> int:
    """Diagnostics sums of device field arrays without allocating (device
    pointers as ints, e.g. torch's data_ptr()); returns the ABI's code."""
    return int(lib().lbm_diag_reduce_noalloc(rho, ux, uy, T, int(n), float(cv), float(rho_l),
                                             float(rho_g), out7, stream))


class Batch:
    """Batched stepping of many domains (``lbm_batch``)."""

    def __init__(self, stream=None):
        h = _vp()
        _check(lib().lbm_batch_create(stream, ctypes.byref(h)))
        self._h = h
        self.members = []

    def attach(self, d: Domain):
        _check(lib().lbm_batch_attach(self._h, d.handle), d.handle)
        self.members.append(d)

    def detach(self, d: Domain):
        _check(lib().lbm_batch_detach(self._h, d.handle), d.handle)
        self.members.remove(d)

    def __len__(self):
        return int(lib().lbm_batch_size(self._h))

    def step(self, n: int = 1):
        _check(lib().lbm_batch_step(self._h, int(n)))

    def sync(self):
        return lib().lbm_batch_sync(self._h)

    def errors_async(self, host_ptr: int):
        """Queues a copy of the members' error words (attach order) into the
        pinned host buffer at host_ptr (len(self) int32); valid once the
        batch stream has passed this point."""
        _check(lib().lbm_batch_errors_async(self._h, ctypes.c_void_p(host_ptr)))

    def autotune(self, steps_per_trial: int = 5):
        """Times load path x threads x rows on a shadow batch of the members'
        shapes (members untouched) and applies the fastest; returns tile()."""
        _check(lib().lbm_batch_autotune(self._h, int(steps_per_trial)))
        return self.tile()

    def tile(self):
        """(threads, rows, staged) of the batch's launches."""
        t, r, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib().lbm_batch_get_tile(self._h, ctypes.byref(t), ctypes.byref(r), ctypes.byref(g))
        return t.value, r.value, bool(g.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
