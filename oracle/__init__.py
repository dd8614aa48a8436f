"""FP64 CPU oracle of the coupled D2Q9 pseudopotential + D2Q5 thermal LBM step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It wraps ``lbm_oracle.c`` (plain C, double precision) through ctypes
and shares no code with the CUDA library in ``paper_2205_00686_gb300``.

The pins that tie this oracle to the paper live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "lbm_oracle.c"), os.path.join(_HERE, "lbm_oracle_analysis.c"),
         os.path.join(_HERE, "lbm_oracle3d.c")]
_HDR = os.path.join(_HERE, "lbm_oracle.h")
LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
# the same sources built with -fopenmp: the per-node loops of a step run on
# all host cores (OMP_NUM_THREADS); each node's arithmetic and every sum's
# order are unchanged, so its results are bit-identical to the serial build
LIB_OMP_PATH = os.path.join(_HERE, "liblbm_oracle_omp.so")

PERIODIC, WALL, OPEN = 0, 1, 2
T_PERIODIC, T_DIRICHLET, T_ADIABATIC = 0, 1, 2
EDGE_W, EDGE_E, EDGE_S, EDGE_N = 0, 1, 2, 3
# names of the per-node work arrays of orc_work, in the order of its codes
WORK = ("rho", "T", "psi", "Fmx", "Fmy", "Fx", "Fy", "ux", "uy", "divu", "dTx", "dTy",
        "Q", "Pn", "S", "fstar", "gstar", "ghost_psi_S", "ghost_psi_N")


def _build_one(path: str, extra, force: bool) -> str:
    newest = max(os.path.getmtime(f) for f in _SRCS + [_HDR])
    if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
        return path
    tmp = path + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", *extra,
           "-shared", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction): the
    serial library and its OpenMP build."""
    _build_one(LIB_OMP_PATH, ["-fopenmp"], force)
    return _build_one(LIB_PATH, [], force)


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "a", "b", "R", "omega", "G", "sigma", "nu", "s0", "s_e", "s_eps", "s_j", "s_q",
        "lambda_", "cv", "w_dot", "vs0", "vs3", "vs4", "gravity")] + [
        ("frozen_flow", ctypes.c_int), ("frozen_thermal", ctypes.c_int)]


class BC(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int * 4), ("therm", ctypes.c_int * 4),
                ("T_edge", ctypes.c_double * 4), ("theta_deg", ctypes.c_double),
                ("heater_x0", ctypes.c_int), ("heater_x1", ctypes.c_int),
                ("T_heater", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "mass", "energy", "liquid_mass", "liquid_area", "liquid_area_smooth",
        "diameter", "diameter_smooth", "max_u")] + [
        ("step", ctypes.c_long), ("nonfinite", ctypes.c_int)]


class BC3(ctypes.Structure):
    _fields_ = [("flow_z", ctypes.c_int), ("therm", ctypes.c_int * 2),
                ("T_edge", ctypes.c_double * 2), ("theta_deg", ctypes.c_double)]


class Contact(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "theta_deg", "xc", "yc", "radius", "base_width", "height")] + [
        ("n_points", ctypes.c_int)]


class Component(ctypes.Structure):
    _fields_ = [("label", ctypes.c_longlong), ("area", ctypes.c_longlong),
                ("sum_y", ctypes.c_longlong), ("y_min", ctypes.c_int), ("y_max", ctypes.c_int),
                ("touches_w", ctypes.c_int), ("touches_e", ctypes.c_int),
                ("touches_s", ctypes.c_int), ("touches_n", ctypes.c_int)]


_libs = {}
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib(omp: bool = False):
    """The serial oracle library, or (omp=True) its OpenMP build."""
    if omp not in _libs:
        build()
        L = ctypes.CDLL(LIB_OMP_PATH if omp else LIB_PATH)
        P, B = ctypes.POINTER(Params), ctypes.POINTER(BC)
        L.orc_Tc.restype = ctypes.c_double
        L.orc_Tc.argtypes = [P]
        for fn in ("orc_p_eos", "orc_dpdT", "orc_psi2"):
            getattr(L, fn).restype = ctypes.c_double
            getattr(L, fn).argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.orc_maxwell.argtypes = [P, ctypes.c_double, _dp, _dp]
        L.orc_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_meq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_geq.argtypes = [P, ctypes.c_double, _dp]
        L.orc_matrices.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_set_defaults.argtypes = [P]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, P, B, ctypes.POINTER(ctypes.c_int)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_fields.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_get_populations.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.orc_set_populations.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_long,
                                          ctypes.c_double]
        L.orc_step_count.restype = ctypes.c_long
        L.orc_step_count.argtypes = [ctypes.c_void_p]
        L.orc_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.POINTER(Diag)]
        L.orc_last_error.argtypes = [ctypes.c_void_p]
        L.orc_reconfigure.argtypes = [ctypes.c_void_p, P, B]
        L.orc_work.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        B3 = ctypes.POINTER(BC3)
        _i19 = ctypes.POINTER(ctypes.c_int)
        L.orc3_velocities.argtypes = [_i19, _i19, _i19, _dp]
        L.orc3_matrices.argtypes = [_dp, _dp, _dp, _dp]
        L.orc3_feq.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.orc3_force_term.argtypes = [ctypes.c_double] * 6 + [_dp]
        L.orc3_create.restype = ctypes.c_void_p
        L.orc3_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, B3,
                                  ctypes.POINTER(ctypes.c_int)]
        L.orc3_destroy.argtypes = [ctypes.c_void_p]
        L.orc3_init.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp]
        L.orc3_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc3_fields.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp]
        L.orc3_get_populations.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.orc3_set_populations.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_long,
                                           ctypes.c_double]
        L.orc3_step_count.restype = ctypes.c_long
        L.orc3_step_count.argtypes = [ctypes.c_void_p]
        L.orc3_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.POINTER(Diag)]
        L.orc_interface_points.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.orc_circle_fit.argtypes = [_dp, _dp, ctypes.c_int, _dp]
        L.orc_contact_angle.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, ctypes.POINTER(Contact)]
        L.orc_components.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, _ip,
                                     ctypes.POINTER(Component), ctypes.c_int, _ip]
        _libs[omp] = L
    return _libs[omp]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def make_params(d: dict) -> Params:
    p = Params()
    lib().orc_set_defaults(ctypes.byref(p))
    for k, v in d.items():
        name = "lambda_" if k == "lambda" else k
        if any(name == f[0] for f in Params._fields_):
            setattr(p, name, v)
    return p


def make_bc(d: dict) -> BC:
    b = BC()
    for e in range(4):
        b.flow[e] = int(d["flow"][e])
        b.therm[e] = int(d["therm"][e])
        b.T_edge[e] = float(d.get("T_edge", (0.0,) * 4)[e])
    b.theta_deg = float(d.get("theta_deg", 90.0))
    b.heater_x0 = int(d.get("heater_x0", 0))
    b.heater_x1 = int(d.get("heater_x1", 0))
    b.T_heater = float(d.get("T_heater", 0.0))
    return b


# ---- closed forms -------------------------------------------------------

def Tc(params: dict) -> float:
    return lib().orc_Tc(ctypes.byref(make_params(params)))


def p_eos(params: dict, rho: float, T: float) -> float:
    return lib().orc_p_eos(ctypes.byref(make_params(params)), rho, T)


def dpdT(params: dict, rho: float, T: float) -> float:
    return lib().orc_dpdT(ctypes.byref(make_params(params)), rho, T)


def psi2(params: dict, rho: float, T: float) -> float:
    return lib().orc_psi2(ctypes.byref(make_params(params)), rho, T)


def maxwell(params: dict, T: float):
    rg, rl = ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_maxwell(ctypes.byref(make_params(params)), T, ctypes.byref(rg),
                           ctypes.byref(rl))
    if rc:
        raise ValueError("no coexistence at T=%g" % T)
    return rg.value, rl.value


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _ptr(out))
    return out


def meq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_meq(rho, ux, uy, _ptr(out))
    return out


def geq(params: dict, T: float) -> np.ndarray:
    out = np.zeros(5)
    lib().orc_geq(ctypes.byref(make_params(params)), T, _ptr(out))
    return out


def matrices():
    M, Mi, Mh, Mhi = np.zeros(81), np.zeros(81), np.zeros(25), np.zeros(25)
    lib().orc_matrices(_ptr(M), _ptr(Mi), _ptr(Mh), _ptr(Mhi))
    return M.reshape(9, 9), Mi.reshape(9, 9), Mh.reshape(5, 5), Mhi.reshape(5, 5)


# ---- interface analyses on a density field ------------------------------

def interface_points(rho, rho_mid: float, skip_rows: int = 0):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    n = lib().orc_interface_points(_ptr(rho), nx, ny, rho_mid, skip_rows, None, None, 0)
    if n < 0:
        raise OracleError(n)
    px, py = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    lib().orc_interface_points(_ptr(rho), nx, ny, rho_mid, skip_rows, _ptr(px), _ptr(py), n)
    return px[:n], py[:n]


def circle_fit(px, py):
    px = np.ascontiguousarray(px, dtype=np.float64)
    py = np.ascontiguousarray(py, dtype=np.float64)
    out = np.zeros(3)
    rc = lib().orc_circle_fit(_ptr(px), _ptr(py), len(px), _ptr(out))
    if rc:
        raise OracleError(rc)
    return tuple(out)


def contact_angle(rho, rho_l: float, rho_g: float, skip_rows: int = 3) -> dict:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    c = Contact()
    rc = lib().orc_contact_angle(_ptr(rho), nx, ny, rho_l, rho_g, skip_rows, ctypes.byref(c))
    if rc:
        raise OracleError(rc)
    return {k: getattr(c, k) for k, _ in Contact._fields_}


def components(rho, threshold: float, below: bool = True, periodic_x: bool = False,
               periodic_y: bool = False):
    """Returns (labels [ny][nx] int32, list of component dicts sorted by label)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    labels = np.zeros((ny, nx), dtype=np.int32)
    n = ctypes.c_int(0)
    cap = min(nx * ny, 4096)
    while True:
        comps = (Component * max(cap, 1))()
        rc = lib().orc_components(_ptr(rho), nx, ny, int(periodic_x), int(periodic_y),
                                  threshold, int(below), labels.ctypes.data_as(_ip), comps, cap,
                                  ctypes.byref(n))
        if rc:
            raise OracleError(rc)
        if n.value <= cap:
            break
        cap = n.value
    out = [{k: getattr(comps[i], k) for k, _ in Component._fields_} for i in range(n.value)]
    return labels, out


# ---- simulation ----------------------------------------------------------

class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__("oracle error %d" % code)
        self.code = code


class Sim:
    """One FP64 CPU simulation of an nx x ny domain (omp=True: the OpenMP
    build, same results on all host cores)."""

    def __init__(self, nx: int, ny: int, params: dict, bc: dict, omp: bool = False):
        self.nx, self.ny = nx, ny
        self._L = lib(omp)
        self._p = make_params(params)
        self._b = make_bc(bc)
        err = ctypes.c_int(0)
        self._h = self._L.orc_create(nx, ny, ctypes.byref(self._p), ctypes.byref(self._b),
                                     ctypes.byref(err))
        if not self._h:
            raise OracleError(err.value)

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    __del__ = close

    def init(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx)
                for a in (rho, ux, uy, T)]
        rc = self._L.orc_init(self._h, *[_ptr(a) for a in arrs])
        if rc:
            raise OracleError(rc)

    def step(self, n: int = 1, check: bool = True) -> int:
        rc = self._L.orc_step(self._h, int(n))
        if rc and check:
            raise OracleError(rc)
        return rc

    @property
    def step_count(self) -> int:
        return self._L.orc_step_count(self._h)

    def fields(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        self._L.orc_fields(self._h, *[_ptr(a) for a in out])
        return tuple(out)

    def populations(self):
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros((5, self.ny, self.nx))
        P = np.zeros((self.ny, self.nx))
        self._L.orc_get_populations(self._h, _ptr(f), _ptr(g), _ptr(P))
        return f, g, P

    def set_populations(self, f, g, P, step: int, rho_ave_prev: float):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        rc = self._L.orc_set_populations(self._h, _ptr(f), _ptr(g), _ptr(P), int(step),
                                       float(rho_ave_prev))
        if rc:
            raise OracleError(rc)

    def diagnostics(self, rho_l: float, rho_g: float, sessile: bool = False) -> dict:
        d = Diag()
        self._L.orc_diagnostics(self._h, rho_l, rho_g, int(sessile), ctypes.byref(d))
        return {k: getattr(d, k) for k, _ in Diag._fields_}

    def work(self, name: str) -> np.ndarray:
        """One per-node quantity as the last step computed it (test hook):
        rho, T, psi, Fmx, Fmy, Fx, Fy, ux, uy, divu, dTx, dTy, Q, Pn, S,
        fstar [9][ny][nx], gstar [5][ny][nx], ghost_psi_S / ghost_psi_N [nx]."""
        code = WORK.index(name)
        if name == "fstar":
            out = np.zeros((9, self.ny, self.nx))
        elif name == "gstar":
            out = np.zeros((5, self.ny, self.nx))
        elif name.startswith("ghost"):
            out = np.zeros(self.nx)
        else:
            out = np.zeros((self.ny, self.nx))
        rc = self._L.orc_work(self._h, code, _ptr(out))
        if rc:
            raise OracleError(rc)
        return out

    @property
    def last_error(self) -> int:
        return self._L.orc_last_error(self._h)

    def reconfigure(self, params: dict, bc: dict):
        self._p = make_params(params)
        self._b = make_bc(bc)
        rc = self._L.orc_reconfigure(self._h, ctypes.byref(self._p), ctypes.byref(self._b))
        if rc:
            raise OracleError(rc)


# ---- three-dimensional form ------------------------------------------------

def make_bc3(d: dict) -> BC3:
    b = BC3()
    b.flow_z = int(d["flow_z"])
    for e in range(2):
        b.therm[e] = int(d["therm"][e])
        b.T_edge[e] = float(d.get("T_edge", (0.0, 0.0))[e])
    b.theta_deg = float(d.get("theta_deg", 90.0))
    return b


def velocities3():
    cx, cy, cz = (ctypes.c_int * 19)(), (ctypes.c_int * 19)(), (ctypes.c_int * 19)()
    w = np.zeros(19)
    lib().orc3_velocities(cx, cy, cz, _ptr(w))
    return np.array(list(cx)), np.array(list(cy)), np.array(list(cz)), w


def matrices3():
    M, Mi, Mh, Mhi = np.zeros(361), np.zeros(361), np.zeros(49), np.zeros(49)
    lib().orc3_matrices(_ptr(M), _ptr(Mi), _ptr(Mh), _ptr(Mhi))
    return M.reshape(19, 19), Mi.reshape(19, 19), Mh.reshape(7, 7), Mhi.reshape(7, 7)


def feq3(rho, ux, uy, uz):
    out = np.zeros(19)
    lib().orc3_feq(rho, ux, uy, uz, _ptr(out))
    return out


def force_term3(ux, uy, uz, Fx, Fy, Fz):
    out = np.zeros(19)
    lib().orc3_force_term(ux, uy, uz, Fx, Fy, Fz, _ptr(out))
    return out


class Sim3:
    """One FP64 CPU simulation of an nx x ny x nz domain (3-D form)."""

    def __init__(self, nx: int, ny: int, nz: int, params: dict, bc3: dict):
        self.nx, self.ny, self.nz = nx, ny, nz
        self._p = make_params(params)
        self._b = make_bc3(bc3)
        err = ctypes.c_int(0)
        self._h = lib().orc3_create(nx, ny, nz, ctypes.byref(self._p), ctypes.byref(self._b),
                                    ctypes.byref(err))
        if not self._h:
            raise OracleError(err.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc3_destroy(self._h)
            self._h = None

    __del__ = close

    def _shape(self):
        return (self.nz, self.ny, self.nx)

    def init(self, rho, ux, uy, uz, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self._shape())
                for a in (rho, ux, uy, uz, T)]
        rc = lib().orc3_init(self._h, *[_ptr(a) for a in arrs])
        if rc:
            raise OracleError(rc)

    def step(self, n: int = 1, check: bool = True) -> int:
        rc = lib().orc3_step(self._h, int(n))
        if rc and check:
            raise OracleError(rc)
        return rc

    @property
    def step_count(self) -> int:
        return lib().orc3_step_count(self._h)

    def fields(self):
        out = [np.zeros(self._shape()) for _ in range(5)]
        lib().orc3_fields(self._h, *[_ptr(a) for a in out])
        return tuple(out)

    def populations(self):
        f = np.zeros((19,) + self._shape())
        g = np.zeros((7,) + self._shape())
        P = np.zeros(self._shape())
        lib().orc3_get_populations(self._h, _ptr(f), _ptr(g), _ptr(P))
        return f, g, P

    def set_populations(self, f, g, P, step: int, rho_ave_prev: float):
        f, g, P = (np.ascontiguousarray(a, dtype=np.float64) for a in (f, g, P))
        rc = lib().orc3_set_populations(self._h, _ptr(f), _ptr(g), _ptr(P), int(step),
                                        float(rho_ave_prev))
        if rc:
            raise OracleError(rc)

    def diagnostics(self, rho_l: float, rho_g: float, sessile: bool = False) -> dict:
        d = Diag()
        lib().orc3_diagnostics(self._h, rho_l, rho_g, int(sessile), ctypes.byref(d))
        return {k: getattr(d, k) for k, _ in Diag._fields_}
