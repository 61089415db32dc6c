"""ctypes wrapper around the plain C oracle (``lbsq_oracle.c``).

Test infrastructure only (see the header of ``lbsq_oracle.c``).  The C file
is compiled with gcc, ``-O2 -ffp-contract=off`` (no fused multiply-add, so
every product and sum is rounded exactly as written) and OpenMP when the
compiler has it.  Nothing here imports the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbsq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbsq_oracle.so")
_lock = threading.Lock()
_lib = None

_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)
_LP = C.POINTER(C.c_int64)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (skipped when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def load_oracle():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        sig = {
            "oracle_velocities": (None, [_IP]),
            "oracle_weights": (None, [_DP]),
            "oracle_opposite": (C.c_int32, [C.c_int32]),
            "oracle_feq": (None, [C.c_double, _DP, _DP]),
            "oracle_feq_inc": (None, [C.c_double, C.c_double, _DP, _DP]),
            "oracle_collide_inc": (None, [_DP, C.c_double, C.c_double, C.c_double, _DP]),
            "oracle_moments": (None, [_DP, _DP, _DP]),
            "oracle_lambda_odd": (C.c_double, [C.c_double, C.c_double]),
            "oracle_collide": (None, [_DP, C.c_double, C.c_double, _DP]),
            "oracle_slip": (None, [_DP, _DP, C.c_double, C.c_double, _DP]),
            "oracle_inside": (C.c_int32, [_DP, C.c_double]),
            "oracle_min_image": (C.c_double, [C.c_double, C.c_int32]),
            "oracle_wca": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "oracle_num_threads": (C.c_int32, []),
            "oracle_set_num_threads": (None, [C.c_int32]),
            "osim_create": (C.c_void_p, [C.c_int32, C.c_int32, C.c_int32,
                                         C.c_double, C.c_double, C.c_double]),
            "osim_destroy": (None, [C.c_void_p]),
            "osim_error": (C.c_int32, [C.c_void_p]),
            "osim_step_count": (C.c_int64, [C.c_void_p]),
            "osim_set_body_force": (None, [C.c_void_p, _DP]),
            "osim_add_tube": (C.c_int32, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
            "osim_set_contact": (None, [C.c_void_p, C.c_double, C.c_double]),
            "osim_set_force_average": (None, [C.c_void_p, C.c_int32]),
            "osim_set_incompressible": (None, [C.c_void_p, C.c_int32]),
            "osim_set_link_at_node": (None, [C.c_void_p, C.c_int32]),
            "osim_set_conversion": (None, [C.c_void_p, C.c_int32]),
            "osim_set_local_density": (None, [C.c_void_p, C.c_int32]),
            "osim_set_psm": (None, [C.c_void_p, C.c_int32]),
            "osim_get_eps": (None, [C.c_void_p, _DP]),
            "oracle_psm_fraction": (C.c_double, [_DP, C.c_double]),
            "osim_set_equilibrium": (None, [C.c_void_p, _DP, _DP]),
            "osim_set_populations": (None, [C.c_void_p, _DP]),
            "osim_get_populations": (None, [C.c_void_p, _DP]),
            "osim_get_owner": (None, [C.c_void_p, _IP]),
            "osim_add_sphere": (C.c_int32, [C.c_void_p, _DP, _DP, C.c_double,
                                            C.c_double, C.c_double, C.c_int32,
                                            C.c_double]),
            "osim_add_plane_wall": (C.c_int32, [C.c_void_p, C.c_int32,
                                                C.c_int32, _DP]),
            "osim_step": (None, [C.c_void_p, C.c_int64]),
            "osim_get_fields": (None, [C.c_void_p, _DP, _DP]),
            "osim_get_totals": (None, [C.c_void_p, _DP, _DP]),
            "osim_get_force_torque": (C.c_int32, [C.c_void_p, C.c_int32, _DP, _DP]),
            "osim_get_stresslet": (C.c_int32, [C.c_void_p, C.c_int32, _DP]),
            "osim_get_object_state": (C.c_int32, [C.c_void_p, C.c_int32, _DP,
                                                  _DP, _DP, _DP]),
            "osim_get_links": (C.c_int64, [C.c_void_p, C.c_int32, _LP, C.c_int64]),
            "osim_get_pending_conversion": (C.c_int32, [C.c_void_p, C.c_int32, _DP, _DP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


# ---------------------------------------------------------------- point functions

def velocities() -> np.ndarray:
    c = np.zeros((19, 3), dtype=np.int32)
    load_oracle().oracle_velocities(c.ctypes.data_as(_IP))
    return c


def weights() -> np.ndarray:
    w = np.zeros(19)
    load_oracle().oracle_weights(w.ctypes.data_as(_DP))
    return w


def opposite(i: int) -> int:
    return int(load_oracle().oracle_opposite(i))


def feq(rho: float, u) -> np.ndarray:
    u, up = _d(u)
    out = np.zeros(19)
    load_oracle().oracle_feq(float(rho), up, out.ctypes.data_as(_DP))
    return out


def feq_inc(rho: float, rho0: float, u) -> np.ndarray:
    u, up = _d(u)
    out = np.zeros(19)
    load_oracle().oracle_feq_inc(float(rho), float(rho0), up, out.ctypes.data_as(_DP))
    return out


def moments(f):
    f, fp = _d(f)
    rho = np.zeros(1)
    j = np.zeros(3)
    load_oracle().oracle_moments(fp, rho.ctypes.data_as(_DP), j.ctypes.data_as(_DP))
    return float(rho[0]), j


def lambda_odd(lambda_e: float, magic: float) -> float:
    return float(load_oracle().oracle_lambda_odd(lambda_e, magic))


def collide(f, lambda_e: float, lambda_o: float) -> np.ndarray:
    f, fp = _d(f)
    out = np.zeros(19)
    load_oracle().oracle_collide(fp, lambda_e, lambda_o, out.ctypes.data_as(_DP))
    return out


def collide_inc(f, lambda_e: float, lambda_o: float, rho0: float) -> np.ndarray:
    f, fp = _d(f)
    out = np.zeros(19)
    load_oracle().oracle_collide_inc(fp, lambda_e, lambda_o, float(rho0), out.ctypes.data_as(_DP))
    return out


def slip(d, e, B1: float, B2: float) -> np.ndarray:
    d, dp = _d(d)
    e, ep = _d(e)
    out = np.zeros(3)
    load_oracle().oracle_slip(dp, ep, B1, B2, out.ctypes.data_as(_DP))
    return out


def inside(d, R: float) -> bool:
    d, dp = _d(d)
    return bool(load_oracle().oracle_inside(dp, R))


def psm_fraction(d, R: float) -> float:
    """Solid fraction of the unit cell at offset d from a sphere's centre."""
    d, dp = _d(d)
    return float(load_oracle().oracle_psm_fraction(dp, R))


def min_image(d: float, n: int) -> float:
    return float(load_oracle().oracle_min_image(d, n))


def wca(r: float, sigma: float, eps: float) -> float:
    return float(load_oracle().oracle_wca(r, sigma, eps))


def num_threads() -> int:
    return int(load_oracle().oracle_num_threads())


def set_num_threads(n: int) -> None:
    load_oracle().oracle_set_num_threads(int(n))


# ---------------------------------------------------------------- simulation

class OracleSim:
    """One periodic D3Q19 lattice with spheres and plane walls (FP64, CPU)."""

    def __init__(self, nx: int, ny: int, nz: int, lambda_e: float = 1.0,
                 collision: str = "bgk", magic: float = 3.0 / 16.0,
                 rho0: float = 1.0):
        self._lib = load_oracle()
        lo = lambda_e if collision == "bgk" else lambda_odd(lambda_e, magic)
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.rho0 = rho0
        self.lambda_e, self.lambda_o = lambda_e, lo
        self._h = self._lib.osim_create(nx, ny, nz, lambda_e, lo, rho0)
        if not self._h:
            raise ValueError("invalid lattice")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.osim_destroy(h)
            self._h = None

    # -- set-up
    def add_sphere(self, pos, e, R, B1=0.0, beta=0.0, mobile=True, density=None):
        pos, pp = _d(pos)
        e, ep = _d(e)
        dens = self.rho0 if density is None else density
        rc = self._lib.osim_add_sphere(self._h, pp, ep, float(R), float(B1),
                                       float(beta), int(bool(mobile)), float(dens))
        if rc < 0:
            raise ValueError(f"add_sphere failed ({-rc})")
        return int(rc)

    def add_plane_wall(self, axis: int, index: int, vel=(0.0, 0.0, 0.0)):
        vel, vp = _d(vel)
        rc = self._lib.osim_add_plane_wall(self._h, axis, index, vp)
        if rc < 0:
            raise ValueError(f"add_plane_wall failed ({-rc})")
        return int(rc)

    def add_tube(self, cx: float, cy: float, r: float):
        """Round tube along z: nodes at distance >= r from the axis (cx, cy) are
        a wall at rest (the paper's tube flow, Sec. V)."""
        rc = self._lib.osim_add_tube(self._h, float(cx), float(cy), float(r))
        if rc < 0:
            raise ValueError(f"add_tube failed ({-rc})")
        return int(rc)

    def set_body_force(self, g):
        g, gp = _d(g)
        self._lib.osim_set_body_force(self._h, gp)

    def set_contact(self, sigma: float, eps: float):
        self._lib.osim_set_contact(self._h, sigma, eps)

    def set_force_average(self, on: bool = True):
        self._lib.osim_set_force_average(self._h, 1 if on else 0)

    def set_link_at_node(self, on: bool = True):
        self._lib.osim_set_link_at_node(self._h, 1 if on else 0)

    def set_psm(self, on: bool = True):
        """Couple spheres by partially saturated cells (see osim_set_psm);
        call before adding spheres."""
        self._lib.osim_set_psm(self._h, 1 if on else 0)

    def eps(self) -> np.ndarray:
        out = np.empty(self.N)
        self._lib.osim_get_eps(self._h, out.ctypes.data_as(_DP))
        return out

    def set_local_density(self, on: bool = True):
        """The bounce-back shift with the fluid node's density (see osim_set_local_density)."""
        self._lib.osim_set_local_density(self._h, 1 if on else 0)

    def set_conversion(self, mode: int):
        """Alternative readings of the cell conversion (see osim_set_conversion)."""
        self._lib.osim_set_conversion(self._h, int(mode))

    def set_incompressible(self, on: bool = True):
        self._lib.osim_set_incompressible(self._h, 1 if on else 0)

    def set_equilibrium(self, rho, u):
        rho, rp = _d(np.reshape(rho, -1))
        u, up = _d(np.reshape(u, (3, -1)))
        self._lib.osim_set_equilibrium(self._h, rp, up)

    def set_populations(self, f):
        f, fp = _d(np.reshape(f, (19, -1)))
        self._lib.osim_set_populations(self._h, fp)

    # -- stepping
    def step(self, n: int = 1):
        self._lib.osim_step(self._h, int(n))
        err = self._lib.osim_error(self._h)
        if err:
            raise RuntimeError(f"oracle error {err}")

    @property
    def steps(self) -> int:
        return int(self._lib.osim_step_count(self._h))

    # -- outputs (arrays are x-fastest: index x + nx*(y + ny*z))
    def populations(self) -> np.ndarray:
        f = np.zeros((19, self.N))
        self._lib.osim_get_populations(self._h, f.ctypes.data_as(_DP))
        return f

    def owner(self) -> np.ndarray:
        o = np.zeros(self.N, dtype=np.int32)
        self._lib.osim_get_owner(self._h, o.ctypes.data_as(_IP))
        return o

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        self._lib.osim_get_fields(self._h, rho.ctypes.data_as(_DP), u.ctypes.data_as(_DP))
        return rho, u

    def totals(self):
        m = np.zeros(1)
        j = np.zeros(3)
        self._lib.osim_get_totals(self._h, m.ctypes.data_as(_DP), j.ctypes.data_as(_DP))
        return float(m[0]), j

    def force_torque(self, oid: int):
        F = np.zeros(3)
        T = np.zeros(3)
        if self._lib.osim_get_force_torque(self._h, oid, F.ctypes.data_as(_DP),
                                           T.ctypes.data_as(_DP)):
            raise ValueError("bad id")
        return F, T

    def stresslet(self, oid: int) -> np.ndarray:
        S = np.zeros(6)
        if self._lib.osim_get_stresslet(self._h, oid, S.ctypes.data_as(_DP)):
            raise ValueError("bad id")
        return S

    def state(self, oid: int):
        p, v, e, w = (np.zeros(3) for _ in range(4))
        if self._lib.osim_get_object_state(self._h, oid, p.ctypes.data_as(_DP),
                                           v.ctypes.data_as(_DP), e.ctypes.data_as(_DP),
                                           w.ctypes.data_as(_DP)):
            raise ValueError("bad id")
        return p, v, e, w

    def pending_conversion(self, oid: int):
        F = np.zeros(3)
        T = np.zeros(3)
        if self._lib.osim_get_pending_conversion(self._h, oid, F.ctypes.data_as(_DP),
                                                 T.ctypes.data_as(_DP)):
            raise ValueError("bad id")
        return F, T

    def links(self, oid: int = 0) -> np.ndarray:
        n = self._lib.osim_get_links(self._h, oid, None, 0)
        out = np.zeros(n, dtype=np.int64)
        self._lib.osim_get_links(self._h, oid, out.ctypes.data_as(_LP), n)
        return out
