"""Thin ctypes binding of the C ABI in ``include/lbsq.h``.

The functions carry the C names (``lb_create``, ``lb_step``, ...) and only
marshal arguments: every step of the method runs in the CUDA library.  There
is no fallback: if ``liblbsq.so`` cannot be loaded the import of this module
fails loudly.  PyTorch, when present, supplies the stream the context runs on
and its caching allocator for the context's device memory.

``Lattice`` wraps one context with numpy-returning getters.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LB_OK, LB_ERR_INVALID, LB_ERR_OOM, LB_ERR_CUDA, LB_ERR_OVERLAP = 0, 1, 2, 3, 4
LB_ERR_DIVERGED, LB_ERR_TIMEOUT, LB_ERR_STATE, LB_ERR_CAPACITY = 5, 6, 7, 8
LB_EQ_COMPRESSIBLE, LB_EQ_INCOMPRESSIBLE = 0, 1
LB_ROUND_DEFAULT, LB_ROUND_NEAREST, LB_ROUND_STOCHASTIC = -1, 0, 1
ROUNDING = {"default": LB_ROUND_DEFAULT, "nearest": LB_ROUND_NEAREST, "stochastic": LB_ROUND_STOCHASTIC}
LB_COUPLE_LINKS, LB_COUPLE_PSM = 0, 1
COUPLING = {"links": LB_COUPLE_LINKS, "psm": LB_COUPLE_PSM}
LB_BGK, LB_TRT = 0, 1
LB_F64, LB_F32, LB_F16DEV, LB_BF16DEV = 0, 1, 2, 3
STORAGE = {"f64": LB_F64, "f32": LB_F32, "f16dev": LB_F16DEV, "bf16dev": LB_BF16DEV}
STORAGE_BYTES = {LB_F64: 8, LB_F32: 4, LB_F16DEV: 2, LB_BF16DEV: 2}
STATUS = {0: "LB_OK", 1: "LB_ERR_INVALID", 2: "LB_ERR_OOM", 3: "LB_ERR_CUDA", 4: "LB_ERR_OVERLAP",
          5: "LB_ERR_DIVERGED", 6: "LB_ERR_TIMEOUT", 7: "LB_ERR_STATE", 8: "LB_ERR_CAPACITY"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class lb_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class lb_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("collision", C.c_int32), ("lambda_e", C.c_double), ("magic", C.c_double),
                ("rho0", C.c_double), ("storage", C.c_int32), ("dev_scale_log2", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p),
                ("allocator", C.POINTER(lb_allocator)), ("equilibrium", C.c_int32), ("rounding", C.c_int32)]


class lb_server_params(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", C.c_void_p), ("hbm_budget_bytes", C.c_size_t),
                ("max_resident", C.c_int32), ("round_steps", C.c_int32), ("tile_units", C.c_int32),
                ("allocator", C.POINTER(lb_allocator))]


class lb_request(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("storage", C.c_int32), ("collision", C.c_int32), ("lambda_e", C.c_double),
                ("magic", C.c_double), ("rho0", C.c_double), ("pos", C.c_double * 3), ("e", C.c_double * 3),
                ("R", C.c_double), ("B1", C.c_double), ("beta", C.c_double), ("obstacle", C.c_double * 4),
                ("wca_sigma", C.c_double), ("wca_eps", C.c_double), ("steps", C.c_int64)]


class lb_result(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("steps_done", C.c_int64),
                ("pos", C.c_double * 3), ("vel", C.c_double * 3), ("e", C.c_double * 3),
                ("omega", C.c_double * 3), ("F", C.c_double * 3), ("T", C.c_double * 3),
                ("mean_speed", C.c_double), ("mean_vel", C.c_double * 3)]


LB_REQ_QUEUED, LB_REQ_RUNNING, LB_REQ_DONE, LB_REQ_FAILED = 0, 1, 2, 3


class LBError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {msg}".strip())


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)
_LP = C.POINTER(C.c_int64)
_CTX = C.c_void_p

# name -> (restype, argtypes); every name is declared in include/lbsq.h
SIGNATURES = {
    "lb_params_default": (None, [C.POINTER(lb_params)]),
    "lb_create": (C.c_int, [C.POINTER(lb_params), C.POINTER(_CTX)]),
    "lb_destroy": (C.c_int, [_CTX]),
    "lb_add_squirmer": (C.c_int, [_CTX, _DP, _DP, C.c_double, C.c_double, C.c_double, C.c_int32,
                                  C.c_double, _IP]),
    "lb_add_wall": (C.c_int, [_CTX, C.c_int32, _DP, C.c_int32, _IP]),
    "lb_set_contact": (C.c_int, [_CTX, C.c_double, C.c_double]),
    "lb_set_force_average": (C.c_int, [_CTX, C.c_int32]),
    "lb_set_link_options": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "lb_set_coupling": (C.c_int, [_CTX, C.c_int32]),
    "lb_get_solid_fraction": (C.c_int, [_CTX, _DP]),
    "lb_set_fields": (C.c_int, [_CTX, _DP, _DP]),
    "lb_set_populations": (C.c_int, [_CTX, _DP]),
    "lb_get_populations": (C.c_int, [_CTX, _DP]),
    "lb_step": (C.c_int, [_CTX, C.c_int64]),
    "lb_sync": (C.c_int, [_CTX]),
    "lb_step_count": (C.c_int64, [_CTX]),
    "lb_get_fields": (C.c_int, [_CTX, _DP, _DP]),
    "lb_get_fields_device": (C.c_int, [_CTX, C.c_void_p, C.c_void_p]),
    "lb_get_owner": (C.c_int, [_CTX, _IP]),
    "lb_get_force_torque": (C.c_int, [_CTX, C.c_int32, _DP, _DP]),
    "lb_get_object_state": (C.c_int, [_CTX, C.c_int32, _DP, _DP, _DP, _DP]),
    "lb_get_stresslet": (C.c_int, [_CTX, C.c_int32, _DP]),
    "lb_get_mass": (C.c_int, [_CTX, _DP, _DP]),
    "lb_get_links": (C.c_int, [_CTX, C.c_int32, _LP, C.c_int64, _LP]),
    "lb_checkpoint_size": (C.c_int, [_CTX, C.POINTER(C.c_size_t)]),
    "lb_checkpoint": (C.c_int, [_CTX, C.c_void_p, C.c_size_t]),
    "lb_restore": (C.c_int, [_CTX, C.c_void_p, C.c_size_t]),
    "lb_last_error": (C.c_char_p, [_CTX]),
    "lb_kernel_launches": (C.c_int64, [_CTX]),
    "lb_set_sweep_variant": (C.c_int, [_CTX, C.c_int32]),
    "lb_profile_begin": (C.c_int, [_CTX]),
    "lb_profile_end": (C.c_int, [_CTX, _DP, _LP]),
    "lb_fluid_totals_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "lb_server_params_default": (None, [C.POINTER(lb_server_params)]),
    "lb_server_create": (C.c_int, [C.POINTER(lb_server_params), C.POINTER(C.c_void_p)]),
    "lb_server_destroy": (C.c_int, [C.c_void_p]),
    "lb_server_submit": (C.c_int, [C.c_void_p, C.POINTER(lb_request), _LP]),
    "lb_server_advance": (C.c_int, [C.c_void_p, _IP, _IP]),
    "lb_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(lb_result)]),
    "lb_server_info": (C.c_int, [C.c_void_p, _IP, _IP, C.POINTER(C.c_size_t), _DP]),
    "lb_server_last_error": (C.c_char_p, [C.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load liblbsq.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library missing: {_build.LIB} (run __graft_entry__.build())")
    lib = C.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(ctx, status: int, where: str):
    if status != LB_OK:
        msg = ""
        if ctx:
            raw = load().lb_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise LBError(status, where, msg)


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


# ------------------------------------------------------------ C-named functions

def lb_params_default() -> lb_params:
    p = lb_params()
    load().lb_params_default(C.byref(p))
    return p


def lb_create(p: lb_params):
    ctx = _CTX()
    _check(None, load().lb_create(C.byref(p), C.byref(ctx)), "lb_create")
    return ctx


def lb_destroy(ctx):
    _check(None, load().lb_destroy(ctx), "lb_destroy")


def lb_add_squirmer(ctx, pos, e, R, B1, beta, mobile=1, density=1.0) -> int:
    oid = C.c_int32()
    pos, e = _f64(pos, 3), _f64(e, 3)
    _check(ctx, load().lb_add_squirmer(ctx, _dp(pos), _dp(e), float(R), float(B1), float(beta),
                                       int(mobile), float(density), C.byref(oid)), "lb_add_squirmer")
    return oid.value


def lb_add_wall(ctx, kind: int, params=()) -> int:
    oid = C.c_int32()
    prm = _f64(params) if len(params) else np.zeros(1)
    _check(ctx, load().lb_add_wall(ctx, int(kind), _dp(prm), len(params), C.byref(oid)), "lb_add_wall")
    return oid.value


def lb_set_contact(ctx, sigma: float, eps: float):
    _check(ctx, load().lb_set_contact(ctx, float(sigma), float(eps)), "lb_set_contact")


def lb_set_force_average(ctx, on: bool):
    _check(ctx, load().lb_set_force_average(ctx, int(bool(on))), "lb_set_force_average")


def lb_set_link_options(ctx, density_of_node: bool, velocity_at_node: bool):
    _check(ctx, load().lb_set_link_options(ctx, int(bool(density_of_node)), int(bool(velocity_at_node))),
           "lb_set_link_options")


def lb_set_coupling(ctx, coupling: int):
    _check(ctx, load().lb_set_coupling(ctx, int(coupling)), "lb_set_coupling")


def lb_get_solid_fraction(ctx, n: int):
    eps = np.empty(n, np.float64)
    _check(ctx, load().lb_get_solid_fraction(ctx, _dp(eps)), "lb_get_solid_fraction")
    return eps


def lb_set_fields(ctx, rho, u):
    rho = _f64(rho)
    u = _f64(u, 3 * rho.size)
    _check(ctx, load().lb_set_fields(ctx, _dp(rho), _dp(u)), "lb_set_fields")


def lb_set_populations(ctx, f):
    f = _f64(f)
    _check(ctx, load().lb_set_populations(ctx, _dp(f)), "lb_set_populations")


def lb_get_populations(ctx, N: int) -> np.ndarray:
    f = np.empty((19, N))
    _check(ctx, load().lb_get_populations(ctx, _dp(f)), "lb_get_populations")
    return f


def lb_step(ctx, n: int):
    _check(ctx, load().lb_step(ctx, int(n)), "lb_step")


def lb_sync(ctx):
    _check(ctx, load().lb_sync(ctx), "lb_sync")


def lb_step_count(ctx) -> int:
    return int(load().lb_step_count(ctx))


def lb_get_fields(ctx, N: int):
    rho = np.empty(N)
    u = np.empty((3, N))
    _check(ctx, load().lb_get_fields(ctx, _dp(rho), _dp(u)), "lb_get_fields")
    return rho, u


def lb_get_fields_device(ctx, rho_ptr: int, u_ptr: int):
    _check(ctx, load().lb_get_fields_device(ctx, C.c_void_p(rho_ptr), C.c_void_p(u_ptr)),
           "lb_get_fields_device")


def lb_get_owner(ctx, N: int) -> np.ndarray:
    o = np.empty(N, dtype=np.int32)
    _check(ctx, load().lb_get_owner(ctx, o.ctypes.data_as(_IP)), "lb_get_owner")
    return o


def lb_get_force_torque(ctx, oid: int):
    F, T = np.empty(3), np.empty(3)
    _check(ctx, load().lb_get_force_torque(ctx, int(oid), _dp(F), _dp(T)), "lb_get_force_torque")
    return F, T


def lb_get_object_state(ctx, oid: int):
    p, v, e, w = (np.empty(3) for _ in range(4))
    _check(ctx, load().lb_get_object_state(ctx, int(oid), _dp(p), _dp(v), _dp(e), _dp(w)),
           "lb_get_object_state")
    return p, v, e, w


def lb_get_stresslet(ctx, oid: int) -> np.ndarray:
    S = np.empty(6)
    _check(ctx, load().lb_get_stresslet(ctx, int(oid), _dp(S)), "lb_get_stresslet")
    return S


def lb_get_mass(ctx):
    m = np.empty(1)
    j = np.empty(3)
    _check(ctx, load().lb_get_mass(ctx, _dp(m), _dp(j)), "lb_get_mass")
    return float(m[0]), j


def lb_get_links(ctx, oid: int = 0) -> np.ndarray:
    cnt = C.c_int64()
    _check(ctx, load().lb_get_links(ctx, int(oid), None, 0, C.byref(cnt)), "lb_get_links")
    out = np.empty(cnt.value, dtype=np.int64)
    if cnt.value:
        _check(ctx, load().lb_get_links(ctx, int(oid), out.ctypes.data_as(_LP), cnt.value,
                                        C.byref(cnt)), "lb_get_links")
    return out


def lb_checkpoint(ctx) -> bytes:
    n = C.c_size_t()
    _check(ctx, load().lb_checkpoint_size(ctx, C.byref(n)), "lb_checkpoint_size")
    buf = C.create_string_buffer(n.value)
    _check(ctx, load().lb_checkpoint(ctx, buf, n.value), "lb_checkpoint")
    return buf.raw


def lb_restore(ctx, blob: bytes) -> None:
    buf = C.create_string_buffer(bytes(blob), len(blob))
    _check(ctx, load().lb_restore(ctx, buf, len(blob)), "lb_restore")


def lb_last_error(ctx) -> str:
    raw = load().lb_last_error(ctx)
    return raw.decode() if raw else ""


def lb_kernel_launches(ctx) -> int:
    return int(load().lb_kernel_launches(ctx))


KERNEL_KINDS = ("sweep", "links", "classify", "convert", "rebuild", "tick")


def lb_set_sweep_variant(ctx, variant: int):
    _check(ctx, load().lb_set_sweep_variant(ctx, int(variant)), "lb_set_sweep_variant")


def lb_profile_begin(ctx):
    _check(ctx, load().lb_profile_begin(ctx), "lb_profile_begin")


def lb_profile_end(ctx):
    t = np.zeros(6)
    n = np.zeros(6, dtype=np.int64)
    _check(ctx, load().lb_profile_end(ctx, _dp(t), n.ctypes.data_as(_LP)), "lb_profile_end")
    return {k: (float(t[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def lb_fluid_totals_static(f_ptr: int, owner_ptr: int, n_cells: int, out_ptr: int, stream_ptr: int = 0):
    """Allocation-free fluid mass and momentum of caller-owned device buffers
    (see include/lbsq.h); pointers are raw device addresses."""
    _check(None, load().lb_fluid_totals_static(C.c_void_p(f_ptr), C.c_void_p(owner_ptr or None), int(n_cells),
                                                C.c_void_p(out_ptr), C.c_void_p(stream_ptr or None)),
           "lb_fluid_totals_static")


# ------------------------------------------------------------ serving

def _scheck(srv, status, where):
    if status != LB_OK:
        raw = load().lb_server_last_error(srv) if srv else b""
        raise LBError(status, where, raw.decode() if raw else "")


def lb_server_params_default() -> lb_server_params:
    p = lb_server_params()
    load().lb_server_params_default(C.byref(p))
    return p


def lb_server_create(p: lb_server_params):
    srv = C.c_void_p()
    _scheck(None, load().lb_server_create(C.byref(p), C.byref(srv)), "lb_server_create")
    return srv


def lb_server_destroy(srv):
    _scheck(None, load().lb_server_destroy(srv), "lb_server_destroy")


def lb_server_submit(srv, req: lb_request) -> int:
    t = C.c_int64()
    _scheck(srv, load().lb_server_submit(srv, C.byref(req), C.byref(t)), "lb_server_submit")
    return t.value


def lb_server_advance(srv):
    r, q = C.c_int32(), C.c_int32()
    _scheck(srv, load().lb_server_advance(srv, C.byref(r), C.byref(q)), "lb_server_advance")
    return r.value, q.value


def lb_server_poll(srv, ticket: int) -> lb_result:
    out = lb_result()
    _scheck(srv, load().lb_server_poll(srv, int(ticket), C.byref(out)), "lb_server_poll")
    return out


def lb_server_info(srv):
    tz, bps, used, cu = C.c_int32(), C.c_int32(), C.c_size_t(), C.c_double()
    _scheck(srv, load().lb_server_info(srv, C.byref(tz), C.byref(bps), C.byref(used), C.byref(cu)),
            "lb_server_info")
    return {"tile_units": tz.value, "blocks_per_sm": bps.value, "bytes_used": used.value,
            "cell_updates": cu.value}


def make_request(geometry=0, shape=(32, 32, 32), storage="f32", collision="trt", lambda_e=1.0,
                 magic=3.0 / 16.0, rho0=1.0, pos=None, e=(0.0, 0.0, 1.0), R=4.0, B1=0.005, beta=0.0,
                 obstacle=(0.0, 0.0, 0.0, 0.0), wca=(1.0, 0.0), steps=100) -> lb_request:
    r = lb_request()
    r.geometry = int(geometry)
    r.nx, r.ny, r.nz = (int(v) for v in shape)
    r.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    r.collision = LB_TRT if collision == "trt" else LB_BGK
    r.lambda_e, r.magic, r.rho0 = float(lambda_e), float(magic), float(rho0)
    pos = pos if pos is not None else tuple(v / 2.0 for v in shape)
    for a in range(3):
        r.pos[a] = float(pos[a])
        r.e[a] = float(e[a])
    r.R, r.B1, r.beta = float(R), float(B1), float(beta)
    for a in range(4):
        r.obstacle[a] = float(obstacle[a])
    r.wca_sigma, r.wca_eps = float(wca[0]), float(wca[1])
    r.steps = int(steps)
    return r


class Server:
    """Many squirmer simulations resident on one GPU, advanced together."""

    def __init__(self, budget_bytes=8 << 30, max_resident=64, round_steps=64, tile_units=0, device=0,
                 use_torch=True):
        p = lb_server_params_default()
        p.device = int(device)
        p.hbm_budget_bytes = int(budget_bytes)
        p.max_resident = int(max_resident)
        p.round_steps = int(round_steps)
        p.tile_units = int(tile_units)
        self._stream = None
        self._alloc = None
        if use_torch:
            import torch
            self._stream = torch.cuda.Stream(device=device)
            p.stream = C.c_void_p(self._stream.cuda_stream)
            self._alloc = TorchAllocator(device, self._stream.cuda_stream)
            p.allocator = C.pointer(self._alloc.struct)
        self.params = p
        self.srv = lb_server_create(p)

    def close(self):
        if getattr(self, "srv", None):
            lb_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def submit(self, req: lb_request) -> int:
        return lb_server_submit(self.srv, req)

    def advance(self):
        return lb_server_advance(self.srv)

    def poll(self, ticket: int) -> lb_result:
        return lb_server_poll(self.srv, ticket)

    def info(self):
        return lb_server_info(self.srv)


# ------------------------------------------------------------ torch plumbing

class TorchAllocator:
    """lb_allocator backed by PyTorch's caching allocator on one stream."""

    def __init__(self, device: int, stream_ptr: int):
        import torch
        self._torch = torch
        self.device = device
        self.stream_ptr = stream_ptr
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = lb_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, _user):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream_ptr))
        except Exception:  # noqa: BLE001 -- the C side turns NULL into LB_ERR_OOM
            return None

    def _do_free(self, ptr, _nbytes, _user):
        if ptr:
            self._torch.cuda.caching_allocator_delete(int(ptr))


class Lattice:
    """One lattice context.  ``storage`` in {'f64','f32','f16dev','bf16dev'};
    ``collision`` in {'bgk','trt'}; ``equilibrium`` in {'compressible',
    'incompressible'}; ``rounding`` in {'default', 'nearest', 'stochastic'}
    (BF16 stores).  With ``use_torch`` the context runs on a torch stream
    and takes its device memory from torch's caching allocator."""

    def __init__(self, shape, collision="bgk", lambda_e=1.0, magic=3.0 / 16.0, rho0=1.0,
                 storage="f64", device=0, use_torch=True, dev_scale_log2=-1, equilibrium="compressible",
                 rounding="default"):
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        p = lb_params_default()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.collision = LB_TRT if collision == "trt" else LB_BGK
        p.lambda_e, p.magic, p.rho0 = float(lambda_e), float(magic), float(rho0)
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.dev_scale_log2 = int(dev_scale_log2)
        if equilibrium not in ("compressible", "incompressible"):
            raise ValueError(f"equilibrium {equilibrium!r}")
        p.equilibrium = LB_EQ_INCOMPRESSIBLE if equilibrium == "incompressible" else LB_EQ_COMPRESSIBLE
        p.rounding = ROUNDING[rounding]
        p.device = int(device)
        self._stream = None
        self._alloc = None
        if use_torch:
            import torch
            self._stream = torch.cuda.Stream(device=device)
            p.stream = C.c_void_p(self._stream.cuda_stream)
            self._alloc = TorchAllocator(device, self._stream.cuda_stream)
            p.allocator = C.pointer(self._alloc.struct)
        self.params = p
        self.ctx = lb_create(p)

    def close(self):
        if getattr(self, "ctx", None):
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # set-up
    def add_squirmer(self, pos, e, R, B1=0.0, beta=0.0, mobile=True, density=1.0):
        return lb_add_squirmer(self.ctx, pos, e, R, B1, beta, int(bool(mobile)), density)

    def add_plane_wall(self, axis, index, vel=None):
        prm = [axis, index] if vel is None else [axis, index, *vel]
        return lb_add_wall(self.ctx, 0, prm)

    def add_tube(self):
        return lb_add_wall(self.ctx, 1, [])

    def add_obstacle(self, pos, radius):
        return lb_add_wall(self.ctx, 2, [*pos, radius])

    def add_round_tube(self, cx, cy, radius):
        """Round tube along z: nodes at distance >= radius from (cx, cy) are a
        wall at rest (lb_add_wall kind 3)."""
        return lb_add_wall(self.ctx, 3, [cx, cy, radius])

    def set_contact(self, sigma, eps):
        lb_set_contact(self.ctx, sigma, eps)

    def set_force_average(self, on=True):
        lb_set_force_average(self.ctx, on)

    def set_link_options(self, density_of_node=False, velocity_at_node=False):
        lb_set_link_options(self.ctx, density_of_node, velocity_at_node)

    def set_coupling(self, coupling="links"):
        """'links' (bounce-back on links, the default) or 'psm' (partially
        saturated cells); before the first sphere (see lb_set_coupling)."""
        lb_set_coupling(self.ctx, COUPLING[coupling] if isinstance(coupling, str) else int(coupling))

    def set_fields(self, rho, u):
        lb_set_fields(self.ctx, np.reshape(rho, -1), np.reshape(u, (3, -1)))

    def set_populations(self, f):
        lb_set_populations(self.ctx, np.reshape(f, (19, -1)))

    # stepping
    def step(self, n=1):
        lb_step(self.ctx, n)

    def sync(self):
        lb_sync(self.ctx)

    @property
    def steps(self):
        return lb_step_count(self.ctx)

    @property
    def launches(self):
        return lb_kernel_launches(self.ctx)

    # outputs
    def populations(self):
        return lb_get_populations(self.ctx, self.N)

    def fields(self):
        return lb_get_fields(self.ctx, self.N)

    def owner(self):
        return lb_get_owner(self.ctx, self.N)

    def solid_fraction(self):
        return lb_get_solid_fraction(self.ctx, self.N)

    def force_torque(self, oid):
        return lb_get_force_torque(self.ctx, oid)

    def state(self, oid):
        return lb_get_object_state(self.ctx, oid)

    def stresslet(self, oid):
        return lb_get_stresslet(self.ctx, oid)

    def mass(self):
        return lb_get_mass(self.ctx)

    def links(self, oid=0):
        return lb_get_links(self.ctx, oid)

    def checkpoint(self):
        """The run so far as bytes (see lb_checkpoint)."""
        return lb_checkpoint(self.ctx)

    def restore(self, blob):
        """Continue from a checkpoint of a lattice set up the same way."""
        lb_restore(self.ctx, blob)

    def set_sweep_variant(self, variant):
        lb_set_sweep_variant(self.ctx, variant)

    def profile_begin(self):
        lb_profile_begin(self.ctx)

    def profile_end(self):
        return lb_profile_end(self.ctx)
