"""ctypes binding of the cgl C ABI (include/cgl.h).

Argument marshalling only: every step of the scheme runs in the CUDA
kernels of libcgl.so.  Loading fails loudly if the library is missing; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcgl.so")

OK = 0
EINVAL, ECUDA, EOOM, EIDP, ENONFINITE, EDT, ETIMEOUT = -1, -2, -3, -4, -5, -6, -7
BC_PERIODIC, BC_OUTFLOW, BC_FIXED, BC_WALL = 0, 1, 2, 3
SIDES = ("W", "E", "S", "N")
FLUX_ADVECTION, FLUX_BURGERS, FLUX_KPP, FLUX_EULER = 0, 1, 2, 3
MODE_LO, MODE_HO, MODE_WENO, MODE_WENO_L = 0, 1, 2, 3
FL_NONE, FL_LIMITED, FL_LOW = 0, 1, 2
FP64, FP32_MIXED = 0, 1
OPT_FP64_LIMITER = 1
OPT_UNFUSED_SWEEPS = 2
OPT_SUBCELL_DT = 4
OPT_AEC_Q1 = 8
OPT_DTE_REDUCE = 16
BATCH_PERSISTENT, BATCH_PHASES = 0, 1
BASIS_BERNSTEIN, BASIS_LGL = 0, 1
FIELD_UE, FIELD_DTE, FIELD_UBL, FIELD_UBE, FIELD_GAMMA, FIELD_NU, FIELD_BETA = 0, 1, 2, 3, 4, 5, 6
FIELD_GX, FIELD_GY, FIELD_R, FIELD_UDOT = 16, 17, 18, 19


class cgl_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("p", C.c_int32), ("bc_x", C.c_int32),
                ("bc_y", C.c_int32), ("basis", C.c_int32), ("x0", C.c_double),
                ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double)]


class cgl_problem(C.Structure):
    _fields_ = [("flux", C.c_int32), ("mode", C.c_int32), ("flux_limiter", C.c_int32),
                ("k_g", C.c_int32), ("k_u", C.c_int32), ("options", C.c_int32),
                ("vx", C.c_double), ("vy", C.c_double), ("gamma_gas", C.c_double),
                ("umin", C.c_double), ("umax", C.c_double), ("pos_eps", C.c_double),
                ("q", C.c_double), ("r", C.c_double), ("weno_eps", C.c_double),
                ("w_lin", C.c_double), ("gamma_eps", C.c_double), ("cfl", C.c_double),
                ("lambda_floor", C.c_double), ("ubc", C.c_double * 4)]


class cgl_boundary(C.Structure):
    _fields_ = [("kind_lo", C.c_int32 * 4), ("kind_hi", C.c_int32 * 4), ("s0", C.c_double * 4),
                ("s1", C.c_double * 4), ("state_lo", (C.c_double * 4) * 4), ("state_hi", (C.c_double * 4) * 4)]


class cgl_step_info(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_last", C.c_double), ("steps", C.c_int64),
                ("violations", C.c_int64), ("clamps", C.c_int64), ("cfl_violations", C.c_int64),
                ("mass", C.c_double * 4), ("umin", C.c_double * 4), ("umax", C.c_double * 4),
                ("ubar_outside", C.c_int64), ("dte_reduced", C.c_int64)]

    def as_dict(self, nc=4):
        return dict(t=self.t, dt_last=self.dt_last, steps=self.steps, violations=self.violations,
                    clamps=self.clamps, cfl_violations=self.cfl_violations,
                    mass=list(self.mass)[:nc], umin=list(self.umin)[:nc], umax=list(self.umax)[:nc],
                    ubar_outside=self.ubar_outside, dte_reduced=self.dte_reduced)


class CglError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cgl error {status}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes)
_PROTOS = [
    ("cgl_last_error", C.c_char_p, []),
    ("cgl_version", C.c_char_p, []),
    ("cgl_problem_defaults", C.c_int, [C.POINTER(cgl_problem), C.c_int32]),
    ("cgl_debug_tables", C.c_int, [C.c_int32, C.POINTER(C.c_double), C.c_size_t, C.POINTER(C.c_size_t)]),
    ("cgl_debug_basis_tables", C.c_int,
     [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_size_t, C.POINTER(C.c_size_t)]),
    ("cgl_mesh_create", C.c_int, [C.POINTER(cgl_mesh_desc), C.POINTER(C.c_void_p)]),
    ("cgl_mesh_destroy", None, [C.c_void_p]),
    ("cgl_mesh_sizes", C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("cgl_state_create", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("cgl_state_create_external", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                                            C.c_void_p, C.POINTER(C.c_void_p)]),
    ("cgl_set_state_nodal", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("cgl_state_destroy", None, [C.c_void_p]),
    ("cgl_set_problem", C.c_int, [C.c_void_p, C.POINTER(cgl_problem)]),
    ("cgl_set_boundary", C.c_int, [C.c_void_p, C.c_void_p]),
    ("cgl_set_state", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t]),
    ("cgl_get_state", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t]),
    ("cgl_set_state_async", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t]),
    ("cgl_get_state_async", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t]),
    ("cgl_sync", C.c_int, [C.c_void_p]),
    ("cgl_set_base_state", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t]),
    ("cgl_set_time", C.c_int, [C.c_void_p, C.c_double]),
    ("cgl_get_time", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("cgl_step", C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(cgl_step_info)]),
    ("cgl_stage", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.POINTER(cgl_step_info)]),
    ("cgl_time_step", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("cgl_get_field", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.c_size_t]),
    ("cgl_kernel_name", C.c_char_p, [C.c_int32]),
    ("cgl_profile", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    ("cgl_launches_per_step", C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    ("cgl_step_async", C.c_int, [C.c_void_p, C.c_int32]),
    ("cgl_get_counters", C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    ("cgl_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    ("cgl_batch_destroy", None, [C.c_void_p]),
    ("cgl_batch_step", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    ("cgl_batch_step_async", C.c_int, [C.c_void_p, C.c_int32]),
    ("cgl_batch_info", C.c_int, [C.c_void_p] + [C.POINTER(C.c_int32)] * 5),
    ("cgl_batch_set_tiles", C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    ("cgl_batch_get_tiles", C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    ("cgl_batch_autotune", C.c_int, [C.c_void_p, C.c_int32, C.c_char_p]),
    ("cgl_batch_load_tuning", C.c_int, [C.c_void_p, C.c_char_p]),
    ("cgl_batch_debug", C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    ("cgl_batch_set_form", C.c_int, [C.c_void_p, C.c_int32]),
    ("cgl_batch_get_form", C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    ("cgl_gradient_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("cgl_measure_peaks", C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
]


def lib():
    """Load libcgl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built: run `python -m paper_2509_04673_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _PROTOS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(st):
    if st != OK:
        raise CglError(st, lib().cgl_last_error().decode())
    return st


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def problem_struct(prob) -> cgl_problem:
    """Fill a cgl_problem from a dict / dataclass with the same field names."""
    d = prob if isinstance(prob, dict) else prob.as_dict()
    p = cgl_problem()
    check(lib().cgl_problem_defaults(C.byref(p), int(d.get("flux", 0))))
    for name, typ in cgl_problem._fields_:
        if name in ("reserved",) or name not in d:
            continue
        if name == "ubc":
            vals = list(d["ubc"]) + [0.0] * 4
            p.ubc = (C.c_double * 4)(*[float(v) for v in vals[:4]])
        elif typ is C.c_int32:
            setattr(p, name, int(d[name]))
        else:
            setattr(p, name, float(d[name]))
    return p


def boundary_struct(bnd) -> cgl_boundary:
    """Fill a cgl_boundary from {side: {"kind": (lo, hi), "state": (lo, hi),
    "s0": s0, "s1": s1}} for the sides W, E, S, N."""
    b = cgl_boundary()
    for k, side in enumerate(SIDES):
        sd = bnd[side]
        b.kind_lo[k], b.kind_hi[k] = int(sd["kind"][0]), int(sd["kind"][1])
        b.s0[k], b.s1[k] = float(sd["s0"]), float(sd["s1"])
        for slot, arr in ((0, b.state_lo), (1, b.state_hi)):
            vals = [float(v) for v in list(sd["state"][slot])] + [0.0] * 4
            for c in range(4):
                arr[k][c] = vals[c]
    return b


class Mesh:
    def __init__(self, mesh):
        d = mesh if isinstance(mesh, dict) else mesh.as_dict()
        desc = cgl_mesh_desc(int(d["nx"]), int(d["ny"]), int(d["p"]), int(d["bc_x"]), int(d["bc_y"]),
                             int(d.get("basis", 0)),
                             float(d["x0"]), float(d["x1"]), float(d["y0"]), float(d["y1"]))
        h = C.c_void_p()
        check(lib().cgl_mesh_create(C.byref(desc), C.byref(h)))
        self.h = h
        nnx, nny, ne = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().cgl_mesh_sizes(h, C.byref(nnx), C.byref(nny), C.byref(ne)))
        self.nnx, self.nny, self.E = nnx.value, nny.value, ne.value
        self.nx, self.ny, self.p = int(d["nx"]), int(d["ny"]), int(d["p"])

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cgl_mesh_destroy(self.h)
            self.h = None


# u0(x, y, comp, ctx) for cgl_set_state_nodal
NODAL_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_double, C.c_int32, C.c_void_p)


class State:
    """u_device / u_bytes: optional caller-owned device buffer that holds the
    nodal state in place (cgl_state_create_external)."""

    def __init__(self, mesh: Mesh, ncomp: int, precision: int = FP64, stream=None, u_device=None, u_bytes=0):
        self.mesh = mesh
        self.nc = ncomp
        h = C.c_void_p()
        s = C.c_void_p(stream) if stream else None
        if u_device:
            check(lib().cgl_state_create_external(mesh.h, ncomp, precision, C.c_void_p(u_device), int(u_bytes), s,
                                                  C.byref(h)))
        else:
            check(lib().cgl_state_create(mesh.h, ncomp, precision, s, C.byref(h)))
        self.h = h

    def set_state_nodal(self, u0):
        """u_j(0) = u0(x_j, y_j, comp) at the nodal points (host callback)."""
        cb = NODAL_FN(lambda x, y, c, ctx: float(u0(x, y, c)))
        check(lib().cgl_set_state_nodal(self.h, C.cast(cb, C.c_void_p), None))

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cgl_state_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def shape(self):
        return (self.nc, self.mesh.nny, self.mesh.nnx)

    def set_problem(self, prob):
        """Set the problem; a "boundary" entry (per-side table) is passed on
        to cgl_set_boundary, its absence restores the mesh's conditions."""
        p = problem_struct(prob)
        d = prob if isinstance(prob, dict) else prob.as_dict()
        check(lib().cgl_set_boundary(self.h, None))
        check(lib().cgl_set_problem(self.h, C.byref(p)))
        self.set_boundary(d.get("boundary"))

    def set_boundary(self, bnd):
        if bnd is None:
            check(lib().cgl_set_boundary(self.h, None))
        else:
            b = boundary_struct(bnd)
            check(lib().cgl_set_boundary(self.h, C.byref(b)))

    def set_state(self, u):
        a = np.ascontiguousarray(u, dtype=np.float64).reshape(self.shape)
        check(lib().cgl_set_state(self.h, _dptr(a), a.size))

    def set_base_state(self, u):
        a = np.ascontiguousarray(u, dtype=np.float64).reshape(self.shape)
        check(lib().cgl_set_base_state(self.h, _dptr(a), a.size))

    def get_state(self, out=None):
        """The state as float64 [comp][gy][gx]; `out` (C-contiguous float64 of
        that shape, e.g. pinned host memory) receives it in place."""
        a = np.empty(self.shape, dtype=np.float64) if out is None else out
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != self.nc * self.mesh.nny * self.mesh.nnx:
            raise ValueError("out must be C-contiguous float64 of the state's shape")
        check(lib().cgl_get_state(self.h, _dptr(a), a.size))
        return a

    def _host_array(self, a):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != self.nc * self.mesh.nny * self.mesh.nnx:
            raise ValueError("host buffer must be C-contiguous float64 of the state's shape")
        return a

    def set_state_async(self, host):
        """Enqueue the copy of `host` (page-locked float64 [comp][gy][gx])
        into the state (cgl_set_state_async); keep `host` untouched until sync()."""
        a = self._host_array(host)
        check(lib().cgl_set_state_async(self.h, _dptr(a), a.size))

    def get_state_async(self, out):
        """Enqueue the copy of the state into `out` (page-locked float64 of the
        state's shape, cgl_get_state_async); valid after sync()."""
        a = self._host_array(out)
        check(lib().cgl_get_state_async(self.h, _dptr(a), a.size))
        return a

    def sync(self):
        """Wait for the state's work and pipelined copies (cgl_sync)."""
        check(lib().cgl_sync(self.h))

    def set_time(self, t):
        check(lib().cgl_set_time(self.h, float(t)))

    def get_time(self):
        t = C.c_double()
        check(lib().cgl_get_time(self.h, C.byref(t)))
        return t.value

    def step(self, nsteps, t_end=math.inf, raise_on_idp=True):
        info = cgl_step_info()
        st = lib().cgl_step(self.h, int(nsteps), float(t_end), C.byref(info))
        if st != OK and not (st == EIDP and not raise_on_idp):
            check(st)
        return info.as_dict(self.nc)

    def step_async(self, nsteps):
        check(lib().cgl_step_async(self.h, int(nsteps)))

    def counters(self):
        c = np.zeros(4, dtype=np.int64)
        check(lib().cgl_get_counters(self.h, c.ctypes.data_as(C.POINTER(C.c_int64))))
        return dict(violations=int(c[0]), clamps=int(c[1]), cfl_violations=int(c[2]), nonfinite=int(c[3]))

    def stage(self, dt, a, b, raise_on_idp=True):
        info = cgl_step_info()
        st = lib().cgl_stage(self.h, float(dt), float(a), float(b), C.byref(info))
        if st != OK and not (st == EIDP and not raise_on_idp):
            check(st)
        return info.as_dict(self.nc)

    def time_step(self):
        dt = C.c_double()
        check(lib().cgl_time_step(self.h, C.byref(dt)))
        return dt.value

    def profile(self, nsteps):
        """Per-kernel device time (ms) and launch counts over nsteps steps."""
        nk = 32
        ms = np.zeros(nk)
        ln = np.zeros(nk, dtype=np.int64)
        check(lib().cgl_profile(self.h, int(nsteps), nk, _dptr(ms),
                                ln.ctypes.data_as(C.POINTER(C.c_int64))))
        names = [lib().cgl_kernel_name(i).decode() for i in range(nk)]
        return {names[i]: (float(ms[i]), int(ln[i])) for i in range(nk) if names[i]}

    def launches_per_step(self):
        k = C.c_int64()
        check(lib().cgl_launches_per_step(self.h, C.byref(k)))
        return k.value

    def get_field(self, field):
        E, NN = self.mesh.E, self.mesh.nnx * self.mesh.nny
        n = {FIELD_UE: self.nc * E, FIELD_DTE: E, FIELD_UBL: self.nc * E, FIELD_UBE: self.nc * E,
             FIELD_GAMMA: E, FIELD_NU: E, FIELD_BETA: E}.get(field, self.nc * NN)
        a = np.empty(n, dtype=np.float64)
        check(lib().cgl_get_field(self.h, int(field), _dptr(a), n))
        return a


def debug_tables(p: int, basis: int = 0) -> dict:
    """The library's host tables of degree p on the given basis (no GPU needed)."""
    need = C.c_size_t()
    check(lib().cgl_debug_basis_tables(p, basis, None, 0, C.byref(need)))
    buf = np.empty(need.value)
    check(lib().cgl_debug_basis_tables(p, basis, _dptr(buf), buf.size, None))
    n1, nq = p + 1, p + 2
    out, k = {}, 0
    for name, shape in (("M", (n1, n1)), ("C", (n1, n1)), ("D", (n1, n1)), ("Ep", (n1, n1)),
                        ("Em", (n1, n1)), ("xq", (nq,)), ("wq", (nq,)), ("Bq", (nq, n1)),
                        ("dBq", (nq, n1)), ("A2", (n1 * n1, n1 * n1)), ("wl", (n1,)), ("xn", (n1,))):
        sz = int(np.prod(shape))
        out[name] = buf[k:k + sz].reshape(shape)
        k += sz
    return out


class Batch:
    """Many independent FP32-mixed scalar states stepped together (one
    persistent launch per SSP stage, CUDA graph per step)."""

    def __init__(self, states):
        self.states = list(states)
        arr = (C.c_void_p * len(self.states))(*[s.h for s in self.states])
        h = C.c_void_p()
        check(lib().cgl_batch_create(arr, len(self.states), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cgl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self, nsteps):
        v = C.c_int64()
        check(lib().cgl_batch_step(self.h, int(nsteps), C.byref(v)))
        return v.value

    def step_async(self, nsteps):
        check(lib().cgl_batch_step_async(self.h, int(nsteps)))

    def info(self):
        vals = [C.c_int32() for _ in range(5)]
        check(lib().cgl_batch_info(self.h, *[C.byref(v) for v in vals]))
        return dict(zip(("grid", "block", "elem_tiles", "node_tiles", "graph"), [v.value for v in vals]))

    def tiles(self):
        t = (C.c_int32 * 5)()
        check(lib().cgl_batch_get_tiles(self.h, t))
        return list(t)

    def set_tiles(self, tiles):
        t = (C.c_int32 * 5)(*[int(x) for x in tiles])
        check(lib().cgl_batch_set_tiles(self.h, t))

    def autotune(self, steps=2, json_path=None):
        check(lib().cgl_batch_autotune(self.h, int(steps), json_path.encode() if json_path else None))
        return self.tiles()

    def load_tuning(self, json_path):
        check(lib().cgl_batch_load_tuning(self.h, json_path.encode()))

    def debug(self, phantom_blocks, spin_limit):
        check(lib().cgl_batch_debug(self.h, int(phantom_blocks), int(spin_limit)))

    def set_form(self, form):
        check(lib().cgl_batch_set_form(self.h, int(form)))

    def form(self):
        v = C.c_int32()
        check(lib().cgl_batch_get_form(self.h, C.byref(v)))
        return v.value


def gradient_noalloc(mesh: Mesh, u_dev_ptr: int, g_dev_ptr: int, stream=None):
    """Lumped gradient projection into caller-owned device memory without any
    allocation by the library (see cgl_gradient_noalloc in include/cgl.h)."""
    check(lib().cgl_gradient_noalloc(mesh.h, C.c_void_p(u_dev_ptr), C.c_void_p(g_dev_ptr),
                                     C.c_void_p(stream) if stream else None))


def measure_peaks() -> dict:
    """Measured float64 / float32 FMA rates of the current device (FLOP/s)."""
    a, b = C.c_double(), C.c_double()
    check(lib().cgl_measure_peaks(C.byref(a), C.byref(b)))
    return {"fp64_flops": a.value, "fp32_flops": b.value}
