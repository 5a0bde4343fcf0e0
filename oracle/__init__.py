"""Python access to the FP64 CPU oracle (amr_oracle.c) -- test infrastructure.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It never imports the CUDA package, and the CUDA package
never imports it.

The shared library is compiled on first use (gcc -O2 -ffp-contract=off
-fopenmp), or ahead of time by `build()`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amr_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None

KIND_SRL, KIND_F2C, KIND_BC, KIND_C2F = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile amr_oracle.c into _build/liborc.so if missing or stale."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _OUT)
    return _OUT


class Params(C.Structure):
    _fields_ = [("ndim", C.c_int), ("N", C.c_int), ("ng", C.c_int), ("nvar", C.c_int),
                ("ntrees", C.c_int * 3), ("periodic", C.c_int * 3),
                ("lo", C.c_double * 3), ("len", C.c_double * 3),
                ("max_level", C.c_int), ("gamma", C.c_double), ("cfl", C.c_double),
                ("bc_type", C.c_int * 6), ("bc_val", (C.c_double * 8) * 6),
                ("limiter", C.c_int), ("flux", C.c_int), ("gravity", C.c_double * 3), ("diagonal", C.c_int),
                ("physics", C.c_int), ("velocity", C.c_double * 3)]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            vp = C.c_void_p
            lib.orc_mesh_new.restype = vp
            lib.orc_mesh_new.argtypes = [P(Params), C.c_int]
            lib.orc_mesh_free.argtypes = [vp]
            lib.orc_n_blocks.restype = C.c_int
            lib.orc_n_blocks.argtypes = [vp]
            lib.orc_get_blocks.argtypes = [vp, vp, vp]
            lib.orc_adapt.restype = vp
            lib.orc_adapt.argtypes = [vp, vp]
            lib.orc_check_balance.restype = C.c_int
            lib.orc_check_balance.argtypes = [vp]
            lib.orc_pattern.restype = C.c_int64
            lib.orc_pattern.argtypes = [vp, vp, C.c_int64]
            lib.orc_fill_ghosts.restype = C.c_int
            lib.orc_fill_ghosts.argtypes = [vp, vp, vp]
            lib.orc_stage.restype = C.c_int
            lib.orc_stage.argtypes = [vp, vp, vp, C.c_int, vp, vp, C.c_double]
            lib.orc_max_speed.restype = C.c_double
            lib.orc_max_speed.argtypes = [vp, vp]
            lib.orc_limited_slope.restype = C.c_double
            lib.orc_limited_slope.argtypes = [C.c_int, C.c_double, C.c_double]
            lib.orc_cell_faces.restype = None
            lib.orc_cell_faces.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, vp, vp]
            lib.orc_weno5.restype = C.c_double
            lib.orc_weno5.argtypes = [C.c_double] * 5
            lib.orc_face_flux.restype = None
            lib.orc_face_flux.argtypes = [P(Params), C.c_int, vp, vp, vp]
            lib.orc_conserved.argtypes = [vp, vp, vp]
            lib.orc_lohner_flags.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, C.c_double, vp]
            lib.orc_lohner_scores.argtypes = [vp, vp, C.c_double, C.c_double, vp]
            lib.orc_transfer.restype = C.c_int
            lib.orc_transfer.argtypes = [vp, vp, vp, vp]
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_get_threads.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def params_from_spec(spec) -> Params:
    p = Params()
    p.ndim, p.N, p.ng, p.nvar = spec.ndim, spec.N, spec.ng, spec.nvar
    for d in range(3):
        p.ntrees[d] = int(spec.ntrees[d]) if d < spec.ndim else 1
        p.periodic[d] = int(spec.periodic[d]) if d < spec.ndim else 1
        p.lo[d] = float(spec.lo[d])
        p.len[d] = float(spec.length[d])
    p.max_level = spec.max_level
    p.gamma, p.cfl = spec.gamma, spec.cfl
    for f in range(6):
        p.bc_type[f] = int(spec.bc_type[f])
        for v in range(8):
            p.bc_val[f][v] = float(spec.bc_val[f][v]) if v < len(spec.bc_val[f]) else 0.0
    p.limiter = int(getattr(spec, "limiter", 0))
    p.flux = int(getattr(spec, "flux", 0))
    gv = getattr(spec, "gravity", (0.0, 0.0, 0.0))
    for d in range(3):
        p.gravity[d] = float(gv[d]) if d < spec.ndim else 0.0
    p.diagonal = int(getattr(spec, "diagonal_ghosts", 0))
    p.physics = int(getattr(spec, "physics", 0))
    vel = getattr(spec, "velocity", (0.0, 0.0, 0.0))
    for d in range(3):
        p.velocity[d] = float(vel[d]) if d < spec.ndim else 0.0
    return p


def limited_slope(limiter: int, a: float, b: float) -> float:
    """The MUSCL slope limiter (0 minmod, 1 MC, 2 van Leer) on one pair of
    one-sided differences."""
    return float(_lib_handle().orc_limited_slope(int(limiter), float(a), float(b)))


def cell_faces(limiter: int, wm: float, w0: float, wp: float):
    """(minus, plus): the values of cell w0 at its left and right faces from
    its neighbours (limiters 0 minmod, 1 MC, 2 van Leer, 4 Koren, 5 WENO3,
    6 first-order upwind)."""
    lo, hi = C.c_double(), C.c_double()
    _lib_handle().orc_cell_faces(int(limiter), float(wm), float(w0), float(wp), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def weno5(a, b, c, d, e) -> float:
    """The WENO5 face value right of c from the five cells a..e."""
    return float(_lib_handle().orc_weno5(float(a), float(b), float(c), float(d), float(e)))


def face_flux(spec, n: int, wL, wR) -> np.ndarray:
    """The numerical flux (spec.flux: 0 Rusanov, 1 HLL) along dimension n
    between primitive states wL and wR (Euler, or the advected scalar)."""
    V = spec.nvar
    a = np.ascontiguousarray(wL, dtype=np.float64)
    b = np.ascontiguousarray(wR, dtype=np.float64)
    F = np.zeros(V)
    p = params_from_spec(spec)
    _lib_handle().orc_face_flux(C.byref(p), int(n), a.ctypes.data, b.ctypes.data, F.ctypes.data)
    return F


def set_threads(n: int) -> None:
    _lib_handle().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_lib_handle().orc_get_threads())


class Mesh:
    """A leaf list of the oracle forest (Sec. 2.2) plus the problem spec."""

    def __init__(self, spec, init_level: int = 0, _handle=None):
        self.spec = spec
        self._lib = _lib_handle()
        self._p = params_from_spec(spec)
        self._h = _handle if _handle is not None else self._lib.orc_mesh_new(C.byref(self._p), int(init_level))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_mesh_free(h)
            self._h = None

    @property
    def n(self) -> int:
        return int(self._lib.orc_n_blocks(self._h))

    def blocks(self):
        n = self.n
        lev = np.zeros(n, dtype=np.int32)
        g = np.zeros((n, 3), dtype=np.int64)
        self._lib.orc_get_blocks(self._h, _ptr(lev), _ptr(g))
        return lev, g

    def adapt(self, flags) -> "Mesh":
        f = np.ascontiguousarray(flags, dtype=np.int8)
        assert f.shape == (self.n,)
        return Mesh(self.spec, _handle=self._lib.orc_adapt(self._h, _ptr(f)))

    def balanced(self) -> bool:
        return bool(self._lib.orc_check_balance(self._h))

    def pattern(self) -> np.ndarray:
        """Canonical ghost pattern [n, 6] int32 (kind, face, dst, src, offset, aux)."""
        cnt = self._lib.orc_pattern(self._h, None, 0)
        if cnt < 0:
            raise RuntimeError("oracle: ghost classification failed (2:1 balance broken)")
        out = np.zeros((max(cnt, 1), 6), dtype=np.int32)
        self._lib.orc_pattern(self._h, _ptr(out), cnt)
        return out[:cnt]

    def new_state(self) -> np.ndarray:
        return np.zeros((self.n, self.spec.nvar, self.spec.ncell))

    def fill_ghosts(self, u: np.ndarray, bc_data: np.ndarray | None = None) -> None:
        assert u.dtype == np.float64 and u.flags.c_contiguous
        bd = None if bc_data is None else np.ascontiguousarray(bc_data, dtype=np.float64)
        rc = self._lib.orc_fill_ghosts(self._h, _ptr(u), None if bd is None else _ptr(bd))
        if rc != 0:
            raise RuntimeError("oracle: ghost fill failed")

    def stage(self, ud, uo, prev, weights, dt_eff) -> int:
        """uo = dt_eff F(ud) + sum_i weights[i] prev[i] (Eq. 5), with flux fixing."""
        arr = (C.c_void_p * max(1, len(prev)))(*[p.ctypes.data for p in prev])
        w = np.ascontiguousarray(weights, dtype=np.float64)
        return int(self._lib.orc_stage(self._h, _ptr(ud), _ptr(uo), len(prev),
                                       C.cast(arr, C.c_void_p), _ptr(w), float(dt_eff)))

    def max_speed(self, u) -> float:
        return float(self._lib.orc_max_speed(self._h, _ptr(u)))

    def dt(self, u) -> float:
        return self.spec.cfl / self.max_speed(u)

    def conserved(self, u) -> np.ndarray:
        s = np.zeros(self.spec.nvar)
        self._lib.orc_conserved(self._h, _ptr(u), _ptr(s))
        return s

    def lohner_flags(self, u, c_ref=5e-2, c_deref=6.25e-3, eps=1e-2, eps_abs=1e-10) -> np.ndarray:
        f = np.zeros(self.n, dtype=np.int8)
        self._lib.orc_lohner_flags(self._h, _ptr(u), c_ref, c_deref, eps, eps_abs, _ptr(f))
        return f

    def lohner_scores(self, u, eps=1e-2, eps_abs=1e-10) -> np.ndarray:
        """Largest criterion value of each block (what lohner_flags compares
        with the thresholds)."""
        sc = np.zeros(self.n, dtype=np.float64)
        self._lib.orc_lohner_scores(self._h, _ptr(u), eps, eps_abs, _ptr(sc))
        return sc

    def transfer(self, u_old, new_mesh: "Mesh") -> np.ndarray:
        out = new_mesh.new_state()
        rc = self._lib.orc_transfer(self._h, _ptr(u_old), new_mesh._h, _ptr(out))
        if rc != 0:
            raise RuntimeError("oracle: a block changed by more than one level")
        return out


def heun_step(mesh: Mesh, u0: np.ndarray, u1: np.ndarray, dt: float | None = None, bc_data=None) -> float:
    """One step of Heun's method, Eq. 6-7, with ghost fills before each stage.

    dt defaults to CFL / max speed of u0 (Sec. 3.2).  Returns the dt used."""
    mesh.fill_ghosts(u0, bc_data)
    if dt is None:
        dt = mesh.dt(u0)
    if mesh.stage(u0, u1, [u0], [1.0], dt):
        raise FloatingPointError("oracle: non-physical state in stage 1")
    mesh.fill_ghosts(u1, bc_data)
    if mesh.stage(u1, u0, [u0, u1], [0.5, 0.5], 0.5 * dt):
        raise FloatingPointError("oracle: non-physical state in stage 2")
    return dt


def rk_combine(L, u: np.ndarray, dt: float, scheme: str) -> np.ndarray:
    """One step of an explicit Runge-Kutta method for u' = L(u) (Sec. 3.1
    lists Heun's method and higher-order SSP and classical schemes):
      heun  u1 = u + dt L(u);  u+ = (u + u1 + dt L(u1)) / 2            (Eq. 6-7)
      ssp3  Shu & Osher's three-stage SSP method, in their convex form:
            u1 = u + dt L(u);  u2 = 3/4 u + 1/4 (u1 + dt L(u1));
            u+ = 1/3 u + 2/3 (u2 + dt L(u2))
      ssp43 the optimal four-stage, third-order SSP method (Spiteri & Ruuth):
            u1 = u + dt/2 L(u);  u2 = u1 + dt/2 L(u1);
            u3 = 2/3 u + 1/3 (u2 + dt/2 L(u2));  u+ = u3 + dt/2 L(u3)
      rk4   the classical method: k1 = L(u), k2 = L(u + dt/2 k1),
            k3 = L(u + dt/2 k2), k4 = L(u + dt k3),
            u+ = u + dt/6 (k1 + 2 k2 + 2 k3 + k4)
    L is any function of one array; returns the new array."""
    if scheme == "heun":
        u1 = u + dt * L(u)
        return 0.5 * u + 0.5 * (u1 + dt * L(u1))
    if scheme == "ssp3":
        u1 = u + dt * L(u)
        u2 = 0.75 * u + 0.25 * (u1 + dt * L(u1))
        return u / 3.0 + 2.0 / 3.0 * (u2 + dt * L(u2))
    if scheme == "ssp43":
        u1 = u + 0.5 * dt * L(u)
        u2 = u1 + 0.5 * dt * L(u1)
        u3 = 2.0 / 3.0 * u + 1.0 / 3.0 * (u2 + 0.5 * dt * L(u2))
        return u3 + 0.5 * dt * L(u3)
    if scheme == "rk4":
        k1 = L(u)
        k2 = L(u + 0.5 * dt * k1)
        k3 = L(u + 0.5 * dt * k2)
        k4 = L(u + dt * k3)
        return u + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    raise ValueError(scheme)


def flux_operator(mesh: Mesh, bc_data=None):
    """L(u): ghost fill, then the flux divergence of Eq. 5 with flux fixing
    (one stage with no previous states and dt_eff = 1)."""
    def L(u):
        mesh.fill_ghosts(u, bc_data)
        out = np.zeros_like(u)
        if mesh.stage(u, out, [], [], 1.0):
            raise FloatingPointError("oracle: non-physical state")
        return out
    return L


def rk_step(mesh: Mesh, u0: np.ndarray, scheme: str, dt: float | None = None, bc_data=None) -> float:
    """One time step of `scheme` on u0 in place (interior cells); dt defaults
    to CFL / max speed of u0 (Sec. 3.2).  Returns the dt used."""
    if dt is None:
        dt = mesh.dt(u0)
    u0[...] = rk_combine(flux_operator(mesh, bc_data), u0, dt, scheme)
    return dt


def run_heun(mesh: Mesh, u0: np.ndarray, nsteps: int, bc_data=None) -> list:
    u1 = np.zeros_like(u0)
    return [heun_step(mesh, u0, u1, bc_data=bc_data) for _ in range(nsteps)]
