"""Python binding of the B300 block-AMR library (include/amr.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libamr_b300.so.  There is no CPU fallback -- importing works on a
machine without a GPU, but creating a forest there fails with AmrError.

Device memory, streams and pinned host buffers come from PyTorch; torch
tensors are passed to the library as raw pointers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

AMR_OK, AMR_EINVAL, AMR_ENOMEM, AMR_ECAPACITY, AMR_ECUDA = 0, 1, 2, 3, 4
AMR_ETIMEOUT, AMR_EBOUNDS, AMR_ENONPHYS, AMR_ESTATE = 5, 6, 7, 8
PHYS_EULER, PHYS_ADVECTION = 0, 1
AMR_STEP_GRAPH, AMR_STEP_GATHER, AMR_STEP_SSP3, AMR_STEP_RK4, AMR_STEP_SSP43 = 1, 2, 4, 8, 16
# the amr_phase order of the per-phase timing
PHASES = ("ghost_r1", "ghost_r2", "stage", "fluxfix", "dt", "conserved", "flags", "transfer", "mesh_host",
          "pattern_host")
STATUS_NAMES = {0: "AMR_OK", 1: "AMR_EINVAL", 2: "AMR_ENOMEM", 3: "AMR_ECAPACITY", 4: "AMR_ECUDA",
                5: "AMR_ETIMEOUT", 6: "AMR_EBOUNDS", 7: "AMR_ENONPHYS", 8: "AMR_ESTATE"}
KIND_SRL, KIND_F2C, KIND_BC, KIND_C2F = 0, 1, 2, 3

EXPORTED = [
    "amr_create_forest", "amr_destroy_forest", "amr_n_blocks", "amr_get_blocks", "amr_build_ghost_pattern",
    "amr_get_ghost_pattern", "amr_set_state", "amr_get_state", "amr_state_ptr", "amr_set_bc_data",
    "amr_fill_ghosts", "amr_compute_dt", "amr_set_dt", "amr_get_dt", "amr_advance_stage", "amr_step",
    "amr_conserved", "amr_flag", "amr_flag_and_regrid", "amr_sync_status", "amr_last_error",
    "amr_launch_count", "amr_conserved_static", "amr_create_batch", "amr_n_instances", "amr_instance_blocks",
    "amr_get_dts", "amr_conserved_all", "amr_autotune", "amr_features", "amr_mlp_create", "amr_mlp_destroy",
    "amr_mlp_n_params", "amr_mlp_get_params", "amr_mlp_set_params", "amr_mlp_forward", "amr_mlp_gradient",
    "amr_mlp_train", "amr_mlp_adamw_step", "amr_mlp_set_precision", "amr_mlp_flags", "amr_get_config", "amr_save", "amr_load", "amr_write_xdmf", "amr_set_launch_shape",
    "amr_trace", "amr_trace_read",
]


class AmrError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS_NAMES.get(status, str(status)), (": " + msg) if msg else ""))


AllocFn = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FreeFn = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("ndim", C.c_int), ("block_n", C.c_int), ("n_ghost", C.c_int), ("n_var", C.c_int),
                ("ntrees", C.c_int * 3), ("periodic", C.c_int * 3),
                ("lo", C.c_double * 3), ("len", C.c_double * 3),
                ("max_level", C.c_int), ("max_blocks", C.c_int), ("n_states", C.c_int), ("precision", C.c_int),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("bc", C.c_int * 6), ("bc_val", (C.c_double * 8) * 6),
                ("dev_alloc", AllocFn), ("dev_free", FreeFn), ("alloc_ctx", C.c_void_p),
                ("host_only", C.c_int), ("limiter", C.c_int), ("flux", C.c_int), ("gravity", C.c_double * 3),
                ("diagonal_ghosts", C.c_int), ("physics", C.c_int), ("velocity", C.c_double * 3)]


class GhostEntry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("face", C.c_int32), ("dst", C.c_int32), ("src", C.c_int32),
                ("offset", C.c_int32), ("aux", C.c_int32)]


class Stage(C.Structure):
    _fields_ = [("s_out", C.c_int), ("s_deriv", C.c_int), ("n_prev", C.c_int), ("s_prev", C.c_int * 4),
                ("w_prev", C.c_double * 4), ("w_dt", C.c_double), ("update_dt", C.c_int), ("gather_halo", C.c_int)]


class FlagParams(C.Structure):
    _fields_ = [("c_refine", C.c_double), ("c_derefine", C.c_double), ("eps", C.c_double), ("eps_abs", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libamr_b300.so (building it first if asked and missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise AmrError(AMR_ESTATE, "libamr_b300.so is not built (run paper_2605_07612_b300.build)")
        _build.build()
    lib = C.CDLL(path)
    P, vp, i64 = C.POINTER, C.c_void_p, C.c_int64
    sig = {
        "amr_create_forest": [P(Config), C.c_int, P(vp)],
        "amr_get_config": [vp, C.c_int, P(Config)],
        "amr_set_launch_shape": [vp, C.c_int],
        "amr_save": [vp, C.c_char_p, vp],
        "amr_load": [C.c_char_p, vp, P(vp), vp],
        "amr_write_xdmf": [vp, C.c_int, C.c_char_p, vp],
        "amr_destroy_forest": [vp],
        "amr_n_blocks": [vp, P(i64)],
        "amr_get_blocks": [vp, vp, vp, i64, P(i64)],
        "amr_build_ghost_pattern": [vp],
        "amr_get_ghost_pattern": [vp, vp, i64, P(i64)],
        "amr_set_state": [vp, C.c_int, vp, C.c_int, vp],
        "amr_get_state": [vp, C.c_int, vp, C.c_int, vp],
        "amr_state_ptr": [vp, C.c_int, P(vp)],
        "amr_set_bc_data": [vp, vp, i64],
        "amr_fill_ghosts": [vp, C.c_int, vp],
        "amr_compute_dt": [vp, C.c_int, vp],
        "amr_set_dt": [vp, C.c_double, vp],
        "amr_get_dt": [vp, P(C.c_double), vp],
        "amr_advance_stage": [vp, P(Stage), vp],
        "amr_step": [vp, C.c_int, C.c_int, vp],
        "amr_conserved": [vp, C.c_int, vp, vp],
        "amr_flag": [vp, C.c_int, P(FlagParams), vp, vp],
        "amr_flag_and_regrid": [vp, P(FlagParams), vp, P(C.c_int), vp],
        "amr_sync_status": [vp, vp],
        "amr_launch_count": [vp, P(i64)],
        "amr_trace": [vp, C.c_int],
        "amr_trace_read": [vp, vp, vp, C.c_int],
        "amr_create_batch": [vp, vp, C.c_int, P(vp)],
        "amr_n_instances": [vp, P(C.c_int)],
        "amr_instance_blocks": [vp, C.c_int, P(i64), P(i64)],
        "amr_get_dts": [vp, vp, vp],
        "amr_conserved_all": [vp, C.c_int, vp, vp],
        "amr_autotune": [vp, P(C.c_int), P(C.c_double), vp],
        "amr_features": [vp, C.c_int, vp, P(C.c_int), vp],
        "amr_mlp_create": [C.c_int, C.c_uint64, P(vp)],
        "amr_mlp_destroy": [vp],
        "amr_mlp_n_params": [vp, P(i64)],
        "amr_mlp_get_params": [vp, vp, i64],
        "amr_mlp_set_params": [vp, vp, i64],
        "amr_mlp_forward": [vp, vp, i64, vp, vp],
        "amr_mlp_gradient": [vp, vp, vp, i64, vp, vp],
        "amr_mlp_train": [vp, vp, vp, i64, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64, P(C.c_double), vp],
        "amr_mlp_adamw_step": [vp, vp, C.c_double, C.c_double, vp],
        "amr_mlp_set_precision": [vp, C.c_int],
        "amr_mlp_flags": [vp, vp, C.c_int, P(FlagParams), C.c_double, vp, P(i64), vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.amr_last_error.argtypes = [vp]
    lib.amr_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def spec_from_config(c: Config):
    """The synth.MeshSpec of a configuration (inverse of config_from_spec)."""
    import synth
    D = int(c.ndim)
    return synth.MeshSpec(ndim=D, N=int(c.block_n), ng=int(c.n_ghost), ntrees=tuple(int(c.ntrees[d]) for d in range(3)),
                          periodic=tuple(int(c.periodic[d]) for d in range(3)), lo=tuple(float(c.lo[d]) for d in range(3)),
                          length=tuple(float(c.len[d]) for d in range(3)), max_level=int(c.max_level),
                          gamma=float(c.gamma), cfl=float(c.cfl), bc_type=tuple(int(c.bc[f]) for f in range(6)),
                          bc_val=tuple(tuple(float(c.bc_val[f][v]) for v in range(8)) for f in range(6)),
                          limiter=int(c.limiter), flux=int(c.flux), gravity=tuple(float(c.gravity[d]) for d in range(3)),
                          diagonal_ghosts=int(c.diagonal_ghosts), physics=int(c.physics),
                          velocity=tuple(float(c.velocity[d]) for d in range(3)))


def config_from_spec(spec, max_blocks, n_states=2, precision=64, host_only=False) -> Config:
    c = Config()
    c.host_only = 1 if host_only else 0
    c.limiter = int(getattr(spec, "limiter", 0))
    c.flux = int(getattr(spec, "flux", 0))
    gv = getattr(spec, "gravity", (0.0, 0.0, 0.0))
    for d in range(3):
        c.gravity[d] = float(gv[d]) if d < spec.ndim else 0.0
    c.diagonal_ghosts = int(getattr(spec, "diagonal_ghosts", 0))
    c.physics = int(getattr(spec, "physics", 0))
    vel = getattr(spec, "velocity", (0.0, 0.0, 0.0))
    for d in range(3):
        c.velocity[d] = float(vel[d]) if d < spec.ndim else 0.0
    c.ndim, c.block_n, c.n_ghost, c.n_var = spec.ndim, spec.N, spec.ng, spec.nvar
    for d in range(3):
        c.ntrees[d] = int(spec.ntrees[d]) if d < spec.ndim else 1
        c.periodic[d] = int(spec.periodic[d]) if d < spec.ndim else 1
        c.lo[d] = float(spec.lo[d])
        c.len[d] = float(spec.length[d])
    c.max_level = spec.max_level
    c.max_blocks = int(max_blocks)
    c.n_states = int(n_states)
    c.precision = int(precision)
    c.gamma, c.cfl = float(spec.gamma), float(spec.cfl)
    for f in range(6):
        c.bc[f] = int(spec.bc_type[f])
        for v in range(8):
            c.bc_val[f][v] = float(spec.bc_val[f][v]) if v < len(spec.bc_val[f]) else 0.0
    return c


class Forest:
    """A forest of blocks on the current CUDA device (Sec. 2.2-2.3)."""

    def __init__(self, spec, init_level=0, max_blocks=None, n_states=2, precision=64, config: Config | None = None,
                 host_only=False, batch=None):
        """A forest of one mesh (spec, init_level), or -- with batch = list of
        (spec, init_level, max_blocks) -- of several independent instances
        advanced together (amr_create_batch)."""
        self.lib = load()
        self.precision = precision
        self.dtype = np.float64 if precision == 64 else np.float32
        h = C.c_void_p()
        if batch is not None:
            cfgs = (Config * len(batch))()
            levels = (C.c_int * len(batch))()
            for i, (sp, lvl, mb) in enumerate(batch):
                if mb is None:
                    mb = int(np.prod([sp.ntrees[d] << lvl for d in range(sp.ndim)]))
                cfgs[i] = config_from_spec(sp, mb, n_states, precision, host_only)
                levels[i] = int(lvl)
            self.spec = batch[0][0]
            self.specs = [b[0] for b in batch]
            self.cfg = cfgs[0]
            self.n_states = n_states
            st = self.lib.amr_create_batch(cfgs, levels, len(batch), C.byref(h))
            if st != AMR_OK:
                raise AmrError(st, "amr_create_batch")
            self.h = h
            return
        self.spec = spec
        self.specs = [spec]
        if config is None:
            if max_blocks is None:
                max_blocks = int(np.prod([spec.ntrees[d] << init_level for d in range(spec.ndim)]))
            config = config_from_spec(spec, max_blocks, n_states, precision, host_only)
        self.cfg = config
        self.max_blocks = config.max_blocks
        self.n_states = config.n_states
        st = self.lib.amr_create_forest(C.byref(config), int(init_level), C.byref(h))
        if st != AMR_OK:
            raise AmrError(st, "amr_create_forest")
        self.h = h

    # ---- checkpoint, restart, output
    def save(self, path, stream=None):
        """Checkpoint: meshes, configurations, dt and slot 0 (amr_save)."""
        self._check(self.lib.amr_save(self.h, os.fsencode(path), _stream_ptr(stream)), "amr_save")

    @classmethod
    def load(cls, path, n_states=None, host_only=False, stream=None) -> "Forest":
        """Restart from a checkpoint written by save() (amr_load)."""
        lib = load()
        opts = None
        if n_states is not None or host_only:
            opts = Config()
            opts.n_states = int(n_states) if n_states is not None else 2
            opts.host_only = 1 if host_only else 0
        h = C.c_void_p()
        st = lib.amr_load(os.fsencode(path), C.byref(opts) if opts is not None else None, C.byref(h), _stream_ptr(stream))
        if st != AMR_OK:
            raise AmrError(st, "amr_load(%s)" % path)
        self = cls.__new__(cls)
        self.lib = lib
        self.h = h
        n = C.c_int()
        self._check(lib.amr_n_instances(h, C.byref(n)), "amr_n_instances")
        self.specs = []
        for i in range(n.value):
            c = Config()
            self._check(lib.amr_get_config(h, i, C.byref(c)), "amr_get_config")
            self.specs.append(spec_from_config(c))
        self.spec = self.specs[0]
        self.cfg = c
        self.precision = int(c.precision)
        self.dtype = np.float64 if self.precision == 64 else np.float32
        self.n_states = int(c.n_states)
        self.max_blocks = int(c.max_blocks)
        return self

    def get_config(self, inst=0) -> Config:
        c = Config()
        self._check(self.lib.amr_get_config(self.h, int(inst), C.byref(c)), "amr_get_config")
        return c

    def write_xdmf(self, s, base, stream=None):
        """XDMF output of slot s: base.xmf (grid description) and base.bin."""
        self._check(self.lib.amr_write_xdmf(self.h, int(s), os.fsencode(base), _stream_ptr(stream)), "amr_write_xdmf")

    @property
    def n_instances(self) -> int:
        n = C.c_int()
        self._check(self.lib.amr_n_instances(self.h, C.byref(n)), "amr_n_instances")
        return int(n.value)

    def instance_blocks(self, inst):
        """(first block, number of blocks) of an instance."""
        a, b = C.c_int64(), C.c_int64()
        self._check(self.lib.amr_instance_blocks(self.h, int(inst), C.byref(a), C.byref(b)), "amr_instance_blocks")
        return int(a.value), int(b.value)

    def get_dts(self, stream=None) -> np.ndarray:
        out = np.zeros(self.n_instances)
        self._check(self.lib.amr_get_dts(self.h, out.ctypes.data, _stream_ptr(stream)), "amr_get_dts")
        return out

    def conserved_all(self, s, stream=None) -> np.ndarray:
        out = np.zeros((self.n_instances, self.spec.nvar))
        self._check(self.lib.amr_conserved_all(self.h, s, out.ctypes.data, _stream_ptr(stream)), "amr_conserved_all")
        return out

    # ---- plumbing
    def _check(self, st, what):
        if st != AMR_OK:
            msg = self.lib.amr_last_error(self.h)
            raise AmrError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            self.lib.amr_destroy_forest(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- mesh
    @property
    def n(self) -> int:
        n = C.c_int64()
        self._check(self.lib.amr_n_blocks(self.h, C.byref(n)), "amr_n_blocks")
        return int(n.value)

    def blocks(self):
        n = self.n
        lev = np.zeros(max(n, 1), dtype=np.int32)
        g = np.zeros((max(n, 1), 3), dtype=np.int64)
        cnt = C.c_int64()
        self._check(self.lib.amr_get_blocks(self.h, lev.ctypes.data, g.ctypes.data, n, C.byref(cnt)), "amr_get_blocks")
        return lev[:n], g[:n]

    def build_ghost_pattern(self):
        self._check(self.lib.amr_build_ghost_pattern(self.h), "amr_build_ghost_pattern")

    def pattern(self) -> np.ndarray:
        cnt = C.c_int64()
        self._check(self.lib.amr_get_ghost_pattern(self.h, None, 0, C.byref(cnt)), "amr_get_ghost_pattern")
        out = np.zeros((max(cnt.value, 1), 6), dtype=np.int32)
        self._check(self.lib.amr_get_ghost_pattern(self.h, out.ctypes.data, cnt.value, C.byref(cnt)), "amr_get_ghost_pattern")
        return out[:cnt.value]

    # ---- state
    def state_shape(self):
        return (self.n, self.spec.nvar, self.spec.ncell)

    def set_state(self, s, arr, stream=None):
        """arr: numpy array (host) or torch tensor (host or CUDA) with n*V*S^d elements."""
        if isinstance(arr, np.ndarray):
            a = np.ascontiguousarray(arr, dtype=self.dtype)
            assert a.size == self.n * self.spec.nvar * self.spec.ncell
            self._check(self.lib.amr_set_state(self.h, s, a.ctypes.data, 0, _stream_ptr(stream)), "amr_set_state")
        else:
            assert arr.is_contiguous() and arr.numel() == self.n * self.spec.nvar * self.spec.ncell
            on_dev = 1 if arr.is_cuda else 0
            self._check(self.lib.amr_set_state(self.h, s, arr.data_ptr(), on_dev, _stream_ptr(stream)), "amr_set_state")

    def get_state(self, s, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self.state_shape(), dtype=self.dtype)
        if isinstance(out, np.ndarray):
            self._check(self.lib.amr_get_state(self.h, s, out.ctypes.data, 0, _stream_ptr(stream)), "amr_get_state")
        else:
            on_dev = 1 if out.is_cuda else 0
            self._check(self.lib.amr_get_state(self.h, s, out.data_ptr(), on_dev, _stream_ptr(stream)), "amr_get_state")
        return out

    def state_ptr(self, s) -> int:
        p = C.c_void_p()
        self._check(self.lib.amr_state_ptr(self.h, s, C.byref(p)), "amr_state_ptr")
        return int(p.value)

    def set_bc_data(self, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        self._check(self.lib.amr_set_bc_data(self.h, v.ctypes.data, v.size), "amr_set_bc_data")

    # ---- the hot path
    def fill_ghosts(self, s, stream=None):
        self._check(self.lib.amr_fill_ghosts(self.h, s, _stream_ptr(stream)), "amr_fill_ghosts")

    def compute_dt(self, s, stream=None):
        self._check(self.lib.amr_compute_dt(self.h, s, _stream_ptr(stream)), "amr_compute_dt")

    def set_dt(self, dt, stream=None):
        self._check(self.lib.amr_set_dt(self.h, float(dt), _stream_ptr(stream)), "amr_set_dt")

    def get_dt(self, stream=None) -> float:
        d = C.c_double()
        self._check(self.lib.amr_get_dt(self.h, C.byref(d), _stream_ptr(stream)), "amr_get_dt")
        return float(d.value)

    def advance_stage(self, s_out, s_deriv, prev, weights, w_dt, update_dt=False, gather=False, stream=None):
        st = Stage()
        st.s_out, st.s_deriv, st.n_prev = s_out, s_deriv, len(prev)
        for i, (p, w) in enumerate(zip(prev, weights)):
            st.s_prev[i] = p
            st.w_prev[i] = float(w)
        st.w_dt = float(w_dt)
        st.update_dt = 1 if update_dt else 0
        st.gather_halo = 1 if gather else 0
        self._check(self.lib.amr_advance_stage(self.h, C.byref(st), _stream_ptr(stream)), "amr_advance_stage")

    def step(self, n_steps=1, use_graph=False, gather=False, stream=None, scheme="heun"):
        """n_steps time steps; scheme 'heun' (2 slots), 'ssp3' (3), 'ssp43' (3) or 'rk4' (4)."""
        flags = (AMR_STEP_GRAPH if use_graph else 0) | (AMR_STEP_GATHER if gather else 0)
        flags |= {"heun": 0, "ssp3": AMR_STEP_SSP3, "ssp43": AMR_STEP_SSP43, "rk4": AMR_STEP_RK4}[scheme]
        self._check(self.lib.amr_step(self.h, int(n_steps), flags, _stream_ptr(stream)), "amr_step")

    def conserved(self, s, stream=None) -> np.ndarray:
        out = np.zeros(self.spec.nvar)
        self._check(self.lib.amr_conserved(self.h, s, out.ctypes.data, _stream_ptr(stream)), "amr_conserved")
        return out

    def flag(self, s, c_ref=5e-2, c_deref=6.25e-3, eps=1e-2, eps_abs=1e-10, stream=None) -> np.ndarray:
        p = FlagParams(c_ref, c_deref, eps, eps_abs)
        out = np.zeros(max(self.n, 1), dtype=np.int8)
        self._check(self.lib.amr_flag(self.h, s, C.byref(p), out.ctypes.data, _stream_ptr(stream)), "amr_flag")
        return out[:self.n]

    def regrid(self, flags=None, c_ref=5e-2, c_deref=6.25e-3, eps=1e-2, eps_abs=1e-10, stream=None) -> bool:
        p = FlagParams(c_ref, c_deref, eps, eps_abs)
        ch = C.c_int()
        fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.int8)
        self._check(self.lib.amr_flag_and_regrid(self.h, C.byref(p), None if fl is None else fl.ctypes.data,
                                                 C.byref(ch), _stream_ptr(stream)), "amr_flag_and_regrid")
        return bool(ch.value)

    def autotune(self, stream=None):
        """Picks the fastest stage launch shape for this mesh; returns (choice, ms)."""
        ch, ms = C.c_int(), C.c_double()
        self._check(self.lib.amr_autotune(self.h, C.byref(ch), C.byref(ms), _stream_ptr(stream)), "amr_autotune")
        return int(ch.value), float(ms.value)

    def set_launch_shape(self, choice):
        """Stage launch shape by autotune choice code (amr_set_launch_shape)."""
        self._check(self.lib.amr_set_launch_shape(self.h, int(choice)), "amr_set_launch_shape")

    def features(self, s, out=None, stream=None):
        """Block features of slot s as a CUDA tensor [F, n_blocks] (torch)."""
        import torch
        F = C.c_int()
        self._check(self.lib.amr_features(self.h, s, None, C.byref(F), _stream_ptr(stream)), "amr_features")
        if out is None:
            out = torch.empty((F.value, self.n), dtype=torch.float32, device="cuda")
        self._check(self.lib.amr_features(self.h, s, out.data_ptr(), C.byref(F), _stream_ptr(stream)), "amr_features")
        return out

    def mlp_flags(self, model, s, tau=0.9, c_ref=5e-2, c_deref=6.25e-3, eps=1e-2, eps_abs=1e-10, stream=None):
        """(flags, number of blocks that fell back to the criterion)."""
        p = FlagParams(c_ref, c_deref, eps, eps_abs)
        out = np.zeros(max(self.n, 1), dtype=np.int8)
        nf = C.c_int64()
        self._check(self.lib.amr_mlp_flags(self.h, model.h, s, C.byref(p), float(tau), out.ctypes.data, C.byref(nf),
                                           _stream_ptr(stream)), "amr_mlp_flags")
        return out[:self.n], int(nf.value)

    def sync_status(self, stream=None) -> int:
        return int(self.lib.amr_sync_status(self.h, _stream_ptr(stream)))

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.amr_launch_count(self.h, C.byref(n)), "amr_launch_count")
        return int(n.value)

    def trace(self, on=True):
        """Per-phase timing on or off (steps then run without a CUDA graph)."""
        self._check(self.lib.amr_trace(self.h, int(bool(on))), "amr_trace")

    def trace_read(self, reset=True) -> dict:
        """{phase name: (total ms, records)} of everything traced so far."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        n = np.zeros(len(PHASES), dtype=np.int64)
        self._check(self.lib.amr_trace_read(self.h, ms.ctypes.data, n.ctypes.data, int(bool(reset))), "amr_trace_read")
        return {p: (float(ms[i]), int(n[i])) for i, p in enumerate(PHASES)}


class Mlp:
    """Learned refinement-flag predictor (amr_mlp_*): F -> 64 -> 64 -> 3."""

    def __init__(self, n_features, seed=0):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.amr_mlp_create(int(n_features), C.c_uint64(seed), C.byref(h))
        if st != AMR_OK:
            raise AmrError(st, "amr_mlp_create")
        self.h = h
        self.F = n_features
        n = C.c_int64()
        self.lib.amr_mlp_n_params(self.h, C.byref(n))
        self.P = int(n.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.amr_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != AMR_OK:
            raise AmrError(st, what)

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.P, dtype=np.float32)
        self._check(self.lib.amr_mlp_get_params(self.h, out.ctypes.data, self.P), "amr_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.amr_mlp_set_params(self.h, p.ctypes.data, self.P), "amr_mlp_set_params")

    def forward(self, x, stream=None):
        """x: CUDA float32 tensor [F, n] -> probabilities [n, 3] (CUDA tensor)."""
        import torch
        n = x.shape[1]
        prob = torch.empty((n, 3), dtype=torch.float32, device=x.device)
        self._check(self.lib.amr_mlp_forward(self.h, x.data_ptr(), n, prob.data_ptr(), _stream_ptr(stream)), "amr_mlp_forward")
        return prob

    def gradient(self, x, y, stream=None):
        """(loss, gradient) of the mean cross-entropy; x [F, n], y [n] int8 classes (CUDA tensors)."""
        import torch
        g = torch.empty(self.P + 1, dtype=torch.float32, device=x.device)
        self._check(self.lib.amr_mlp_gradient(self.h, x.data_ptr(), y.data_ptr(), x.shape[1], g.data_ptr(),
                                              _stream_ptr(stream)), "amr_mlp_gradient")
        g = g.cpu().numpy()
        return float(g[-1]), g[:-1]

    def set_precision(self, bits):
        """16: BF16 tensor-core passes (default); 32: FP32 CUDA-core passes."""
        self._check(self.lib.amr_mlp_set_precision(self.h, int(bits)), "amr_mlp_set_precision")

    def adamw_step(self, grad, lr, weight_decay=0.0, stream=None):
        """One AdamW step with a caller-supplied gradient (CUDA float32 tensor [P])."""
        self._check(self.lib.amr_mlp_adamw_step(self.h, grad.data_ptr(), float(lr), float(weight_decay), _stream_ptr(stream)),
                    "amr_mlp_adamw_step")

    def train(self, x, y, epochs=20, batch=256, lr=3e-3, weight_decay=1e-4, seed=0, stream=None) -> float:
        loss = C.c_double()
        self._check(self.lib.amr_mlp_train(self.h, x.data_ptr(), y.data_ptr(), x.shape[1], int(epochs), int(batch), float(lr),
                                           float(weight_decay), C.c_uint64(seed), C.byref(loss), _stream_ptr(stream)),
                    "amr_mlp_train")
        return float(loss.value)
