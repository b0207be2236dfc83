"""Thin ctypes binding of include/cpic.h (argument marshalling only).

Every function of the C ABI is exposed under the same name and returns the status code;
``check`` turns a non-zero status into an exception carrying cpic_last_error(). The
``Run`` class wraps one run handle for convenience (numpy in, numpy out; torch tensors may
be passed for device pointers). No arithmetic of the method happens here: if the compiled
library is missing, ``load`` raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpic.so")

CPIC_OK = 0
CPIC_ERR_INVALID, CPIC_ERR_OOM, CPIC_ERR_CUDA, CPIC_ERR_NOT_CONVERGED = -1, -2, -3, -4
CPIC_ERR_TIMEOUT, CPIC_ERR_NONFINITE, CPIC_ERR_BUSY, CPIC_ERR_STATE = -5, -6, -7, -8
CPIC_ERR_CAPACITY, CPIC_ERR_NOT_BUILT, CPIC_ERR_CANCELLED = -9, -10, -11
CPIC_BC_PERIODIC, CPIC_BC_DIRICHLET, CPIC_BC_NEUMANN = 0, 1, 2
CPIC_PBC_PERIODIC, CPIC_PBC_ABSORB, CPIC_PBC_REFLECT = 0, 1, 2
CPIC_MAP_SINE, CPIC_MAP_ANNULUS, CPIC_MAP_SPHERE_AXISYM, CPIC_MAP_SHELL = 1, 2, 3, 4
CPIC_SOLVER_MG, CPIC_SOLVER_BICGSTAB = 0, 1
CPIC_BATCH_AUTO, CPIC_BATCH_BRANCHES, CPIC_BATCH_PERSISTENT = 0, 1, 2
MAX_SPECIES = 4
GYRO_BORIS, GYRO_CYCLOTRONIC = 0, 1  # cpic_set_gyro_integrator kinds
MG_COARSE_REDISCRETIZED, MG_COARSE_GALERKIN = 0, 1  # cpic_set_multigrid
MG_INTERP_BILINEAR, MG_INTERP_OPERATOR = 0, 1
MG_SMOOTH_POINT, MG_SMOOTH_LINE = 0, 1


class cpic_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("field_bc", ctypes.c_int32 * 6),
        ("field_bc_value", ctypes.c_double * 6),
        ("particle_bc", ctypes.c_int32 * 6),
        ("dt", ctypes.c_double),
        ("background", ctypes.c_double),
        ("axisymmetric", ctypes.c_int32),
        ("n_species", ctypes.c_int32),
        ("q", ctypes.c_double * MAX_SPECIES),
        ("m", ctypes.c_double * MAX_SPECIES),
        ("w", ctypes.c_double * MAX_SPECIES),
        ("capacity", ctypes.c_int64 * MAX_SPECIES),
        ("sort_interval", ctypes.c_int32),
        ("mg_max_cycles", ctypes.c_int32),
        ("mg_rtol", ctypes.c_double),
    ]


class cpic_diag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("field_energy", ctypes.c_double),
        ("kinetic_energy", ctypes.c_double),
        ("n_particles", ctypes.c_int64 * MAX_SPECIES),
        ("absorbed", (ctypes.c_int64 * 6) * MAX_SPECIES),
        ("injected", ctypes.c_int64 * MAX_SPECIES),
        ("dropped", ctypes.c_int64 * MAX_SPECIES),
        ("nonfinite", ctypes.c_int64),
        ("mg_cycles", ctypes.c_int32),
        ("mg_residual", ctypes.c_double),
        ("pc_face_only", ctypes.c_int32),
        ("object_potential", ctypes.c_double),
        ("object_charge", ctypes.c_double),
    ]


CPIC_REQ_CYLINDER = 0
CPIC_REQ_SPHERE = 1


class cpic_server_opts(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_size_t),
        ("max_active", ctypes.c_int32),
        ("steps_per_slice", ctypes.c_int32),
        ("sort_interval", ctypes.c_int32),
    ]


class cpic_request(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("particles_per_species", ctypes.c_int64),
        ("phi_object", ctypes.c_double),
        ("density", ctypes.c_double),
        ("temperature", ctypes.c_double),
        ("mass_ratio", ctypes.c_double),
        ("r_object", ctypes.c_double),
        ("r_outer", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("steps", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class cpic_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("ticket", ctypes.c_uint64),
        ("steps", ctypes.c_int32),
        ("queue_s", ctypes.c_double),
        ("latency_s", ctypes.c_double),
        ("particle_steps", ctypes.c_int64),
        ("field_energy", ctypes.c_double),
        ("kinetic_energy", ctypes.c_double),
        ("n_particles", ctypes.c_int64 * 2),
        ("absorbed_object", ctypes.c_int64 * 2),
        ("absorbed_outer", ctypes.c_int64 * 2),
        ("injected", ctypes.c_int64 * 2),
        ("current_object", ctypes.c_double * 2),
        ("mg_cycles", ctypes.c_int32),
        ("message", ctypes.c_char * 160),
    ]


TUNE_CANDIDATES = 5


class cpic_tuning(ctypes.Structure):
    _fields_ = [
        ("sort_interval", ctypes.c_int32),
        ("interval", ctypes.c_int32 * TUNE_CANDIDATES),
        ("ms_per_step", ctypes.c_float * TUNE_CANDIDATES),
        ("chunk", ctypes.c_int32),
        ("chunks", ctypes.c_int32 * TUNE_CANDIDATES),
        ("ms_chunk", ctypes.c_float * TUNE_CANDIDATES),
        ("tile", ctypes.c_int32),
        ("ms_tile", ctypes.c_float * 2),
    ]


_lib = None
P = ctypes.c_void_p
_SIGS = {
    "cpic_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "cpic_last_error": ([], ctypes.c_char_p),
    "cpic_abi_version": ([], ctypes.c_int),
    "cpic_kernel_launches": ([], ctypes.c_int64),
    "cpic_query_footprint": ([ctypes.POINTER(cpic_config), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "cpic_create": ([ctypes.POINTER(cpic_config), P, ctypes.c_size_t, P, ctypes.POINTER(P)], ctypes.c_int),
    "cpic_destroy": ([P], ctypes.c_int),
    "cpic_set_stream": ([P, P], ctypes.c_int),
    "cpic_set_map_vertices": ([P, P], ctypes.c_int),
    "cpic_set_map_analytic": ([P, ctypes.c_int, P, ctypes.c_int], ctypes.c_int),
    "cpic_load_particles": ([P, ctypes.c_int, ctypes.c_int64, P, P, P], ctypes.c_int),
    "cpic_get_particles": ([P, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), P, P, P], ctypes.c_int),
    "cpic_set_floating": ([P, ctypes.c_int, ctypes.c_double], ctypes.c_int),
    "cpic_get_collection": ([P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64], ctypes.c_int),
    "cpic_set_magnetic_field": ([P, P], ctypes.c_int),
    "cpic_set_gyro_integrator": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_set_multigrid": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "cpic_set_injection": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, ctypes.c_uint64],
                           ctypes.c_int),
    "cpic_initialize": ([P], ctypes.c_int),
    "cpic_step": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_step_particles": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_load_maxwellian": ([P, ctypes.c_int, ctypes.c_int64, ctypes.c_double, P, ctypes.c_uint64], ctypes.c_int),
    "cpic_batch_create": ([ctypes.c_int, P, ctypes.POINTER(P)], ctypes.c_int),
    "cpic_batch_destroy": ([P], ctypes.c_int),
    "cpic_batch_add": ([P, P], ctypes.c_int),
    "cpic_batch_remove": ([P, P], ctypes.c_int),
    "cpic_batch_size": ([P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cpic_batch_step": ([P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "cpic_batch_set_mode": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_batch_synchronize": ([P], ctypes.c_int),
    "cpic_get_config": ([P, P], ctypes.c_int),
    "cpic_set_sort_interval": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_set_solver": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_set_push_tuning": ([P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "cpic_autotune": ([P, ctypes.c_int, P], ctypes.c_int),
    "cpic_checkpoint": ([P, ctypes.c_char_p], ctypes.c_int),
    "cpic_restore": ([ctypes.c_char_p, P, ctypes.c_size_t, P, ctypes.POINTER(P)], ctypes.c_int),
    "cpic_server_start": ([P, ctypes.POINTER(P)], ctypes.c_int),
    "cpic_server_submit": ([P, P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "cpic_server_poll": ([P, ctypes.c_uint64, P], ctypes.c_int),
    "cpic_server_cancel": ([P, ctypes.c_uint64], ctypes.c_int),
    "cpic_server_stats": ([P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "cpic_server_stop": ([P], ctypes.c_int),
    "cpic_vertex_field": ([P], ctypes.c_int),
    "cpic_push": ([P], ctypes.c_int),
    "cpic_deposit": ([P], ctypes.c_int),
    "cpic_kick": ([P, ctypes.c_double], ctypes.c_int),
    "cpic_inject": ([P], ctypes.c_int),
    "cpic_sort": ([P], ctypes.c_int),
    "cpic_solve_field": ([P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cpic_get_diag": ([P, ctypes.POINTER(cpic_diag)], ctypes.c_int),
    "cpic_get_phi": ([P, P], ctypes.c_int),
    "cpic_set_phi": ([P, P], ctypes.c_int),
    "cpic_get_charge": ([P, ctypes.c_int, P], ctypes.c_int),
    "cpic_get_vertex_tables": ([P, P, P], ctypes.c_int),
    "cpic_get_geometry": ([P, P, P], ctypes.c_int),
    "cpic_synchronize": ([P], ctypes.c_int),
    "cpic_sort_cells_noalloc": ([ctypes.c_int, P, ctypes.c_int64, P, P, P, P, P, P, P, P], ctypes.c_int),
    "cpic_profile": ([P, ctypes.c_int], ctypes.c_int),
    "cpic_profile_read": ([P, P, P], ctypes.c_int),
}
PHASES = ("field", "push", "inject", "sort", "solve")


class CpicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cpic status {status}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load libcpic.so (built by paper_1311_2286_gb300/build.py). Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def check(status: int):
    if status != CPIC_OK:
        msg = load().cpic_last_error()
        raise CpicError(status, msg.decode() if msg else "")
    return status


def __getattr__(name):
    if name.startswith("cpic_") and name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def make_config(dim, n, field_bc, field_bc_value, particle_bc, dt, species, background=0.0,
                axisymmetric=False, sort_interval=0, mg_max_cycles=0, mg_rtol=0.0):
    """species: list of (q, m, w, capacity)."""
    c = cpic_config()
    c.dim = dim
    for a in range(3):
        c.n[a] = n[a] if a < len(n) else 1
    for f in range(6):
        c.field_bc[f] = field_bc[f] if f < len(field_bc) else 0
        c.field_bc_value[f] = field_bc_value[f] if f < len(field_bc_value) else 0.0
        c.particle_bc[f] = particle_bc[f] if f < len(particle_bc) else 0
    c.dt = dt
    c.background = background
    c.axisymmetric = 1 if axisymmetric else 0
    c.n_species = len(species)
    for s, (q, m, w, cap) in enumerate(species):
        c.q[s], c.m[s], c.w[s], c.capacity[s] = q, m, w, cap
    c.sort_interval = sort_interval
    c.mg_max_cycles = mg_max_cycles
    c.mg_rtol = mg_rtol
    return c


def config_from_workload(wl, sort_interval=0, mg_max_cycles=0, mg_rtol=0.0):
    return make_config(wl.dim, wl.n, wl.field_bc, wl.field_bc_value, wl.particle_bc, wl.dt,
                       [(s.q, s.m, s.w, max(s.capacity, p.n)) for s, p in zip(wl.species, wl.particles)],
                       background=wl.background, axisymmetric=wl.omega_axisym, sort_interval=sort_interval,
                       mg_max_cycles=mg_max_cycles, mg_rtol=mg_rtol)


class Run:
    """One simulation run (owns its cpic_run handle)."""

    def __init__(self, cfg: cpic_config, arena=None, stream=None):
        lib = load()
        self.cfg = cfg
        self.D = cfg.dim
        self.n = tuple(cfg.n[a] for a in range(cfg.dim))
        self.ncell = int(np.prod(self.n))
        self.nvert = int(np.prod([x + 1 for x in self.n]))
        self._arena = arena
        h = ctypes.c_void_p()
        nbytes = 0
        if arena is not None:
            nbytes = arena.numel() * arena.element_size() if hasattr(arena, "numel") else arena.nbytes
        check(lib.cpic_create(ctypes.byref(cfg), _ptr(arena), nbytes, stream, ctypes.byref(h)))
        self.h = h

    @staticmethod
    def footprint(cfg: cpic_config) -> int:
        n = ctypes.c_size_t()
        check(load().cpic_query_footprint(ctypes.byref(cfg), ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            check(load().cpic_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup
    def set_stream(self, stream):
        check(load().cpic_set_stream(self.h, stream))

    def set_map_vertices(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        check(load().cpic_set_map_vertices(self.h, _ptr(X)))

    def set_map_analytic(self, map_id, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        check(load().cpic_set_map_analytic(self.h, map_id, _ptr(p), p.size))

    def load_particles(self, sp, cell, t, v):
        if hasattr(cell, "data_ptr"):
            n = cell.shape[0]
            check(load().cpic_load_particles(self.h, sp, n, _ptr(cell), _ptr(t), _ptr(v)))
            return
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        check(load().cpic_load_particles(self.h, sp, cell.shape[0], _ptr(cell), _ptr(t), _ptr(v)))

    def load_maxwellian(self, sp, n, vth, seed, drift=None):
        """Device-side Maxwellian load of species sp, uniform in physical space."""
        d = None if drift is None else np.ascontiguousarray(drift, dtype=np.float64)
        check(load().cpic_load_maxwellian(self.h, sp, n, vth, _ptr(d), seed))

    def set_injection(self, sp, face, density, vth, seed, drift=None):
        d = None if drift is None else np.ascontiguousarray(drift, dtype=np.float64)
        check(load().cpic_set_injection(self.h, sp, face, density, vth, _ptr(d), seed))

    # ---- cycle
    def initialize(self):
        check(load().cpic_initialize(self.h))

    def step(self, nsteps=1):
        check(load().cpic_step(self.h, nsteps))

    def set_sort_interval(self, interval):
        check(load().cpic_set_sort_interval(self.h, interval))

    def set_solver(self, solver):
        """CPIC_SOLVER_MG (V-cycle iteration) or CPIC_SOLVER_BICGSTAB (V-cycle-preconditioned
        BiCGStab) for the kernel-chain field solve."""
        check(load().cpic_set_solver(self.h, solver))

    def autotune(self, trial_steps=8):
        """Choose the sort interval, the push chunk size and the deposit tiling by timing
        fixed-field particle steps (state restored after every trial)."""
        t = cpic_tuning()
        check(load().cpic_autotune(self.h, trial_steps, ctypes.byref(t)))
        return {"sort_interval": t.sort_interval, "interval": list(t.interval), "ms_per_step": list(t.ms_per_step),
                "chunk": t.chunk, "chunks": list(t.chunks), "ms_chunk": list(t.ms_chunk),
                "tile": t.tile, "ms_tile": list(t.ms_tile)}

    def set_push_tuning(self, chunk=0, tile=1):
        """Push kernel knobs: particles per block chunk (0: one wave of blocks) and deposit
        tiling (1: shared-memory tile, 0: direct)."""
        check(load().cpic_set_push_tuning(self.h, chunk, tile))

    def checkpoint(self, path):
        check(load().cpic_checkpoint(self.h, os.fsencode(path)))

    @classmethod
    def restore(cls, path, stream=None):
        """A run created from a checkpoint file (owns its device memory)."""
        h = P()
        check(load().cpic_restore(os.fsencode(path), None, 0, stream, ctypes.byref(h)))
        cfg = cpic_config()
        run = cls.__new__(cls)
        run._arena = None
        run.h = h
        check(load().cpic_get_config(h, ctypes.byref(cfg)))
        run.cfg = cfg
        run.D = cfg.dim
        run.n = tuple(cfg.n[a] for a in range(cfg.dim))
        run.ncell = int(np.prod(run.n))
        run.nvert = int(np.prod([x + 1 for x in run.n]))
        return run

    def set_magnetic_field(self, B):
        """cpic_set_magnetic_field: uniform B0 (3 components in the velocity components' order;
        an axisymmetric run's (v_r, v_z, v_theta) takes (0, B_z, 0) only)."""
        b = np.ascontiguousarray(B, dtype=np.float64)
        check(load().cpic_set_magnetic_field(self.h, _ptr(b)))

    def set_multigrid(self, coarse="rediscretized", smoother="point", interpolation="bilinear"):
        """cpic_set_multigrid: coarse "rediscretized" | "galerkin", smoother "point" | "line",
        interpolation "bilinear" | "operator"."""
        c = {"rediscretized": MG_COARSE_REDISCRETIZED, "galerkin": MG_COARSE_GALERKIN}[coarse]
        i = {"bilinear": MG_INTERP_BILINEAR, "operator": MG_INTERP_OPERATOR}[interpolation]
        m = {"point": MG_SMOOTH_POINT, "line": MG_SMOOTH_LINE}[smoother]
        check(load().cpic_set_multigrid(self.h, c, i, m))

    def set_gyro_integrator(self, kind):
        """cpic_set_gyro_integrator: "boris" or "cyclotronic" (exact gyration in B0)."""
        k = {"boris": GYRO_BORIS, "cyclotronic": GYRO_CYCLOTRONIC}[kind] if isinstance(kind, str) else int(kind)
        check(load().cpic_set_gyro_integrator(self.h, k))

    def collection(self, sp, face=0):
        """cpic_get_collection: particles of species sp removed at face 0/1 so far, per face
        cell (2D: along axis 1; 3D: j + n1 k)."""
        n = self.cfg.n[1] * (self.cfg.n[2] if self.D == 3 else 1)
        out = np.zeros(n, dtype=np.int64)
        check(load().cpic_get_collection(self.h, sp, face, _ptr(out), n))
        return out

    def set_floating(self, face=0, charge0=0.0):
        """cpic_set_floating: the face's conductor floats (Gauss's-law potential from its
        collected charge)."""
        check(load().cpic_set_floating(self.h, face, charge0))

    def step_particles(self, nsteps=1):
        """Particle steps with the field held fixed (no field solve)."""
        check(load().cpic_step_particles(self.h, nsteps))

    def vertex_field(self):
        check(load().cpic_vertex_field(self.h))

    def push(self):
        check(load().cpic_push(self.h))

    def deposit(self):
        check(load().cpic_deposit(self.h))

    def kick(self, fraction):
        check(load().cpic_kick(self.h, fraction))

    def inject(self):
        check(load().cpic_inject(self.h))

    def sort(self):
        check(load().cpic_sort(self.h))

    def solve_field(self, rtol=1e-10, max_cycles=50, allow_not_converged=False):
        c = ctypes.c_int()
        r = ctypes.c_double()
        st = load().cpic_solve_field(self.h, rtol, max_cycles, ctypes.byref(c), ctypes.byref(r))
        if not (allow_not_converged and st == CPIC_ERR_NOT_CONVERGED):
            check(st)
        return c.value, r.value

    def synchronize(self):
        check(load().cpic_synchronize(self.h))

    def profile(self, enable=True):
        check(load().cpic_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{phase: (ms, count)} accumulated since the last read."""
        ms = np.zeros(len(PHASES), np.float64)
        cnt = np.zeros(len(PHASES), np.int64)
        check(load().cpic_profile_read(self.h, _ptr(ms), _ptr(cnt)))
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    # ---- data out
    def diag(self) -> dict:
        d = cpic_diag()
        check(load().cpic_get_diag(self.h, ctypes.byref(d)))
        ns = self.cfg.n_species
        return {
            "step": d.step, "W_E": d.field_energy, "W_K": d.kinetic_energy,
            "n": [d.n_particles[s] for s in range(ns)],
            "absorbed": [[d.absorbed[s][f] for f in range(2 * self.D)] for s in range(ns)],
            "injected": [d.injected[s] for s in range(ns)], "dropped": [d.dropped[s] for s in range(ns)],
            "nonfinite": d.nonfinite, "mg_cycles": d.mg_cycles, "mg_residual": d.mg_residual,
            "pc_face_only": d.pc_face_only, "object_potential": d.object_potential,
            "object_charge": d.object_charge,
        }

    def phi(self):
        out = np.empty(self.ncell, np.float64)
        check(load().cpic_get_phi(self.h, _ptr(out)))
        return out.reshape(tuple(reversed(self.n)))

    def set_phi(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        check(load().cpic_set_phi(self.h, _ptr(phi)))

    def charge(self, sp):
        out = np.empty(self.ncell, np.int64)
        check(load().cpic_get_charge(self.h, sp, _ptr(out)))
        return out.reshape(tuple(reversed(self.n)))

    def vertex_tables(self):
        """cpic_get_vertex_tables: the mover's FP32 k and G, numpy vertex layout."""
        k = np.empty(self.nvert * self.D * self.D, np.float32)
        g = np.empty(self.nvert * self.D, np.float32)
        check(load().cpic_get_vertex_tables(self.h, _ptr(k), _ptr(g)))
        vshape = tuple(reversed([x + 1 for x in self.n]))
        return k.reshape(vshape + (self.D, self.D)), g.reshape(vshape + (self.D,))

    def geometry(self):
        k = np.empty(self.nvert * self.D * self.D, np.float64)
        jc = np.empty(self.ncell, np.float64)
        check(load().cpic_get_geometry(self.h, _ptr(k), _ptr(jc)))
        vshape = tuple(reversed([x + 1 for x in self.n]))
        return k.reshape(vshape + (self.D, self.D)), jc.reshape(tuple(reversed(self.n)))

    def particles(self, sp):
        cap = int(self.cfg.capacity[sp])
        cell = np.empty(cap, np.int32)
        t = np.empty(self.D * cap, np.float32)
        v = np.empty(3 * cap, np.float32)
        n = ctypes.c_int64()
        check(load().cpic_get_particles(self.h, sp, cap, ctypes.byref(n), _ptr(cell), _ptr(t), _ptr(v)))
        m = n.value
        return cell[:m].copy(), t[: self.D * m].reshape(self.D, m).copy(), v[: 3 * m].reshape(3, m).copy()


def run_from_workload(wl, sort_interval=0, analytic=None, mg_rtol=0.0, mg_max_cycles=0, arena=None, stream=None):
    """Create a run for a workload (map from its vertex array unless analytic=(id, params)),
    load its particles and injection sources."""
    cfg = config_from_workload(wl, sort_interval=sort_interval, mg_rtol=mg_rtol, mg_max_cycles=mg_max_cycles)
    run = Run(cfg, arena=arena, stream=stream)
    if analytic is None:
        run.set_map_vertices(wl.vertices)
    else:
        run.set_map_analytic(*analytic)
    for s, ps in enumerate(wl.particles):
        run.load_particles(s, ps.cell, ps.t, ps.v)
    for inj in wl.injection:
        s, face, dens, vth, seed = inj[:5]
        run.set_injection(s, face, dens, vth, seed, drift=inj[5] if len(inj) > 5 else None)
    if getattr(wl, "B0", None) is not None:
        run.set_magnetic_field(wl.B0)
        run.set_gyro_integrator(getattr(wl, "gyro", "boris"))
    return run


def cylinder_run_device(n1, n2, npart_per_species, phi_obj, seed, sort_interval=4, arena=None, stream=None,
                        inject=True, r0=1.0, R=40.0):
    """A cylinder-in-plasma run (annulus map, both species) loaded on the device with
    cpic_load_maxwellian and initialised."""
    from . import workloads as wl

    w = wl.cylinder(n1=n1, n2=n2, r0=r0, R=R, npart_per_species=npart_per_species, phi_obj=phi_obj, seed=seed,
                    inject=inject, host_particles=False)
    cfg = config_from_workload(w, sort_interval=sort_interval)
    if arena is None:
        import torch

        arena = torch.empty(Run.footprint(cfg), dtype=torch.uint8, device="cuda")
    run = Run(cfg, arena=arena, stream=stream)
    run.set_map_analytic(CPIC_MAP_ANNULUS, [r0, R])
    for s, sp in enumerate(w.species):
        run.load_maxwellian(s, npart_per_species, sp.vth, seed=seed * 16 + s)
    run.sort()  # the load draws cells in random order: start in cell order
    for (s, face, dens, vth, sd) in w.injection:
        run.set_injection(s, face, dens, vth, sd)
    run.initialize()
    return run


def sphere_run_device(n1, n2, n3, npart_per_species, phi_obj=-5.0, seed=2, sort_interval=4, arena=None,
                      stream=None, r0=1.0, R=30.0, theta_c=None, inject=False, host_map=False):
    """A 3D sphere-in-plasma run (shell map, reflecting polar caps) loaded on the device
    with cpic_load_maxwellian and initialised; with inject, Maxwellian flux injection of both
    species through the outer boundary. host_map: the map is given as the host vertex array
    of workloads.shell_vertices (cpic_set_map_vertices) instead of being evaluated on the
    device (cpic_set_map_analytic)."""
    import math

    from . import workloads as wl

    theta_c = math.pi / 32 if theta_c is None else theta_c
    w = wl.sphere(n1=n1, n2=n2, n3=n3, r0=r0, R=R, theta_c=theta_c, npart_per_species=npart_per_species,
                  phi_obj=phi_obj, seed=seed, host_particles=False, inject=inject)
    cfg = config_from_workload(w, sort_interval=sort_interval)
    if arena is None:
        import torch

        arena = torch.empty(Run.footprint(cfg), dtype=torch.uint8, device="cuda")
    run = Run(cfg, arena=arena, stream=stream)
    if host_map:
        run.set_map_vertices(w.vertices)
    else:
        run.set_map_analytic(CPIC_MAP_SHELL, [r0, R, theta_c])
    for s, sp in enumerate(w.species):
        run.load_maxwellian(s, npart_per_species, sp.vth, seed=seed * 16 + s)
    run.sort()  # the load draws cells in random order: start in cell order
    for (s, face, dens, vth, sd) in w.injection:
        run.set_injection(s, face, dens, vth, sd)
    run.initialize()
    run._keep = arena
    return run


class Batch:
    """Many runs stepped together (one CUDA graph launch per batch step)."""

    def __init__(self, max_runs, stream=None):
        h = P()
        check(load().cpic_batch_create(max_runs, stream, ctypes.byref(h)))
        self.h = h
        self.runs = []

    def add(self, run):
        check(load().cpic_batch_add(self.h, run.h))
        self.runs.append(run)

    def remove(self, run):
        check(load().cpic_batch_remove(self.h, run.h))
        self.runs.remove(run)

    def __len__(self):
        n = ctypes.c_int()
        check(load().cpic_batch_size(self.h, ctypes.byref(n)))
        return n.value

    def step(self, nsteps=1, solve=True):
        check(load().cpic_batch_step(self.h, nsteps, 1 if solve else 0))

    def set_mode(self, mode):
        check(load().cpic_batch_set_mode(self.h, mode))

    def synchronize(self):
        check(load().cpic_batch_synchronize(self.h))

    def close(self):
        if self.h:
            load().cpic_batch_destroy(self.h)
            self.h = None


def make_request(n1=64, n2=128, particles_per_species=100_000, phi_object=-5.0, density=1.0, temperature=1.0,
                 mass_ratio=1836.0, r_object=1.0, r_outer=40.0, dt=0.1, steps=100, seed=1, kind=CPIC_REQ_CYLINDER):
    q = cpic_request()
    q.kind = kind
    q.n[0], q.n[1], q.n[2] = n1, n2, 1
    q.particles_per_species = particles_per_species
    q.phi_object = phi_object
    q.density = density
    q.temperature = temperature
    q.mass_ratio = mass_ratio
    q.r_object, q.r_outer = r_object, r_outer
    q.dt = dt
    q.steps = steps
    q.seed = seed
    return q


def run_for_request(req, sort_interval=4, stream=None, start=True):
    """A stand-alone run set up exactly as the server sets up request `req` (cpic_request):
    the device-evaluated map, cpic_load_maxwellian of both species with the request's
    seeds, flux injection at the outer boundary, a cell sort and (with start) the start-up
    solve. Stepping it with cpic_step gives the served result."""
    import math

    from . import workloads as wl

    sph = req.kind == CPIC_REQ_SPHERE
    pps = req.particles_per_species
    if sph:
        w = wl.sphere(n1=req.n[0], n2=req.n[1], n3=req.n[2], r0=req.r_object, R=req.r_outer,
                      npart_per_species=pps, phi_obj=req.phi_object, mass_ratio=req.mass_ratio, dt=req.dt,
                      host_particles=False)
    else:
        w = wl.cylinder(n1=req.n[0], n2=req.n[1], r0=req.r_object, R=req.r_outer, npart_per_species=pps,
                        phi_obj=req.phi_object, mass_ratio=req.mass_ratio, dt=req.dt, host_particles=False)
    for sp in w.species:
        sp.w = sp.w * req.density
    cfg = config_from_workload(w, sort_interval=sort_interval)
    for s in range(2):
        cfg.capacity[s] = pps + pps // 2 + 1024
    run = Run(cfg, stream=stream)
    if sph:
        run.set_map_analytic(CPIC_MAP_SHELL, [req.r_object, req.r_outer, math.pi / 32])
    else:
        run.set_map_analytic(CPIC_MAP_ANNULUS, [req.r_object, req.r_outer])
    vth = [math.sqrt(req.temperature), math.sqrt(req.temperature / req.mass_ratio)]
    for s in range(2):
        run.load_maxwellian(s, pps, vth[s], seed=req.seed * 16 + s)
    for s in range(2):
        run.set_injection(s, 1, req.density, vth[s], req.seed * 1000 + 7 + s)
    run.sort()
    if start:
        run.initialize()
    return run


class Server:
    """Request loop with continuous batching (cpic_server_*)."""

    def __init__(self, hbm_budget=0, max_active=0, steps_per_slice=0, sort_interval=0):
        o = cpic_server_opts(hbm_budget, max_active, steps_per_slice, sort_interval)
        h = P()
        check(load().cpic_server_start(ctypes.byref(o), ctypes.byref(h)))
        self.h = h

    def submit(self, req) -> int:
        t = ctypes.c_uint64()
        check(load().cpic_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """The result as a dict once done, else None."""
        r = cpic_result()
        st = load().cpic_server_poll(self.h, ticket, ctypes.byref(r))
        if st == CPIC_ERR_BUSY:
            return None
        check(st)
        out = {k: getattr(r, k) for k, _ in cpic_result._fields_}
        for k in ("n_particles", "absorbed_object", "absorbed_outer", "injected", "current_object"):
            out[k] = list(out[k])
        out["message"] = r.message.decode(errors="replace")
        return out

    def cancel(self, ticket) -> int:
        """cpic_server_cancel: the status (CPIC_OK, CPIC_ERR_STATE when already done)."""
        return load().cpic_server_cancel(self.h, ticket)

    def wait(self, ticket, timeout=600.0, interval=1e-3):
        import time

        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} not done after {timeout} s")
            time.sleep(interval)

    def stats(self):
        q, a, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        check(load().cpic_server_stats(self.h, ctypes.byref(q), ctypes.byref(a), ctypes.byref(f)))
        return {"queued": q.value, "active": a.value, "pool_free": f.value}

    def stop(self):
        if self.h:
            load().cpic_server_stop(self.h)
            self.h = None
