"""The PIC cycle composed from the oracle's steps (Sec. II: mover, P->G, field solve, G->P).

Step order (reading of the four-step cycle of Sec. II and the leapfrog of eq. (step1)):
state at step n is (xi^n, v^{n-1/2}) for every particle and phi^n;
  1. G^n = vertex field of phi^n (spec G);
  2. push every particle (eqs. (step1)-(step4)) to (xi^{n+1}, v^{n+1/2}); remove and tally
     the absorbed ones; W_K^n = sum_s 1/2 m_s w_s sum_p v^{n-1/2} . v^{n+1/2};
  3. inject new particles (spec I, step index n);
  4. deposit rho^{n+1} (eq. (pg)) and solve for phi^{n+1} (spec P);
  History entry n holds W_E^n = 1/2 sum_c phi^n_c Q^n_c (before the push) and W_K^n.
Start-up: deposit and solve at xi^0, then v^{-1/2} = v^0 - dt/2 (q/m) E(xi^0).

Two precisions: "fp64" uses the FP64 mover and the exact FP64 b2 deposit; "fp32" replays
the FP32 operation sequence of spec R with FP32 tables and the fixed-point deposit of
spec Q (the results a GPU implementation of the same specs must reproduce bit for bit
given the same potential). The FP64 mover and deposit run either as numpy array
operations (engine "numpy") or as the same definitions in C loops (engine "c",
oracle/pic64.c, optionally on several OpenMP threads), for long runs. The direct solve's
factorisation is kept for the run.
W_K uses the kicked velocity v^{n+1/2} (before any specular reflection), as spec D reads.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import deposit as dep
from . import gradient, inject, mover, poisson
from .geometry import build_geometry

BC_PERIODIC = poisson.BC_PERIODIC


def unpack_cells(cell, D):
    """Per-axis cell indices (D, n) from the packed int32 cell word of the particle format
    (2D: i | j << 16; 3D: i | j << 10 | k << 20)."""
    c = np.asarray(cell).astype(np.int64)
    if D == 2:
        return np.stack([c & 0xFFFF, c >> 16])
    return np.stack([c & 0x3FF, (c >> 10) & 0x3FF, c >> 20])


@dataclass
class SpeciesState:
    q: float
    m: float
    w: float
    idx: np.ndarray  # (D, n) int64
    t: np.ndarray  # (D, n)
    v: np.ndarray  # (3, n)
    absorbed: np.ndarray  # per face counts


class OraclePIC:
    def __init__(self, wl, precision: str = "fp64", engine: str = "numpy", threads: int = 1):
        self.wl = wl
        self.engine = engine
        self.threads = threads
        self.D = wl.dim
        self.n = tuple(wl.n)
        self.precision = precision
        self.bc = list(wl.field_bc)
        self.bcval = list(wl.field_bc_value)
        self.pbc = list(wl.particle_bc)
        periodic = [self.bc[2 * a] == BC_PERIODIC for a in range(self.D)]
        self.periodic = periodic
        self.geom = build_geometry(wl.vertices, periodic, axisym=wl.omega_axisym)
        self._solver = None  # assembled and factorised on the first solve
        self.floating = None  # (face, charge0) of a floating conductor
        self.object_potential = 0.0
        self.object_charge = 0.0
        self.dt = wl.dt
        self.step_index = 0
        self.species = []
        for s, ps in zip(wl.species, wl.particles):
            idx = unpack_cells(ps.cell, self.D)
            if precision == "fp64":
                t, v = ps.t.astype(np.float64), ps.v.astype(np.float64)
            else:
                t, v = ps.t.copy(), ps.v.copy()
            self.species.append(SpeciesState(s.q, s.m, s.w, idx, t, v, np.zeros(2 * self.D, np.int64)))
        self.injection = list(wl.injection)
        self.phi = np.zeros(self.geom.Jc.shape)
        self.history = []
        self.injected = [0] * len(self.species)
        self._face_area = {}
        # collection tally: particles removed at faces 0 / 1 per face cell (transverse indices
        # of the corrector point, clamped into the face; 3D: j + n1 k)
        ncol = self.n[1] * (self.n[2] if self.D == 3 else 1)
        self.collect = np.zeros((len(self.species), 2, ncol), dtype=np.int64)
        self.B0 = getattr(wl, "B0", None)  # uniform magnetic field: Boris kick
        # the cyclotronic integrator (exact gyration) in place of the Boris step
        self.gyro = getattr(wl, "gyro", "boris") == "cyclotronic" and self.B0 is not None and bool(np.any(self.B0))
        # axisymmetric runs: the vertex table of the cylindrical radius (component 0 of the map)
        self.R = np.ascontiguousarray(self.geom.X[..., 0]) if self.geom.axisym else None

    # ---- steps ---------------------------------------------------------------------
    def charge(self):
        """Q_c (numpy cell layout)."""
        Q = self.wl.background * self.geom.Jc
        # axisymmetric runs: a macro-particle is a ring of charge q w (Omega_c Q_c must hold
        # the ring charge / 2 pi)
        ring = 1.0 / (2.0 * np.pi * self.geom.omega_c) if self.geom.axisym else 1.0
        for sp in self.species:
            if self.precision == "fp64":
                if self.engine == "c":
                    C = dep.deposit_exact_c(sp.idx, sp.t, self.n, self.periodic, self.threads)
                else:
                    C = dep.deposit_exact(sp.idx, sp.t, self.n, self.periodic)
                Q = Q + (sp.q * sp.w) * C * ring
            else:
                C = dep.deposit_fixed(sp.idx, sp.t, self.n, self.periodic)
                Q = Q + (sp.q * sp.w) * np.ldexp(C.astype(np.float64), -dep.QF) * ring
        return Q

    def solve(self):
        self.Q = self.charge()
        if self._solver is None:
            bv = list(self.bcval)
            if self.floating is not None:
                bv[self.floating[0]] = 0.0  # the conductor's potential is added below
            self.M, self.bbc = poisson.assemble(self.geom, self.bc, bv)
            self._solver = poisson.DirectSolver(self.geom, self.M, self.bbc, self.bc)
        self.phi = self._solver(self.Q)
        if self.floating is not None:
            face, q0 = self.floating
            qobj = q0
            for sp in self.species:
                qobj += sp.q * sp.w * float(sp.absorbed[face])
            if self.geom.axisym:  # Gauss's law on the ring-charge scale of the right-hand side
                qobj_rhs = qobj / (2.0 * np.pi)
            else:
                qobj_rhs = qobj
            V = -(qobj_rhs + self._face_flux(self.phi, face, 0.0)) / self._cpsi
            self.phi = self.phi + V * self._psi
            self.bcval[face] = V  # the vertex field's Dirichlet value on that face
            self.object_potential, self.object_charge = V, qobj
        return self.phi

    def _face_flux(self, u, face, ub):
        """sum over the cells at face `face` (axis 0) of the Dirichlet face flux
        2 a^{00} (u_c - ub), in cell-index order (axis 1 fastest)."""
        a00 = self.geom.face[0][0]  # numpy face layout, axis 0 last
        col_f = 0 if face == 0 else self.n[0]
        col_c = 0 if face == 0 else self.n[0] - 1
        af = a00[..., col_f].ravel()
        uc = u[..., col_c].ravel()
        acc = 0.0
        for x, y in zip(af, uc):
            acc += 2.0 * x * (y - ub)
        return acc

    def set_floating(self, face, charge0=0.0):
        """The conductor at Dirichlet face `face` (0 or 1, the ends of axis 0) floats
        (Sec. III.A-B: the object charges up with the particles it collects). Gauss's law
        for the conductor: its charge Q = charge0 + sum_s q_s w_s (absorbed at the face) is
        minus the outward flux of grad phi through its surface, which in the finite-volume
        scheme (spec P) is the Dirichlet face flux 2 a^{00} (phi_c - V) summed over the
        face's cells. Every solve takes phi_0 with the conductor at 0 and adds V psi, psi
        the charge-free potential with the conductor at 1 and every other Dirichlet face at
        0; V = -(Q + G0) / Cpsi with G0, Cpsi the face flux sums of phi_0 (about 0) and of
        psi (about 1)."""
        bv = [0.0] * len(self.bcval)
        bv[face] = 1.0
        M1, b1 = poisson.assemble(self.geom, self.bc, bv)
        self._psi = poisson.DirectSolver(self.geom, M1, b1, self.bc)(np.zeros(self.geom.Jc.shape))
        self._cpsi = self._face_flux(self._psi, face, 1.0)
        self.floating = (face, float(charge0))
        self._solver = None

    def field_tables(self):
        G = gradient.vertex_gradient(self.phi, self.bc, self.bcval)
        if self.precision == "fp64":
            return self.geom.k, G
        return self.geom.k.astype(np.float32), G.astype(np.float32)

    def initialize(self):
        self.solve()
        k, G = self.field_tables()
        for sp in self.species:
            qm = sp.q / sp.m
            if self.precision == "fp64":
                sp.v = mover.kick64(sp.idx, sp.t, sp.v, k, G, -0.5 * self.dt * qm,
                                    B=None if self.gyro else self.B0, axisym=self.geom.axisym)
            else:
                sp.v = mover.kick32(sp.idx, sp.t, sp.v, k, G, self.n, np.float32(-0.5 * self.dt * qm),
                                    boris=None if self.gyro else
                                    mover.boris_constants32(self.dt, qm, self.B0, -0.5, axisym=self.geom.axisym))

    def step(self, solve: bool = True):
        """One PIC cycle. solve=False holds the field fixed (mover, injection and deposit
        only: the fixed-field mover runs of Sec. III)."""
        we = 0.5 * float(np.sum(self.phi * self.Q))
        k, G = self.field_tables()
        ke = []
        for s, sp in enumerate(self.species):
            qm = sp.q / sp.m
            if self.precision == "fp64" and self.engine == "c":
                sp.idx = np.ascontiguousarray(sp.idx, dtype=np.int64)
                sp.t = np.ascontiguousarray(sp.t, dtype=np.float64)
                sp.v = np.ascontiguousarray(sp.v, dtype=np.float64)
                idx, t, v, face, vdot = mover.push64_c(sp.idx, sp.t, sp.v, k, G, self.dt, qm, self.n, self.pbc,
                                                       self.threads, inplace=True, B=self.B0, R=self.R,
                                                       gyro=self.gyro)
                ke.append(0.5 * sp.m * sp.w * float(np.sum(vdot)))
            elif self.precision == "fp64":
                vold = sp.v
                idx, t, v, face, vk = mover.push64(sp.idx, sp.t, sp.v, k, G, self.dt, qm, self.n, self.pbc,
                                                   return_kicked=True, B=self.B0, R=self.R, gyro=self.gyro)
                ke.append(0.5 * sp.m * sp.w * float(np.sum(vold * vk)))
            else:
                idx, t, v, face, kefp = mover.push32(
                    sp.idx, sp.t, sp.v, k, G, self.n, self.pbc,
                    np.float32(self.dt * qm), np.float32(0.5 * self.dt), np.float32(self.dt),
                    boris=None if self.gyro else mover.boris_constants32(self.dt, qm, self.B0,
                                                                         axisym=self.geom.axisym),
                    R32=None if self.R is None else self.R.astype(np.float32),
                    gyro=mover.gyro_constants32(self.dt, qm, self.B0, self.geom.axisym) if self.gyro else None)
                ke.append(0.5 * sp.m * sp.w * float(np.ldexp(float(kefp.sum()), -24)))
            alive = face < 0
            if np.all(alive):
                sp.idx, sp.t, sp.v = idx.astype(np.int64, copy=False), t, v
                continue
            sp.absorbed += np.bincount(face[~alive], minlength=2 * self.D)[: 2 * self.D]
            for f in (0, 1):
                hit = face == f
                if np.any(hit):
                    b = np.clip(idx[1][hit], 0, self.n[1] - 1)
                    if self.D == 3:
                        b = b + self.n[1] * np.clip(idx[2][hit], 0, self.n[2] - 1)
                    self.collect[s, f] += np.bincount(b, minlength=self.collect.shape[2])
            sp.idx = np.compress(alive, idx, axis=1).astype(np.int64, copy=False)
            sp.t, sp.v = np.compress(alive, t, axis=1), np.compress(alive, v, axis=1)
        for inj in self.injection:
            s, face, dens, vth, seed = inj[:5]
            drift = tuple(inj[5]) if len(inj) > 5 else (0.0, 0.0, 0.0)
            sp = self.species[s]
            side = face % 2
            dweights = None
            if self.D == 2 and any(drift):  # a drifting Maxwellian: per-segment flux weights
                key = ("drift", s, side)
                if key not in self._face_area:
                    rings = inject.face_ring_areas_2d(self.geom.X, side) if self.geom.axisym else None
                    self._face_area[key] = inject.face_drift_weights_2d(self.geom.X, self.geom.k, side, drift, vth,
                                                                        rings)
                dweights = self._face_area[key]
            if side not in self._face_area:
                if self.geom.axisym:
                    self._face_area[side] = inject.face_area_axisym(self.geom.X, side)
                else:
                    self._face_area[side] = (inject.face_length_2d(self.geom.X, side) if self.D == 2
                                             else inject.face_area_3d(self.geom.X, side))
            area = self._face_area[side]
            if dweights is not None:
                tot = 0.0
                for x in dweights:
                    tot += float(x)
                rate = dens * tot * self.dt / sp.w
            else:
                rate = inject.rate_per_step(dens, vth, area, self.dt, sp.w)
            cnt = inject.count_at_step(rate, self.step_index)
            if cnt == 0:
                continue
            if self.D == 2:
                rings = inject.face_ring_areas_2d(self.geom.X, side) if self.geom.axisym else None
                idx, t32, v32, _ = inject.inject_2d(self.geom.k, self.n, side, cnt, self.step_index, s, seed,
                                                    vth, drift, self.dt, ring_areas=rings, drift_weights=dweights)
            else:
                idx, t32, v32, _ = inject.inject_3d(self.geom.X, self.geom.k, self.n, side, cnt, self.step_index, s,
                                                    seed, vth, (0.0, 0.0, 0.0), self.dt)
            self.injected[s] += idx.shape[1]
            if self.precision == "fp64":
                t32, v32 = t32.astype(np.float64), v32.astype(np.float64)
            sp.idx = np.concatenate([sp.idx, idx], axis=1)
            sp.t = np.concatenate([sp.t, t32], axis=1)
            sp.v = np.concatenate([sp.v, v32], axis=1)
        if solve:
            self.solve()
        else:
            self.Q = self.charge()
        self.step_index += 1
        self.history.append({"step": self.step_index, "W_E": we, "W_K": sum(ke),
                             "object_potential": self.object_potential, "object_charge": self.object_charge,
                             "n": [sp.idx.shape[1] for sp in self.species],
                             "absorbed": [sp.absorbed.copy() for sp in self.species]})
        return self.history[-1]
