"""Seeded synthetic inputs: analytic maps sampled at vertices, particle loads, grids.

This module is shared by the CUDA path's tests and bench and by the oracle's tests.
It holds none of the method's arithmetic (no metric, no interpolation, no push):
only the map x(xi) evaluated at vertices (the mesh is an input of the method, Sec. II.A,
eq. (map)) and seeded random particle states.

Array layout (the C-ABI layout): logical axis a (xi, eta, zeta) = numpy axis D-1-a, so a
2D cell array has shape (N2, N1) and index [j, i]; vertex arrays have N_a + 1 entries per
axis, including the periodic image of vertex 0, and a trailing component axis:
(N2+1, N1+1, 2) in 2D, (N3+1, N2+1, N1+1, 3) in 3D.

Particle state (structure of arrays): ``cell`` int32 packed per-axis cell indices
(2D: i | j << 16; 3D: i | j << 10 | k << 20; -1 = dead), ``t`` float32 (D, n) in-cell
offsets in [0, 1), ``v`` float32 (3, n) physical velocity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi

# ---------------------------------------------------------------------------------------
# maps x(xi) at vertices
# ---------------------------------------------------------------------------------------


def _logical_vertices(n):
    """Logical vertex coordinates xi_a = i_a / N_a for each axis, as 1-D arrays."""
    return [np.arange(na + 1, dtype=np.float64) / na for na in n]


def map2_vertices(n1: int, n2: int, eps: float) -> np.ndarray:
    """Sine-distorted square, Sec. II.B.4 eq. (map2):
    x = xi + eps sin(2 pi xi) sin(2 pi eta), y = eta + eps sin(2 pi xi) sin(2 pi eta).
    Periodic in both axes with period vectors (1, 0) and (0, 1)."""
    xi, eta = _logical_vertices((n1, n2))
    XI, ETA = np.meshgrid(xi, eta, indexing="xy")  # shape (n2+1, n1+1)
    s = eps * np.sin(TWO_PI * XI) * np.sin(TWO_PI * ETA)
    X = np.empty((n2 + 1, n1 + 1, 2))
    X[..., 0] = XI + s
    X[..., 1] = ETA + s
    # exact periodic images (sin(2 pi) is not exactly 0 in floating point)
    X[:, n1, 0] = X[:, 0, 0] + 1.0
    X[:, n1, 1] = X[:, 0, 1]
    X[n2, :, 0] = X[0, :, 0]
    X[n2, :, 1] = X[0, :, 1] + 1.0
    return X


def map2_jacobian_exact(xi, eta, eps):
    """Closed-form Jacobian of eq. (map2): J = 1 + 2 pi eps sin(2 pi (xi + eta))."""
    return 1.0 + TWO_PI * eps * np.sin(TWO_PI * (xi + eta))


def annulus_vertices(n1: int, n2: int, r0: float, R: float) -> np.ndarray:
    """Body-fitted annulus around a cylinder: r = r0 (R/r0)^xi, theta = 2 pi eta.
    xi is radial (object at xi = 0, outer boundary at xi = 1); eta is periodic with a zero
    period vector."""
    xi, eta = _logical_vertices((n1, n2))
    XI, ETA = np.meshgrid(xi, eta, indexing="xy")
    r = r0 * (R / r0) ** XI
    th = TWO_PI * ETA
    X = np.empty((n2 + 1, n1 + 1, 2))
    X[..., 0] = r * np.cos(th)
    X[..., 1] = r * np.sin(th)
    X[n2] = X[0]
    return X


def sphere_axisym_vertices(n1: int, n2: int, r1: float, r2: float) -> np.ndarray:
    """Spherical shell in the (r, z) half plane, Sec. II.B.3 eqs. (r), (z):
    r = [r1 + (r2 - r1) xi] sin(pi (1 - eta)), z = [r1 + (r2 - r1) xi] cos(pi (1 - eta)).
    Component 0 is the cylindrical radius r (the geometric factor Omega = r)."""
    xi, eta = _logical_vertices((n1, n2))
    XI, ETA = np.meshgrid(xi, eta, indexing="xy")
    rad = r1 + (r2 - r1) * XI
    ang = math.pi * (1.0 - ETA)
    X = np.empty((n2 + 1, n1 + 1, 2))
    X[..., 0] = rad * np.sin(ang)
    X[..., 1] = rad * np.cos(ang)
    X[0, :, 0] = 0.0  # on the axis
    X[n2, :, 0] = 0.0
    return X


def shell_vertices(n1: int, n2: int, n3: int, r0: float, R: float, theta_c: float) -> np.ndarray:
    """3D spherical shell with geometric radial stretching: r = r0 (R/r0)^xi,
    polar angle theta = theta_c + (pi - 2 theta_c) eta (polar caps cut out), azimuth
    phi = 2 pi zeta (periodic, zero period vector)."""
    xi, eta, zeta = _logical_vertices((n1, n2, n3))
    ZE, ET, XI = np.meshgrid(zeta, eta, xi, indexing="ij")  # (n3+1, n2+1, n1+1)
    r = r0 * (R / r0) ** XI
    th = theta_c + (math.pi - 2.0 * theta_c) * ET
    ph = TWO_PI * ZE
    X = np.empty((n3 + 1, n2 + 1, n1 + 1, 3))
    X[..., 0] = r * np.sin(th) * np.cos(ph)
    X[..., 1] = r * np.sin(th) * np.sin(ph)
    X[..., 2] = r * np.cos(th)
    X[n3] = X[0]
    return X


# ---------------------------------------------------------------------------------------
# particle state helpers (format only)
# ---------------------------------------------------------------------------------------


def pack_cells(idx: np.ndarray) -> np.ndarray:
    """Pack per-axis cell indices, shape (D, n), into the int32 cell word."""
    D = idx.shape[0]
    idx = idx.astype(np.int64)
    if D == 2:
        w = idx[0] | (idx[1] << 16)
    else:
        w = idx[0] | (idx[1] << 10) | (idx[2] << 20)
    return w.astype(np.int32)


def unpack_cells(cell: np.ndarray, D: int) -> np.ndarray:
    """Inverse of pack_cells for live particles (cell >= 0)."""
    c = cell.astype(np.int64)
    if D == 2:
        return np.stack([c & 0xFFFF, c >> 16])
    return np.stack([c & 0x3FF, (c >> 10) & 0x3FF, c >> 20])


def split_logical(u: np.ndarray, n) -> tuple[np.ndarray, np.ndarray]:
    """Split float64 cell-unit coordinates u (D, n) with 0 <= u_a < N_a into integer cells and
    float32 offsets in [0, 1)."""
    c = np.floor(u).astype(np.int64)
    t = (u - c).astype(np.float32)
    one = t >= np.float32(1.0)
    t[one] = np.float32(0.0)
    c[one] += 1
    for a, na in enumerate(n):
        c[a] %= na
    return c, t


@dataclass
class ParticleSet:
    """One species' particles in the C-ABI format."""

    cell: np.ndarray  # int32 (n,)
    t: np.ndarray  # float32 (D, n)
    v: np.ndarray  # float32 (3, n)

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])


def _from_logical(u, n, v):
    c, t = split_logical(u, n)
    return ParticleSet(pack_cells(c), np.ascontiguousarray(t), np.ascontiguousarray(v.astype(np.float32)))


def maxwellian(rng: np.random.Generator, npart: int, vth: float, drift=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Isotropic Maxwellian velocities, shape (3, n), float64."""
    v = rng.standard_normal((3, npart)) * vth
    return v + np.asarray(drift, dtype=np.float64)[:, None]


def load_uniform_logical(rng, n, npart, vth):
    """Positions uniform in logical space (equal counts per cell on average)."""
    D = len(n)
    u = rng.random((D, npart)) * np.asarray(n, dtype=np.float64)[:, None]
    return _from_logical(u, n, maxwellian(rng, npart, vth))


def load_map2(rng, n1, n2, eps, npart, vth, amp=0.0, mode=1):
    """Particles uniform in PHYSICAL space on the map2 square (density proportional to the
    closed-form Jacobian in logical space), with an optional density perturbation
    1 + amp cos(2 pi mode x) in physical x. Rejection sampling in (xi, eta)."""
    jmax = (1.0 + TWO_PI * abs(eps)) * (1.0 + abs(amp))
    out = []
    have = 0
    while have < npart:
        m = int((npart - have) * 1.5 * jmax) + 64
        xi = rng.random(m)
        eta = rng.random(m)
        s = eps * np.sin(TWO_PI * xi) * np.sin(TWO_PI * eta)
        x = xi + s
        dens = map2_jacobian_exact(xi, eta, eps) * (1.0 + amp * np.cos(TWO_PI * mode * x))
        keep = rng.random(m) * jmax < dens
        out.append(np.stack([xi[keep], eta[keep]]))
        have += int(keep.sum())
    u = np.concatenate(out, axis=1)[:, :npart] * np.array([[n1], [n2]], dtype=np.float64)
    return _from_logical(u, (n1, n2), maxwellian(rng, npart, vth))


def load_annulus(rng, n1, n2, r0, R, npart, vth, drift=(0.0, 0.0, 0.0)):
    """Particles uniform in physical space in the annulus r0 < r < R of annulus_vertices:
    area element ~ r^2 d(xi) d(eta), so xi has density ~ (R/r0)^(2 xi) (inverse CDF)."""
    L = math.log(R / r0)
    U = rng.random(npart)
    xi = np.log1p(U * ((R / r0) ** 2 - 1.0)) / (2.0 * L)
    eta = rng.random(npart)
    u = np.stack([xi * n1, eta * n2])
    u[0] = np.minimum(u[0], np.nextafter(n1, 0))
    return _from_logical(u, (n1, n2), maxwellian(rng, npart, vth, drift))


def load_shell(rng, n, r0, R, theta_c, npart, vth):
    """Particles uniform in physical space inside the 3D shell of shell_vertices:
    volume element ~ r^3 sin(theta) d(xi) d(eta) d(zeta)."""
    n1, n2, n3 = n
    L = math.log(R / r0)
    U = rng.random(npart)
    xi = np.log1p(U * ((R / r0) ** 3 - 1.0)) / (3.0 * L)
    # theta in [theta_c, pi - theta_c] with density ~ sin(theta)
    c0 = math.cos(theta_c)
    ct = c0 - rng.random(npart) * 2.0 * c0
    th = np.arccos(ct)
    eta = (th - theta_c) / (math.pi - 2.0 * theta_c)
    zeta = rng.random(npart)
    u = np.stack([xi * n1, eta * n2, zeta * n3])
    u[0] = np.minimum(u[0], np.nextafter(n1, 0))
    u[1] = np.clip(u[1], 0.0, np.nextafter(n2, 0))
    return _from_logical(u, n, maxwellian(rng, npart, vth))


# ---------------------------------------------------------------------------------------
# named workloads (shapes of the paper's test problems)
# ---------------------------------------------------------------------------------------

# boundary condition codes shared with include/cpic.h (a format, not arithmetic)
BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
PBC_PERIODIC, PBC_ABSORB, PBC_REFLECT = 0, 1, 2


@dataclass
class Species:
    q: float
    m: float
    w: float
    vth: float
    capacity: int = 0


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    vertices: np.ndarray
    field_bc: list  # 2*dim entries (face = 2*axis + side)
    field_bc_value: list
    particle_bc: list
    dt: float
    species: list
    particles: list  # ParticleSet per species
    background: float = 0.0  # uniform immobile charge density
    omega_axisym: bool = False
    injection: list = field(default_factory=list)  # (species, face, density, vth, seed)
    sort_interval: int = 0
    B0: tuple = None  # uniform magnetic field (velocity components), None: unmagnetised
    gyro: str = "boris"  # magnetised push: "boris" or "cyclotronic" (exact gyration)


def langmuir_map2(n1=32, n2=32, eps=0.05, ppc=64, vth=0.05, amp=0.01, dt=0.1, seed=0):
    """Doubly periodic Langmuir test on the map2 square: electrons (q/m = -1) uniform in
    physical space with a 1% cos(2 pi x) perturbation, immobile neutralising ions
    (background density +1), omega_pe = 1."""
    rng = np.random.default_rng(seed)
    npart = n1 * n2 * ppc
    w = 1.0 / npart  # unit box area, n0 = 1
    ps = load_map2(rng, n1, n2, eps, npart, vth, amp=amp)
    return Workload(
        name=f"langmuir_map2_{n1}x{n2}_eps{eps}",
        dim=2,
        n=(n1, n2),
        vertices=map2_vertices(n1, n2, eps),
        field_bc=[BC_PERIODIC] * 4,
        field_bc_value=[0.0] * 4,
        particle_bc=[PBC_PERIODIC] * 4,
        dt=dt,
        species=[Species(q=-1.0, m=1.0, w=w, vth=vth, capacity=npart)],
        particles=[ps],
        background=1.0,
    )


def planar_wall(n1=128, n2=128, Lx=20.0, Ly=5.0, ppc=64, mass_ratio=1836.0, ion_drift=-2.1, dt=0.05, seed=12,
                capacity_factor=1.6):
    """The conducting planar wall of Sec. III.A (Test A, eq. (map3): x = Lx xi, y = Ly eta):
    the wall at xi = 0 (absorbing; floating when the run says so, else grounded), phi = 0 at
    xi = 1, eta periodic; the box starts empty and both species are injected at xi = 1 each
    step from a unit-density plasma, electrons from a Maxwellian at rest, ions (T_i = T_e)
    from one drifting at ion_drift ion thermal speeds along x (toward the wall). The weight
    gives about ppc particles per cell and species at unit density."""
    xi, eta = _logical_vertices((n1, n2))
    XI, ETA = np.meshgrid(xi, eta, indexing="xy")
    X = np.empty((n2 + 1, n1 + 1, 2))
    X[..., 0] = Lx * XI
    X[..., 1] = Ly * ETA
    w = Lx * Ly / (ppc * n1 * n2)
    vti = 1.0 / math.sqrt(mass_ratio)
    cap = int(capacity_factor * ppc * n1 * n2)
    sp = [Species(-1.0, 1.0, w, 1.0, cap), Species(1.0, mass_ratio, w, vti, cap)]
    empty = [ParticleSet(np.zeros(0, np.int32), np.zeros((2, 0), np.float32), np.zeros((3, 0), np.float32))
             for _ in sp]
    return Workload(
        name=f"planar_wall_{n1}x{n2}",
        dim=2,
        n=(n1, n2),
        vertices=X,
        field_bc=[BC_DIRICHLET, BC_DIRICHLET, BC_PERIODIC, BC_PERIODIC],
        field_bc_value=[0.0, 0.0, 0.0, 0.0],
        particle_bc=[PBC_ABSORB, PBC_ABSORB, PBC_PERIODIC, PBC_PERIODIC],
        dt=dt,
        species=sp,
        particles=empty,
        injection=[(0, 1, 1.0, 1.0, seed * 1000 + 1), (1, 1, 1.0, vti, seed * 1000 + 2, (ion_drift * vti, 0.0, 0.0))],
    )


def two_stream_map2(n1=64, n2=64, eps=0.05, ppc=256, v0=0.0975, vth=0.002, amp=1e-3, dt=0.05, seed=0):
    """Two-stream configuration on the doubly periodic map2 square: two equal cold electron
    beams (each half of the unit density) drifting at +v0 and -v0 along x through immobile
    neutralising ions, with a small cos(2 pi x) density perturbation as the seed. The beams
    are loaded as pairs at the same position (equal and opposite drift), so the seed is
    the only initial current-free perturbation."""
    rng = np.random.default_rng(seed)
    half = n1 * n2 * ppc // 2
    ps = load_map2(rng, n1, n2, eps, half, vth, amp=amp)
    cell = np.concatenate([ps.cell, ps.cell])
    t = np.concatenate([ps.t, ps.t], axis=1)
    v = np.concatenate([ps.v, ps.v], axis=1).astype(np.float64)
    v[0, :half] += v0
    v[0, half:] -= v0
    npart = 2 * half
    return Workload(
        name=f"two_stream_map2_{n1}x{n2}_eps{eps}",
        dim=2,
        n=(n1, n2),
        vertices=map2_vertices(n1, n2, eps),
        field_bc=[BC_PERIODIC] * 4,
        field_bc_value=[0.0] * 4,
        particle_bc=[PBC_PERIODIC] * 4,
        dt=dt,
        species=[Species(q=-1.0, m=1.0, w=1.0 / npart, vth=vth, capacity=npart)],
        particles=[ParticleSet(cell, t, v.astype(np.float32))],
        background=1.0,
    )


def cylinder(n1=128, n2=256, r0=1.0, R=40.0, npart_per_species=2_000_000, phi_obj=-5.0,
             mass_ratio=1836.0, dt=0.1, seed=1, inject=True, capacity_factor=1.5, host_particles=True):
    """2D cylinder in plasma on the log-polar annulus: object at xi = 0 held at phi_obj and
    absorbing, outer boundary at xi = 1 (phi = 0, absorbing, Maxwellian flux injection),
    eta periodic. Electrons (q = -1, m = 1, vth = 1) and ions (q = +1, m = mass_ratio,
    T_i = T_e). Loaded uniform in physical space at density 1. host_particles=False leaves
    the particle sets empty (the run is loaded on the device with cpic_load_maxwellian)."""
    rng = np.random.default_rng(seed)
    area = math.pi * (R * R - r0 * r0)
    w = area / npart_per_species
    vti = 1.0 / math.sqrt(mass_ratio)
    cap = int(npart_per_species * capacity_factor)
    sp = [Species(-1.0, 1.0, w, 1.0, cap), Species(1.0, mass_ratio, w, vti, cap)]
    if host_particles:
        parts = [load_annulus(rng, n1, n2, r0, R, npart_per_species, s.vth) for s in sp]
    else:
        parts = [ParticleSet(np.zeros(0, np.int32), np.zeros((2, 0), np.float32), np.zeros((3, 0), np.float32))
                 for _ in sp]
    inj = []
    if inject:
        inj = [(0, 1, 1.0, 1.0, seed * 1000 + 7), (1, 1, 1.0, vti, seed * 1000 + 8)]
    return Workload(
        name=f"cylinder_{n1}x{n2}_{2 * npart_per_species}",
        dim=2,
        n=(n1, n2),
        vertices=annulus_vertices(n1, n2, r0, R),
        field_bc=[BC_DIRICHLET, BC_DIRICHLET, BC_PERIODIC, BC_PERIODIC],
        field_bc_value=[phi_obj, 0.0, 0.0, 0.0],
        particle_bc=[PBC_ABSORB, PBC_ABSORB, PBC_PERIODIC, PBC_PERIODIC],
        dt=dt,
        species=sp,
        particles=parts,
        injection=inj,
    )


def sphere(n1=128, n2=128, n3=128, r0=1.0, R=30.0, theta_c=math.pi / 32, npart_per_species=32_000_000,
           phi_obj=-5.0, mass_ratio=1836.0, dt=0.1, seed=2, capacity_factor=1.5, host_particles=True,
           inject=False):
    """3D sphere in plasma on the shell map r = r0 (R/r0)^xi, theta = theta_c + (pi -
    2 theta_c) eta, phi = 2 pi zeta (polar caps cut out): object at xi = 0 held at phi_obj
    and absorbing, outer boundary at 0 and absorbing, polar caps Neumann for the field and
    specular for particles, zeta periodic. Electrons and ions (T_i = T_e), uniform in
    physical space at density 1; with inject, both species enter as Maxwellian flux through
    the outer boundary (face 1) at density 1."""
    rng = np.random.default_rng(seed)
    vol = (4.0 / 3.0) * math.pi * (R**3 - r0**3) * math.cos(theta_c)
    w = vol / npart_per_species
    vti = 1.0 / math.sqrt(mass_ratio)
    cap = int(npart_per_species * capacity_factor)
    sp = [Species(-1.0, 1.0, w, 1.0, cap), Species(1.0, mass_ratio, w, vti, cap)]
    n = (n1, n2, n3)
    if host_particles:
        parts = [load_shell(rng, n, r0, R, theta_c, npart_per_species, s.vth) for s in sp]
    else:
        parts = [ParticleSet(np.zeros(0, np.int32), np.zeros((3, 0), np.float32), np.zeros((3, 0), np.float32))
                 for _ in sp]
    inj = []
    if inject:
        inj = [(0, 1, 1.0, 1.0, seed * 1000 + 7), (1, 1, 1.0, vti, seed * 1000 + 8)]
    return Workload(
        name=f"sphere_{n1}x{n2}x{n3}_{2 * npart_per_species}",
        dim=3,
        n=n,
        vertices=shell_vertices(n1, n2, n3, r0, R, theta_c),
        field_bc=[BC_DIRICHLET, BC_DIRICHLET, BC_NEUMANN, BC_NEUMANN, BC_PERIODIC, BC_PERIODIC],
        field_bc_value=[phi_obj, 0.0, 0.0, 0.0, 0.0, 0.0],
        particle_bc=[PBC_ABSORB, PBC_ABSORB, PBC_REFLECT, PBC_REFLECT, PBC_PERIODIC, PBC_PERIODIC],
        dt=dt,
        species=sp,
        particles=parts,
        injection=inj,
    )


def sphere_axisym(n1=128, n2=128, r1=1.0, r2=10.0, npart_per_species=1_000_000, phi_obj=-2.5, mass_ratio=1836.0,
                  dt=0.1, seed=6, inject=True, capacity_factor=1.5):
    """Sphere in plasma in 2D cylindrical geometry with azimuthal symmetry (Sec. III.B: the
    spherical-shell map of eqs. (r), (z), Omega = r): sphere of radius r1 at xi = 0 (held at
    phi_obj and absorbing, or floating), outer sphere r2 at xi = 1 (phi = 0, absorbing,
    Maxwellian flux injection of both species), the z axis at eta = 0, 1 (Neumann field,
    specular particles). Macro-particles are rings around the axis, loaded uniform in the
    3D shell (r_sph^3 uniform, cos of the polar angle uniform) with equal weights;
    velocities (v_r, v_z, v_theta) Maxwellian; T_i = T_e."""
    rng = np.random.default_rng(seed)
    vol = (4.0 / 3.0) * math.pi * (r2**3 - r1**3)
    w = vol / npart_per_species
    vti = 1.0 / math.sqrt(mass_ratio)
    cap = int(npart_per_species * capacity_factor)
    sp = [Species(-1.0, 1.0, w, 1.0, cap), Species(1.0, mass_ratio, w, vti, cap)]
    parts = []
    for s in sp:
        rs = np.cbrt(r1**3 + rng.random(npart_per_species) * (r2**3 - r1**3))
        polar = np.arccos(1.0 - 2.0 * rng.random(npart_per_species))
        u = np.stack([(rs - r1) / (r2 - r1) * n1, (1.0 - polar / math.pi) * n2])
        u[0] = np.clip(u[0], 0.0, np.nextafter(n1, 0))
        u[1] = np.clip(u[1], 0.0, np.nextafter(n2, 0))
        parts.append(_from_logical(u, (n1, n2), maxwellian(rng, npart_per_species, s.vth)))
    inj = [(0, 1, 1.0, 1.0, seed * 1000 + 7), (1, 1, 1.0, vti, seed * 1000 + 8)] if inject else []
    return Workload(
        name=f"sphere_axisym_{n1}x{n2}_{2 * npart_per_species}",
        dim=2,
        n=(n1, n2),
        vertices=sphere_axisym_vertices(n1, n2, r1, r2),
        field_bc=[BC_DIRICHLET, BC_DIRICHLET, BC_NEUMANN, BC_NEUMANN],
        field_bc_value=[phi_obj, 0.0, 0.0, 0.0],
        particle_bc=[PBC_ABSORB, PBC_ABSORB, PBC_REFLECT, PBC_REFLECT],
        dt=dt,
        species=sp,
        particles=parts,
        omega_axisym=True,
        injection=inj,
    )


def box_reflect(n1=32, n2=32, npart=50_000, vth=1.0, dt=0.1, seed=7):
    """2D unit square (uniform map) with specular walls on axis 0 (Neumann field) and a
    periodic axis 1; one electron species at a neutralising background."""
    rng = np.random.default_rng(seed)
    X = map2_vertices(n1, n2, 0.0)
    u = np.stack([rng.random(npart) * n1, rng.random(npart) * n2])
    u[0] = np.minimum(u[0], np.nextafter(n1, 0))
    ps = _from_logical(u, (n1, n2), maxwellian(rng, npart, vth))
    w = 1.0 / npart
    return Workload(
        name=f"box_reflect_{n1}x{n2}",
        dim=2,
        n=(n1, n2),
        vertices=X,
        field_bc=[BC_NEUMANN, BC_NEUMANN, BC_PERIODIC, BC_PERIODIC],
        field_bc_value=[0.0, 0.0, 0.0, 0.0],
        particle_bc=[PBC_REFLECT, PBC_REFLECT, PBC_PERIODIC, PBC_PERIODIC],
        dt=dt,
        species=[Species(-1.0, 1.0, w, vth, int(npart * 1.5))],
        particles=[ps],
        background=1.0,
    )


def random_field(rng, shape, scale=1.0):
    """A smooth-ish random cell-centred potential for frozen-field mover tests."""
    base = rng.standard_normal(shape)
    # a few passes of neighbour averaging (periodic) to make it smooth
    for _ in range(3):
        acc = base.copy()
        for ax in range(base.ndim):
            acc += np.roll(base, 1, axis=ax) + np.roll(base, -1, axis=ax)
        base = acc / (1 + 2 * base.ndim)
    return scale * base


def batch_specs(nruns, seed=1000):
    """Independent cylinder runs of uneven size (the batched configuration): cells
    N1 x N2 uniform in {32..256} x {64..512} in steps of 16 (so that the multigrid
    hierarchy halves down to its dense coarse solve of at most 512 cells), particles per
    species uniform in [10^4, 2 10^6], object potential uniform in [-10, +2], run i
    seeded seed + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nruns):
        n1 = int(rng.integers(2, 17)) * 16
        n2 = int(rng.integers(4, 33)) * 16
        npart = int(rng.integers(10_000, 2_000_001))
        phi = float(rng.uniform(-10.0, 2.0))
        out.append(dict(n1=n1, n2=n2, npart_per_species=npart, phi_obj=phi, seed=seed + i))
    return out
