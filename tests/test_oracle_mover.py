"""Pins of the oracle's hybrid mover (Sec. II.B.4) in FP64 and of its FP32 replay."""
import math

import numpy as np
import pytest

from oracle import geometry, gradient, mover, poisson
from paper_1311_2286_gb300 import workloads as wl

P, Dr = poisson.BC_PERIODIC, poisson.BC_DIRICHLET
PP, PA = mover.PBC_PERIODIC, mover.PBC_ABSORB


def _uniform(n1, n2):
    return geometry.build_geometry(wl.map2_vertices(n1, n2, 0.0), [True, True])


def test_free_streaming_on_uniform_map():
    """With zero field, xi advances by dt k v = dt N v in cell units (eq. (hybridx))."""
    n = (16, 8)
    g = _uniform(*n)
    rng = np.random.default_rng(0)
    idx = np.stack([rng.integers(0, 16, 100), rng.integers(0, 8, 100)])
    t = rng.random((2, 100))
    v = rng.standard_normal((3, 100)) * 0.3
    G = np.zeros(g.k.shape[:-1])
    i2, t2, v2, face = mover.push64(idx, t, v, g.k, G, 0.1, -1.0, n, [PP] * 4)
    for a in range(2):
        u0 = idx[a] + t[a] + 0.1 * n[a] * v[a]
        np.testing.assert_allclose(i2[a] + t2[a], np.mod(u0, n[a]), atol=1e-12)
    np.testing.assert_array_equal(v2, v)
    assert np.all(face == -1)


def test_kick_in_uniform_logical_field():
    """G = const on the uniform map: E = -k^T G = -N G, v^{n+1/2} = v + dt (q/m) E."""
    n = (8, 8)
    g = _uniform(*n)
    G = np.zeros(g.k.shape[:-1])
    G[..., 0] = 0.02
    G[..., 1] = -0.01
    idx = np.array([[2, 5], [3, 1]])
    t = np.array([[0.1, 0.9], [0.4, 0.2]])
    v = np.zeros((3, 2))
    _, _, v2, _ = mover.push64(idx, t, v, g.k, G, 0.1, -1.0, n, [PP] * 4)
    np.testing.assert_allclose(v2[0], -1.0 * 0.1 * (-8 * 0.02), rtol=1e-12)
    np.testing.assert_allclose(v2[1], -1.0 * 0.1 * (-8 * -0.01), rtol=1e-12)
    assert np.all(v2[2] == 0)


def test_reversibility_uniform_map():
    """P6: on the uniform map with a frozen field the push is time reversible: N steps,
    then restart from (x^N, -v^{N+1/2}) for N steps, returns to x^0 within 1e-12."""
    n = (16, 16)
    g = _uniform(*n)
    rng = np.random.default_rng(5)
    phi = wl.random_field(rng, (16, 16), 0.05)
    G = gradient.vertex_gradient(phi, [P] * 4, [0.0] * 4)
    npart = 200
    idx0 = np.stack([rng.integers(0, 16, npart), rng.integers(0, 16, npart)])
    t0 = rng.random((2, npart))
    v0 = rng.standard_normal((3, npart)) * 0.05
    idx, t, v = idx0, t0, v0
    steps, dt, qm = 40, 0.1, -1.0
    for _ in range(steps):
        idx, t, v, _ = mover.push64(idx, t, v, g.k, G, dt, qm, n, [PP] * 4)
    # v^{N+1/2} from one more kick at x^N
    vN = mover.kick64(idx, t, v, g.k, G, dt * qm)
    idx, t, v = idx, t, -vN
    for _ in range(steps):
        idx, t, v, _ = mover.push64(idx, t, v, g.k, G, dt, qm, n, [PP] * 4)
    u_back = idx + t
    u0 = idx0 + t0
    dist = np.abs(((u_back - u0) + 8) % 16 - 8)
    assert np.max(dist) < 1e-12


def _map2_x(u, n, eps):
    xi, eta = u[0] / n, u[1] / n
    s = eps * np.sin(2 * np.pi * xi) * np.sin(2 * np.pi * eta)
    return np.stack([xi + s, eta + s])


def test_predictor_corrector_second_order_on_distorted_map():
    """Sec. II.B.4: on a non-orthogonal mesh the predictor-corrector regains second-order
    accuracy in time. With E = 0 the logical trajectory solves du/dt = k(u) v; against a
    fine-dt reference on the same grid the error drops 4x when dt halves, and the end point
    mapped through the exact map lies on the straight physical line x0 + v T up to the
    metric's O(h^2) error."""
    n, eps = 512, 0.1
    g = geometry.build_geometry(wl.map2_vertices(n, n, eps), [True, True])
    G = np.zeros(g.k.shape[:-1])
    rng = np.random.default_rng(6)
    npart = 64
    u0 = rng.random((2, npart)) * n
    v = np.zeros((3, npart))
    v[0] = 0.25
    v[1] = -0.15
    T = 0.4

    def run(dt):
        idx = np.floor(u0).astype(np.int64)
        t = u0 - idx
        for _ in range(int(round(T / dt))):
            idx, t, _, _ = mover.push64(idx, t, v, g.k, G, dt, 0.0, (n, n), [PP] * 4)
        return idx + t

    ref = run(0.00125)
    e = []
    for dt in (0.02, 0.01):
        d = (run(dt) - ref + n / 2) % n - n / 2
        e.append(np.max(np.abs(d)))
    assert 3.6 < e[0] / e[1] < 4.4
    x_end = _map2_x(ref, n, eps)
    x_ref = _map2_x(u0, n, eps) + T * v[:2]
    d = (x_end - x_ref + 0.5) % 1.0 - 0.5
    assert np.max(np.abs(d)) < 4.0 / n ** 2


def test_absorption_faces_and_edge_cases():
    """Leaving through xi < 0 or xi >= 1 removes the particle (Sec. II.B.4); an offset of
    exactly 0 on cell 0 stays inside, a coordinate of exactly N leaves."""
    n = (8, 8)
    g = _uniform(*n)
    G = np.zeros(g.k.shape[:-1])
    pbc = [PA, PA, PP, PP]
    idx = np.array([[0, 7, 0, 7, 3], [1, 2, 3, 4, 5]])
    t = np.array([[0.1, 0.9, 0.5, 0.5, 0.5], [0.5, 0.5, 0.5, 0.5, 0.5]])
    v = np.zeros((3, 5))
    # displacement dt*N*v in cell units: -0.2, +0.2, exactly -0.5 (lands on 0), +0.5 (lands on 8)
    v[0] = np.array([-0.25, 0.25, -0.625, 0.625, 0.0])
    _, t2, _, face = mover.push64(idx, t, v, g.k, G, 0.1, 0.0, n, pbc)
    assert list(face) == [0, 1, -1, 1, -1]
    assert t2[0, 2] == 0.0


def test_replay32_matches_fp64_single_step():
    """The FP32 replay of spec R agrees with the FP64 mover to the single-step tolerance
    (normwise 1e-5 on global xi and on v) on the distorted map with a random field."""
    n = (32, 32)
    g = geometry.build_geometry(wl.map2_vertices(32, 32, 0.05), [True, True])
    rng = np.random.default_rng(7)
    phi = wl.random_field(rng, (32, 32), 0.3)
    G = gradient.vertex_gradient(phi, [P] * 4, [0.0] * 4)
    ps = wl.load_uniform_logical(rng, n, 20000, 0.5)
    idx = np.stack([ps.cell & 0xFFFF, ps.cell >> 16]).astype(np.int64)
    i64, t64, v64, f64 = mover.push64(idx, ps.t.astype(np.float64), ps.v.astype(np.float64), g.k, G, 0.1, -1.0, n, [PP] * 4)
    i32, t32, v32, f32, ke = mover.push32(idx, ps.t, ps.v, g.k.astype(np.float32), G.astype(np.float32), n, [PP] * 4,
                                          np.float32(-0.1), np.float32(0.05), np.float32(0.1))
    u64 = (i64 + t64) / 32.0
    u32 = (i32 + t32.astype(np.float64)) / 32.0
    du = np.abs(u32 - u64)
    du = np.minimum(du, 1.0 - du)
    assert np.max(du) / np.max(np.abs(u64)) < 1e-5
    assert np.max(np.abs(v32 - v64)) / np.max(np.abs(v64)) < 1e-5
    ke64 = np.sum(ps.v.astype(np.float64) * v32.astype(np.float64), axis=0)
    # spec D: FP32 product rounded to 2^-24 units; within FP32 rounding of the exact product
    assert np.all(np.abs(ke - np.ldexp(ke64, 24)) <= np.abs(np.ldexp(ke64, 24)) * 2e-7 + 1)


def test_replay32_axisym_matches_fp64_single_step():
    """The FP32 replay of the axisymmetric mover (meridional displacement and frame turn)
    agrees with the FP64 form to the single-step FP32 tolerance on the spherical-shell map
    with a random radial-plus-noise field, including particles near the axis."""
    n = (32, 32)
    w = wl.sphere_axisym(32, 32, npart_per_species=20_000, seed=9, inject=False)
    g = geometry.build_geometry(w.vertices, [False, False], axisym=True)
    rng = np.random.default_rng(3)
    phi = wl.random_field(rng, (32, 32), 0.3) + np.linspace(-3, 0, 32)
    G = gradient.vertex_gradient(phi, w.field_bc, w.field_bc_value)
    ps = w.particles[0]
    idx = wl.unpack_cells(ps.cell, 2)
    R = g.X[..., 0]
    i64, t64, v64, f64 = mover.push64(idx, ps.t.astype(np.float64), ps.v.astype(np.float64), g.k, G, 0.1, -1.0, n,
                                      w.particle_bc, R=R)
    i32, t32, v32, f32, ke = mover.push32(idx, ps.t, ps.v, g.k.astype(np.float32), G.astype(np.float32), n,
                                          w.particle_bc, np.float32(-0.1), np.float32(0.05), np.float32(0.1),
                                          R32=R.astype(np.float32))
    same = (f64 == f32)
    assert same.mean() > 0.999
    alive = same & (f64 < 0)
    u64 = (i64 + t64)[:, alive]
    u32 = (i32 + t32.astype(np.float64))[:, alive]
    assert np.max(np.abs(u32 - u64)) < 32 * 2e-5
    assert np.max(np.abs(v32 - v64)[:, alive]) / np.max(np.abs(v64)) < 2e-5


def test_replay32_deterministic_and_absorbs():
    n = (16, 16)
    g = _uniform(*n)
    G32 = np.zeros(g.k.shape[:-1], np.float32)
    idx = np.array([[0, 15], [3, 4]])
    t = np.array([[0.1, 0.9], [0.5, 0.5]], np.float32)
    v = np.zeros((3, 2), np.float32)
    v[0] = [-0.5, 0.5]
    a = mover.push32(idx, t, v, g.k.astype(np.float32), G32, n, [PA, PA, PP, PP], np.float32(0), np.float32(0.05), np.float32(0.1))
    b = mover.push32(idx, t, v, g.k.astype(np.float32), G32, n, [PA, PA, PP, PP], np.float32(0), np.float32(0.05), np.float32(0.1))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert list(a[3]) == [0, 1] and list(a[0][0]) == [-1, 16]  # removed: their corrector cells


def test_reflection_is_an_elastic_wall_on_the_uniform_map():
    """Spec B on the uniform map (k = N I, the textbook Cartesian case): a particle that
    crosses a reflecting wall ends at the mirror image of its unreflected position, with the
    normal velocity component reversed and the tangential one unchanged; |v| is kept. The
    FP32 replay takes the same decisions."""
    n = (8, 8)
    X = wl.map2_vertices(8, 8, 0.0)
    g = geometry.build_geometry(X, [False, True])
    k = g.k
    G = np.zeros(k.shape[:-1])
    pbc = [mover.PBC_REFLECT, mover.PBC_REFLECT, mover.PBC_PERIODIC, mover.PBC_PERIODIC]
    # cell units: x moves by dt * 8 * vx cells per step
    idx = np.array([[0, 7, 3], [2, 5, 4]])
    t = np.array([[0.25, 0.75, 0.5], [0.5, 0.5, 0.5]])
    v = np.array([[-1.0, 1.0, 0.2], [0.3, -0.4, 0.0], [0.1, 0.0, 0.0]])
    dt = 0.05  # 0.4 cells of motion for |vx| = 1
    i1, t1, v1, face = mover.push64(idx, t, v, k, G, dt, 0.0, n, pbc)
    assert np.all(face == -1)
    u_free = idx[0] + t[0] + dt * 8 * v[0]
    u_ref = np.where(u_free < 0, -u_free, np.where(u_free >= 8, 16 - u_free, u_free))
    np.testing.assert_allclose(i1[0] + t1[0], u_ref, atol=1e-12)
    np.testing.assert_allclose(v1[0], np.where((u_free < 0) | (u_free >= 8), -v[0], v[0]), atol=1e-15)
    np.testing.assert_allclose(v1[1:], v[1:], atol=1e-15)
    np.testing.assert_allclose(np.sum(v1 ** 2, axis=0), np.sum(v ** 2, axis=0), rtol=1e-14)
    # FP32 replay: same cells and removal decisions, values to FP32 rounding
    i32, t32, v32, f32, _ = mover.push32(idx, t.astype(np.float32), v.astype(np.float32), k.astype(np.float32),
                                         G.astype(np.float32), n, pbc, np.float32(0.0), np.float32(dt / 2),
                                         np.float32(dt))
    assert np.array_equal(f32, face) and np.array_equal(i32, i1)
    np.testing.assert_allclose(t32, t1, atol=1e-6)
    np.testing.assert_allclose(v32, v1, atol=1e-6)


def test_reflection_on_a_curved_cap_keeps_speed_and_flips_the_normal():
    """Spec B on the 3D shell's polar cap: the reflected velocity has the same speed and its
    component along the cap's normal (row 1 of k, i.e. grad eta) is reversed."""
    w = wl.sphere(6, 8, 8, npart_per_species=10, seed=3)
    g = geometry.build_geometry(w.vertices, [False, False, True])
    k = g.k
    G = np.zeros(k.shape[:-1])
    # particles next to the theta = theta_c cap moving towards it (decreasing eta)
    npart = 6
    idx = np.stack([np.arange(npart) % 6, np.zeros(npart, int), np.arange(npart) % 8])
    t = np.stack([np.full(npart, 0.5), np.full(npart, 0.05), np.full(npart, 0.5)])
    # physical velocity along -grad(eta) at the particle
    kp = mover.gather(k, idx, t)
    nrm = kp[:, 1, :] / np.linalg.norm(kp[:, 1, :], axis=1)[:, None]
    v = (-3.0 * nrm).T.copy()
    i1, t1, v1, face, vk = mover.push64(idx, t, v, k, G, 0.1, 0.0, w.n, w.particle_bc, return_kicked=True)
    assert np.all(face < 0)
    assert np.all((i1[1] >= 0) & (i1[1] < w.n[1]))
    hit = np.any(v1 != vk, axis=0)  # reflected (the inner cells reach the cap in one step)
    assert 0 < np.sum(hit) < npart
    np.testing.assert_allclose(np.linalg.norm(v1, axis=0), np.linalg.norm(vk, axis=0), rtol=1e-13)
    # the component along grad(eta) was negative (towards the cap) and is now positive
    assert np.all(np.sum(vk.T * kp[:, 1, :], axis=1) < 0)
    assert np.all(np.sum(v1.T * kp[:, 1, :], axis=1)[hit] > 0)


@pytest.mark.parametrize("case", ["map2", "cylinder", "box_reflect", "sphere3d", "sphere_axisym"])
def test_c_loop_mover_and_deposit_equal_the_numpy_forms(case):
    """oracle/pic64.c restates push64 and deposit_exact as loops (for long runs): the push
    is bit-identical to the numpy form (same operation order: positions, faces, velocities
    and the v.v products), also on several threads, including absorption, reflection and
    3D; the deposit agrees to FP64 rounding of the summation order. The pins of the numpy
    forms (uniform-map limit, reversibility, second order, elastic walls) therefore hold for
    the C loops too."""
    from oracle import deposit as dep
    from oracle import geometry, gradient
    from paper_1311_2286_gb300 import workloads as wl

    w = {"map2": lambda: wl.langmuir_map2(32, 32, eps=0.1, ppc=20, vth=0.3, seed=1),
         "cylinder": lambda: wl.cylinder(32, 64, npart_per_species=50_000, seed=2, inject=False),
         "box_reflect": lambda: wl.box_reflect(16, 16, 20_000, vth=2.0),
         "sphere3d": lambda: wl.sphere(12, 10, 8, npart_per_species=20_000, seed=3),
         "sphere_axisym": lambda: wl.sphere_axisym(24, 24, npart_per_species=30_000, seed=4, inject=False)}[case]()
    per = [w.field_bc[2 * a] == 0 for a in range(w.dim)]
    g = geometry.build_geometry(w.vertices, per, axisym=w.omega_axisym)
    R = g.X[..., 0] if w.omega_axisym else None
    phi = wl.random_field(np.random.default_rng(0), tuple(reversed(w.n)), 0.5)
    if case in ("cylinder", "sphere3d", "sphere_axisym"):
        phi = phi + np.linspace(-5, 0, w.n[0])
    G = gradient.vertex_gradient(phi, w.field_bc, w.field_bc_value)
    ps = w.particles[0]
    idx = wl.unpack_cells(ps.cell, w.dim)
    t, v = ps.t.astype(np.float64), ps.v.astype(np.float64)
    a = mover.push64(idx, t, v, g.k, G, w.dt, -1.0, w.n, w.particle_bc, return_kicked=True, R=R)
    for threads in (1, 3):
        b = mover.push64_c(idx, t, v, g.k, G, w.dt, -1.0, w.n, w.particle_bc, threads=threads, R=R)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        assert np.array_equal(np.sum(a[4] * v, axis=0), b[4])
    if case in ("cylinder", "sphere3d", "sphere_axisym"):
        assert np.any(a[3] >= 0)  # the case removes particles
    if case in ("box_reflect", "sphere3d", "sphere_axisym"):
        assert np.any(np.any(a[2] != a[4], axis=0) & (a[3] < 0))  # and reflects some
    alive = a[3] < 0
    e1 = dep.deposit_exact(a[0][:, alive], a[1][:, alive], w.n, per)
    for threads in (1, 4):
        e2 = dep.deposit_exact_c(a[0][:, alive], a[1][:, alive], w.n, per, threads=threads)
        assert np.max(np.abs(e1 - e2)) <= 1e-12 * np.max(np.abs(e1))


# ------------------------------------------------------------------ uniform B0 (Boris step)

def _uniform_tables(n, G0):
    """Uniform map (k = N I in cell units) and a uniform logical field G0 at every vertex."""
    from oracle import geometry
    from paper_1311_2286_gb300 import workloads as wl

    X = wl.map2_vertices(n, n, 0.0)
    g = geometry.build_geometry(X, [True, True])
    G = np.broadcast_to(np.asarray(G0, dtype=np.float64), g.k.shape[:-2] + (2,)).copy()
    return g.k, G


def test_boris_gyration_phase_and_speed():
    """Eq. (step1) with a uniform B0 and no E (Boris rotation): the speed is kept to rounding
    and the velocity turns by exactly 2 atan(omega_c dt / 2) per step, clockwise for
    q B_z > 0 (the force q v x B), in the FP64 mover, the C loops and the FP32 replay."""
    n = 16
    k, G = _uniform_tables(n, (0.0, 0.0))
    qm, Bz, dt, N = 1.7, 0.8, 0.3, 40
    idx = np.array([[3], [5]])
    t = np.array([[0.25], [0.5]])
    v0 = np.array([[0.02], [0.0], [0.013]])
    v = v0.copy()
    i, tt = idx, t
    for _ in range(N):
        i, tt, v, face = mover.push64(i, tt, v, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=(0.0, 0.0, Bz))
    theta = 2.0 * math.atan(qm * Bz * dt / 2.0)
    ang = math.atan2(v[1, 0], v[0, 0])
    assert abs(((ang + N * theta) + math.pi) % (2 * math.pi) - math.pi) < 1e-12
    assert abs(math.hypot(v[0, 0], v[1, 0]) - 0.02) < 1e-15 and v[2, 0] == 0.013
    b = mover.push64_c(idx, t, v0, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=(0.0, 0.0, Bz))
    a = mover.push64(idx, t, v0, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=(0.0, 0.0, Bz))
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[1], b[1])
    bc = mover.boris_constants32(dt, qm, (0.0, 0.0, Bz))
    r = mover.push32(idx.astype(np.int32), t.astype(np.float32), v0.astype(np.float32), k.astype(np.float32),
                     G.astype(np.float32), (n, n), [0, 0, 0, 0], np.float32(dt * qm), np.float32(dt / 2),
                     np.float32(dt), boris=bc)
    np.testing.assert_allclose(r[2].astype(np.float64), a[2], rtol=0, atol=1e-7)


def test_boris_exb_drift():
    """Uniform E (from a uniform logical field on the uniform map) perpendicular to a uniform
    B: averaged over whole gyrations the velocity is the E x B drift E x B / B^2 (the Boris
    step keeps it exactly), and v_z is untouched."""
    n = 64
    G0 = np.array([0.01, -0.004])  # cell units: E = -k^T G = -N G0
    k, G = _uniform_tables(n, G0)
    qm, Bz, dt = -1.0, 2.0, 0.05
    E = -n * G0
    drift = np.array([E[1] * Bz, -E[0] * Bz]) / Bz**2
    idx = np.array([[10], [20]])
    t = np.array([[0.5], [0.5]])
    v = np.array([[0.3], [0.1], [0.05]])
    omega = abs(qm * Bz)
    period_steps = 2 * math.pi / (2 * math.atan(omega * dt / 2))
    N = int(round(25 * period_steps))
    acc = np.zeros(2)
    i, tt = idx, t
    vs = []
    for _ in range(N):
        i, tt, v, face = mover.push64(i, tt, v, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=(0.0, 0.0, Bz))
        vs.append(v[:2, 0].copy())
    vs = np.array(vs)
    # average over an integer number of gyrations (the nearest whole number of steps)
    mean = vs[: int(round(24 * period_steps))].mean(axis=0)
    assert np.max(np.abs(mean - drift)) < 2e-3 * np.linalg.norm(drift) + 1e-3 * 0.3, (mean, drift)
    assert v[2, 0] == 0.05


# ------------------------------------------------------------------ cyclotronic integrator

def _helix(x0, v0, b, w, t):
    """Exact motion in a uniform field alone: dv/dt = w (v x b), |b| = 1, from (x0, v0)."""
    vpar = np.dot(v0, b) * b
    vperp = v0 - vpar
    u = np.cross(v0, b)
    x = x0 + vpar * t + (math.sin(w * t) / w) * vperp + ((1.0 - math.cos(w * t)) / w) * u
    v = vpar + math.cos(w * t) * vperp + math.sin(w * t) * u
    return x, v


def test_cyclotronic_gyration_is_exact():
    """The cyclotronic push (plain electric kick, then the exact gyration flow over dt)
    follows the helix of a uniform field exactly, at any w dt (here 1.3 rad per step, with
    B oblique to the 2D plane): after 37 steps position and velocity equal the closed form
    to rounding, while the Boris step at the same dt is off by a phase error of order 0.1
    per gyration. The C loops and the FP32 replay agree with the FP64 form."""
    n = 16
    k, G = _uniform_tables(n, (0.0, 0.0))
    B = np.array([0.3, -0.4, 1.2])
    qm, N = -1.0, 37
    bm = float(np.linalg.norm(B))
    dt = 1.3 / bm
    w = qm * bm
    x0 = np.array([5.25 / n, 7.5 / n, 0.0])
    v0 = np.array([0.011, -0.006, 0.004])
    idx = np.array([[5], [7]])
    t = np.array([[0.25], [0.5]])
    i, tt, v = idx, t, v0[:, None].copy()
    ib, tb, vb = idx, t, v0[:, None].copy()
    for _ in range(N):
        i, tt, v, face = mover.push64(i, tt, v, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=B, gyro=True)
        ib, tb, vb, _f = mover.push64(ib, tb, vb, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=B)
    xe, ve = _helix(x0, v0, B / bm, w, N * dt)
    pos = (i[:, 0] + tt[:, 0]) / n
    dpos = (pos - xe[:2] + 0.5) % 1.0 - 0.5
    assert np.max(np.abs(dpos)) < 1e-13, dpos
    assert np.max(np.abs(v[:, 0] - ve)) < 1e-14, v[:, 0] - ve
    assert np.max(np.abs(vb[:, 0] - ve)) > 1e-3  # Boris: the phase error of 2 atan(w dt / 2)
    a = mover.push64(idx, t, v0[:, None], k, G, dt, qm, (n, n), [0, 0, 0, 0], B=B, gyro=True, return_kicked=True)
    c = mover.push64_c(idx, t, v0[:, None], k, G, dt, qm, (n, n), [0, 0, 0, 0], B=B, gyro=True)
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]) and np.array_equal(a[2], c[2])
    r = mover.push32(idx.astype(np.int32), t.astype(np.float32), v0[:, None].astype(np.float32),
                     k.astype(np.float32), G.astype(np.float32), (n, n), [0, 0, 0, 0], np.float32(dt * qm),
                     np.float32(dt / 2), np.float32(dt), gyro=mover.gyro_constants32(dt, qm, B))
    np.testing.assert_allclose(r[2].astype(np.float64), a[2], rtol=0, atol=1e-8)
    np.testing.assert_allclose(r[1].astype(np.float64), a[1], rtol=0, atol=1e-6)


def test_cyclotronic_exb_drift_is_exact():
    """Uniform E perpendicular to a uniform B: over a whole number of gyrations the
    cyclotronic push moves the particle by exactly (E x B / B^2) times the elapsed time,
    whatever dt (here w dt = pi/4, 8 steps per gyration, 5 gyrations), for any initial
    velocity: the kick-plus-exact-gyration composition has the E x B drift as its fixed
    point. The parallel velocity is untouched."""
    n = 64
    G0 = np.array([0.0001, -0.00004])  # a drift of (0.02, 0.05) over the run: no wrap
    k, G = _uniform_tables(n, G0)
    E = -n * G0
    qm, Bz = -1.0, 2.0
    dt = (math.pi / 4) / abs(qm * Bz)
    drift = np.array([E[1] * Bz, -E[0] * Bz]) / Bz**2
    idx = np.array([[10], [20]])
    t = np.array([[0.5], [0.5]])
    v = np.array([[0.3], [0.1], [0.05]])
    i, tt = idx, t
    N = 40
    for _ in range(N):
        i, tt, v, face = mover.push64(i, tt, v, k, G, dt, qm, (n, n), [0, 0, 0, 0], B=(0.0, 0.0, Bz), gyro=True)
    disp = ((i + tt) - (idx + t))[:, 0] / n
    np.testing.assert_allclose(disp, drift * N * dt, rtol=1e-9, atol=1e-14)
    assert v[2, 0] == 0.05


def test_axisym_gyration_sense_and_circle():
    """An axisymmetric run with B along the axis: a positive particle moving in +theta
    (v = (v_r, v_z, v_theta) = (0, v_z, v_theta), B = +B_z) is pushed outward (q v x B
    along +r): the velocity components' basis (r, z, theta) is left-handed, so the push must
    take v x B as the component cross product with -B. The cyclotronic push then follows
    the exact 3D circle (projected on the meridional plane, velocity in the moving frame)
    to the b1 map's interpolation error, and the Boris push turns the same way."""
    n = 128
    X = wl.sphere_axisym_vertices(n, n, 1.0, 10.0)
    g = geometry.build_geometry(X, [False, False], axisym=True)
    G = np.zeros(g.X.shape[:2] + (2,))
    qm, Bz, dt, m = 1.0, 0.5, 0.4, 40
    r0, z0 = 5.0, 1.0
    v0 = np.array([0.0, 0.1, 0.4])  # (v_r, v_z, v_theta)
    R = math.hypot(r0, z0)
    u = np.array([[(R - 1.0) / 9.0 * n], [(1.0 - math.atan2(r0, z0) / math.pi) * n]])
    c = np.floor(u).astype(np.int64)
    B = (0.0, Bz, 0.0)
    pbc = [1, 1, 2, 2]
    _, _, vb, _ = mover.push64(c, u - c, v0[:, None], g.k, G, dt, qm, (n, n), pbc, B=B, R=g.X[..., 0])
    _, _, vc, _ = mover.push64(c, u - c, v0[:, None], g.k, G, dt, qm, (n, n), pbc, B=B, R=g.X[..., 0], gyro=True)
    assert vb[0, 0] > 0.0 and vc[0, 0] > 0.0  # outward
    i, tt, v = c, u - c, v0[:, None].copy()
    for _ in range(m):
        i, tt, v, face = mover.push64(i, tt, v, g.k, G, dt, qm, (n, n), pbc, B=B, R=g.X[..., 0], gyro=True)
        assert face[0] == -1
    # Cartesian: x along r at the start, y along theta, z along the axis
    xe, ve = _helix(np.array([r0, 0.0, z0]), np.array([v0[0], v0[2], v0[1]]), np.array([0.0, 0.0, 1.0]),
                    qm * Bz, m * dt)
    a = math.atan2(xe[1], xe[0])
    rz = mover.gather(X, i, tt)[0]
    assert abs(rz[0] - math.hypot(xe[0], xe[1])) < 10.0 / n**2 and abs(rz[1] - xe[2]) < 10.0 / n**2
    vr = math.cos(a) * ve[0] + math.sin(a) * ve[1]
    vth = -math.sin(a) * ve[0] + math.cos(a) * ve[1]
    assert np.max(np.abs(v[:, 0] - np.array([vr, ve[2], vth]))) < 2.0 / n**2
    # C loops and FP32 replay of one axisymmetric cyclotronic step
    a64 = mover.push64(c, u - c, v0[:, None], g.k, G, dt, qm, (n, n), pbc, B=B, R=g.X[..., 0], gyro=True)
    c64 = mover.push64_c(c, u - c, v0[:, None], g.k, G, dt, qm, (n, n), pbc, B=B, R=g.X[..., 0], gyro=True)
    assert all(np.array_equal(x, y) for x, y in zip(a64[:3], c64[:3]))
    r32 = mover.push32(c.astype(np.int32), (u - c).astype(np.float32), v0[:, None].astype(np.float32),
                       g.k.astype(np.float32), G.astype(np.float32), (n, n), pbc, np.float32(dt * qm),
                       np.float32(dt / 2), np.float32(dt), R32=g.X[..., 0].astype(np.float32),
                       gyro=mover.gyro_constants32(dt, qm, B, axisym=True))
    np.testing.assert_allclose(r32[2].astype(np.float64), a64[2], rtol=0, atol=2e-7)
