"""Pins of the vertex field (spec G), the b-splines and the fixed-point deposit (spec Q)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import deposit as dep
from oracle import geometry, gradient, mover, poisson
from paper_1311_2286_gb300 import workloads as wl

P, Dr, N_ = poisson.BC_PERIODIC, poisson.BC_DIRICHLET, poisson.BC_NEUMANN


# ------------------------------------------------------------------ spec G (vertex field)

def test_gradient_of_linear_potential_is_exact():
    """phi = a i + b j (cell units): every interior vertex has G = (a, b) exactly."""
    n1, n2 = 9, 7
    i = np.arange(n1)[None, :]
    j = np.arange(n2)[:, None]
    phi = 0.75 * i - 1.25 * j + 0.0 * i * j
    G = gradient.vertex_gradient(phi, [Dr, Dr, Dr, Dr], [0.0] * 4)
    np.testing.assert_array_equal(G[1:-1, 1:-1, 0], 0.75)
    np.testing.assert_array_equal(G[1:-1, 1:-1, 1], -1.25)


def test_gradient_second_order_and_periodic_images():
    errs = []
    for n in (16, 32, 64):
        x = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(x, x, indexing="xy")
        phi = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        G = gradient.vertex_gradient(phi, [P] * 4, [0.0] * 4)
        xv = np.arange(n + 1) / n
        XV, YV = np.meshgrid(xv, xv, indexing="xy")
        gx = 2 * np.pi * np.cos(2 * np.pi * XV) * np.cos(2 * np.pi * YV) / n
        errs.append(np.max(np.abs(G[..., 0] - gx)) * n)
        assert np.array_equal(G[:, -1], G[:, 0]) and np.array_equal(G[-1, :], G[0, :])
    assert errs[0] / errs[1] > 3.7 and errs[1] / errs[2] > 3.9


def test_gradient_tangential_zero_on_dirichlet_face():
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((6, 8))
    G = gradient.vertex_gradient(phi, [Dr, Dr, P, P], [-5.0, 0.0, 0, 0])
    assert np.max(np.abs(G[:, 0, 1])) < 1e-15 and np.max(np.abs(G[:, -1, 1])) < 1e-15


def test_physical_field_of_uniform_potential_on_distorted_map():
    """E = -k^T G gathered with b1 weights (eqs. (vvp), (Wvp)) reproduces a uniform physical
    field E0 from phi = -E0 . x on the non-orthogonal map2 grid, at second order."""
    E0 = np.array([0.3, -0.7])
    errs = []
    for n in (16, 32, 64):
        X = wl.map2_vertices(n, n, 0.1)
        g = geometry.build_geometry(X, [True, True])
        xc = (np.arange(n) + 0.5) / n
        XI, ETA = np.meshgrid(xc, xc, indexing="xy")
        s = 0.1 * np.sin(2 * np.pi * XI) * np.sin(2 * np.pi * ETA)
        # phi = -E0.x is not periodic; use ghosts built from the map's own periodic shift:
        # take phi' = -E0.(x - xi_vec) which is periodic, and add the logical part exactly
        phi_p = -(E0[0] * s + E0[1] * s)
        G = gradient.vertex_gradient(phi_p, [P] * 4, [0.0] * 4)
        G[..., 0] += -E0[0] / n
        G[..., 1] += -E0[1] / n
        rng = np.random.default_rng(4)
        idx = np.stack([rng.integers(0, n, 500), rng.integers(0, n, 500)])
        t = rng.random((2, 500))
        kp = mover.gather(g.k, idx, t)
        gp = mover.gather(G, idx, t)
        E = -np.einsum("pa,pab->pb", gp, kp)
        errs.append(np.max(np.abs(E - E0)))
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.6


# ------------------------------------------------------------------ b-splines (eqs. b1, b2)

def test_b2_partition_of_unity_and_printed_constant():
    """Eq. (b2) with the restored 1/2 sums to one over the three nearest cell centres and is
    continuous at |xi| = 1/2, 3/2; the printed form (without 1/2) is neither."""
    d = np.linspace(-0.5, 0.4999, 1001)
    s = dep.b2(d - 1) + dep.b2(d) + dep.b2(d + 1)
    np.testing.assert_allclose(s, 1.0, rtol=0, atol=1e-14)
    assert abs(dep.b2(0.5 - 1e-12) - dep.b2(0.5 + 1e-12)) < 1e-10
    assert abs(dep.b2(1.5 - 1e-9)) < 1e-15
    printed = dep.b2_as_printed(d - 1) + dep.b2_as_printed(d) + dep.b2_as_printed(d + 1)
    assert np.min(np.abs(printed - 1.0)) > 0.2
    assert abs(dep.b2_as_printed(0.5 - 1e-12) - dep.b2_as_printed(0.5 + 1e-12)) > 0.4


def test_b1_interpolation_partition():
    d = np.linspace(0, 1, 11)
    np.testing.assert_allclose(dep.b1(d) + dep.b1(d - 1), 1.0)


# ------------------------------------------------------------------ spec Q

def test_axis_weights_are_exact_b2_values():
    """W[m] = b2 at the sub-cell centre d = s / 2^(K+1), scaled by 2^(2K+3), exactly
    (rational arithmetic), and they sum to 2^(2K+3)."""
    t = np.array([0.0, 1e-9, 0.25, 0.5, 0.73, np.nextafter(np.float32(1), np.float32(0))], dtype=np.float32)
    W = dep.axis_weights(t)
    K = dep.QK
    for p in range(t.size):
        u = math.floor(Fraction(float(t[p])) * 2 ** K)
        s = 2 * u + 1 - 2 ** K
        d = Fraction(s, 2 ** (K + 1))
        b2 = lambda x: Fraction(3, 4) - x * x if abs(x) < Fraction(1, 2) else Fraction(1, 2) * (Fraction(3, 2) - abs(x)) ** 2
        for m in (-1, 0, 1):
            assert Fraction(int(W[m + 1][p])) == b2(d - m) * 2 ** (2 * K + 3)
        assert sum(int(W[m][p]) for m in range(3)) == 2 ** (2 * K + 3)


@pytest.mark.parametrize("D", [2, 3])
def test_node_weights_sum_exactly_and_approximate_b2(D):
    rng = np.random.default_rng(D)
    t = rng.random((D, 4000)).astype(np.float32)
    t[:, :3] = np.float32(0.0)
    t[:, 3] = np.nextafter(np.float32(1), np.float32(0))
    q = dep.node_weights(t)
    total = sum(q.values())
    assert np.all(total == 1 << dep.QF)
    d = t.astype(np.float64) - 0.5
    for m, qm in q.items():
        exact = np.ones(t.shape[1])
        for a in range(D):
            exact = exact * dep.b2(d[a] - m[a])
        assert np.all(qm >= 0) and np.all(qm < 1 << dep.QF)
        # per axis: the offset is quantised to the centre of its 2^-16 sub-interval (b2 has
        # slope <= 1, so it moves by <= 2^-17) and the weight rounded to 2^-16 (error
        # <= 2^-17, twice that for the centre); each product rounded to 2^-24 (the centre
        # takes the other 3^D - 1 roundings)
        axis_err = 2.0 ** -17 + 2.0 ** -16
        assert np.max(np.abs(qm / 2.0 ** dep.QF - exact)) < D * axis_err + 3 ** D * 2.0 ** -25


@pytest.mark.parametrize("D", [2, 3])
def test_axis_weights_fixed_are_rounded_b2_and_sum_exactly(D):
    """The 16-bit per-axis weights are the nearest multiples of 2^-16 of the exact b2
    values of the quantised offset (outer nodes), the centre takes the remainder; every
    node weight but the centre is the exact product rounded to 2^-24 (halves up), the
    centre the remainder (rational arithmetic)."""
    rng = np.random.default_rng(40 + D)
    t = np.concatenate([np.array([0.0, 0.5, np.nextafter(np.float32(1), np.float32(0))], dtype=np.float32),
                        rng.random(200).astype(np.float32)])
    B = dep.QB
    w = dep.axis_weights_fixed(t)
    K = dep.QK
    for p in range(t.size):
        u = math.floor(Fraction(float(t[p])) * 2 ** K)
        d = Fraction(2 * u + 1 - 2 ** K, 2 ** (K + 1))
        for m in (-1, 1):
            exact = (Fraction(1, 2) * (Fraction(3, 2) - abs(d - m)) ** 2) * 2 ** B
            assert abs(Fraction(int(w[m + 1][p])) - exact) <= Fraction(1, 2)
        assert int(w[0][p]) + int(w[1][p]) + int(w[2][p]) == 2 ** B
    tt = np.stack([t] * D)
    q = dep.node_weights(tt)
    r = D * B - dep.QF
    centre = (0,) * D
    rest = np.zeros(t.size, dtype=object)
    for m, qm in q.items():
        if m == centre:
            continue
        for p in range(0, t.size, 17):
            prod = Fraction(1)
            for a in range(D):
                prod *= int(w[m[a] + 1][p])
            x = prod / 2 ** r
            # round half up: the nearest integer, ties upwards
            assert Fraction(int(qm[p])) - Fraction(1, 2) < x <= Fraction(int(qm[p])) + Fraction(1, 2)
        rest = rest + qm.astype(object)
    assert np.array_equal(q[centre].astype(object), (1 << dep.QF) - rest)


@pytest.mark.parametrize("D", [2, 3])
def test_deposit_conserves_charge_exactly(D):
    """P5: every particle deposits exactly 2^QF units, also when its stencil folds onto a
    non-periodic boundary cell."""
    rng = np.random.default_rng(10 + D)
    n = (6, 5, 4)[:D]
    npart = 3000
    idx = np.stack([rng.integers(0, n[a], npart) for a in range(D)])
    t = rng.random((D, npart)).astype(np.float32)
    periodic = [False, True, True][:D]
    C = dep.deposit_fixed(idx, t, n, periodic)
    assert C.dtype == np.int64 and int(C.sum()) == npart << dep.QF
    E = dep.deposit_exact(idx, t, n, periodic)
    assert abs(E.sum() - npart) < 1e-9
    assert np.max(np.abs(C / 2.0 ** dep.QF - E)) < npart * 2.0 ** -14


def test_deposit_uniform_grid_textbook_tsc():
    """P1: on the uniform grid one particle's deposit is the tensor product of textbook TSC
    weights (0.5 (0.5 - d)^2, 0.75 - d^2, 0.5 (0.5 + d)^2)."""
    idx = np.array([[3], [2]])
    t = np.array([[0.3], [0.85]], dtype=np.float32)
    E = dep.deposit_exact(idx, t, (8, 8), [True, True])
    d = t[:, 0].astype(np.float64) - 0.5
    w = [np.array([0.5 * (0.5 - x) ** 2, 0.75 - x * x, 0.5 * (0.5 + x) ** 2]) for x in d]
    ref = np.zeros((8, 8))
    for a, b in itertools.product(range(3), range(3)):
        ref[2 + b - 1, 3 + a - 1] = w[0][a] * w[1][b]
    np.testing.assert_allclose(E, ref, atol=1e-15)


def _potential_error_of_quantisation(w):
    """Relative L2 difference of the potentials solved from the spec-Q deposit and from the
    unquantised FP64 deposit of the same particles (the solve is linear, so the difference
    is the solve of the charge difference with homogeneous boundary values)."""
    per = [w.field_bc[2 * a] == P for a in range(w.dim)]
    g = geometry.build_geometry(w.vertices, per)
    M, bbc = poisson.assemble(g, w.field_bc, w.field_bc_value)
    M0, b0 = poisson.assemble(g, w.field_bc, [0.0] * len(w.field_bc_value))
    dQ = np.zeros(g.Jc.shape)
    Qe = w.background * g.Jc
    for sp, ps in zip(w.species, w.particles):
        idx = wl.unpack_cells(ps.cell, w.dim)
        Cf = dep.deposit_fixed(idx, ps.t, w.n, per)
        Ce = dep.deposit_exact(idx, ps.t.astype(np.float64), w.n, per)
        dQ += sp.q * sp.w * (np.ldexp(Cf.astype(np.float64), -dep.QF) - Ce)
        Qe += sp.q * sp.w * Ce
    phi = poisson.solve(g, M, bbc, Qe, w.field_bc)
    dphi = poisson.solve(g, M0, b0, dQ, w.field_bc)
    return np.linalg.norm(dphi) / np.linalg.norm(phi)


@pytest.mark.parametrize("case", ["cylinder_128x256_4M", "shell_24x24x24_414k"])
def test_quantised_deposit_potential_within_fp32_state_tolerance(case):
    """Spec Q's effect on the field: at the cylinder configuration's full size (128 x 256,
    2M + 2M particles) and on a 3D shell with the sphere configuration's particles per cell
    (about 30), the potential solved from the fixed-point deposit is within 1e-5 relative
    L2 (the single-step FP32 state tolerance) of the one solved from the exact FP64 b2
    deposit of the same particles."""
    if case.startswith("cylinder"):
        w = wl.cylinder(n1=128, n2=256, npart_per_species=2_000_000, seed=1, inject=False)
    else:
        w = wl.sphere(24, 24, 24, npart_per_species=207_000, seed=2)
    err = _potential_error_of_quantisation(w)
    assert err <= 1e-5, err
