"""Pins of the oracle's axisymmetric (Omega = r) path: the 2D (r, z) meridional plane of
a problem with azimuthal symmetry (Sec. II.B, the spherical-shell map of Sec. II.B.3 and
the sphere-in-plasma run of Sec. III.B). Each check is fixed by the physics, not by the
oracle: Gauss's law for a charged sphere, straight-line free streaming in 3D, the ring
density of a uniformly loaded shell and the surface of revolution of the injection face."""
import math

import numpy as np
import pytest

from oracle import inject, mover
from oracle import geometry
from paper_1311_2286_gb300 import workloads as wl


def _empty(w):
    w.particles = [wl.ParticleSet(np.zeros(0, np.int32), np.zeros((2, 0), np.float32),
                                  np.zeros((3, 0), np.float32)) for _ in w.species]
    return w


def test_floating_sphere_capacitance():
    """A sphere of radius 1 carrying charge Q inside a grounded sphere of radius 10 floats
    to V = Q (1/r1 - 1/r2) / (4 pi) (eps0 = 1) and the charge-free potential between them
    is V (1/r - 1/r2) / (1/r1 - 1/r2). This fixes the 2 pi of Gauss's law on the
    ring-charge scale and the Omega = r face coefficients; the discrete value converges at
    second order."""
    from oracle.pic import OraclePIC

    Q = 0.61
    exact = Q * (1.0 - 0.1) / (4.0 * math.pi)
    errs = []
    for n in (16, 32, 64):
        w = _empty(wl.sphere_axisym(n, n, npart_per_species=1, phi_obj=2.0, inject=False))
        pic = OraclePIC(w, "fp64")
        pic.set_floating(0, Q)
        pic.solve()
        errs.append(abs(pic.object_potential - exact))
        rad = 1.0 + 9.0 * (np.arange(n) + 0.5) / n
        prof = pic.phi.mean(axis=0)  # every polar row holds the same radial profile
        np.testing.assert_allclose(prof, exact * (1.0 / rad - 0.1) / 0.9, rtol=0, atol=4e-2 * exact)
        # spherical symmetry: the rows agree with each other
        assert np.max(np.abs(pic.phi - prof[None, :])) < 2e-2 * exact
    assert errs[2] < 5e-3 * exact, errs
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def _physical(X, idx, t):
    """(r, z) of logical positions by b1 interpolation of the vertex table."""
    return mover.gather(X, idx.astype(np.int64), t)


@pytest.mark.parametrize("n", [64, 128])
def test_axisym_free_streaming_is_a_straight_line(n):
    """With no field a ring particle moves on a straight line in 3D: after m steps
    (x, y, z) = (r0 + m dt v_r, m dt v_theta, z0 + m dt v_z), so r = sqrt(x^2 + y^2), and
    its velocity in the cylindrical frame at the end is the Cartesian velocity turned by
    the azimuth atan2(y, x). r v_theta is conserved. The test follows particles through
    the axis region and checks all three against the closed form; the error is the map's
    b1 interpolation error, and halves at least as the grid doubles."""
    X = wl.sphere_axisym_vertices(n, n, 1.0, 10.0)
    g = geometry.build_geometry(X, [False, False], axisym=True)
    G = np.zeros(g.X.shape[:2] + (2,))
    r0 = np.array([3.0, 2.0, 6.0, 0.7])
    z0 = np.array([1.0, -2.5, 0.5, 4.0])
    v0 = np.array([[0.3, -0.5, -0.2, 0.4],   # v_r
                   [0.5, 0.1, 0.3, -0.6],    # v_z
                   [0.2, 0.7, -0.9, 0.05]])  # v_theta
    # logical coordinates of (r0, z0) on the spherical-shell map
    R = np.hypot(r0, z0)
    polar = np.arctan2(r0, z0)
    u = np.stack([(R - 1.0) / 9.0 * n, (1.0 - polar / math.pi) * n])
    c = np.floor(u).astype(np.int64)
    t = u - c
    idx, v = c, v0.copy()
    dt, m = 0.05, 60
    for _ in range(m):
        idx, t, v, face = mover.push64(idx, t, v, g.k, G, dt, 0.0, (n, n), [3, 3, 2, 2], R=g.X[..., 0])
        assert np.all(face == -1)
    x = r0 + m * dt * v0[0]
    y = m * dt * v0[2]
    z = z0 + m * dt * v0[1]
    a = np.arctan2(y, x)
    rz = _physical(X, idx, t)
    err_pos = np.max(np.abs(rz - np.stack([np.hypot(x, y), z], axis=1)))
    vr = np.cos(a) * v0[0] + np.sin(a) * v0[2]
    vth = np.cos(a) * v0[2] - np.sin(a) * v0[0]
    err_v = np.max(np.abs(np.stack([vr, v0[1], vth]) - v))
    assert err_pos < 10.0 / n**2, err_pos
    assert err_v < 1.0 / n**2, err_v
    # speed is kept exactly up to rounding (a pure rotation of (v_r, v_theta))
    np.testing.assert_allclose(np.sum(v * v, axis=0), np.sum(v0 * v0, axis=0), rtol=1e-13)
    # angular momentum r v_theta against its initial value
    np.testing.assert_allclose(rz[:, 0] * v[2], r0 * v0[2], rtol=0, atol=10.0 / n**2)


def test_axisym_free_streaming_converges():
    """The end-point error of the free-streaming check falls at least 3x per grid
    doubling (second order in the cell size of the b1 map)."""
    errs = []
    for n in (32, 64, 128):
        X = wl.sphere_axisym_vertices(n, n, 1.0, 10.0)
        g = geometry.build_geometry(X, [False, False], axisym=True)
        G = np.zeros(g.X.shape[:2] + (2,))
        r0, z0 = np.array([2.5]), np.array([1.5])
        v0 = np.array([[0.4], [-0.3], [0.6]])
        R = np.hypot(r0, z0)
        u = np.stack([(R - 1.0) / 9.0 * n, (1.0 - np.arctan2(r0, z0) / math.pi) * n])
        c = np.floor(u).astype(np.int64)
        idx, t, v = c, u - c, v0.copy()
        for _ in range(40):
            idx, t, v, _f = mover.push64(idx, t, v, g.k, G, 0.05, 0.0, (n, n), [3, 3, 2, 2], R=g.X[..., 0])
        x, y, z = r0 + 2.0 * v0[0], 2.0 * v0[2], z0 + 2.0 * v0[1]
        rz = _physical(X, idx, t)
        errs.append(float(np.max(np.abs(rz - np.stack([np.hypot(x, y), z], axis=1)))))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_ring_density_of_uniform_shell():
    """Rings loaded uniformly in the 3D shell at density 1 (the sphere workload's loading)
    give Q_c = q n J_c in every cell once each ring's charge is spread over its ring
    volume 2 pi r J_c: the oracle's charge Q_c / (q J_c) averages 1 in radial and polar
    bands alike (a missing 2 pi, a missing 1/r or a loading that is not uniform in volume
    fails one band by far more than the sampling noise)."""
    from oracle.pic import OraclePIC

    n = 16
    w = wl.sphere_axisym(n, n, npart_per_species=400_000, inject=False, seed=11)
    w.species = w.species[:1]
    w.particles = w.particles[:1]
    w.background = 0.0
    pic = OraclePIC(w, "fp64")
    dens = pic.charge() / (w.species[0].q * pic.geom.Jc)  # (n2, n1)
    # interior bands (the b2 shape spills charge into the boundary cells' neighbours)
    for band in (dens[2:-2, 2:6], dens[2:-2, 6:10], dens[2:-2, 10:14], dens[2:5, 2:-2], dens[6:10, 2:-2],
                 dens[11:14, 2:-2]):
        assert abs(band.mean() - 1.0) < 0.03, band.mean()


def test_axisym_injection_face_and_segment_weights():
    """The injection face xi = 1 is the sphere r = 10: its surface of revolution sums to
    4 pi 100 up to the polygon's O(h^2) error, and the ring-area draw picks each face
    segment with probability proportional to 2 pi r_mid |dX| (chi-square over all segments,
    a uniform-in-segment draw fails by orders of magnitude)."""
    n = 32
    X = wl.sphere_axisym_vertices(n, n, 1.0, 10.0)
    area = inject.face_area_axisym(X, 1)
    assert abs(area / (4.0 * math.pi * 100.0) - 1.0) < 2.0 / n**2
    rings = inject.face_ring_areas_2d(X, 1)
    g = geometry.build_geometry(X, [False, False], axisym=True)
    cnt = 200_000
    idx, t32, v32, keep = inject.inject_2d(g.k, (n, n), 1, cnt, 0, 0, 1234, 1.0, (0.0, 0.0, 0.0), 1e-4,
                                           ring_areas=rings)
    assert keep.mean() > 0.99
    obs = np.bincount(idx[1], minlength=n).astype(np.float64)
    expect = rings / rings.sum() * obs.sum()
    chi2 = float(np.sum((obs - expect) ** 2 / expect))
    assert chi2 < n + 6.0 * math.sqrt(2.0 * n), chi2
    # injected particles enter through the face, inward: v_r of the radial direction < 0
    assert np.all(idx[0] == n - 1)
