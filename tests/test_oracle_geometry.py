"""Pins of the oracle's metric (spec M) against closed forms and the paper's printed facts."""
import math

import numpy as np
import pytest

from oracle import geometry
from paper_1311_2286_gb300 import workloads as wl


def _cell_centres(n1, n2):
    xi = (np.arange(n1) + 0.5) / n1
    eta = (np.arange(n2) + 0.5) / n2
    XI, ETA = np.meshgrid(xi, eta, indexing="xy")
    return XI, ETA


@pytest.mark.parametrize("eps", [0.05, 0.1])
def test_map2_jacobian_closed_form_second_order(eps):
    """P2: FD J_c of map2 converges at second order to J = 1 + 2 pi eps sin 2 pi (xi + eta)
    (eq. (map2)); cell units: J_c = J / (N1 N2)."""
    errs = []
    for n in (32, 64, 128):
        g = geometry.build_geometry(wl.map2_vertices(n, n, eps), [True, True])
        XI, ETA = _cell_centres(n, n)
        exact = wl.map2_jacobian_exact(XI, ETA, eps) / (n * n)
        errs.append(np.max(np.abs(g.Jc - exact)) * n * n)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_map2_cell_size_ratio_matches_paper():
    """Sec. II.B.4: at eps = 0.1 the ratio of the largest to smallest cell is 4.4;
    closed form (1 + 2 pi eps)/(1 - 2 pi eps) = 4.38."""
    g = geometry.build_geometry(wl.map2_vertices(256, 256, 0.1), [True, True])
    ratio = g.Jc.max() / g.Jc.min()
    closed = (1 + 2 * math.pi * 0.1) / (1 - 2 * math.pi * 0.1)
    assert abs(ratio - closed) / closed < 2e-3
    assert round(ratio, 1) == 4.4


def test_map2_inverse_jacobi_second_order():
    """k = j^-1 (eq. (jcon)) at vertices vs the analytic inverse of eq. (map2)'s Jacobi
    matrix, in cell units (k_cell = N k)."""
    eps = 0.1
    errs = []
    for n in (32, 64, 128):
        g = geometry.build_geometry(wl.map2_vertices(n, n, eps), [True, True])
        xi = np.arange(n + 1) / n
        XI, ETA = np.meshgrid(xi, xi, indexing="xy")
        a = 2 * math.pi * eps * np.cos(2 * math.pi * XI) * np.sin(2 * math.pi * ETA)
        b = 2 * math.pi * eps * np.sin(2 * math.pi * XI) * np.cos(2 * math.pi * ETA)
        j = np.empty(XI.shape + (2, 2))
        j[..., 0, 0] = 1 + a
        j[..., 0, 1] = b
        j[..., 1, 0] = a
        j[..., 1, 1] = 1 + b
        kex = np.linalg.inv(j) * n
        errs.append(np.max(np.abs(g.k - kex)) / n)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_uniform_map_reduces_to_cartesian():
    """P1: with eps = 0 the map is the identity; in cell units k = N I, J_c = 1/(N1 N2),
    face coefficients a^{uu} = N1/N2, a^{vv} = N2/N1, cross terms 0."""
    n1, n2 = 16, 24
    X = wl.map2_vertices(n1, n2, 0.0)
    g = geometry.build_geometry(X, [True, True])
    np.testing.assert_allclose(g.k[..., 0, 0], n1, rtol=1e-12)
    np.testing.assert_allclose(g.k[..., 1, 1], n2, rtol=1e-12)
    assert np.max(np.abs(g.k[..., 0, 1])) < 1e-9 and np.max(np.abs(g.k[..., 1, 0])) < 1e-9
    np.testing.assert_allclose(g.Jc, 1.0 / (n1 * n2), rtol=1e-12)
    np.testing.assert_allclose(g.face[0][0], n1 / n2, rtol=1e-12)
    np.testing.assert_allclose(g.face[1][1], n2 / n1, rtol=1e-12)
    assert np.max(np.abs(g.face[0][1])) < 1e-12 and np.max(np.abs(g.face[1][0])) < 1e-12


def test_annulus_area_and_orthogonality():
    """The cell Jacobian of a bilinear cell is its exact polygon area: the sum equals the
    area of the inscribed polygonal annulus (closed form), and the log-polar map is
    orthogonal (g^{12} = 0, eq. (gcon))."""
    n1, n2, r0, R = 32, 64, 1.0, 40.0
    g = geometry.build_geometry(wl.annulus_vertices(n1, n2, r0, R), [False, True])
    poly = 0.5 * n2 * math.sin(2 * math.pi / n2) * (R * R - r0 * r0)
    assert abs(g.Jc.sum() - poly) / poly < 1e-12
    assert np.max(np.abs(g.face[0][1])) < 1e-9 * np.max(np.abs(g.face[0][0]))
    assert np.max(np.abs(g.face[1][0])) < 1e-9 * np.max(np.abs(g.face[1][1]))


def test_periodic_vertex_tables_are_exact_images():
    """On a periodic axis vertex N repeats vertex 0 bit for bit (the device table relies on
    it)."""
    g = geometry.build_geometry(wl.map2_vertices(16, 16, 0.07), [True, True])
    assert np.array_equal(g.k[:, -1], g.k[:, 0]) and np.array_equal(g.k[-1, :], g.k[0, :])


def test_shell_volume_and_orthogonality():
    """3D shell: the cell Jacobians sum to the shell segment's volume at second order. The
    spherical map is orthogonal in the continuum; the discrete face metric built from chord
    averages is orthogonal up to O(h^2), so the cross coefficients decay at second order
    (and vanish exactly on the faces normal to the periodic azimuth)."""
    r0, R, tc = 1.0, 30.0, math.pi / 32
    exact = 2 * math.pi / 3 * (R ** 3 - r0 ** 3) * 2 * math.cos(tc)
    errs, cross = [], []
    for n in (8, 16, 32):
        X = wl.shell_vertices(n, n, n, r0, R, tc)
        g = geometry.build_geometry(X, [False, False, True])
        errs.append(abs(g.Jc.sum() - exact) / exact)
        worst = 0.0
        for a in range(3):
            for b in range(3):
                if a != b:
                    worst = max(worst, np.max(np.abs(g.face[a][b])) / np.max(np.abs(g.face[a][a])))
        cross.append(worst)
        assert np.max(np.abs(g.face[2][0])) < 1e-12 * np.max(np.abs(g.face[2][2]))
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.6
    assert cross[0] / cross[1] > 3.5 and cross[1] / cross[2] > 3.8


def test_inverse3_against_numpy():
    rng = np.random.default_rng(0)
    m = rng.standard_normal((50, 3, 3)) + 3 * np.eye(3)
    k, det = geometry.inverse3(m)
    np.testing.assert_allclose(k, np.linalg.inv(m), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(det, np.linalg.det(m), rtol=1e-12)
