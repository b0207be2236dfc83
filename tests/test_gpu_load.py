"""Device-side Maxwellian loading (cpic_load_maxwellian) against its definition:
cells drawn with probability J_c / sum J_c (uniform physical density), offsets uniform in
each cell, velocities vth N(0, 1) + drift. Statistical checks with fixed seeds, plus
determinism (same seed -> same particles)."""
import numpy as np
import pytest

from paper_1311_2286_gb300 import workloads as wl
from oracle import geometry as ogeo

pytestmark = pytest.mark.gpu


def _run(cpic, n1, n2, npart):
    w = wl.cylinder(n1=n1, n2=n2, npart_per_species=16, seed=5, inject=False, capacity_factor=npart / 16 + 2)
    run = cpic.run_from_workload(w)
    return w, run


def test_maxwellian_load_statistics(cpic):
    n1, n2, N = 32, 64, 400_000
    w, run = _run(cpic, n1, n2, N)
    vth, drift = 0.7, (0.3, -0.2, 0.1)
    run.load_maxwellian(0, N, vth, seed=1234, drift=drift)
    cell, t, v = run.particles(0)
    assert cell.shape == (N,)
    i, j = cell & 0xFFFF, cell >> 16
    assert i.min() >= 0 and i.max() < n1 and j.min() >= 0 and j.max() < n2
    # cell probabilities from the oracle's own cell Jacobians (independent of the device)
    per = [w.field_bc[2 * a] == wl.BC_PERIODIC for a in range(w.dim)]
    g = ogeo.build_geometry(w.vertices, per, axisym=w.omega_axisym)
    Jc = np.asarray(g.Jc, dtype=np.float64).reshape(n2, n1)
    p = (Jc / Jc.sum()).ravel()
    counts = np.bincount(i + n1 * j, minlength=n1 * n2).astype(np.float64)
    expected = N * p
    chi2 = np.sum((counts - expected) ** 2 / expected)
    dof = n1 * n2 - 1
    assert abs(chi2 - dof) < 6 * np.sqrt(2 * dof), (chi2, dof)
    # offsets uniform in [0, 1)
    assert t.min() >= 0.0 and t.max() < 1.0
    for a in range(2):
        assert abs(t[a].mean() - 0.5) < 5 / np.sqrt(12 * N)
        assert abs(t[a].var() - 1 / 12) < 0.01 / 12 * 5
    # velocities
    for a in range(3):
        m, s2 = v[a].mean(), v[a].var()
        assert abs(m - drift[a]) < 5 * vth / np.sqrt(N)
        assert abs(s2 / vth**2 - 1) < 5 * np.sqrt(2 / N)
        # fourth moment of a Gaussian: kurtosis 3
        k = np.mean((v[a] - m) ** 4) / s2**2
        assert abs(k - 3) < 0.05
    run.close()


def test_maxwellian_load_is_deterministic(cpic):
    w, run = _run(cpic, 16, 32, 50_000)
    run.load_maxwellian(1, 50_000, 0.05, seed=99)
    a = run.particles(1)
    run.load_maxwellian(1, 50_000, 0.05, seed=99)
    b = run.particles(1)
    run.load_maxwellian(1, 50_000, 0.05, seed=100)
    c = run.particles(1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[2], c[2])
    run.close()


def test_maxwellian_load_axisym_is_uniform_in_volume(cpic):
    """An axisymmetric run loads rings uniform in the 3D volume: cells with probability
    Omega_c J_c / sum Omega_c J_c (the ring volume 2 pi r J_c, up to the constant)."""
    n1, n2, N = 16, 32, 300_000
    w = wl.sphere_axisym(n1, n2, npart_per_species=16, seed=5, inject=False, capacity_factor=N / 16 + 2)
    run = cpic.run_from_workload(w)
    run.load_maxwellian(0, N, 1.0, seed=77)
    cell, t, v = run.particles(0)
    i, j = cell & 0xFFFF, cell >> 16
    g = ogeo.build_geometry(w.vertices, [False, False], axisym=True)
    wgt = (np.asarray(g.omega_c) * np.asarray(g.Jc)).reshape(n2, n1)
    p = (wgt / wgt.sum()).ravel()
    counts = np.bincount(i + n1 * j, minlength=n1 * n2).astype(np.float64)
    expected = N * p
    chi2 = np.sum((counts - expected) ** 2 / expected)
    dof = n1 * n2 - 1
    assert abs(chi2 - dof) < 6 * np.sqrt(2 * dof), (chi2, dof)
    run.close()
