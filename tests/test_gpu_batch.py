"""Batched runs (row a11): a run stepped inside a batch gives bit-identical particles (as
sets: the order inside a cell after a sort is unspecified), charge, potential and
diagnostics to the same run stepped alone, for full cycles and for fixed-field particle
steps, across sort steps, and after members are removed."""
import numpy as np
import pytest

from paper_1311_2286_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SPECS = [dict(n1=16, n2=32, npart_per_species=3001, seed=41, phi_obj=-5.0),
         dict(n1=32, n2=64, npart_per_species=12007, seed=42, phi_obj=-2.0),
         dict(n1=24, n2=48, npart_per_species=5003, seed=43, phi_obj=1.0)]


def _make(cpic, spec):
    w = wl.cylinder(inject=True, **spec)
    return cpic.run_from_workload(w, sort_interval=3)


def _records(cell, t, v):
    # the order of particles inside a cell after a sort is unspecified: compare sets
    return np.sort(np.rec.fromarrays([cell, t[0], t[1], v[0], v[1], v[2]]))


def _state(run):
    out = [run.phi(), run.diag()]
    for s in range(2):
        out.append(_records(*run.particles(s)))
        out.append(run.charge(s))
    return out


def _same(a, b):
    pa, pb = a[0], b[0]
    assert np.array_equal(pa, pb)
    da, db = a[1], b[1]
    for k in da:
        assert np.array_equal(np.asarray(da[k]), np.asarray(db[k])), k
    for x, y in zip(a[2:], b[2:]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("solve", [True, False])
def test_batch_equals_alone(cpic, solve, mode):
    nsteps = 7  # crosses two sorts (interval 3)
    alone = []
    for spec in SPECS:
        r = _make(cpic, spec)
        r.initialize()
        (r.step if solve else r.step_particles)(nsteps)
        alone.append(_state(r))
        r.close()
    runs = [_make(cpic, spec) for spec in SPECS]
    b = cpic.Batch(8)
    b.set_mode(mode)
    for r in runs:
        r.initialize()
        b.add(r)
    assert len(b) == len(SPECS)
    b.step(nsteps, solve=solve)
    b.synchronize()
    for r, ref in zip(runs, alone):
        _same(_state(r), ref)
    b.close()
    for r in runs:
        r.close()


def test_batch_remove_and_continue(cpic):
    """Removing a member mid-run: the remaining members continue exactly as alone."""
    ref = _make(cpic, SPECS[1])
    ref.initialize()
    ref.step(5)
    want = _state(ref)
    ref.close()
    runs = [_make(cpic, spec) for spec in SPECS]
    b = cpic.Batch(4)
    for r in runs:
        r.initialize()
        b.add(r)
    b.step(2)
    b.remove(runs[0])
    b.remove(runs[2])
    b.step(3)
    b.synchronize()
    _same(_state(runs[1]), want)
    b.close()
    for r in runs:
        r.close()


def test_mixed_batch_equals_alone(cpic):
    """A batch whose 2D cylinder members share the persistent particle launch while a 3D
    sphere, a magnetised 2D run and an axisymmetric floating-sphere run with the cyclotronic
    push (which cannot join it) push in their own branches: every member ends bit-identical
    to the same run stepped alone (full cycles, across sorts)."""
    def makers():
        def sphere():
            w = wl.sphere(16, 12, 8, npart_per_species=4000, seed=44, inject=True)
            return cpic.run_from_workload(w, sort_interval=2)

        def magnetized():
            w = wl.cylinder(inject=True, **SPECS[1])
            w.B0 = (0.0, 0.0, 0.7)
            return cpic.run_from_workload(w, sort_interval=3)

        def axisym_floating():  # Test C's kind of run: rings, cyclotronic push, floating sphere
            w = wl.sphere_axisym(24, 24, npart_per_species=20_000, seed=45, dt=0.05)
            w.B0 = (0.0, 5.0, 0.0)
            w.gyro = "cyclotronic"
            run = cpic.run_from_workload(w, sort_interval=2)
            run.set_floating(0, 0.0)
            return run

        return [lambda: _make(cpic, SPECS[0]), sphere, magnetized, axisym_floating, lambda: _make(cpic, SPECS[2])]

    def state3(run):
        d = run.diag()
        parts = [np.sort(np.rec.fromarrays([c, *t, *v])) for c, t, v in (run.particles(s) for s in range(2))]
        return run.phi(), d, parts, [run.charge(s) for s in range(2)]

    alone = []
    for mk in makers():
        r = mk()
        r.initialize()
        r.step(5)
        alone.append(state3(r))
        r.close()
    runs = [mk() for mk in makers()]
    b = cpic.Batch(8)
    b.set_mode(cpic.CPIC_BATCH_PERSISTENT)
    for r in runs:
        r.initialize()
        b.add(r)
    b.step(5)
    b.synchronize()
    for r, ref in zip(runs, alone):
        got = state3(r)
        assert np.array_equal(got[0], ref[0])
        for k in ("step", "n", "absorbed", "injected", "W_E", "W_K", "mg_cycles", "object_potential", "object_charge"):
            assert got[1][k] == ref[1][k], k
        for x, y in zip(got[2] + got[3], ref[2] + ref[3]):
            assert np.array_equal(x, y)
    b.close()
    for r in runs:
        r.close()
