"""Checkpoint/restore and the autotuner: a restored run continues the saved one exactly;
autotuning leaves the simulation unchanged (its trial steps are undone) and sets one of its
candidate sort intervals, chunk sizes and deposit paths; the push knobs change no result."""
import os

import numpy as np
import pytest

from paper_1311_2286_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _records(cell, t, v):
    return np.sort(np.rec.fromarrays([cell] + [t[a] for a in range(t.shape[0])] + [v[0], v[1], v[2]]))


def _state(run, nsp):
    d = run.diag()
    out = [run.phi(), {k: np.asarray(v) for k, v in d.items()}]
    for s in range(nsp):
        out.append(_records(*run.particles(s)))
        out.append(run.charge(s))
    return out


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    for k in a[1]:
        assert np.array_equal(a[1][k], b[1][k]), k
    for x, y in zip(a[2:], b[2:]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("case", ["cylinder", "sphere3d", "axisym_floating_cyclotronic"])
def test_checkpoint_restore_continues_exactly(cpic, tmp_path, case):
    """A restored run continues bit for bit: the 2D cylinder, the 3D sphere, and an
    axisymmetric floating sphere with a field along the axis, the cyclotronic push and the
    Galerkin / operator-induced / line-relaxation multigrid (every setting the file keeps)."""
    if case == "cylinder":
        w = wl.cylinder(n1=32, n2=64, npart_per_species=20_000, seed=61, inject=True)
    elif case == "sphere3d":
        w = wl.sphere(16, 16, 16, npart_per_species=20_000, seed=62)
    else:
        w = wl.sphere_axisym(24, 24, npart_per_species=20_000, seed=63, dt=0.05)
        w.B0 = (0.0, 5.0, 0.0)
        w.gyro = "cyclotronic"
    a = cpic.run_from_workload(w, sort_interval=3)
    if case == "axisym_floating_cyclotronic":
        a.set_multigrid("galerkin", "line", "operator")
        a.set_floating(0, 0.0)
    a.initialize()
    a.step(5)
    path = os.path.join(tmp_path, "run.ckpt")
    a.checkpoint(path)
    a.step(7)
    want = _state(a, len(w.species))
    a.close()
    b = cpic.Run.restore(path)
    b.step(7)
    _same(_state(b, len(w.species)), want)
    b.close()


def test_restore_rejects_foreign_file(cpic, tmp_path):
    path = os.path.join(tmp_path, "junk.ckpt")
    with open(path, "wb") as f:
        f.write(b"not a checkpoint" * 10)
    with pytest.raises(cpic.CpicError) as e:
        cpic.Run.restore(path)
    assert e.value.status == cpic.CPIC_ERR_INVALID


def test_autotune_leaves_the_run_unchanged(cpic):
    w = wl.cylinder(n1=32, n2=64, npart_per_species=40_000, seed=63, inject=True)
    a = cpic.run_from_workload(w, sort_interval=4)
    a.initialize()
    a.step(3)
    t = a.autotune(trial_steps=6)
    assert t["sort_interval"] in (1, 2, 4, 8, 16)
    assert all(ms > 0 for ms in t["ms_per_step"])
    assert t["chunk"] in t["chunks"] and t["chunks"] == [0, 1024, 2048, 4096, 8192]
    assert all(ms > 0 for ms in t["ms_chunk"]) and all(ms > 0 for ms in t["ms_tile"])
    assert t["tile"] in (0, 1)
    a.step(6)
    got = _state(a, 2)
    chosen = t["sort_interval"]
    a.close()
    # the same run without autotuning, stepped with the interval it chose (the push knobs
    # change no result: the deposit is integer and the per-particle arithmetic is the same)
    c = cpic.run_from_workload(w, sort_interval=4)
    c.initialize()
    c.step(3)
    c.set_sort_interval(chosen)
    c.step(6)
    _same(got, _state(c, 2))
    c.close()


@pytest.mark.parametrize("chunk,tile", [(0, 0), (1024, 1), (256, 1), (8192, 0)])
def test_push_tuning_changes_no_result(cpic, chunk, tile):
    """Any chunk size and either deposit path give the same particles, charge and counters
    as the defaults (one wave of blocks, tiled deposit), in 2D and 3D."""
    outs = []
    for knobs in (None, (chunk, tile)):
        w = wl.cylinder(n1=32, n2=64, npart_per_species=40_000, seed=64, inject=True)
        r = cpic.run_from_workload(w, sort_interval=2)
        r.initialize()
        if knobs:
            r.set_push_tuning(*knobs)
        r.step(5)
        outs.append(_state(r, 2))
        r.close()
    _same(outs[0], outs[1])
    outs = []
    for knobs in (None, (chunk, tile)):
        r = cpic.sphere_run_device(16, 16, 16, 20_000, sort_interval=2)
        if knobs:
            r.set_push_tuning(*knobs)
        r.step_particles(4)
        outs.append(([r.particles(s) for s in range(2)], [r.charge(s) for s in range(2)], r.diag()))
        r.close()
    (pa, ca, da), (pb, cb, db) = outs
    for s in range(2):
        ra = np.sort(np.rec.fromarrays([pa[s][0], *pa[s][1], *pa[s][2]]))
        rb = np.sort(np.rec.fromarrays([pb[s][0], *pb[s][1], *pb[s][2]]))
        assert np.array_equal(ra, rb)
        assert np.array_equal(ca[s], cb[s])
    for key in ("n", "absorbed", "W_K"):
        assert da[key] == db[key], key


@pytest.mark.parametrize("interval", [1, 2, 3])
def test_fused_sort_order_matches_gathered_sort(cpic, tmp_path, interval):
    """The sort that leaves its gather to the next direct 3D push (and takes its histogram
    from that step's push and injection) against the sort with its own histogram and gather
    (the tiled push): the same particles (as sets), charge, counters and potential after
    each stretch, with reads, a checkpoint, an explicit sort and a change of push kernel in
    between, several of them while an order is pending, and a restored run continuing."""
    def run_for(tile):
        r = cpic.sphere_run_device(16, 12, 8, 20_000, sort_interval=interval, inject=True)
        r.set_push_tuning(0, tile)
        states = []
        r.step(3)
        states.append(_state(r, 2))
        r.step_particles(interval)  # ends with a sort: with tile 0 its order is pending now
        states.append(_state(r, 2))
        path = str(tmp_path / ("run%d.ck" % tile))
        r.checkpoint(path)
        r.step(interval)
        r.sort()
        r.step(2)
        states.append(_state(r, 2))
        r.set_push_tuning(0, 1 - tile)  # the other push kernel from here on
        r.step(interval + 1)
        states.append(_state(r, 2))
        r.close()
        c = cpic.Run.restore(path)
        c.step(interval + 2)
        states.append(_state(c, 2))
        c.close()
        return states

    for x, y in zip(run_for(0), run_for(1)):
        _same(x, y)
