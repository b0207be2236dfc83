"""Whole PIC cycles on the device (cpic_step: vertex field, push + deposit, injection, sort,
charge -> RHS, multigrid solve, diagnostics) against the oracle's cycle (oracle/pic.py,
FP64 mover, exact b2 deposit, direct solve), run from the same particles.

What is compared (run-level tolerances for the Sec. II four-step cycle and the charging
runs of Sec. III.A-B):
  * the start-up half kick (v^{-1/2}) and the state after one step: <= 1e-5 normwise
    (global xi and v) against FP64;
  * the device's field energy at every step against 1/2 sum_c phi_c Q_c evaluated here in
    FP64 from the device's own potential and charge (FP64 rounding of the same sum);
  * the time-averaged field energy of the run within 1% of the oracle's, and the collected
    current (macro-particles absorbed at the object and at the outer boundary, per species)
    within 1% where the counts allow it: the two runs start from the same particles and
    inject the same Maxwellian draws, so their counts are correlated; the Poisson sigma of
    each count is reported beside the difference, and the tolerance is
    max(1%, 3 sigma of the difference of two independent counts) only where the count is
    too small for 1% to be resolved at all (fewer than 10^5 events: sigma > 0.3%).
The same cylinder run is then stepped inside a batch (next to other runs) and through the
server (continuous batching): both must equal the stand-alone device run bit for bit, so the
batched and served forms meet the same tolerances against the oracle.
"""
import math
import os

import numpy as np
import pytest

from oracle import poisson
from oracle.pic import OraclePIC
from paper_1311_2286_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

THREADS = max(1, len(os.sched_getaffinity(0)))


def _unpack(cell, D):
    return wl.unpack_cells(cell, D)


def _state_error(run, pic, w):
    """max normwise error of the device's global positions and velocities against the
    oracle's, species by species (same particle order: no sort, no removal yet)."""
    ex, ev = 0.0, 0.0
    for s, sp in enumerate(pic.species):
        cell, t, v = run.particles(s)
        assert cell.shape[0] == sp.idx.shape[1]
        u32 = (_unpack(cell, w.dim) + t.astype(np.float64)) / np.array(w.n)[:, None]
        u64 = (sp.idx + sp.t) / np.array(w.n)[:, None]
        du = np.abs(u32 - u64)
        for a in range(w.dim):
            if w.particle_bc[2 * a] == wl.PBC_PERIODIC:
                du[a] = np.minimum(du[a], 1.0 - du[a])
        ex = max(ex, float(np.max(du) / np.max(np.abs(u64))))
        ev = max(ev, float(np.max(np.abs(v.astype(np.float64) - sp.v)) / np.max(np.abs(sp.v))))
    return ex, ev


def _field_energy_from_device(run, w, geom):
    """1/2 sum_c phi_c Q_c in FP64 from the device's potential and fixed-point charge."""
    C = [run.charge(s) for s in range(len(w.species))]
    Q = poisson.charge_in_cells(geom, C, [sp.q * sp.w for sp in w.species], w.background)
    return 0.5 * float(np.sum(run.phi() * Q))


def _run_pair(cpic, w, steps, sort_interval, run=None, floating=None, trace=None):
    """Device and oracle runs of the same workload; returns per-level field energies and
    cumulative absorbed counts of both, and the one-step errors. floating: (face, charge0)
    of a floating conductor on both sides; trace: a list that receives, per level, the
    device's and the oracle's conductor potential."""
    if run is None:
        run = cpic.run_from_workload(w, sort_interval=sort_interval, mg_rtol=1e-12, mg_max_cycles=200)
    pic = OraclePIC(w, "fp64", engine="c", threads=THREADS)
    if floating is not None:
        run.set_floating(*floating)
        pic.set_floating(*floating)
    run.initialize()
    pic.initialize()
    if trace is not None:
        trace.append((run.diag()["object_potential"], pic.object_potential))
    err0 = _state_error(run, pic, w)
    dev_we, dev_we_check, dev_abs = [run.diag()["W_E"]], [_field_energy_from_device(run, w, pic.geom)], []
    err1 = None
    for k in range(steps):
        run.step(1)
        pic.step()
        if k == 0 and sort_interval != 1:
            err1 = _state_error(run, pic, w) if not w.injection else None
        d = run.diag()
        dev_we.append(d["W_E"])
        dev_we_check.append(_field_energy_from_device(run, w, pic.geom))
        dev_abs.append(d["absorbed"])
        if trace is not None:
            trace.append((d["object_potential"], pic.object_potential))
    ora_we = [h["W_E"] for h in pic.history] + [0.5 * float(np.sum(pic.phi * pic.Q))]
    ora_abs = [h["absorbed"] for h in pic.history]
    return run, pic, err0, err1, np.array(dev_we), np.array(dev_we_check), np.array(ora_we), dev_abs, ora_abs


def _current_check(dev_abs, ora_abs, w, first, last, report):
    """Counts absorbed between steps first and last per species and face (object = face 0,
    outer = face 1): relative difference and the Poisson sigma of the difference of two
    independent counts of that size."""
    worst = 0.0
    for s in range(len(w.species)):
        for f in (0, 1):
            nd = int(dev_abs[last - 1][s][f]) - int(dev_abs[first - 1][s][f])
            no = int(ora_abs[last - 1][s][f]) - int(ora_abs[first - 1][s][f])
            if no == 0 and nd == 0:
                continue
            rel = abs(nd - no) / max(no, 1)
            sig = math.sqrt(2.0 / max(no, 1))
            report.append({"species": s, "face": f, "device": nd, "oracle": no, "rel_diff": rel, "sigma": sig})
            tol = 0.01 if no >= 100_000 else max(0.01, 3.0 * sig)
            assert rel <= tol, report[-1]
            worst = max(worst, rel)
    return worst


def test_langmuir_cycle_matches_oracle(cpic):
    """The doubly periodic Langmuir configuration at full size (map2 32 x 32, eps 0.05,
    64 electrons per cell, 1% density perturbation, v_th 0.05, dt 0.1, 100 steps, seed 0):
    start-up and one-step state <= 1e-5 against FP64, W_E at every level equal to
    1/2 sum phi Q of the device's own fields, time-averaged W_E and W_K within 1% of the
    oracle's."""
    w = wl.langmuir_map2(32, 32, eps=0.05, ppc=64, vth=0.05, amp=0.01, dt=0.1, seed=0)
    run, pic, err0, err1, we, we_chk, we_ora, _, _ = _run_pair(cpic, w, 100, 0)
    assert err0[0] <= 1e-5 and err0[1] <= 1e-5, err0
    assert err1[0] <= 1e-5 and err1[1] <= 1e-5, err1
    np.testing.assert_allclose(we, we_chk, rtol=1e-12)
    assert abs(we.mean() / we_ora.mean() - 1.0) <= 0.01, (we.mean(), we_ora.mean())
    print("langmuir cycle: errors start-up %s step 1 %s; W_E mean device %.6e oracle %.6e"
          % (err0, err1, we.mean(), we_ora.mean()))
    wk_dev = np.array([run.diag()["W_K"]])
    assert abs(wk_dev[0] / pic.history[-1]["W_K"] - 1.0) <= 0.01
    run.close()


CYL = dict(n1=48, n2=96, r0=1.0, R=10.0, npart_per_species=150_000, phi_obj=-5.0, seed=41, inject=True)
CYL_STEPS = 300


def test_cylinder_cycle_matches_oracle(cpic, record_property):
    """A reduced cylinder-in-plasma run (annulus r = 10^xi, 48 x 96 cells, 150k + 150k
    particles, object at -5, Maxwellian flux injection of both species at r = 10, sort every
    4 steps, 300 steps): W_E at every level equal to 1/2 sum phi Q of the device's fields;
    time-averaged W_E within 1% of the oracle's; collected currents (object and outer
    boundary, both species) within 1% where the counts resolve 1% (sigma reported)."""
    w = wl.cylinder(**CYL)
    run, pic, err0, _, we, we_chk, we_ora, dev_abs, ora_abs = _run_pair(cpic, w, CYL_STEPS, 4)
    assert err0[0] <= 1e-5 and err0[1] <= 1e-5, err0
    np.testing.assert_allclose(we, we_chk, rtol=1e-12)
    assert abs(we.mean() / we_ora.mean() - 1.0) <= 0.01, (we.mean(), we_ora.mean())
    report = []
    _current_check(dev_abs, ora_abs, w, 1, CYL_STEPS, report)
    record_property("currents", report)
    print("cylinder cycle: W_E mean device %.6e oracle %.6e" % (we.mean(), we_ora.mean()))
    for r in report:
        print("cylinder cycle current:", r)
    assert any(r["species"] == 1 and r["face"] == 0 and r["device"] > 0 for r in report)  # ions collected
    run.close()


def test_floating_cylinder_matches_oracle(cpic):
    """Row f1: the reduced cylinder run with the object as a floating conductor (uncharged
    at start; Gauss's-law potential from the charge it collects, Sec. III.A-B) on the
    device and in the oracle: the conductor potential agrees at every level (to 1e-3 of its
    range), its time average within 1%, the object charges negative (electrons are
    collected faster than ions), and the device's field energy is 1/2 sum phi Q of its own
    fields."""
    w = wl.cylinder(**CYL)
    trace = []
    run, pic, err0, _, we, we_chk, we_ora, dev_abs, ora_abs = _run_pair(cpic, w, CYL_STEPS, 4, floating=(0, 0.0),
                                                                         trace=trace)
    v = np.array(trace)
    scale = np.max(np.abs(v[:, 1]))
    assert np.max(np.abs(v[:, 0] - v[:, 1])) <= 1e-3 * scale, np.max(np.abs(v[:, 0] - v[:, 1]))
    assert abs(v[:, 0].mean() / v[:, 1].mean() - 1.0) <= 0.01
    assert v[-1, 1] < -0.5 and run.diag()["object_charge"] < 0.0
    np.testing.assert_allclose(we, we_chk, rtol=1e-12)
    print("floating cylinder: V(end) device %.6f oracle %.6f, mean %.6f / %.6f, max |dV| %.2e"
          % (v[-1, 0], v[-1, 1], v[:, 0].mean(), v[:, 1].mean(), np.max(np.abs(v[:, 0] - v[:, 1]))))
    run.close()


SPH = dict(n1=48, n2=48, npart_per_species=150_000, seed=43, dt=0.1)
SPH_STEPS = 300


@pytest.mark.parametrize("Bz", [0.0, 19.0])
def test_sphere_axisym_cycle_matches_oracle(cpic, record_property, Bz):
    """Row f3: a reduced Test B run (the sphere r1 = 1 in r2 = 10 on the 2D axisymmetric
    (r, z) map, Omega = r, 48 x 48 cells, 150k + 150k rings, the sphere floating from zero
    charge, Maxwellian flux injection at r2, specular z axis, dt 0.1, sort every 4 steps,
    300 steps) on the device and in the oracle: start-up and first-step state <= 1e-5
    against FP64; W_E at every level equal to 1/2 sum phi Q of the device's fields; the
    sphere potential at every level within 1e-3 of its range, its time average within 1%;
    time-averaged W_E within 1%; collected currents within 1% where the counts resolve it.
    With B_z = 19 along the axis (Test C's moderately magnetised field) both sides push
    with the cyclotronic integrator at dt 0.05 (w_ce dt = 0.95)."""
    w = wl.sphere_axisym(**SPH) if Bz == 0.0 else wl.sphere_axisym(**dict(SPH, dt=0.05))
    if Bz:
        w.B0 = (0.0, Bz, 0.0)
        w.gyro = "cyclotronic"
    trace = []
    run, pic, err0, _, we, we_chk, we_ora, dev_abs, ora_abs = _run_pair(cpic, w, SPH_STEPS, 4, floating=(0, 0.0),
                                                                         trace=trace)
    assert err0[0] <= 1e-5 and err0[1] <= 1e-5, err0
    np.testing.assert_allclose(we, we_chk, rtol=1e-12)
    v = np.array(trace)
    scale = np.max(np.abs(v[:, 1]))
    assert np.max(np.abs(v[:, 0] - v[:, 1])) <= 1e-3 * scale, np.max(np.abs(v[:, 0] - v[:, 1]))
    assert abs(v[:, 0].mean() / v[:, 1].mean() - 1.0) <= 0.01
    assert v[-1, 1] < -0.5
    assert abs(we.mean() / we_ora.mean() - 1.0) <= 0.01, (we.mean(), we_ora.mean())
    report = []
    _current_check(dev_abs, ora_abs, w, 1, SPH_STEPS, report)
    record_property("currents", report)
    # collection tally (Fig. 7's diagnostic): per sphere and outer-face cell
    for s in range(len(w.species)):
        for f in (0, 1):
            dev, ora = run.collection(s, f), pic.collect[s, f]
            assert np.abs(dev - ora).sum() <= max(2, 0.005 * ora.sum()), (s, f, dev, ora)
    print("axisymmetric sphere: V(end) device %.6f oracle %.6f, mean %.6f / %.6f, max |dV| %.2e; W_E mean %.6e / %.6e"
          % (v[-1, 0], v[-1, 1], v[:, 0].mean(), v[:, 1].mean(), np.max(np.abs(v[:, 0] - v[:, 1])), we.mean(),
             we_ora.mean()))
    for r in report:
        print("axisymmetric sphere current:", r)
    run.close()


def _polar_fraction(counts):
    """Fraction of the sphere's collection with |cos delta| > 0.8, cos delta = cos[pi (1 -
    eta)] at the face cell's centre (Fig. 7's axis); 0.2 for isotropic collection (the band
    |cos delta| > 0.8 holds a fifth of the sphere's area)."""
    n2 = counts.size
    cd = np.cos(np.pi * (1.0 - (np.arange(n2) + 0.5) / n2))
    tot = counts.sum()
    return float(counts[np.abs(cd) > 0.8].sum()) / max(tot, 1), int(tot)


def test_sphere_floating_potential_test_b(cpic):
    """Test B at the paper's size (Sec. III.B: 128 x 128, r1 = 1, r2 = 10, dt 0.1, plasma of
    density 1 and T_i = T_e, m_i/m_e = 1836, the sphere floating from zero charge, flux
    injection at r2), on the device alone with about 230 rings per cell per species: the
    sphere potential averaged over the last quarter of 4000 steps lies within 8% of the
    OML value -2.50 T_e that the paper's -2.54 is compared with (OML is approximate at
    r1 = lambda_D; the paper's own agreement is 1.6%), and both species are collected
    isotropically over the last tenth (Fig. 7: a fifth of the collection in |cos delta| >
    0.8). Physics, not parity: the parity of this path against the oracle is the test
    above."""
    n = 128
    w = wl.sphere_axisym(n, n, npart_per_species=230 * n * n, seed=8, dt=0.1, capacity_factor=1.6)
    run = cpic.run_from_workload(w, sort_interval=8)
    run.set_floating(0, 0.0)
    run.initialize()
    steps, vs = 4000, []
    for k in range(steps // 50):
        run.step(50)
        vs.append(run.diag()["object_potential"])
        if k == (steps * 9 // 10) // 50 - 1:
            c0 = [run.collection(s, 0) for s in range(2)]
    tail = float(np.mean(vs[-len(vs) // 4:]))
    print("Test B: sphere potential (last quarter of %d steps) %.4f T_e (OML -2.50, paper -2.54)" % (steps, tail))
    assert abs(tail / -2.50 - 1.0) <= 0.08, tail
    # Fig. 7, unmagnetised: both species are collected isotropically over the last tenth
    fr = [_polar_fraction(run.collection(s, 0) - c0[s]) for s in range(2)]
    print("Test B collection over the last tenth: |cos delta| > 0.8 fraction electrons %.3f (%d), ions %.3f (%d)"
          % (fr[0][0], fr[0][1], fr[1][0], fr[1][1]))
    for f, n in fr:
        assert abs(f - 0.2) <= 0.05 and n > 1000, fr
    run.close()


def test_planar_wall_potential_test_a(cpic):
    """Test A (Sec. III.A) at the paper's size: the 20 x 5 box on the uniform 128 x 128 map
    of eq. (map3), empty at start, the wall at xi = 0 floating from zero charge (Gauss's
    law), phi = 0 at xi = 1, eta periodic, electrons (at rest) and ions (T_i = T_e, m_i/m_e =
    1836, drifting at -2.1 v_thi toward the wall) injected at xi = 1 from unit density, dt
    0.05, 64 particles per cell per species at unit density, 24000 steps (the oracle's own
    runs of this box settle by about step 12000). The electrons reach the wall first: the
    early minimum of the wall potential lies within 10% of the paper's -5.7 T_e; the
    potential averaged over the last sixth lies within 4% of the paper's -2.11 T_e (its
    analytic steady state is -2.10), and the final potential is one-dimensional (its spread
    along eta is small next to the wall potential, and it is shielded within the box). Physics, not parity: the parity of this
    path is the drifting injection and floating-conductor tests."""
    w = wl.planar_wall(128, 128, ppc=64)
    run = cpic.run_from_workload(w, sort_interval=8)
    run.set_floating(0, 0.0)
    run.initialize()
    steps, vs = 24000, []
    for k in range(steps // 50):
        run.step(50)
        vs.append(run.diag()["object_potential"])
    vs = np.array(vs)
    tail = float(np.mean(vs[-len(vs) // 6:]))
    spike = float(vs.min())
    phi = run.phi()  # (eta, xi)
    spread = float(np.max(np.std(phi, axis=0)))
    print("Test A: wall potential, last sixth of %d steps %.4f T_e (paper -2.11, analytic -2.10); early minimum "
          "%.3f at step %d (paper -5.7); max spread along eta of the final phi %.4f"
          % (steps, tail, spike, (int(vs.argmin()) + 1) * 50, spread))
    assert abs(tail / -2.11 - 1.0) <= 0.04, tail
    assert abs(spike / -5.7 - 1.0) <= 0.10, spike
    assert spread <= 0.1 * abs(tail), spread
    # the wall is shielded: strongly negative next to it, near zero in the far half of the box
    prof = phi.mean(axis=0)
    assert prof[0] < 0.5 * tail and np.max(np.abs(prof[len(prof) // 2:])) < 0.2 * abs(tail), prof
    run.close()


def test_cylinder_cycle_same_in_batch_and_alone(cpic):
    """The reduced cylinder run stepped inside a batch, next to two other runs, ends in the
    same state as the stand-alone device run that test_cylinder_cycle_matches_oracle
    compares with the oracle (bit for bit: fields, counts, energies, particles as a set)."""
    steps = 60

    def final(run):
        d = run.diag()
        parts = [np.sort(np.rec.fromarrays([c, *t, *v])) for c, t, v in (run.particles(s) for s in range(2))]
        return run.phi(), [run.charge(s) for s in range(2)], d, parts

    alone = cpic.run_from_workload(wl.cylinder(**CYL), sort_interval=4, mg_rtol=1e-12, mg_max_cycles=200)
    alone.initialize()
    alone.step(steps)
    ref = final(alone)
    alone.close()
    import torch

    stream = torch.cuda.Stream()
    cs = __import__("ctypes").c_void_p(stream.cuda_stream)
    target = cpic.run_from_workload(wl.cylinder(**CYL), sort_interval=4, mg_rtol=1e-12, mg_max_cycles=200,
                                    stream=cs)
    target.initialize()
    others = [cpic.cylinder_run_device(32, 64, 40_000 + 1000 * i, -3.0 + i, 70 + i, stream=cs) for i in range(2)]
    batch = cpic.Batch(4, stream=cs)
    for r in [others[0], target, others[1]]:
        batch.add(r)
    batch.step(steps)
    batch.synchronize()
    got = final(target)
    batch.close()
    assert np.array_equal(got[0], ref[0])
    for s in range(2):
        assert np.array_equal(got[1][s], ref[1][s])
        assert np.array_equal(got[3][s], ref[3][s])
    for key in ("step", "n", "absorbed", "injected", "W_E", "W_K", "mg_cycles"):
        assert got[2][key] == ref[2][key], key
    for r in others + [target]:
        r.close()


def _request_run(cpic, req, sort_interval=4):
    """A stand-alone run set up exactly as the server sets up a cylinder request
    (cpic.run_for_request, before its start-up), and the workload the oracle runs from it:
    the particles the device loaded (read back), the same map, boundaries and injection."""
    run = cpic.run_for_request(req, sort_interval=sort_interval, start=False)
    w = wl.cylinder(n1=req.n[0], n2=req.n[1], r0=req.r_object, R=req.r_outer,
                    npart_per_species=req.particles_per_species, phi_obj=req.phi_object, seed=0,
                    mass_ratio=req.mass_ratio, dt=req.dt, inject=True, host_particles=False)
    vth = [math.sqrt(req.temperature), math.sqrt(req.temperature / req.mass_ratio)]
    w.particles = [wl.ParticleSet(*run.particles(s)) for s in range(2)]
    w.injection = [(s, 1, req.density, vth[s], req.seed * 1000 + 7 + s) for s in range(2)]
    return run, w


def test_served_request_matches_oracle(cpic):
    """A served cylinder request (continuous batching next to two other requests) gives the
    result of the same run stepped alone, and that run, started from the particles the
    device loaded for it, meets the cycle tolerances against the oracle: time-averaged W_E
    within 1%, collected currents within 1% where resolved (sigma reported)."""
    steps = 150
    req = cpic.make_request(n1=48, n2=96, particles_per_species=120_000, phi_object=-4.0, r_outer=10.0,
                            steps=steps, seed=77)
    sv = cpic.Server(hbm_budget=2 << 30, max_active=4, steps_per_slice=10)
    noise = [sv.submit(cpic.make_request(n1=32, n2=64, particles_per_species=30_000, steps=40, seed=80 + i))
             for i in range(2)]
    served = sv.wait(sv.submit(req))
    for tk in noise:
        assert sv.wait(tk)["status"] == 0
    sv.stop()
    assert served["status"] == 0 and served["steps"] == steps
    run, w = _request_run(cpic, req)
    run, pic, err0, _, we, we_chk, we_ora, dev_abs, ora_abs = _run_pair(cpic, w, steps, 4, run=run)
    d = run.diag()
    assert served["field_energy"] == d["W_E"] and served["kinetic_energy"] == d["W_K"]
    for s in range(2):
        assert served["absorbed_object"][s] == d["absorbed"][s][0]
        assert served["absorbed_outer"][s] == d["absorbed"][s][1]
        assert served["n_particles"][s] == d["n"][s] and served["injected"][s] == d["injected"][s]
    np.testing.assert_allclose(we, we_chk, rtol=1e-12)
    assert abs(we.mean() / we_ora.mean() - 1.0) <= 0.01, (we.mean(), we_ora.mean())
    report = []
    _current_check(dev_abs, ora_abs, w, 1, steps, report)
    print("served cycle: W_E mean device %.6e oracle %.6e" % (we.mean(), we_ora.mean()))
    for r in report:
        print("served cycle current:", r)
    run.close()


@pytest.mark.parametrize("gyro", ["boris", "cyclotronic"])
def test_magnetized_langmuir_cycle_matches_oracle(cpic, gyro):
    """Row f2 through whole cycles: the cold plasma wave across a uniform B_z = 1 (the
    upper-hybrid oscillation the oracle's pin checks) on the device (generic kernel, Boris
    kick and start-up, or the cyclotronic push and its plain start-up kick) against the
    oracle from the same particles: start-up and one-step state <= 1e-5 against FP64, W_E
    at every level 1/2 sum phi Q of the device's fields, time-averaged W_E within 1%."""
    w = wl.langmuir_map2(32, 32, eps=0.05, ppc=16, vth=0.0, amp=0.05, dt=0.1, seed=0)
    w.B0 = (0.0, 0.0, 1.0)
    w.gyro = gyro
    run = cpic.run_from_workload(w, sort_interval=0, mg_rtol=1e-12, mg_max_cycles=200)
    run, pic, err0, err1, we, we_chk, we_ora, _, _ = _run_pair(cpic, w, 100, 0, run=run)
    assert err0[0] <= 1e-5 and err0[1] <= 1e-5, err0
    assert err1[0] <= 1e-5 and err1[1] <= 1e-5, err1
    np.testing.assert_allclose(we, we_chk, rtol=1e-12)
    assert abs(we.mean() / we_ora.mean() - 1.0) <= 0.01, (we.mean(), we_ora.mean())
    print("magnetized langmuir (%s): W_E mean device %.6e oracle %.6e" % (gyro, we.mean(), we_ora.mean()))
    run.close()


@pytest.mark.parametrize("Bz,expected", [(1.9, -2.51), (19.0, -2.43)])
def test_sphere_floating_potential_test_c(cpic, Bz, expected):
    """Test C (Sec. III.C): the sphere of Test B in a uniform field along the axis, B_z0 =
    1.9 (electron gyroradius 0.53, weakly magnetised) and 19 (0.053, moderately
    magnetised; w_ce dt = 0.95, which the cyclotronic integrator resolves), 128 x 128,
    dt 0.05, on the device with the cyclotronic push over 8000 steps (the physical time of
    Test B's 4000). The paper's own values for these runs are -2.51 T_e and -2.43 T_e
    (averaged over the last sixth), and it finds them within about 10% of another code's
    -2.37 and -2.21; the sphere potential averaged over the last sixth here lies within
    10% of the paper's values (and the potential is less negative in the stronger field).
    The collection over the last tenth (Fig. 7) is isotropic for the ions in both fields
    and for the electrons in the weak one, and peaks at the poles for the electrons in the
    moderate one. Physics, not parity: the parity of this path is the cyclotronic push and
    cycle tests."""
    n = 128
    w = wl.sphere_axisym(n, n, npart_per_species=230 * n * n, seed=9, dt=0.05, capacity_factor=1.6)
    w.B0 = (0.0, Bz, 0.0)
    w.gyro = "cyclotronic"
    run = cpic.run_from_workload(w, sort_interval=8)
    run.set_floating(0, 0.0)
    run.initialize()
    steps, vs = 8000, []
    for k in range(steps // 50):
        run.step(50)
        vs.append(run.diag()["object_potential"])
        if k == (steps * 9 // 10) // 50 - 1:
            c0 = [run.collection(s, 0) for s in range(2)]
    tail = float(np.mean(vs[-len(vs) // 6:]))
    fr = [_polar_fraction(run.collection(s, 0) - c0[s]) for s in range(2)]
    print("Test C (B_z0 %.1f) collection over the last tenth: |cos delta| > 0.8 fraction electrons %.3f (%d), "
          "ions %.3f (%d)" % (Bz, fr[0][0], fr[0][1], fr[1][0], fr[1][1]))
    # Fig. 7: the ions (gyroradius above the sphere's radius) are collected isotropically in
    # both fields, the electrons too in the weak field, while in the moderate field (electron
    # gyroradius 0.05 r1) they reach the sphere mostly along the field, near the poles
    assert abs(fr[1][0] - 0.2) <= 0.05, fr
    if Bz < 5.0:
        assert abs(fr[0][0] - 0.2) <= 0.05, fr
    else:
        assert fr[0][0] >= 0.27, fr
    print("Test C (B_z0 %.1f): sphere potential (last sixth of %d steps) %.4f T_e (paper %.2f)"
          % (Bz, steps, tail, expected))
    assert abs(tail / expected - 1.0) <= 0.10, tail
    run.close()


def test_landau_damping_rate(cpic):
    """Landau damping (the paper's validation tests include it, Sec. III): a 5% density
    perturbation with k lambda_D = 0.5 (wavelength the unit box, vth = 0.5 / 2 pi) on the
    distorted map2 grid (eps 0.05), 64 x 64 cells, 1024 electrons per cell, dt 0.05, 400 full
    cycles on the device. The field energy oscillates at 2 omega and decays as exp(2 gamma
    t); the linear theory of a Maxwellian plasma gives omega = 1.4156, gamma = -0.1533 (in
    omega_pe) at k lambda_D = 0.5. Peaks of W_E fitted between t = 4 (after the initial
    transient) and t = 12 (before the thermal noise floor): omega within 3%, gamma within
    10%."""
    w = wl.langmuir_map2(64, 64, eps=0.05, ppc=1024, vth=0.5 / (2.0 * math.pi), amp=0.05, dt=0.05, seed=7)
    run = cpic.run_from_workload(w, sort_interval=4, mg_rtol=1e-10, mg_max_cycles=100)
    run.initialize()
    we = [run.diag()["W_E"]]
    for _ in range(400):
        run.step(1)
        we.append(run.diag()["W_E"])
    run.close()
    we = np.array(we)
    t = np.arange(we.size) * w.dt
    pk = [i for i in range(1, we.size - 1) if we[i] > we[i - 1] and we[i] >= we[i + 1]]
    tp, wp = t[pk], we[pk]
    lin = (tp > 4.0) & (tp < 12.0)
    slope, _ = np.polyfit(tp[lin], np.log(wp[lin]), 1)
    gamma = 0.5 * slope
    omega = math.pi / np.mean(np.diff(tp[lin]))
    print("Landau damping k lambda_D = 0.5: omega %.4f (theory 1.4156), gamma %.4f (theory -0.1533), %d peaks"
          % (omega, gamma, int(lin.sum())))
    assert abs(omega / 1.4156 - 1.0) <= 0.03, omega
    assert abs(gamma / -0.1533 - 1.0) <= 0.10, gamma


def test_two_stream_growth_rate(cpic):
    """Two-stream instability (the paper's validation tests include it, Sec. III): two cold
    electron beams at +-v0 with k v0 = 0.612 omega_pe for the box's mode (k = 2 pi), where
    the cold two-beam dispersion relation 1 = (1/2)[1/(w - kv0)^2 + 1/(w + kv0)^2] has its
    largest growth rate gamma = omega_pe / (2 sqrt 2) = 0.3536; distorted map2 grid (eps
    0.05), 64 x 64 cells, 256 electrons per cell, dt 0.05, on the device. The field energy
    grows as exp(2 gamma t) from the seeded perturbation until the beams trap (the seed
    also excites the stable roots, which beat with the growing one early on); fitted over
    W_E between 1% and 20% of its saturation maximum: gamma within 10%."""
    w = wl.two_stream_map2(64, 64, eps=0.05, ppc=256, v0=0.612 / (2.0 * math.pi), vth=0.002, amp=1e-3, dt=0.05,
                           seed=8)
    run = cpic.run_from_workload(w, sort_interval=4, mg_rtol=1e-10, mg_max_cycles=100)
    run.initialize()
    we = [run.diag()["W_E"]]
    for _ in range(500):
        run.step(1)
        we.append(run.diag()["W_E"])
    run.close()
    we = np.array(we)
    t = np.arange(we.size) * w.dt
    top = int(np.argmax(we))
    # the last stretch before the maximum with W_E between 1% and 20% of it
    stop = top
    while stop > 0 and we[stop - 1] > 0.2 * we[top]:
        stop -= 1
    first = stop
    while first > 0 and we[first - 1] > 0.01 * we[top]:
        first -= 1
    sel = np.zeros(we.size, bool)
    sel[first:stop] = True
    slope, _ = np.polyfit(t[sel], np.log(we[sel]), 1)
    gamma = 0.5 * slope
    print("two-stream: growth rate %.4f (theory 0.3536) over t = %.2f .. %.2f, W_E %.2e -> %.2e"
          % (gamma, t[sel][0], t[sel][-1], we[0], we.max()))
    assert sel.sum() >= 20
    assert abs(gamma / 0.3536 - 1.0) <= 0.10, gamma
