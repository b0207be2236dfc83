"""Whole-loop pins of the oracle: Langmuir oscillation (P8), energy and charge, injection."""
import math

import numpy as np
import pytest

from oracle import inject, philox
from oracle.pic import OraclePIC
from paper_1311_2286_gb300 import workloads as wl


def _mode_amplitude(pic, eps):
    """sum_p cos(2 pi x_p) over electrons, x_p the physical x of the particle (exact map2)."""
    sp = pic.species[0]
    n1, n2 = pic.n
    xi = (sp.idx[0] + sp.t[0].astype(np.float64)) / n1
    eta = (sp.idx[1] + sp.t[1].astype(np.float64)) / n2
    x = xi + eps * np.sin(2 * np.pi * xi) * np.sin(2 * np.pi * eta)
    return float(np.sum(np.cos(2 * np.pi * x)))


def _run(eps, ppc, vth, amp, steps, precision="fp64", seed=0):
    w = wl.langmuir_map2(32, 32, eps=eps, ppc=ppc, vth=vth, amp=amp, dt=0.1, seed=seed)
    pic = OraclePIC(w, precision)
    pic.initialize()
    amps = [_mode_amplitude(pic, eps)]
    for _ in range(steps):
        pic.step()
        amps.append(_mode_amplitude(pic, eps))
    return pic, np.array(amps)


def _frequency(sig, dt):
    """Frequency of a (nearly) sinusoidal signal from a least-squares fit of
    a cos(w t) + b sin(w t) + c over a grid of w, refined by parabolic interpolation."""
    t = np.arange(sig.size) * dt
    ws = np.linspace(0.5, 2.0, 3001)
    res = []
    for w in ws:
        A = np.stack([np.cos(w * t), np.sin(w * t), np.ones_like(t)], 1)
        coef, r, *_ = np.linalg.lstsq(A, sig, rcond=None)
        res.append(np.sum((A @ coef - sig) ** 2))
    res = np.array(res)
    i = int(np.argmin(res))
    y0, y1, y2 = res[i - 1], res[i], res[i + 1]
    off = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return ws[i] + off * (ws[1] - ws[0])


@pytest.mark.slow
def test_langmuir_cold_frequency_and_energy():
    """P8 (cold): a cold electron plasma oscillates at the leapfrog-modified plasma
    frequency (2/dt) asin(omega_pe dt/2) = 1.0004 omega_pe (within 1%), on the distorted
    map2 grid. Total energy W_E + W_K stays within 2% over 100 steps: the staggered b2/b1
    pair is exactly energy conserving only in 1D (Sec. II.B cites the 1D definition); in 2D
    the deviation measured here is 1.1% and does not change when dt is halved."""
    pic, amps = _run(0.05, 16, 0.0, 0.05, 100)
    w = _frequency(amps - amps.mean(), 0.1)
    target = 2 / 0.1 * math.asin(0.05)
    assert abs(w - target) / target < 0.01, w
    tot = np.array([h["W_E"] + h["W_K"] for h in pic.history])
    assert np.max(np.abs(tot - tot[0])) / abs(tot[0]) < 0.02


@pytest.mark.slow
def test_langmuir_warm_bohm_gross():
    """P8 (warm, v_th = 0.05 so k lambda_D = 0.314): the mode oscillates near the
    Bohm-Gross frequency sqrt(1 + 3 k^2 lambda_D^2) = 1.139 (kinetic value ~1.16); the
    +/- perturbation difference cancels the particle noise."""
    _, ap = _run(0.05, 32, 0.05, 0.05, 100, seed=3)
    _, am = _run(0.05, 32, 0.05, -0.05, 100, seed=3)
    w = _frequency(ap - am, 0.1)
    assert 1.10 < w < 1.20, w


def test_charge_conservation_every_step_fp32_path():
    """P5 along a run: with periodic boundaries the fixed-point charge is exactly
    N 2^24 per species at every step (fp32 path: spec R replay + spec Q)."""
    w = wl.langmuir_map2(16, 16, eps=0.05, ppc=8, vth=0.05, amp=0.01, dt=0.1, seed=2)
    pic = OraclePIC(w, "fp32")
    pic.initialize()
    from oracle import deposit as dep

    for _ in range(5):
        pic.step()
        sp = pic.species[0]
        C = dep.deposit_fixed(sp.idx, sp.t, pic.n, pic.periodic)
        assert int(C.sum()) == sp.idx.shape[1] << dep.QF


# ------------------------------------------------------------------ Philox and injection

def test_philox_known_answer_vectors():
    """Philox4x32-10 reproduces the generator's published known-answer vectors (golden file,
    cited there): a swapped word, a wrong multiplier or key schedule fails this."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(np.array([v[0:4]], np.uint32), np.array([v[4:6]], np.uint32))
        assert [int(x) for x in out[0]] == v[6:10]


def test_thermal_flux_rate_by_brute_force_crossing_count():
    """Spec I's injection rate n vth / sqrt(2 pi) A dt / w is the one-sided Maxwellian flux:
    brute force on a box of uniform Maxwellian plasma (density n, thermal speed vth) next
    to a plane: the macro-particles that cross the plane within dt (x + vx dt > 0 from
    x < 0) number rate_per_step within 4 sigma of Poisson counting; a wrong constant (1/2,
    1/sqrt(pi), 1/4 of the mean speed's flux ...) differs by more than 10%."""
    rng = np.random.default_rng(21)
    vth, dt, dens, A = 1.7, 0.05, 3.0, 2.5
    L = 8.0 * vth * dt  # deeper than any particle can travel in dt (8 sigma)
    npart = 4_000_000
    w = dens * L * A / npart  # physical particles per macro-particle
    crossed = 0
    for _ in range(4):
        x = -L * rng.random(npart)
        vx = vth * rng.standard_normal(npart)
        crossed += int(np.sum(x + vx * dt > 0.0))
    expected = 4 * inject.rate_per_step(dens, vth, A, dt, w)
    assert abs(crossed - expected) < 4.0 * math.sqrt(expected), (crossed, expected)
    assert expected > 1e5


def test_philox_uniformity_and_stream_independence():
    """Statistical pins of the counter-based generator: uniform (chi^2 over 64 bins),
    distinct keys and counters give uncorrelated streams."""
    n = 200000
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    key = np.zeros((n, 2), np.uint32)
    out = philox.philox4x32_10(ctr, key)
    u = philox.uniform01(out)
    assert u.min() > 0 and u.max() < 1
    h, _ = np.histogram(u[:, 0], bins=64, range=(0, 1))
    chi2 = np.sum((h - n / 64) ** 2 / (n / 64))
    assert chi2 < 120  # 63 dof; p ~ 1e-5
    key2 = key.copy()
    key2[:, 0] = 1
    u2 = philox.uniform01(philox.philox4x32_10(ctr, key2))
    assert abs(np.corrcoef(u[:, 0], u2[:, 0])[0, 1]) < 0.01
    assert abs(np.corrcoef(u[:-1, 1], u[1:, 1])[0, 1]) < 0.01
    # all four words are used and distinct
    assert len(np.unique(out[:1000].ravel())) == 4000


def test_injection_counts_and_flux_statistics():
    """Spec I: deterministic count sequence floor((n+1) r) - floor(n r); the normal speed
    of injected particles is flux-weighted (Rayleigh, mean vth sqrt(pi/2)), tangential
    components are Gaussian with std vth, positions are uniform along the face."""
    n1, n2 = 16, 64
    X = wl.annulus_vertices(n1, n2, 1.0, 40.0)
    from oracle.geometry import build_geometry

    g = build_geometry(X, [False, True])
    area = inject.face_length_2d(X, 1)
    assert abs(area - 2 * 40.0 * n2 * math.sin(math.pi / n2)) < 1e-9
    r = inject.rate_per_step(1.0, 1.0, area, 0.1, 0.01)
    counts = [inject.count_at_step(r, s) for s in range(100)]
    assert sum(counts) == math.floor(100 * r)
    idx, t32, v32, keep = inject.inject_2d(g.k, (n1, n2), 1, 40000, 0, 0, 1234, 1.0, (0, 0, 0), 1e-3)
    # a particle whose partial push ends within FP32 rounding of the face is dropped
    assert keep.mean() > 0.999
    # radial unit vector at the particle's angle (outer face, theta = 2 pi eta)
    th = 2 * np.pi * (idx[1] + t32[1].astype(np.float64)) / n2
    vr = v32[0] * np.cos(th) + v32[1] * np.sin(th)
    vt = -v32[0] * np.sin(th) + v32[1] * np.cos(th)
    vn = -vr
    assert np.all(vn > 0)
    assert abs(vn.mean() - math.sqrt(math.pi / 2)) < 0.02
    assert abs(vt.std() - 1.0) < 0.02 and abs(v32[2].std() - 1.0) < 0.02
    assert np.all(idx[0] == n1 - 1)
    hist, _ = np.histogram(idx[1], bins=n2, range=(0, n2))
    assert np.sum((hist - 40000 / n2) ** 2 / (40000 / n2)) < 120


def test_inject_3d_flux_statistics():
    """Spec I in 3D on the shell's outer face: positions uniform in physical area (face-cell
    counts follow the face-cell areas, which go as sin theta), the normal speed is
    Rayleigh (flux-weighted Maxwellian), the tangential components are Gaussian, velocities
    point inward, and the face area tends to the sphere's 4 pi R^2 cos(theta_c)."""
    import math

    from oracle import geometry, inject
    from paper_1311_2286_gb300 import workloads as wl

    n = (8, 16, 24)
    w = wl.sphere(*n, npart_per_species=10, seed=1)
    g = geometry.build_geometry(w.vertices, [False, False, True])
    area = inject.face_area_3d(w.vertices, 1)
    exact = 4 * math.pi * 30.0**2 * math.cos(math.pi / 32)
    assert abs(area / exact - 1) < 0.01  # chord-polygon faces under-estimate by O(h^2)
    cnt, vth = 200_000, 1.3
    idx, t32, v32, keep = inject.inject_3d(w.vertices, g.k, n, 1, cnt, 0, 0, 77, vth, (0, 0, 0), 1e-2)
    assert keep.mean() > 0.999
    areas = inject.face_areas_3d(w.vertices, 1)
    counts = np.bincount(idx[1] + n[1] * idx[2], minlength=n[1] * n[2]).astype(float)
    expected = keep.sum() * areas / areas.sum()
    chi2 = np.sum((counts - expected) ** 2 / expected)
    dof = n[1] * n[2] - 1
    assert abs(chi2 - dof) < 6 * np.sqrt(2 * dof)
    # inward normal = -r_hat at the particle's (theta, phi) on the outer face (analytic
    # shell map); normal speed Rayleigh with scale vth
    i, j, k = idx
    th = math.pi / 32 + (math.pi - math.pi / 16) * (j + t32[1]) / n[1]
    ph = 2 * math.pi * (k + t32[2]) / n[2]
    rhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    vn = -np.sum(v32.T.astype(float) * rhat, axis=1)
    assert np.mean(vn > 0) > 0.995
    assert abs(np.mean(vn) / (vth * math.sqrt(math.pi / 2)) - 1) < 0.02
    vt = v32.T.astype(float) + vn[:, None] * rhat
    assert abs(np.mean(np.sum(vt * vt, axis=1)) / (2 * vth**2) - 1) < 0.03


# ------------------------------------------------------------------ P7: OML currents

def _oml_run(phi_obj, mass_ratio, steps, window, npart=100_000, seed=31):
    """Oracle run of the biased cylinder (annulus r = 10^xi around a cylinder of radius 1
    Debye length, 32 x 64 cells, object held at phi_obj and absorbing, Maxwellian flux
    injection of both species at r = 10, T_i = T_e); time-averaged collected current per
    unit length of each species over the last `window` steps, in units of the OML value."""
    from scipy.special import erfc

    w = wl.cylinder(n1=32, n2=64, r0=1.0, R=10.0, npart_per_species=npart, phi_obj=phi_obj, seed=seed,
                    inject=True, mass_ratio=mass_ratio)
    import os

    pic = OraclePIC(w, "fp64", engine="c", threads=max(1, len(os.sched_getaffinity(0))))
    pic.initialize()
    for _ in range(steps):
        pic.step()
    h = pic.history
    out = {}
    for s, sp in enumerate(w.species):
        vth = 1.0 / math.sqrt(sp.m)
        I0 = vth / math.sqrt(2.0 * math.pi) * 2.0 * math.pi * 1.0  # random current, n = |q| = r0 = 1
        chi = -sp.q * phi_obj  # > 0: attracted
        oml = I0 * (2.0 * math.sqrt(chi / math.pi) + math.exp(chi) * erfc(math.sqrt(chi))) if chi > 0 \
            else I0 * math.exp(chi)
        cnt = int(h[-1]["absorbed"][s][0]) - int(h[-1 - window]["absorbed"][s][0])
        out[s] = (cnt * sp.w / (window * w.dt) / oml, cnt)
    return out


@pytest.mark.slow
def test_oml_currents_to_a_biased_cylinder():
    """P7 (Sec. III.B compares with orbit-motion-limited theory): the oracle's collected
    currents to a cylinder of radius lambda_D biased to -5 kT/e are the OML values within
    +-15% for the attracted ions, I0 [2 sqrt(chi/pi) + e^chi erfc(sqrt(chi))], and +-20% for
    the repelled electrons, I0 e^-chi, with I0 = q n vth / sqrt(2 pi) 2 pi r0 the random
    current. A wrong injection flux constant, a wrong absorption tally or a wrong charge
    normalisation moves these by far more. The ions have m_i/m_e = 25 here (reading): OML
    depends on the mass only through vth, and the lighter ions reach their steady sheath
    within the run (with 1836 the ion current still falls through the run's length)."""
    r = _oml_run(-5.0, 25.0, 1200, 600)
    assert r[1][1] > 20_000 and abs(r[1][0] - 1.0) <= 0.15, r
    assert r[0][1] > 200 and abs(r[0][0] - 1.0) <= 0.20, r


@pytest.mark.slow
def test_oml_current_of_attracted_electrons():
    """P7 with the bias reversed (+2 kT/e): the attracted electrons' collected current is the
    OML value I0 [2 sqrt(chi/pi) + e^chi erfc(sqrt(chi))] within +-15% (electrons reach
    steady state within a few tens of plasma periods)."""
    r = _oml_run(2.0, 1836.0, 600, 300)
    assert r[0][1] > 20_000 and abs(r[0][0] - 1.0) <= 0.15, r


def test_upper_hybrid_frequency_with_uniform_b():
    """Row f2 in the whole loop: a cold electron plasma wave across a uniform B0 = B_z
    (Boris kick) oscillates at the upper-hybrid frequency sqrt(omega_pe^2 + omega_ce^2)
    (sqrt 2 for B_z = 1 in units of omega_pe), within 2% (leapfrog and Boris phase errors
    are O(dt^2) = 0.3% here), on the distorted map2 grid."""
    w = wl.langmuir_map2(32, 32, eps=0.05, ppc=16, vth=0.0, amp=0.05, dt=0.1, seed=0)
    w.B0 = (0.0, 0.0, 1.0)
    pic = OraclePIC(w, "fp64")
    pic.initialize()
    amps = [_mode_amplitude(pic, 0.05)]
    for _ in range(100):
        pic.step()
        amps.append(_mode_amplitude(pic, 0.05))
    amps = np.array(amps)
    wfreq = _frequency(amps - amps.mean(), 0.1)
    assert abs(wfreq / math.sqrt(2.0) - 1.0) < 0.02, wfreq


def test_collection_tally_bins_by_the_transverse_cell():
    """The collection tally (Fig. 7's diagnostic): particles placed in rows j of the first
    column, moving into the object face with no field, are removed there in one step and
    counted in exactly their rows; the tally sums to the absorbed count; particles moving
    the other way are not counted."""
    w = wl.cylinder(n1=16, n2=32, npart_per_species=1, seed=3, inject=False)
    rows = np.array([0, 3, 3, 17, 31, 31, 31], dtype=np.int64)
    m = rows.size
    cell = (0 | (rows << 16)).astype(np.int32)
    t = np.stack([np.full(m, 0.02), np.full(m, 0.5)]).astype(np.float32)
    theta = 2.0 * np.pi * (rows + 0.5) / 32  # the annulus: theta = 2 pi eta
    v = np.zeros((3, m), np.float32)
    v[0], v[1] = -2.0 * np.cos(theta), -2.0 * np.sin(theta)  # radially inward: one step crosses r0
    th1 = 2.0 * np.pi * 5.5 / 32  # a particle of the other species moving outward, mid-domain
    keep = wl.ParticleSet(np.array([8 | (5 << 16)], np.int32), np.full((2, 1), 0.5, np.float32),
                          np.array([[2.0 * np.cos(th1)], [2.0 * np.sin(th1)], [0.0]], np.float32))
    w.particles = [wl.ParticleSet(cell, t, v), keep]
    w.field_bc_value = [0.0] * 4  # no bias, and light macro-particles: a negligible field
    for sp in w.species:
        sp.w = 1e-9
    pic = OraclePIC(w, "fp64")
    pic.solve()
    pic.step(solve=False)
    np.testing.assert_array_equal(pic.collect[0, 0], np.bincount(rows, minlength=32))
    assert pic.collect[0, 0].sum() == pic.species[0].absorbed[0] == m
    assert pic.collect[1].sum() == 0 and pic.collect[0, 1].sum() == 0


@pytest.mark.parametrize("u_over_vth", [2.1, -0.7])
def test_drifting_flux_by_brute_force(u_over_vth):
    """Drifting Maxwellian injection (Sec. III.A's ions, drift 2.1 vth toward the wall): the
    flux density Gamma(u) = vth/sqrt(2 pi) exp(-u^2/2vth^2) + u/2 (1 + erf(u/sqrt(2) vth))
    equals the count of a drifting Maxwellian box's particles crossing a plane within dt
    (within 4 sigma), and the normal speeds the injection draws (inverse CDF by bisection)
    have the distribution of those crossing particles' speeds (two-sample Kolmogorov-Smirnov
    distance below its 1e-3-level critical value); the in-plane tangential drift is added
    to the Gaussian tangential speed."""
    rng = np.random.default_rng(31)
    vth, dt, dens, A = 0.9, 0.05, 2.0, 1.5
    u = u_over_vth * vth
    L = (abs(u) + 8.0 * vth) * dt
    npart = 4_000_000
    w = dens * L * A / npart
    vx = u + vth * rng.standard_normal(npart)
    x = -L * rng.random(npart)
    hit = x + vx * dt > 0.0
    crossed = int(hit.sum())
    expected = dens * inject.drift_flux(u, vth) * A * dt / w
    assert abs(crossed - expected) < 4.0 * math.sqrt(expected), (crossed, expected)
    # injected normal speeds on the xi = 1 face of a uniform rectangle (inward normal -x):
    # a drift (-u, 0.3, 0.2) is u along the inward normal
    n = (8, 16)
    X = np.zeros((n[1] + 1, n[0] + 1, 2))
    X[..., 0] = np.linspace(0.0, 2.0, n[0] + 1)[None, :]
    X[..., 1] = np.linspace(0.0, A, n[1] + 1)[:, None]
    from oracle import geometry
    g = geometry.build_geometry(X, [False, True])
    drift = (-u, 0.3, 0.2)
    wts = inject.face_drift_weights_2d(X, g.k, 1, drift, vth)
    np.testing.assert_allclose(wts.sum(), inject.drift_flux(u, vth) * A, rtol=1e-12)
    cnt = 40_000
    idx, t32, v32, keep = inject.inject_2d(g.k, n, 1, cnt, 0, 0, 77, vth, drift, 1e-6, drift_weights=wts)
    vn = -v32[0].astype(np.float64)
    ref = np.sort(vx[hit])
    got = np.sort(vn)
    allv = np.concatenate([ref, got])
    d = np.max(np.abs(np.searchsorted(ref, allv, side="right") / ref.size
                      - np.searchsorted(got, allv, side="right") / got.size))
    crit = 1.95 * math.sqrt((ref.size + got.size) / (ref.size * got.size))
    assert d < crit, (d, crit)
    assert abs(v32[1].mean() - 0.3) < 5 * vth / math.sqrt(cnt) and abs(v32[2].mean() - 0.2) < 5 * vth / math.sqrt(cnt)


def test_planar_wall_early_spike():
    """Test A (Sec. III.A) on a reduced 32 x 16 grid: the box fills from the source at
    xi = 1, the fast electrons reach the floating wall first and drive it to the paper's
    early minimum of about -5.7 T_e (within 10%) in the first 1600 steps; the ions have not
    arrived yet, so the wall then still sits far below the -2.1 T_e steady state."""
    w = wl.planar_wall(32, 16, ppc=32)
    p = OraclePIC(w, "fp64", engine="c", threads=4)
    p.set_floating(0, 0.0)
    p.initialize()
    vs = []
    for _ in range(1600):
        p.step()
        vs.append(p.history[-1]["object_potential"])
    vs = np.array(vs)
    assert abs(vs.min() / -5.7 - 1.0) <= 0.10, vs.min()
    assert vs[-100:].mean() < -4.0
    assert p.injected[1] > 0 and p.history[-1]["n"][1] > 0


def test_drifting_flux_reduces_to_the_resting_flux():
    """With no drift along the normal the drifting source is the resting one (closed forms):
    Gamma(0) = vth / sqrt(2 pi), the normal-speed CDF is the Rayleigh CDF
    1 - exp(-v^2 / 2 vth^2), so its inverse at q is vth sqrt(-2 ln(1 - q)); and for large
    inward drift the flux tends to u (every particle crosses) and the normal speed to u."""
    vth = 0.7
    assert abs(inject.drift_flux(0.0, vth) - vth / math.sqrt(2.0 * math.pi)) < 1e-15
    for v in (0.1, 0.5, 1.3, 3.0):
        assert abs(inject.drift_normal_cdf(v, 0.0, vth) - (1.0 - math.exp(-v * v / (2.0 * vth * vth)))) < 1e-13
    for q in (0.05, 0.3, 0.5, 0.9, 0.999):
        want = vth * math.sqrt(-2.0 * math.log(1.0 - q))
        assert abs(inject.drift_normal_speed(q, 0.0, vth) - want) < 1e-12 * max(want, 1.0)
    u = 40.0 * vth
    assert abs(inject.drift_flux(u, vth) / u - 1.0) < 1e-12
    assert abs(inject.drift_normal_speed(0.5, u, vth) / u - 1.0) < 1e-2
    # an outflowing drift (u < 0) still injects the inward tail, fewer the faster it flows out
    assert 0.0 < inject.drift_flux(-2.0 * vth, vth) < inject.drift_flux(-1.0 * vth, vth) < inject.drift_flux(0.0, vth)


def test_planar_wall_steady_state():
    """Test A (Sec. III.A) on a reduced 32 x 16 grid with 8 particles per cell and species:
    once the drifting ions have filled the box the floating wall settles at the analytic
    steady state of the paper's comparison, -2.10 T_e (the paper's own run: -2.11); the
    mean over the last sixth of 18000 steps lies within 6% of it (the reduced run's noise),
    and the early minimum (the electrons' arrival) lies well below it."""
    w = wl.planar_wall(32, 16, ppc=8)
    p = OraclePIC(w, "fp64", engine="c", threads=8)
    p.set_floating(0, 0.0)
    p.initialize()
    vs = []
    for k in range(18000):
        p.step()
        if k % 50 == 49:
            vs.append(p.history[-1]["object_potential"])
    vs = np.array(vs)
    tail = float(vs[-len(vs) // 6:].mean())
    assert abs(tail / -2.10 - 1.0) <= 0.06, tail
    assert vs.min() < 2.0 * tail
