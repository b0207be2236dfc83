"""Hybrid mover in FP64 (Sec. II.B.4) and the ctypes wrapper of the FP32 replay.

Particles keep a logical position (cell index + in-cell offset, cell units) and a
physical velocity. One push (eqs. (step1)-(step4), unmagnetised):
  1. b1-gather (eqs. (vvp), (Wvp), (b1)) of the logical field G and of k at xi^n;
     E^alpha = -sum_a G^a k^{a alpha} (reading: the vertex field is logical and is turned
     physical at the particle with the same gathered k that the predictor needs);
  2. v^{n+1/2} = v^{n-1/2} + dt (q/m) E (eq. (step1); B0 = 0, so the Boris rotation is the
     identity; in 2D E has no z component);
  3. predictor xi' = xi^n + dt/2 k(xi^n) v^{n+1/2} (eq. (step2)); in 2D only the in-plane
     velocity moves xi;
  4. k(xi') by b1 interpolation (eq. (step3));
  5. corrector xi^{n+1} = xi^n + dt k(xi') v^{n+1/2} (eq. (step4));
  6. boundaries: periodic axes wrap; on an absorbing axis a cell index < 0 or >= N removes
     the particle (Sec. II.B.4: leaving the domain means a logical coordinate < 0 or > 1;
     an offset of exactly 0 on cell 0 is inside, a coordinate of exactly 1 is outside).
A predictor point outside a non-periodic axis is clamped to the boundary (reading).
Spec B (reflecting axes; the paper reflects at the axis of its spherical runs, Sec. III.B,
without a formula): a corrector position outside a reflecting axis is mirrored in logical
space about the face, u -> -u below and u -> 2N - u above (on the split representation:
cell -1 - c or 2N - 1 - c, offset 1 - t, renormalised), and the velocity is reflected about
the unit normal of that face, n = row a of k(xi') (the k the corrector used) normalised:
v <- v - 2 (v.n) n / (n.n). A particle still outside after one mirror is removed at that
face. The kinetic-energy tally uses the kicked velocity, before any reflection.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os

import numpy as np

PBC_PERIODIC, PBC_ABSORB, PBC_REFLECT = 0, 1, 2


def _vertex_lookup(table, idx):
    """table: numpy vertex layout (..., comps); idx: per-axis vertex indices (D, n)."""
    D = idx.shape[0]
    return table[tuple(idx[D - 1 - x] for x in range(D))]


def gather(table, idx, t):
    """b1 interpolation of a vertex table at (cell idx, offsets t): sum over the 2^D corners
    of prod_a b1 weights times the vertex value."""
    D = idx.shape[0]
    acc = 0.0
    for o in itertools.product((0, 1), repeat=D):
        w = np.ones(idx.shape[1])
        for a in range(D):
            w = w * (t[a] if o[a] else 1.0 - t[a])
        corner = idx + np.asarray(o)[:, None]
        val = _vertex_lookup(table, corner)
        acc = acc + w.reshape((-1,) + (1,) * (val.ndim - 1)) * val
    return acc


def _renorm(x):
    c = np.floor(x)
    f = x - c
    one = f >= 1.0
    f = np.where(one, 0.0, f)
    c = c + one
    return c.astype(np.int64), f


def boris64(v, E3, h, B):
    """Boris step in FP64 (eq. (step1) with a uniform B0, v x B averaged over the step):
    v- = v + h E; v' = v- + v- x t; v+ = v- + v' x s; v + = v+ + h E, with t = h B0,
    s = 2 t / (1 + |t|^2) and h = dt q/m / 2. v, E3: (3, n)."""
    t = h * np.asarray(B, dtype=np.float64)
    s = 2.0 * t / (1.0 + float(np.dot(t, t)))
    vm = v + h * E3
    vp = vm + np.cross(vm.T, t).T
    return vm + np.cross(vp.T, s).T + h * E3


def component_field(B, axisym):
    """The uniform field in the basis of the velocity components. A 2D axisymmetric run
    stores v = (v_r, v_z, v_theta); that basis is left-handed (r x z = -theta), so the
    component formula of a cross product gives minus the physical one there, and v x B is
    taken as the component cross product with -B."""
    B = np.asarray(B, dtype=np.float64)
    return -B if axisym else B


def gyro_constants64(dt, qm, B):
    """Constants of the exact gyration over dt in a uniform field B (component basis):
    (b0, b1, b2, cos th, sin th, f1, f2) with b = B / |B|, th = (q/m) |B| dt (signed by q),
    f1 = sin th / th and f2 = (1 - cos th) / th = 2 sin^2(th/2) / th (1 and 0 at th = 0)."""
    B = [float(x) for x in B]
    bm = math.sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2])
    b = [x / bm for x in B]
    th = float(qm) * bm * float(dt)
    if th == 0.0:
        return (b[0], b[1], b[2], 1.0, 0.0, 1.0, 0.0)
    sh = math.sin(0.5 * th)
    return (b[0], b[1], b[2], math.cos(th), math.sin(th), math.sin(th) / th, 2.0 * sh * sh / th)


def gyro_flow64(v, dt, gc):
    """The exact motion in the uniform magnetic field alone over dt (the cyclotronic
    integrator's gyration flow; Sec. II.B.4 with the reading of the cited cyclotronic
    scheme): with u = v x b, v_par = (v . b) b, v_perp = v - v_par,
      v' = v_par + cos th v_perp + sin th u,
      displacement = dt (v_par + f1 v_perp + f2 u).
    gc: gyro_constants64. Returns (displacement (3, n), v' (3, n))."""
    b = np.asarray(gc[:3], dtype=np.float64)[:, None]
    cs, sn, f1, f2 = gc[3:]
    vpar = v[0] * b[0] + v[1] * b[1] + v[2] * b[2]
    par = vpar * b
    vperp = v - par
    u = np.stack([v[1] * b[2] - v[2] * b[1], v[2] * b[0] - v[0] * b[2], v[0] * b[1] - v[1] * b[0]])
    vnew = (par + cs * vperp) + sn * u
    disp = dt * ((par + f1 * vperp) + f2 * u)
    return disp, vnew


def axisym_frame(rn, d, v):
    """The axisymmetric frame step for a 3D displacement d = (d_r, d_z, d_theta) taken from
    (r, 0, z) in the local Cartesian frame: the new point has x = r + d_r, y = d_theta,
    r' = sqrt(x^2 + y^2); the meridional displacement is (r' - r, d_z) and the velocity v is
    turned into the frame at the new azimuth. Returns (meridional displacement, v)."""
    x = rn + d[0]
    y = d[2]
    r1 = np.sqrt(x * x + y * y)
    safe = r1 > 0.0
    ca = np.where(safe, x / np.where(safe, r1, 1.0), 1.0)
    sa = np.where(safe, y / np.where(safe, r1, 1.0), 0.0)
    vout = v.copy()
    vout[0] = ca * v[0] + sa * v[2]
    vout[2] = ca * v[2] - sa * v[0]
    return np.stack([r1 - rn, d[1]]), vout


def axisym_step(rn, v, dt):
    """The cylindrical part of the axisymmetric mover (2D (r, z) meridional plane, Omega = r,
    azimuthal symmetry; Sec. II.B: the cylindrical Boris mover in its hybrid form; reading):
    the particle moves on a straight line in 3D over the step, from (r, 0, z) with velocity
    (v_r, v_theta, v_z): x = r + dt v_r, y = dt v_theta, r' = sqrt(x^2 + y^2); the meridional
    displacement is (r' - r, dt v_z) and the velocity turns with the frame by the angle
    alpha of (x, y): v_r' = cos a v_r + sin a v_theta, v_theta' = cos a v_theta - sin a v_r
    (the inertial forces; r v_theta is kept). v = (v_r, v_z, v_theta). Returns the
    displacement (2, n) and the velocity (3, n) in the new frame."""
    x = rn + dt * v[0]
    y = dt * v[2]
    r1 = np.sqrt(x * x + y * y)
    safe = r1 > 0.0
    ca = np.where(safe, x / np.where(safe, r1, 1.0), 1.0)
    sa = np.where(safe, y / np.where(safe, r1, 1.0), 0.0)
    disp = np.stack([r1 - rn, dt * v[1]])
    vout = v.copy()
    vout[0] = ca * v[0] + sa * v[2]
    vout[2] = ca * v[2] - sa * v[0]
    return disp, vout


def push64(idx, t, v, k, G, dt, qm, n, pbc, return_kicked=False, B=None, R=None, gyro=False):
    """One FP64 push. idx (D, n) int, t (D, n), v (3, n); k: vertex table (..., a, alpha);
    G: vertex table (..., a); qm: q/m per particle (n,) or scalar; B: uniform magnetic
    field (3,) or None (the kick is then v += dt q/m E; with B, the Boris step); R: for an
    axisymmetric run (2D, Omega = r), the vertex table of the cylindrical radius: the
    position then advances by the meridional displacement of axisym_step instead of dt v,
    predictor xi' = xi^n + 1/2 k(xi^n) disp, corrector xi^{n+1} = xi^n + k(xi') disp, and
    the velocity is turned into the new frame. gyro (with B): the cyclotronic integrator
    instead of the Boris step: v+ = v + dt (q/m) E, then the exact gyration flow over dt
    (gyro_flow64) gives the displacement (which moves xi through the same predictor and
    corrector) and the new velocity; in an axisymmetric run the displacement starts from
    the particle's point in 3D and the frame turns as in axisym_step.
    Returns (idx, t, v, face) with face = -1 alive or 2a+side for removed particles, plus
    the kicked velocity before any reflection (and before the gyration) when return_kicked."""
    D = idx.shape[0]
    idx = idx.astype(np.int64)
    t = np.asarray(t, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    kp = gather(k, idx, t)  # (n, a, alpha)
    gp = gather(G, idx, t)  # (n, a)
    E = -np.einsum("pa,pab->pb", gp, kp)  # (n, alpha), alpha < D
    magnetized = B is not None and bool(np.any(np.asarray(B)))
    gyro = gyro and magnetized
    if magnetized and not gyro:
        E3 = np.zeros_like(v)
        E3[:D] = E.T
        v = boris64(v, E3, 0.5 * dt * np.asarray(qm), component_field(B, R is not None))
    else:
        v[:D] = v[:D] + dt * np.asarray(qm) * E.T
    vk = v.copy()
    dform = gyro or R is not None  # the position moves by a displacement, not dt v
    if gyro:
        assert np.ndim(qm) == 0, "the cyclotronic push takes one q/m"
        d3, vnew = gyro_flow64(v, dt, gyro_constants64(dt, qm, component_field(B, R is not None)))
        if R is not None:
            disp, vrot = axisym_frame(gather(R, idx, t), d3, vnew)
        else:
            disp, vrot = d3[:D], vnew
    elif R is not None:
        disp, vrot = axisym_step(gather(R, idx, t), v, dt)
    if dform:
        d = np.einsum("pab,bp->ap", kp, disp)
        cpred, tpred = _renorm(t + 0.5 * d)
    else:
        # predictor
        d = np.einsum("pab,bp->ap", kp, v[:D])
        cpred, tpred = _renorm(t + 0.5 * dt * d)
    ip = idx + cpred
    for a in range(D):
        if pbc[2 * a] == PBC_PERIODIC:
            ip[a] = np.mod(ip[a], n[a])
        else:
            low = ip[a] < 0
            high = ip[a] >= n[a]
            ip[a] = np.clip(ip[a], 0, n[a] - 1)
            tpred[a] = np.where(low, 0.0, np.where(high, 1.0, tpred[a]))
    kq = gather(k, ip, tpred)
    if dform:
        d2 = np.einsum("pab,bp->ap", kq, disp)
        cn, tn = _renorm(t + d2)
        v = vrot
    else:
        d2 = np.einsum("pab,bp->ap", kq, v[:D])
        cn, tn = _renorm(t + dt * d2)
    inew = idx + cn
    face = np.full(idx.shape[1], -1, dtype=np.int64)
    for a in range(D):
        if pbc[2 * a] == PBC_PERIODIC:
            inew[a] = np.mod(inew[a], n[a])
        elif pbc[2 * a] == PBC_ABSORB:
            lo = (inew[a] < 0) & (face < 0)
            hi = (inew[a] >= n[a]) & (face < 0)
            face[lo] = 2 * a
            face[hi] = 2 * a + 1
    ke_v = vk
    for a in range(D):
        if pbc[2 * a] != PBC_REFLECT:
            continue
        below = (inew[a] < 0) & (face < 0)
        above = (inew[a] >= n[a]) & (face < 0)
        out = below | above
        if not np.any(out):
            continue
        c2 = np.where(below, -inew[a] - 1, 2 * n[a] - 1 - inew[a])
        c_add, t2 = _renorm(1.0 - tn[a])
        c2 = c2 + c_add
        still = out & ((c2 < 0) | (c2 >= n[a]))
        face[still & below] = 2 * a
        face[still & above] = 2 * a + 1
        ok = out & ~still
        inew[a] = np.where(ok, c2, inew[a])
        tn[a] = np.where(ok, t2, tn[a])
        nv = kq[:, a, :]  # (n, alpha): row a of k(xi')
        nn = np.sum(nv * nv, axis=1)
        dot = np.sum(v[:D].T * nv, axis=1)
        sfac = np.where(ok, 2.0 * dot / nn, 0.0)
        v[:D] = v[:D] - (sfac[:, None] * nv).T
    if return_kicked:
        return inew, tn, v, face, ke_v
    return inew, tn, v, face


def kick64(idx, t, v, k, G, coef, B=None, axisym=False):
    """Gather and kick only: v += coef * E (used for the leapfrog start-up half step), coef
    = fraction * dt q/m; with a uniform B, the Boris step over that fraction of dt (the
    cyclotronic integrator's start-up is the plain kick: pass B=None)."""
    D = idx.shape[0]
    v = np.array(v, dtype=np.float64)
    kp = gather(k, idx.astype(np.int64), np.asarray(t, dtype=np.float64))
    gp = gather(G, idx.astype(np.int64), np.asarray(t, dtype=np.float64))
    E = -np.einsum("pa,pab->pb", gp, kp)
    if B is not None and np.any(np.asarray(B)):
        E3 = np.zeros_like(v)
        E3[:D] = E.T
        return boris64(v, E3, 0.5 * np.asarray(coef), component_field(B, axisym))
    v[:D] = v[:D] + np.asarray(coef) * E.T
    return v


# ---------------------------------------------------------------------------------------
# FP32 replay (oracle/replay32.c)
# ---------------------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from .build import build_replay

        path = build_replay()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.replay_push.argtypes = [ctypes.c_int, P, P, ctypes.c_long, P, P, P, P, P,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P, P, P, P]
        lib.replay_push.restype = None
        lib.replay_kick.argtypes = [ctypes.c_int, P, ctypes.c_long, P, P, P, P, P, ctypes.c_float, P]
        lib.replay_kick.restype = None
        _LIB = lib
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def boris_constants32(dt, qm, B, fraction=1.0, axisym=False):
    """FP32 Boris constants (h, t0, t1, t2, s0, s1, s2) of a kick over fraction * dt:
    h = dt q/m / 2, t = h B0, s = 2 t / (1 + |t|^2), computed in FP64 and rounded once;
    None without a field. B0 in the velocity components' basis (component_field)."""
    if B is None or not np.any(np.asarray(B, dtype=np.float64)):
        return None
    h = 0.5 * fraction * dt * qm
    t = h * component_field(B, axisym)
    s = 2.0 * t / (1.0 + float(np.dot(t, t)))
    return np.asarray([h, *t, *s], dtype=np.float32)


def gyro_constants32(dt, qm, B, axisym=False):
    """FP32 constants of the cyclotronic push (b0, b1, b2, cos th, sin th, f1, f2): the FP64
    gyro_constants64 of the field in the velocity components' basis, rounded once; None
    without a field."""
    if B is None or not np.any(np.asarray(B, dtype=np.float64)):
        return None
    return np.asarray(gyro_constants64(dt, qm, component_field(B, axisym)), dtype=np.float32)


def push32(idx, t32, v32, k32, G32, n, pbc, dtqm, hdt, dt, boris=None, R32=None, gyro=None):
    """FP32 replay of one push. Arguments as push64 but float32 tables (numpy vertex
    layout, k32 (..., a, alpha), G32 (..., a)) and float32 coefficients
    dtqm = float32(dt q / m), hdt = float32(dt / 2), dt = float32(dt); boris: the
    boris_constants32 of a magnetised run (None: no field); R32: the FP32 vertex table of the
    cylindrical radius of an axisymmetric run (None: Cartesian); gyro: the gyro_constants32
    of a run with the cyclotronic integrator (boris is then None).
    Returns (idx, t, v, face, ke_fp)."""
    D = idx.shape[0]
    np_ = idx.shape[1]
    idx_c = np.ascontiguousarray(idx, dtype=np.int32).copy()
    t_c = np.ascontiguousarray(t32, dtype=np.float32).copy()
    v_c = np.ascontiguousarray(v32, dtype=np.float32).copy()
    K = np.ascontiguousarray(k32, dtype=np.float32).reshape(-1)
    G = np.ascontiguousarray(G32, dtype=np.float32).reshape(-1)
    nn = np.asarray(list(n) + [1] * (3 - D), dtype=np.int32)
    pb = np.asarray(list(pbc) + [0] * (6 - len(pbc)), dtype=np.int32)
    face = np.empty(np_, dtype=np.int32)
    ke = np.empty(np_, dtype=np.int64)
    bc = None if boris is None else np.ascontiguousarray(boris, dtype=np.float32)
    Rc = None if R32 is None else np.ascontiguousarray(R32, dtype=np.float32).reshape(-1)
    gc = None if gyro is None else np.ascontiguousarray(gyro, dtype=np.float32)
    _lib().replay_push(D, _ptr(nn), _ptr(pb), np_, _ptr(idx_c), _ptr(t_c), _ptr(v_c), _ptr(K), _ptr(G),
                       np.float32(dtqm), np.float32(hdt), np.float32(dt), _ptr(face), _ptr(ke),
                       None if bc is None else _ptr(bc), None if Rc is None else _ptr(Rc),
                       None if gc is None else _ptr(gc))
    return idx_c, t_c, v_c, face, ke


def kick32(idx, t32, v32, k32, G32, n, coef, boris=None):
    D = idx.shape[0]
    idx_c = np.ascontiguousarray(idx, dtype=np.int32)
    t_c = np.ascontiguousarray(t32, dtype=np.float32)
    v_c = np.ascontiguousarray(v32, dtype=np.float32).copy()
    K = np.ascontiguousarray(k32, dtype=np.float32).reshape(-1)
    G = np.ascontiguousarray(G32, dtype=np.float32).reshape(-1)
    nn = np.asarray(list(n) + [1] * (3 - D), dtype=np.int32)
    bc = None if boris is None else np.ascontiguousarray(boris, dtype=np.float32)
    _lib().replay_kick(D, _ptr(nn), idx.shape[1], _ptr(idx_c), _ptr(t_c), _ptr(v_c), _ptr(K), _ptr(G),
                       np.float32(coef), None if bc is None else _ptr(bc))
    return v_c


# ---------------------------------------------------------------------------------------
# FP64 mover as C loops (oracle/pic64.c): the same definition as push64
# ---------------------------------------------------------------------------------------

_LIB64 = None


def _lib64():
    global _LIB64
    if _LIB64 is None:
        from .build import build_pic64

        lib = ctypes.CDLL(build_pic64())
        P = ctypes.c_void_p
        lib.oracle_push64.argtypes = [ctypes.c_int, P, P, ctypes.c_long, P, P, P, P, P, ctypes.c_double,
                                      ctypes.c_double, P, P, ctypes.c_int, P, P, P]
        lib.oracle_push64.restype = None
        lib.oracle_deposit64.argtypes = [ctypes.c_int, P, P, ctypes.c_long, P, P, P, ctypes.c_int]
        lib.oracle_deposit64.restype = ctypes.c_int
        lib.oracle_openmp_threads.argtypes = []
        lib.oracle_openmp_threads.restype = ctypes.c_int
        _LIB64 = lib
    return _LIB64


def openmp_threads():
    """Threads the C loops can use (1 when built without OpenMP)."""
    return int(_lib64().oracle_openmp_threads())


def push64_c(idx, t, v, k, G, dt, qm, n, pbc, threads=1, inplace=False, B=None, R=None, gyro=False):
    """push64 as C loops. qm is a scalar. Returns (idx, t, v, face, vdot) with vdot the
    per-particle v^{n-1/2} . v^{n+1/2} (kicked velocity, before any reflection). With
    inplace, idx (int64), t and v (float64), C-contiguous, are updated and returned."""
    D = idx.shape[0]
    np_ = idx.shape[1]
    if inplace:
        idx_c, t_c, v_c = idx, t, v
        assert idx_c.dtype == np.int64 and t_c.dtype == np.float64 and v_c.dtype == np.float64
        assert idx_c.flags.c_contiguous and t_c.flags.c_contiguous and v_c.flags.c_contiguous
    else:
        idx_c = np.array(idx, dtype=np.int64, order="C")
        t_c = np.array(t, dtype=np.float64, order="C")
        v_c = np.array(v, dtype=np.float64, order="C")
    K = np.ascontiguousarray(k, dtype=np.float64).reshape(-1)
    Gc = np.ascontiguousarray(G, dtype=np.float64).reshape(-1)
    nn = np.asarray(list(n) + [1] * (3 - D), dtype=np.int32)
    pb = np.asarray(list(pbc) + [0] * (6 - len(pbc)), dtype=np.int32)
    face = np.empty(np_, dtype=np.int32)
    vdot = np.empty(np_, dtype=np.float64)
    magnetized = B is not None and bool(np.any(np.asarray(B)))
    Bv, Gy = None, None
    if magnetized and gyro:
        Gy = np.asarray(gyro_constants64(dt, qm, component_field(B, R is not None)), dtype=np.float64)
    elif magnetized:
        Bv = np.ascontiguousarray(component_field(B, R is not None), dtype=np.float64)
    Rc = None if R is None else np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    _lib64().oracle_push64(D, _ptr(nn), _ptr(pb), np_, _ptr(idx_c), _ptr(t_c), _ptr(v_c), _ptr(K), _ptr(Gc),
                           float(dt), float(qm), _ptr(face), _ptr(vdot), int(threads),
                           None if Bv is None else _ptr(Bv), None if Rc is None else _ptr(Rc),
                           None if Gy is None else _ptr(Gy))
    return idx_c, t_c, v_c, face.astype(np.int64), vdot
