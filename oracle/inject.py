"""Spec I: Maxwellian flux injection at a boundary face (Sec. III.A-B: plasma injected from
the outer boundary each step with fluxes from a Maxwellian; Sec. III.B: loaded at t = 0).

Readings (the paper gives no formulas):
  * particles per step from a one-sided Maxwellian flux n vth / sqrt(2 pi) through the
    face's physical length (2D polyline through the face vertices, summed in vertex order),
    rate r = n vth / sqrt(2 pi) * A * dt / w; step n (0-based) injects
    floor((n+1) r) - floor(n r) particles (a deterministic fractional carry);
  * draws: Philox4x32-10 with key (seed low 32 bits, seed high 32 bits) and counter
    (p, n, species, 0) for U0..U3 and (p, n, species, 1) for U4..U7, u -> (u + 1/2) 2^-32;
  * position uniform in the face's logical coordinate: u1 = U0 * N2 (uniform in arc length
    when the face's arc length is linear in eta, as on the annulus);
  * velocity: inward normal speed vth sqrt(-2 ln U1) (flux-weighted), tangential and z
    components vth sqrt(-2 ln U2) (cos 2 pi U3, sin 2 pi U3), plus the drift vector;
    the inward normal is -+ k^{a.}/|k^{a.}| with k linearly interpolated along the face
    from its FP64 vertex values; the tangent is the normal rotated by +90 degrees;
  * partial first push: the particle enters at a uniformly random time within the step:
    u = u_face + U4 dt (k v) (cell units, FP64, velocity already rounded to FP32); then the
    split (cell, FP32 offset) with the 1.0 -> next-cell rule, periodic wrap along the face;
    a particle whose partial push leaves the domain is dropped (not counted).
A drifting Maxwellian (Sec. III.A: the ions of the wall test enter with a drift toward the
wall), 2D faces: with u = drift . n the inward drift of a face point, the one-sided flux
density of a Maxwellian of density 1 drifting at u along the normal is
  Gamma(u) = vth / sqrt(2 pi) exp(-u^2 / 2 vth^2) + (u / 2) (1 + erf(u / (sqrt 2 vth))),
so the rate is n sum_j Gamma(u_j) A_j dt / w over the face segments (u_j at the segment's
midpoint normal, A_j its length, or its surface of revolution in an axisymmetric run), the
segment is drawn by inverse CDF of Gamma(u_j) A_j (U0) and the offset along it is U5; the
normal speed has the flux-weighted density v exp(-(v - u)^2 / 2 vth^2) on v > 0 and is drawn
by inverse CDF, F(v) = 1 - U1, solved by 64 bisections of [0, max(u, 0) + 12 vth] in FP64;
the tangential and out-of-plane components are the Gaussian ones above plus the drift's
tangential and out-of-plane parts. With no drift this is the rule above (Gamma = vth /
sqrt(2 pi), v = vth sqrt(-2 ln U1)), which stays the one used.
3D (faces normal to axis 0 of a 3D map, e.g. the outer shell of the sphere runs):
  * face area: per face cell the quadrilateral area 1/2 |(X11 - X00) x (X01 - X10)| from its
    four vertices, summed in face-cell order (axis 1 fastest); the rate uses the total;
  * position uniform in physical area: the face cell is the first whose inclusive prefix
    of areas exceeds U0 * total (so on the shell the density on the face goes as sin theta),
    the offsets along axes 1 and 2 are U5 and U6;
  * velocity: inward unit normal from row 0 of k (bilinear in the face cell), a tangent
    basis t1 = the coordinate axis least aligned with the normal (lowest index on ties),
    made orthogonal to it and normalised, t2 = n x t1; v = vth sqrt(-2 ln U1) n +
    vth sqrt(-2 ln U2) (cos 2 pi U3 t1 + sin 2 pi U3 t2) + drift;
  * partial first push u = u_face + U4 dt (k v) with k at the face point; a particle that
    leaves axis 0 or axis 1 in its partial push is dropped; a periodic axis 2 wraps.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x32_10, uniform01

INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def face_length_2d(X, side):
    """Physical length of the xi = 0 (side 0) or xi = 1 (side 1) face, summed in order."""
    col = X[:, 0 if side == 0 else -1, :]
    acc = 0.0
    for j in range(col.shape[0] - 1):
        d = col[j + 1] - col[j]
        acc += math.sqrt(d[0] * d[0] + d[1] * d[1])
    return acc


def face_ring_areas_2d(X, side):
    """Axisymmetric runs (2D (r, z) map, Omega = r): the surface of revolution of each face
    segment of the xi = 0 / xi = 1 face, 2 pi r_mid |dX| (r_mid the mean radius of the
    segment's two vertices), in segment order."""
    col = X[:, 0 if side == 0 else -1, :]
    out = np.empty(col.shape[0] - 1)
    for j in range(col.shape[0] - 1):
        d = col[j + 1] - col[j]
        out[j] = 2.0 * math.pi * (0.5 * (col[j, 0] + col[j + 1, 0])) * math.sqrt(d[0] * d[0] + d[1] * d[1])
    return out


def face_area_axisym(X, side):
    acc = 0.0
    for x in face_ring_areas_2d(X, side):
        acc += float(x)
    return acc


def rate_per_step(density, vth, area, dt, w):
    return (((density * vth) * INV_SQRT_2PI) * area) * dt / w


def drift_flux(u, vth):
    """One-sided flux density through a plane of a unit-density Maxwellian (thermal speed
    vth) drifting at u along the plane's inward normal."""
    return vth * INV_SQRT_2PI * math.exp(-u * u / (2.0 * vth * vth)) + 0.5 * u * (1.0 + math.erf(u / (math.sqrt(2.0) * vth)))


def drift_normal_cdf(v, u, vth):
    """CDF on v > 0 of the flux-weighted normal speed density v exp(-(v - u)^2 / 2 vth^2)."""
    s2 = vth * vth
    a = math.sqrt(0.5 * math.pi) * u * vth
    e0 = math.exp(-u * u / (2.0 * s2))
    erf0 = math.erf(u / (math.sqrt(2.0) * vth))
    z = s2 * e0 + a * (1.0 + erf0)
    f = s2 * (e0 - math.exp(-(v - u) * (v - u) / (2.0 * s2))) + a * (math.erf((v - u) / (math.sqrt(2.0) * vth)) + erf0)
    return f / z


def drift_normal_speed(q, u, vth):
    """The normal speed with drift_normal_cdf(v) = q: 64 bisections of [0, max(u, 0) + 12 vth]."""
    lo, hi = 0.0, max(u, 0.0) + 12.0 * vth
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        if drift_normal_cdf(mid, u, vth) < q:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def face_drift_weights_2d(X, k64, side, drift, vth, ring_areas=None):
    """Per face segment (drifting injection): Gamma(u_j) A_j with u_j = drift . n_j, n_j the
    inward unit normal from row 0 of k averaged over the segment's two vertices (FP64), A_j
    the segment's length or its surface of revolution."""
    n1 = X.shape[1] - 1
    col = 0 if side == 0 else n1
    m = X.shape[0] - 1
    sgn = -1.0 if side == 1 else 1.0
    out = np.empty(m)
    for j in range(m):
        kb = 0.5 * (k64[j, col] + k64[j + 1, col])
        ga = kb[0]
        gn = math.sqrt(ga[0] * ga[0] + ga[1] * ga[1])
        nin = sgn * ga / gn
        u = drift[0] * nin[0] + drift[1] * nin[1]
        if ring_areas is not None:
            a = float(ring_areas[j])
        else:
            d = X[j + 1, col] - X[j, col]
            a = math.sqrt(d[0] * d[0] + d[1] * d[1])
        out[j] = drift_flux(u, vth) * a
    return out


def count_at_step(rate, step):
    return int(math.floor((step + 1) * rate) - math.floor(step * rate))


def draws(count, step, species, seed):
    p = np.arange(count, dtype=np.uint64)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    out = []
    for word in (0, 1):
        ctr = np.zeros((count, 4), dtype=np.uint32)
        ctr[:, 0] = p.astype(np.uint32)
        ctr[:, 1] = np.uint32(step & 0xFFFFFFFF)
        ctr[:, 2] = np.uint32(species)
        ctr[:, 3] = np.uint32(word)
        out.append(uniform01(philox4x32_10(ctr, np.broadcast_to(key, (count, 2)))))
    return np.concatenate(out, axis=1)  # (count, 8)


def inject_2d(k64, n, side, count, step, species, seed, vth, drift, dt, ring_areas=None, drift_weights=None):
    """New particles on the face normal to axis 0 (side 0: xi = 0, side 1: xi = 1).
    k64: FP64 vertex table (N2+1, N1+1, a, alpha). Returns (idx (2, m), t32 (2, m),
    v32 (3, m), keep mask over the count draws). ring_areas (axisymmetric runs): the face
    segments' surfaces of revolution; the segment is then drawn by inverse CDF of those
    (the first whose inclusive prefix exceeds U0 * total), the offset along it is U5, the
    out-of-plane component is v_theta, and axis 1 is not periodic (a particle whose partial
    push leaves it is dropped). drift_weights (a drifting Maxwellian: face_drift_weights_2d):
    the segment is drawn by inverse CDF of those, the offset along it from U5, and the normal
    speed from the drifting flux-weighted distribution."""
    n1, n2 = n
    U = draws(count, step, species, seed)
    drifting = drift_weights is not None
    if drifting:
        cdf = np.empty_like(drift_weights)
        acc = 0.0
        for i, x in enumerate(drift_weights):
            acc += float(x)
            cdf[i] = acc
        j = np.minimum(np.searchsorted(cdf, U[:, 0] * acc, side="right"), n2 - 1).astype(np.int64)
        s = U[:, 5]
    elif ring_areas is None:
        u1 = U[:, 0] * n2
        j = np.floor(u1).astype(np.int64)
        j = np.minimum(j, n2 - 1)
        s = u1 - j
    else:
        cdf = np.empty_like(ring_areas)
        acc = 0.0
        for i, x in enumerate(ring_areas):
            acc += float(x)
            cdf[i] = acc
        j = np.minimum(np.searchsorted(cdf, U[:, 0] * acc, side="right"), n2 - 1).astype(np.int64)
        s = U[:, 5]
    col = 0 if side == 0 else n1
    kb = (1.0 - s)[:, None, None] * k64[j, col] + s[:, None, None] * k64[j + 1, col]
    ga = kb[:, 0, :]  # d u^0 / d x
    gn = np.sqrt(ga[:, 0] * ga[:, 0] + ga[:, 1] * ga[:, 1])
    sgn = -1.0 if side == 1 else 1.0
    nin = sgn * ga / gn[:, None]
    tau = np.stack([-nin[:, 1], nin[:, 0]], axis=1)
    rho = vth * np.sqrt(-2.0 * np.log(U[:, 2]))
    vt = rho * np.cos(2.0 * math.pi * U[:, 3])
    vz = rho * np.sin(2.0 * math.pi * U[:, 3])
    v = np.empty((3, count))
    if drifting:
        un = drift[0] * nin[:, 0] + drift[1] * nin[:, 1]
        ut = drift[0] * tau[:, 0] + drift[1] * tau[:, 1]
        vn = np.array([drift_normal_speed(1.0 - U[p, 1], un[p], vth) for p in range(count)])
        vt = vt + ut
        v[0] = vn * nin[:, 0] + vt * tau[:, 0]
        v[1] = vn * nin[:, 1] + vt * tau[:, 1]
    else:
        vn = vth * np.sqrt(-2.0 * np.log(U[:, 1]))
        v[0] = vn * nin[:, 0] + vt * tau[:, 0] + drift[0]
        v[1] = vn * nin[:, 1] + vt * tau[:, 1] + drift[1]
    v[2] = vz + drift[2]
    v32 = v.astype(np.float32)
    vd = v32.astype(np.float64)
    du0 = (U[:, 4] * dt) * (kb[:, 0, 0] * vd[0] + kb[:, 0, 1] * vd[1])
    du1 = (U[:, 4] * dt) * (kb[:, 1, 0] * vd[0] + kb[:, 1, 1] * vd[1])
    u0 = (0.0 if side == 0 else float(n1)) + du0
    uu1 = (j + s) + du1
    out_idx = np.empty((2, count), dtype=np.int64)
    out_t = np.empty((2, count), dtype=np.float32)
    for a, u in enumerate((u0, uu1)):
        c = np.floor(u)
        f32 = (u - c).astype(np.float32)
        one = f32 >= np.float32(1.0)
        f32[one] = np.float32(0.0)
        c = c + one
        out_idx[a] = c.astype(np.int64)
        out_t[a] = f32
    if ring_areas is None:
        out_idx[1] = np.mod(out_idx[1], n2)  # (a periodic face)
        keep = (out_idx[0] >= 0) & (out_idx[0] < n1)
    else:
        keep = (out_idx[0] >= 0) & (out_idx[0] < n1) & (out_idx[1] >= 0) & (out_idx[1] < n2)
    return out_idx[:, keep], out_t[:, keep], v32[:, keep], keep


def face_areas_3d(X, side):
    """Physical areas of the face cells of the xi = 0 (side 0) / xi = 1 (side 1) face of a
    3D vertex map X (N3+1, N2+1, N1+1, 3), as a flat array in face-cell order j + N2 k."""
    F = X[:, :, 0 if side == 0 else -1, :]  # (N3+1, N2+1, 3), [k, j]
    X00, X10 = F[:-1, :-1], F[:-1, 1:]
    X01, X11 = F[1:, :-1], F[1:, 1:]
    a = X11 - X00
    b = X01 - X10
    cx = a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1]
    cy = a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2]
    cz = a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]
    return (0.5 * np.sqrt(cx * cx + cy * cy + cz * cz)).ravel()


def face_area_3d(X, side):
    acc = 0.0
    for x in face_areas_3d(X, side):
        acc += float(x)
    return acc


def inject_3d(X, k64, n, side, count, step, species, seed, vth, drift, dt, periodic2=True):
    """New particles on the 3D face normal to axis 0. k64: FP64 vertex table
    (N3+1, N2+1, N1+1, a, alpha). Returns (idx (3, m), t32 (3, m), v32 (3, m), keep)."""
    n1, n2, n3 = n
    U = draws(count, step, species, seed)
    areas = face_areas_3d(X, side)
    cdf = np.empty_like(areas)
    acc = 0.0
    for i, x in enumerate(areas):
        acc += float(x)
        cdf[i] = acc
    target = U[:, 0] * acc
    cellf = np.searchsorted(cdf, target, side="right")
    cellf = np.minimum(cellf, n2 * n3 - 1)
    j, kk = cellf % n2, cellf // n2
    t1, t2 = U[:, 5], U[:, 6]
    col = 0 if side == 0 else n1
    kf = ((1 - t1) * (1 - t2))[:, None, None] * k64[kk, j, col] + (t1 * (1 - t2))[:, None, None] * k64[kk, j + 1, col] \
        + ((1 - t1) * t2)[:, None, None] * k64[kk + 1, j, col] + (t1 * t2)[:, None, None] * k64[kk + 1, j + 1, col]
    ga = kf[:, 0, :]
    sgn = -1.0 if side == 1 else 1.0
    nin = sgn * ga / np.linalg.norm(ga, axis=1)[:, None]
    e = np.zeros_like(nin)
    e[np.arange(count), np.argmin(np.abs(nin), axis=1)] = 1.0
    t1v = e - np.sum(e * nin, axis=1)[:, None] * nin
    t1v = t1v / np.linalg.norm(t1v, axis=1)[:, None]
    t2v = np.cross(nin, t1v)
    vn = vth * np.sqrt(-2.0 * np.log(U[:, 1]))
    rho = vth * np.sqrt(-2.0 * np.log(U[:, 2]))
    c3, s3 = np.cos(2.0 * math.pi * U[:, 3]), np.sin(2.0 * math.pi * U[:, 3])
    v = (vn[:, None] * nin + (rho * c3)[:, None] * t1v + (rho * s3)[:, None] * t2v).T + np.asarray(drift)[:, None]
    v32 = v.astype(np.float32)
    vd = v32.astype(np.float64)
    du = (U[:, 4] * dt)[None, :] * np.einsum("pab,bp->ap", kf, vd)
    base = [np.full(count, 0.0 if side == 0 else float(n1)), j + t1, kk + t2]
    out_idx = np.empty((3, count), dtype=np.int64)
    out_t = np.empty((3, count), dtype=np.float32)
    for a in range(3):
        u = base[a] + du[a]
        c = np.floor(u)
        f32 = (u - c).astype(np.float32)
        one = f32 >= np.float32(1.0)
        f32[one] = np.float32(0.0)
        c = c + one
        out_idx[a] = c.astype(np.int64)
        out_t[a] = f32
    if periodic2:
        out_idx[2] = np.mod(out_idx[2], n3)
    keep = (out_idx[0] >= 0) & (out_idx[0] < n1) & (out_idx[1] >= 0) & (out_idx[1] < n2)
    return out_idx[:, keep], out_t[:, keep], v32[:, keep], keep
