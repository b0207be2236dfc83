"""Spec M: metric coefficients from the discrete map known at cell vertices.

Sec. II.A: Jacobi matrix j_{alpha beta} = dx^alpha/dxi^beta (eq. jcov), its inverse
k^{alpha beta} = dxi^alpha/dx^beta (eq. jcon), Jacobian J = det j (eq. jac), contravariant
metric g^{ab} (eq. gcon) and the logical-space Poisson operator
(1/(Omega J)) d_i (Omega J g^{ij} d_j phi) (eq. poiscurv). The paper computes the metric by
finite differences of the vertex map (Sec. II.A, last paragraph); the stencils below are
this implementation's reading of that sentence.

Everything is FP64 and in CELL UNITS: logical coordinates u^a = N_a xi^a, so a cell is a
unit square/cube, k is dU/dx (k_cell^{a alpha} = N_a k^{a alpha}) and the Jacobian of a
cell equals its physical area (2D) or volume (3D).

Layout: logical axis a is numpy axis D-1-a (see paper_1311_2286_gb300.workloads).
Floating-point operation order is part of the spec (the device geometry reproduces it
bit for bit): every expression is written with explicit parentheses.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# A cross coefficient a^{ab} (b != a) no larger than this fraction of the face's a^{aa} is
# the rounding residue of an orthogonal map and is set to zero, so that orthogonal maps give
# exact 5-point (2D) / 7-point (3D) operators (reading; applied identically on the device).
CROSS_ROUNDOFF = 1e-12


def _ax(D: int, a: int) -> int:
    return D - 1 - a


def vertex_derivative(X: np.ndarray, a: int, periodic: bool) -> np.ndarray:
    """dX/du^a at every vertex (cell units).

    Interior: central difference (X[v+1] - X[v-1]) * 0.5.
    Non-periodic ends: one-sided second order ((4 X1 - 3 X0) - X2) * 0.5 and
    ((3 XN - 4 X(N-1)) + X(N-2)) * 0.5.
    Periodic axis: the neighbour of vertex 0 is X[N-1] - (X[N] - X[0]) (the period vector
    is taken from the vertex array itself); vertex N copies vertex 0.
    """
    D = X.ndim - 1
    ax = _ax(D, a)
    Xm = np.moveaxis(X, ax, 0)
    n = Xm.shape[0] - 1
    out = np.empty_like(Xm)
    if periodic:
        shift = Xm[n] - Xm[0]
        prev0 = Xm[n - 1] - shift
        out[0] = (Xm[1] - prev0) * 0.5
        out[1:n] = (Xm[2 : n + 1] - Xm[0 : n - 1]) * 0.5
        out[n] = out[0]
    else:
        out[1:n] = (Xm[2 : n + 1] - Xm[0 : n - 1]) * 0.5
        out[0] = ((4.0 * Xm[1] - 3.0 * Xm[0]) - Xm[2]) * 0.5
        out[n] = ((3.0 * Xm[n] - 4.0 * Xm[n - 1]) + Xm[n - 2]) * 0.5
    return np.moveaxis(out, 0, ax)


def jacobi_vertices(X: np.ndarray, periodic) -> np.ndarray:
    """Jacobi matrix j[..., alpha, a] = dx^alpha/du^a at vertices, eq. (jcov) in cell units."""
    D = X.ndim - 1
    return np.stack([vertex_derivative(X, a, bool(periodic[a])) for a in range(D)], axis=-1)


def inverse2(j: np.ndarray):
    """Inverse of 2x2 matrices j[..., alpha, a] -> k[..., a, alpha] and det (Cramer)."""
    det = (j[..., 0, 0] * j[..., 1, 1]) - (j[..., 0, 1] * j[..., 1, 0])
    k = np.empty_like(j)
    k[..., 0, 0] = j[..., 1, 1] / det
    k[..., 0, 1] = (-j[..., 0, 1]) / det
    k[..., 1, 0] = (-j[..., 1, 0]) / det
    k[..., 1, 1] = j[..., 0, 0] / det
    return k, det


def det3(m: np.ndarray) -> np.ndarray:
    """Determinant of 3x3 matrices by expansion along the first row."""
    c0 = (m[..., 1, 1] * m[..., 2, 2]) - (m[..., 1, 2] * m[..., 2, 1])
    c1 = (m[..., 1, 0] * m[..., 2, 2]) - (m[..., 1, 2] * m[..., 2, 0])
    c2 = (m[..., 1, 0] * m[..., 2, 1]) - (m[..., 1, 1] * m[..., 2, 0])
    return ((m[..., 0, 0] * c0) - (m[..., 0, 1] * c1)) + (m[..., 0, 2] * c2)


def inverse3(j: np.ndarray):
    """Inverse of 3x3 matrices by the adjugate: k[a, alpha] = cof(alpha, a) / det."""
    det = det3(j)
    k = np.empty_like(j)
    for a in range(3):
        for al in range(3):
            # cofactor of element (al, a) of j: rows != al, columns != a
            r = [x for x in range(3) if x != al]
            c = [x for x in range(3) if x != a]
            minor = (j[..., r[0], c[0]] * j[..., r[1], c[1]]) - (j[..., r[0], c[1]] * j[..., r[1], c[0]])
            sign = 1.0 if (al + a) % 2 == 0 else -1.0
            k[..., a, al] = (sign * minor) / det
    return k, det


def dot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dot product over the last axis, summed left to right."""
    acc = a[..., 0] * b[..., 0]
    for c in range(1, a.shape[-1]):
        acc = acc + (a[..., c] * b[..., c])
    return acc


def cross(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    out = np.empty_like(a)
    out[..., 0] = (a[..., 1] * b[..., 2]) - (a[..., 2] * b[..., 1])
    out[..., 1] = (a[..., 2] * b[..., 0]) - (a[..., 0] * b[..., 2])
    out[..., 2] = (a[..., 0] * b[..., 1]) - (a[..., 1] * b[..., 0])
    return out


@dataclass
class Geometry:
    """Metric of one logical grid (all FP64, cell units)."""

    dim: int
    n: tuple  # cells per logical axis (N1, N2[, N3])
    periodic: tuple
    X: np.ndarray  # vertices
    j: np.ndarray  # vertex Jacobi matrices [..., alpha, a]
    k: np.ndarray  # vertex inverse Jacobi matrices [..., a, alpha]
    Jc: np.ndarray  # cell Jacobians (cell area / volume)
    omega_c: np.ndarray  # cell geometric factor Omega
    face: list  # per axis a: coefficient arrays coef[b][face index] (Omega J g^{ab})
    axisym: bool = False  # Omega = r (2D cylindrical geometry with azimuthal symmetry)

    def k32(self) -> np.ndarray:
        """FP32 vertex table of k in cell units, [..., a, alpha] (round to nearest)."""
        return self.k.astype(np.float32)


def _cell_average_derivatives(X: np.ndarray) -> list:
    """Cell-centred dX/du^a from the mean of the cell's parallel edges (2 in 2D, 4 in 3D)."""
    D = X.ndim - 1
    out = []
    if D == 2:
        e0a = X[:-1, 1:] - X[:-1, :-1]  # edge (j, i)->(j, i+1)
        e0b = X[1:, 1:] - X[1:, :-1]  # edge (j+1, i)->(j+1, i+1)
        e1a = X[1:, :-1] - X[:-1, :-1]  # edge (j, i)->(j+1, i)
        e1b = X[1:, 1:] - X[:-1, 1:]  # edge (j, i+1)->(j+1, i+1)
        out.append((e0a + e0b) * 0.5)
        out.append((e1a + e1b) * 0.5)
        return out
    # 3D: X[k, j, i]
    e = []
    lo, hi = slice(None, -1), slice(1, None)
    # axis 0 (i): differences along i at the 4 (j,k) corners, summed in a fixed order
    e = [X[lo, lo, hi] - X[lo, lo, lo], X[lo, hi, hi] - X[lo, hi, lo],
         X[hi, lo, hi] - X[hi, lo, lo], X[hi, hi, hi] - X[hi, hi, lo]]
    out.append((((e[0] + e[1]) + e[2]) + e[3]) * 0.25)
    e = [X[lo, hi, lo] - X[lo, lo, lo], X[lo, hi, hi] - X[lo, lo, hi],
         X[hi, hi, lo] - X[hi, lo, lo], X[hi, hi, hi] - X[hi, lo, hi]]
    out.append((((e[0] + e[1]) + e[2]) + e[3]) * 0.25)
    e = [X[hi, lo, lo] - X[lo, lo, lo], X[hi, lo, hi] - X[lo, lo, hi],
         X[hi, hi, lo] - X[lo, hi, lo], X[hi, hi, hi] - X[lo, hi, hi]]
    out.append((((e[0] + e[1]) + e[2]) + e[3]) * 0.25)
    return out


def cell_jacobian(X: np.ndarray) -> np.ndarray:
    """J_c: determinant of the cell-averaged Jacobi matrix. In 2D this is exactly the area of
    the quadrilateral cell (cell units: Delta xi Delta eta = 1)."""
    D = X.ndim - 1
    d = _cell_average_derivatives(X)
    if D == 2:
        return (d[0][..., 0] * d[1][..., 1]) - (d[1][..., 0] * d[0][..., 1])
    m = np.stack(d, axis=-1)  # [..., alpha, a]
    return det3(m)


def cell_omega(X: np.ndarray, axisym: bool) -> np.ndarray:
    """Omega at cell centres: 1 (Cartesian) or r = x^1 averaged over the cell's vertices."""
    D = X.ndim - 1
    shape = tuple(s - 1 for s in X.shape[:-1])
    if not axisym:
        return np.ones(shape)
    r = X[..., 0]
    assert D == 2
    return (((r[:-1, :-1] + r[:-1, 1:]) + r[1:, :-1]) + r[1:, 1:]) * 0.25


def face_coefficients_2d(X, dv, axisym):
    """Face coefficients a^{ab} = Omega J g^{ab} (cell units) on the faces normal to each
    logical axis, eqs. (gcon), (poiscurv).

    xi-face (i, j) lies between cells (i-1, j) and (i, j), arrays of shape (N2, N1+1):
      x_v = X[j+1, i] - X[j, i] (the face edge), x_u = (dX/du[j, i] + dX/du[j+1, i]) * 0.5,
      J = x_u x x_v, a^{uu} = Omega |x_v|^2 / J, a^{uv} = -Omega (x_u . x_v) / J.
    eta-face (i, j) lies between cells (i, j-1) and (i, j), shape (N2+1, N1):
      x_u = X[j, i+1] - X[j, i], x_v = (dX/dv[j, i] + dX/dv[j, i+1]) * 0.5,
      a^{vv} = Omega |x_u|^2 / J, a^{vu} = -Omega (x_u . x_v) / J.
    Omega on a face is 1, or r averaged over the face's two vertices (axisymmetric)."""
    du, dvv = dv
    # xi-faces
    xv = X[1:, :, :] - X[:-1, :, :]
    xu = (du[:-1, :, :] + du[1:, :, :]) * 0.5
    J = (xu[..., 0] * xv[..., 1]) - (xv[..., 0] * xu[..., 1])
    om = (X[:-1, :, 0] + X[1:, :, 0]) * 0.5 if axisym else np.ones(J.shape)
    a_uu = (om * dot(xv, xv)) / J
    a_uv = -((om * dot(xu, xv)) / J)
    # eta-faces
    xu2 = X[:, 1:, :] - X[:, :-1, :]
    xv2 = (dvv[:, :-1, :] + dvv[:, 1:, :]) * 0.5
    J2 = (xu2[..., 0] * xv2[..., 1]) - (xv2[..., 0] * xu2[..., 1])
    om2 = (X[:, :-1, 0] + X[:, 1:, 0]) * 0.5 if axisym else np.ones(J2.shape)
    a_vv = (om2 * dot(xu2, xu2)) / J2
    a_vu = -((om2 * dot(xu2, xv2)) / J2)
    a_uv = np.where(np.abs(a_uv) <= CROSS_ROUNDOFF * np.abs(a_uu), 0.0, a_uv)
    a_vu = np.where(np.abs(a_vu) <= CROSS_ROUNDOFF * np.abs(a_vv), 0.0, a_vu)
    return [[a_uu, a_uv], [a_vu, a_vv]]


def face_coefficients_3d(X, dv):
    """3D face coefficients a^{ab} = J g^{ab} = J a^a . a^b with the contravariant basis
    a^a = (x_b x x_c)/J (cyclic). On the face normal to axis a: the across derivative is
    the mean of the vertex derivatives at the face's 4 vertices, each along derivative
    is the mean of the face's 2 parallel edges. Returns coef[a][b] with face arrays of
    shape (N3, N2, N1+1) for a = 0, (N3, N2+1, N1) for a = 1, (N3+1, N2, N1) for a = 2."""
    lo, hi, al = slice(None, -1), slice(1, None), slice(None)
    out = []
    for a in range(3):
        # index maps: the face is at vertex index along a, cell index along the others
        if a == 0:
            q = [X[lo, lo, al], X[lo, hi, al], X[hi, lo, al], X[hi, hi, al]]  # (k,j) corners
            dq = [dv[0][lo, lo, al], dv[0][lo, hi, al], dv[0][hi, lo, al], dv[0][hi, hi, al]]
            xa = (((dq[0] + dq[1]) + dq[2]) + dq[3]) * 0.25
            xb = ((q[1] - q[0]) + (q[3] - q[2])) * 0.5  # along j
            xc = ((q[2] - q[0]) + (q[3] - q[1])) * 0.5  # along k
            d = [xa, xb, xc]
        elif a == 1:
            q = [X[lo, al, lo], X[lo, al, hi], X[hi, al, lo], X[hi, al, hi]]  # (k,i) corners
            dq = [dv[1][lo, al, lo], dv[1][lo, al, hi], dv[1][hi, al, lo], dv[1][hi, al, hi]]
            xa = (((dq[0] + dq[1]) + dq[2]) + dq[3]) * 0.25
            xi_ = ((q[1] - q[0]) + (q[3] - q[2])) * 0.5  # along i
            xk = ((q[2] - q[0]) + (q[3] - q[1])) * 0.5  # along k
            d = [xi_, xa, xk]
        else:
            q = [X[al, lo, lo], X[al, lo, hi], X[al, hi, lo], X[al, hi, hi]]  # (j,i) corners
            dq = [dv[2][al, lo, lo], dv[2][al, lo, hi], dv[2][al, hi, lo], dv[2][al, hi, hi]]
            xa = (((dq[0] + dq[1]) + dq[2]) + dq[3]) * 0.25
            xi_ = ((q[1] - q[0]) + (q[3] - q[2])) * 0.5  # along i
            xj = ((q[2] - q[0]) + (q[3] - q[1])) * 0.5  # along j
            d = [xi_, xj, xa]
        # contravariant basis times J: A^b = x_{b+1} x x_{b+2}
        A = [cross(d[1], d[2]), cross(d[2], d[0]), cross(d[0], d[1])]
        J = dot(d[0], A[0])
        coef = [dot(A[a], A[b]) / J for b in range(3)]
        for b in range(3):
            if b != a:
                coef[b] = np.where(np.abs(coef[b]) <= CROSS_ROUNDOFF * np.abs(coef[a]), 0.0, coef[b])
        out.append(coef)
    return out


def build_geometry(X: np.ndarray, periodic, axisym: bool = False) -> Geometry:
    """Spec M: all metric quantities of a grid from its vertex map."""
    D = X.ndim - 1
    n = tuple(X.shape[D - 1 - a] - 1 for a in range(D))
    dv = [vertex_derivative(X, a, bool(periodic[a])) for a in range(D)]
    j = np.stack(dv, axis=-1)
    if D == 2:
        k, _ = inverse2(j)
        face = face_coefficients_2d(X, dv, axisym)
    else:
        k, _ = inverse3(j)
        face = face_coefficients_3d(X, dv)
    return Geometry(
        dim=D, n=n, periodic=tuple(bool(p) for p in periodic), X=X, j=j, k=k,
        Jc=cell_jacobian(X), omega_c=cell_omega(X, axisym), face=face, axisym=bool(axisym),
    )
