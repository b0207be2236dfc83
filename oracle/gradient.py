"""Spec G: the logical field at vertices from the cell-centred potential.

Sec. II.B (staggered layout): phi and the density live at cell centres, the electric field
at vertices. The paper gives no formula for the vertex field; this implementation's
reading: in cell units, G^a_v = d phi / d u^a at vertex v is the mean, over the 2^(D-1)
pairs of cells that straddle v along axis a, of the cell difference:
  2D: G^0(i, j) = ((phi(i, j-1) - phi(i-1, j-1)) + (phi(i, j) - phi(i-1, j))) * 0.5
      G^1(i, j) = ((phi(i-1, j) - phi(i-1, j-1)) + (phi(i, j) - phi(i, j-1))) * 0.5
  3D: the 4 differences summed in the order (lo, lo), (hi, lo), (lo, hi), (hi, hi) of the
      two other axes (first other axis fastest), times 0.25.
Cells outside the grid are ghost cells (Dirichlet 2 phi_b - phi_in, Neumann phi_in,
periodic wrap), resolved axis by axis starting from axis 0. The physical field is then
E^alpha = -sum_a G^a k^{a alpha}. G is rounded to FP32 once (round to nearest).
"""
from __future__ import annotations

import numpy as np

from .poisson import BC_DIRICHLET, BC_NEUMANN, BC_PERIODIC


def ghost_extend(phi, bc, bcval):
    """Pad phi (numpy cell layout) by one ghost layer on every side, per the face BCs.
    Axis 0 (xi) is padded first, so corner ghosts apply the later axes' rule to ghosts."""
    D = phi.ndim
    out = phi
    for a in range(D):
        ax = D - 1 - a
        m = np.moveaxis(out, ax, 0)
        first, last = m[0], m[-1]
        res = []
        for side, inner, opposite in ((0, first, last), (1, last, first)):
            kind = bc[2 * a + side]
            if kind == BC_PERIODIC:
                res.append(opposite)
            elif kind == BC_NEUMANN:
                res.append(inner)
            elif kind == BC_DIRICHLET:
                res.append(2.0 * bcval[2 * a + side] - inner)
            else:
                raise ValueError(kind)
        m = np.concatenate([res[0][None], m, res[1][None]], axis=0)
        out = np.moveaxis(m, 0, ax)
    return out


def vertex_gradient(phi, bc, bcval):
    """G[..., a] at all vertices (numpy vertex layout (N2+1, N1+1, D) / (N3+1, ..., D)),
    FP64, cell units."""
    D = phi.ndim
    P = ghost_extend(phi, bc, bcval)  # shape N + 2 per axis; P[g] = phi[g - 1]
    if D == 2:
        # vertex (j, i) touches cells (j-1..j, i-1..i) = P[j..j+1, i..i+1]
        p00 = P[:-1, :-1]  # (j-1, i-1)
        p01 = P[:-1, 1:]  # (j-1, i)
        p10 = P[1:, :-1]  # (j, i-1)
        p11 = P[1:, 1:]  # (j, i)
        g0 = ((p01 - p00) + (p11 - p10)) * 0.5
        g1 = ((p10 - p00) + (p11 - p01)) * 0.5
        return np.stack([g0, g1], axis=-1)
    # 3D: vertex (k, j, i) touches P[k..k+1, j..j+1, i..i+1]
    c = {}
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                c[(di, dj, dk)] = P[dk : P.shape[0] - 1 + dk, dj : P.shape[1] - 1 + dj, di : P.shape[2] - 1 + di]
    out = []
    for a in range(3):
        others = [b for b in range(3) if b != a]
        acc = None
        for ob in (0, 1):  # second other axis (slow)
            for oa in (0, 1):  # first other axis (fast)
                lo = [0, 0, 0]
                hi = [0, 0, 0]
                lo[others[0]] = hi[others[0]] = oa
                lo[others[1]] = hi[others[1]] = ob
                hi[a] = 1
                d = c[tuple(hi)] - c[tuple(lo)]
                acc = d if acc is None else acc + d
        out.append(acc * 0.25)
    return np.stack(out, axis=-1)
