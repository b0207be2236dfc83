"""Spec Q: b2 charge assignment, Sec. II.B.1 eqs. (pg), (Wpc), (b2), in 64-bit fixed point.

Eq. (b2) as printed gives (3/2 - |xi|)^2 for 1/2 < |xi| < 3/2; that branch is
discontinuous at |xi| = 1/2 and the weights do not sum to one. Reading: the standard
quadratic B-spline 1/2 (3/2 - |xi|)^2 (Birdsall & Langdon, the reference the paper cites
for its assignment functions). b2 is assigned to the 3^D cell centres around the particle
(density lives at cell centres, Sec. II.B).

Fixed-point spec (constants QK = 16, QB = 16, QF = 24):
  per axis: u = floor(t * 2^QK) (exact for an FP32 offset), s = 2u + 1 - 2^QK (odd,
  |s| < 2^QK), integer weights for nodes m = -1, 0, +1:
    W[-1] = (2^QK - s)^2,  W[0] = 2 (3 * 2^(2 QK) - s^2),  W[+1] = (2^QK + s)^2,
  which are b2 at the sub-cell centre offset d = s / 2^(QK+1) scaled by 2^(2 QK + 3) and
  sum to exactly 2^(2 QK + 3);
  per-axis weights at QB bits, outer ones rounded to nearest (halves up), the centre one
  the remainder:  w[+-1] = (W[+-1] + 2^(h-1)) >> h  with h = 2 QK + 3 - QB,
                  w[0] = 2^QB - w[-1] - w[+1]   (so the three sum to exactly 2^QB);
  node weights: the exact product p(m) = prod_a w_a[m_a] (eq. (Wpc) builds the
  multidimensional weight as a product of one-dimensional ones), rounded to QF bits for
  every node but the centre, q(m) = (p(m) + 2^(r-1)) >> r with r = D QB - QF, and the
  centre node m = 0 takes the remainder q(0) = 2^QF - sum_{m != 0} q(m), so the 3^D node
  weights of a particle sum to exactly 2^QF (charge conservation is exact, P5) and every
  node weight is below 2^QF.
  Node cells outside a non-periodic axis fold onto the boundary cell (charge kept);
  periodic axes wrap.
Resolution: offsets to 2^-16 of a cell, per-axis weights to 2^-17, node weights to 2^-25 of
one particle; the resulting potential differs from the one of the unquantised FP64 deposit
by a few 1e-7 (2D) to a few 1e-6 (3D) relative L2, pinned by the tests.
"""
from __future__ import annotations

import itertools

import numpy as np

QK = 16
QB = 16
QF = 24


def b1(x):
    """Linear B-spline, eq. (b1)."""
    ax = np.abs(x)
    return np.where(ax < 1.0, 1.0 - ax, 0.0)


def b2(x):
    """Quadratic B-spline, eq. (b2) with the 1/2 of the outer branch restored."""
    ax = np.abs(x)
    return np.where(ax < 0.5, 0.75 - ax * ax, np.where(ax < 1.5, 0.5 * (1.5 - ax) ** 2, 0.0))


def b2_as_printed(x):
    """Eq. (b2) exactly as printed (outer branch without the 1/2): used only by the test
    that documents the garbled constant."""
    ax = np.abs(x)
    return np.where(ax < 0.5, 0.75 - ax * ax, np.where(ax < 1.5, (1.5 - ax) ** 2, 0.0))


def axis_weights(t32: np.ndarray):
    """Integer per-axis weights W[m+1] (int64 arrays) from float32 offsets t in [0, 1)."""
    t32 = np.asarray(t32, dtype=np.float32)
    u = np.floor(t32.astype(np.float64) * float(1 << QK)).astype(np.int64)
    s = 2 * u + 1 - (1 << QK)
    one = np.int64(1 << QK)
    return [(one - s) ** 2, 2 * (3 * one * one - s * s), (one + s) ** 2]


def axis_weights_fixed(t32: np.ndarray):
    """Per-axis weights w[m+1] at QB bits (int64 arrays), summing to 2^QB."""
    h = 2 * QK + 3 - QB
    W = axis_weights(t32)
    wm = (W[0] + (1 << (h - 1))) >> h
    wp = (W[2] + (1 << (h - 1))) >> h
    return [wm, (1 << QB) - wm - wp, wp]


def node_products(t32: np.ndarray):
    """Exact products p(m) = prod_a w_a[m_a] of the per-axis weights (int64; at most 48
    bits). Returns dict offset tuple -> int64 array (n,)."""
    D = t32.shape[0]
    w = [axis_weights_fixed(t32[a]) for a in range(D)]
    out = {}
    for m in itertools.product((-1, 0, 1), repeat=D):
        q = np.ones(t32.shape[1], dtype=np.int64)
        for a in range(D):
            q = q * w[a][m[a] + 1]
        out[m] = q
    return out


def node_weights(t32: np.ndarray):
    """Fixed-point node weights for particles with offsets t32 (D, n): the products rounded
    to QF bits, the centre node the remainder. Returns dict offset tuple (m0, m1[, m2]) ->
    int64 array (n,)."""
    D = t32.shape[0]
    r = D * QB - QF
    p = node_products(t32)
    centre = (0,) * D
    out = {}
    rest = np.zeros(t32.shape[1], dtype=np.int64)
    for m, pm in p.items():
        if m == centre:
            continue
        q = (pm + (1 << (r - 1))) >> r
        out[m] = q
        rest = rest + q
    out[centre] = (1 << QF) - rest
    return dict(sorted(out.items()))


def deposit_fixed(idx: np.ndarray, t32: np.ndarray, n, periodic) -> np.ndarray:
    """Accumulate int64 charge counts (numpy cell layout) for live particles with per-axis
    cell indices idx (D, n) and float32 offsets t32 (D, n)."""
    D = len(n)
    C = np.zeros(int(np.prod(n)), dtype=np.int64)
    for m, q in node_weights(t32).items():
        lin = np.zeros(idx.shape[1], dtype=np.int64)
        for a in reversed(range(D)):
            c = idx[a].astype(np.int64) + m[a]
            if periodic[a]:
                c = np.mod(c, n[a])
            else:
                c = np.clip(c, 0, n[a] - 1)
            lin = lin * n[a] + c
        np.add.at(C, lin, q)
    return C.reshape(tuple(reversed(n)))


def deposit_exact(idx: np.ndarray, t: np.ndarray, n, periodic) -> np.ndarray:
    """FP64 b2 deposit (no quantisation), same folding rules: eq. (pg) numerator with unit
    charge per particle."""
    D = len(n)
    C = np.zeros(int(np.prod(n)), dtype=np.float64)
    d = np.asarray(t, dtype=np.float64) - 0.5  # offset from the cell centre
    for m in itertools.product((-1, 0, 1), repeat=D):
        w = np.ones(idx.shape[1])
        lin = np.zeros(idx.shape[1], dtype=np.int64)
        for a in range(D):
            w = w * b2(d[a] - m[a])
        for a in reversed(range(D)):
            c = idx[a].astype(np.int64) + m[a]
            c = np.mod(c, n[a]) if periodic[a] else np.clip(c, 0, n[a] - 1)
            lin = lin * n[a] + c
        np.add.at(C, lin, w)
    return C.reshape(tuple(reversed(n)))


def deposit_exact_c(idx: np.ndarray, t: np.ndarray, n, periodic, threads: int = 1) -> np.ndarray:
    """deposit_exact as C loops (oracle/pic64.c); with threads > 1 each thread deposits a
    contiguous block of particles into its own grid, added in thread order."""
    from .mover import _lib64, _ptr

    D = len(n)
    C = np.zeros(int(np.prod(n)), dtype=np.float64)
    idx_c = np.ascontiguousarray(idx, dtype=np.int64)
    t_c = np.ascontiguousarray(t, dtype=np.float64)
    nn = np.asarray(list(n) + [1] * (3 - D), dtype=np.int32)
    per = np.asarray(list(periodic) + [0] * (3 - D), dtype=np.int32)
    if _lib64().oracle_deposit64(D, _ptr(nn), _ptr(per), idx_c.shape[1], _ptr(idx_c), _ptr(t_c), _ptr(C),
                                 int(threads)) != 0:
        raise MemoryError("oracle_deposit64: per-thread grids")
    return C.reshape(tuple(reversed(n)))
