"""Spec P: conservative finite-volume logical-space Poisson problem and its direct solve.

Sec. II.B.3: second-order conservative discretisation of eq. (poiscurv), boundary
conditions imposed through ghost cells; Sec. II.B (normalised units, eps0 = 1).

Integrating eq. (poiscurv) over a cell (cell units, unit logical volume) gives
  sum over faces of the outward flux  Omega J g^{ab} d_b phi  =  -Omega_c Q_c,
with Q_c the charge in the cell. The flux through the face normal to axis a is
  F = a^{aa} (phi_right - phi_left) + sum_{b != a} a^{ab} D_b phi,
  D_b phi = ((phi_R(+b) + phi_L(+b)) - (phi_R(-b) + phi_L(-b))) / 4,
with a^{ab} = Omega J g^{ab} from spec M. Ghost cells (reading of "boundary conditions
via ghost cells"): Dirichlet ghost = 2 phi_b - phi_in, Neumann ghost = phi_in, periodic
wraps. On a Dirichlet boundary face the flux is a^{aa} * 2 (phi_in - phi_b) (normal part;
the tangential derivative of a constant boundary value is zero); on a Neumann face the flux
is zero.

The assembled system is M phi = Omega Q + b_bc with M = -(divergence operator), so M is
positive (semi)definite for orthogonal maps. For a singular problem (no Dirichlet face)
the right-hand side is projected onto the range by subtracting a uniform physical charge
density, and the gauge sum_c J_c phi_c = 0 is imposed (reading: the paper is silent).
The solve is a sparse direct factorisation (scipy SuperLU), a library primitive.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
FIXED_POINT_BITS = 24  # spec Q: one particle deposits exactly 2^24 charge units


def _lin(idx, n):
    """Linear cell index i + N1 (j + N2 k) of per-axis index arrays."""
    lin = np.zeros_like(idx[0])
    for a in reversed(range(len(n))):
        lin = lin * n[a] + idx[a]
    return lin


def _resolve(idx, n, bc, bcval):
    """Ghost resolution of cells idx (list of per-axis arrays; at most one axis out of
    range per cell). Returns (linear index, coefficient, constant)."""
    D = len(n)
    idx = [x.copy() for x in idx]
    coef = np.ones(idx[0].shape)
    const = np.zeros(idx[0].shape)
    for a in range(D):
        for side, bad in ((0, idx[a] < 0), (1, idx[a] >= n[a])):
            if not bad.any():
                continue
            kind = bc[2 * a + side]
            if kind == BC_PERIODIC:
                idx[a][bad] = np.mod(idx[a][bad], n[a])
            else:
                idx[a][bad] = 0 if side == 0 else n[a] - 1
                if kind == BC_DIRICHLET:
                    coef[bad] *= -1.0
                    const[bad] = 2.0 * bcval[2 * a + side]
    return _lin(idx, n), coef, const


def _face_indices(n, a, periodic):
    """Per-axis index arrays of all faces normal to axis a (face index along a is the
    vertex index; a periodic axis omits the duplicate face N_a)."""
    D = len(n)
    ranges = []
    for b in range(D):
        if b == a:
            ranges.append(np.arange(n[a] if periodic else n[a] + 1))
        else:
            ranges.append(np.arange(n[b]))
    grids = np.meshgrid(*ranges, indexing="ij")
    return [g.ravel() for g in grids]


def _coef_at(coef, idx, D):
    """Fetch a face coefficient array (numpy layout, axis a = numpy axis D-1-a)."""
    return coef[tuple(idx[D - 1 - x] for x in range(D))]


def assemble(geom, bc, bcval):
    """Assemble M (CSR) and b_bc with M phi = Omega Q + b_bc (see module docstring)."""
    D, n = geom.dim, geom.n
    N = int(np.prod(n))
    rows, cols, vals = [], [], []
    bbc = np.zeros(N)

    def add(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for a in range(D):
        per = bc[2 * a] == BC_PERIODIC
        f = _face_indices(n, a, per)
        c_aa = _coef_at(geom.face[a][a], f, D)
        left = [x.copy() for x in f]
        left[a] = f[a] - 1
        right = [x.copy() for x in f]
        interior = np.ones(f[0].shape, bool) if per else (f[a] > 0) & (f[a] < n[a])
        lo = (~interior) & (f[a] == 0)
        hi = (~interior) & (f[a] == n[a])
        # ---- interior (or periodic) faces
        sel = interior
        fl = [x[sel] for x in left]
        fr = [x[sel] for x in right]
        Lc, _, _ = _resolve(fl, n, bc, bcval)
        Rc, _, _ = _resolve(fr, n, bc, bcval)
        terms = [(Rc, np.ones(Lc.shape), np.zeros(Lc.shape), c_aa[sel]),
                 (Lc, -np.ones(Lc.shape), np.zeros(Lc.shape), c_aa[sel])]
        for b in range(D):
            if b == a:
                continue
            c_ab = _coef_at(geom.face[a][b], f, D)[sel] * 0.25
            for sgn in (+1, -1):
                for base in (fr, fl):
                    m = [x.copy() for x in base]
                    m[b] = m[b] + sgn
                    idx, cf, cst = _resolve(m, n, bc, bcval)
                    terms.append((idx, cf * sgn, cst * sgn, c_ab))
        for tgt, cf, cst, cc in terms:
            add(Lc, tgt, -(cc * cf))
            add(Rc, tgt, cc * cf)
            np.add.at(bbc, Lc, cc * cst)
            np.add.at(bbc, Rc, -(cc * cst))
        # ---- boundary faces
        for side, sel_b in ((0, lo), (1, hi)):
            if not sel_b.any():
                continue
            kind = bc[2 * a + side]
            if kind != BC_DIRICHLET:
                continue  # Neumann: zero flux
            cell = [x[sel_b].copy() for x in (right if side == 0 else left)]
            ci = _lin(cell, n)
            cc = 2.0 * c_aa[sel_b]
            add(ci, ci, cc)
            np.add.at(bbc, ci, cc * bcval[2 * a + side])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    M = sp.csr_matrix((v, (r, c)), shape=(N, N))
    M.sum_duplicates()
    return M, bbc


def charge_in_cells(geom, charge_counts, qw, background):
    """Q_c: sum_s q_s w_s C_{s,c} 2^-F plus a uniform background density times the cell
    volume J_c (eq. (pg) with the J_c of the density cancelled against the cell volume).
    charge_counts: list of int64 arrays (numpy cell layout), one per species.
    Axisymmetric runs (Omega = r): a macro-particle is a ring of charge q w around the axis,
    so its charge density is q w / (2 pi r J) and the right-hand side Omega_c Q_c needs
    Q_c = (sum of ring charges) / (2 pi Omega_c) for the particles."""
    Q = background * geom.Jc
    scale = 1.0 / (2.0 * np.pi * geom.omega_c) if geom.axisym else 1.0
    for C, f in zip(charge_counts, qw):
        Q = Q + (f * np.ldexp(C.astype(np.float64), -FIXED_POINT_BITS)) * scale
    return Q


def is_singular(bc, D):
    return not any(bc[f] == BC_DIRICHLET for f in range(2 * D))


def solve(geom, M, bbc, Q, bc):
    """Solve M phi = Omega Q + b_bc directly (FP64). Returns phi in numpy cell layout."""
    D = geom.dim
    rhs = (geom.omega_c * Q).ravel(order="C") + bbc
    J = geom.Jc.ravel(order="C")
    if is_singular(bc, D):
        rhs = rhs - (rhs.sum() / J.sum()) * J
        N = rhs.size
        Jcol = sp.csr_matrix(J.reshape(N, 1))
        Big = sp.bmat([[M, Jcol], [Jcol.T, None]], format="csc")
        sol = spla.spsolve(Big, np.concatenate([rhs, [0.0]]))
        phi = sol[:N]
    else:
        phi = spla.spsolve(M.tocsc(), rhs)
    return phi.reshape(geom.Jc.shape)


class DirectSolver:
    """solve() with the sparse LU factorisation (scipy SuperLU, a library primitive) kept
    between calls: the operator of a run does not change, only the charge does."""

    def __init__(self, geom, M, bbc, bc):
        self.geom, self.bbc, self.bc = geom, bbc, bc
        self.singular = is_singular(bc, geom.dim)
        self.J = geom.Jc.ravel(order="C")
        if self.singular:
            N = self.J.size
            Jcol = sp.csr_matrix(self.J.reshape(N, 1))
            self.lu = spla.splu(sp.bmat([[M, Jcol], [Jcol.T, None]], format="csc"))
        else:
            self.lu = spla.splu(M.tocsc())

    def __call__(self, Q):
        rhs = (self.geom.omega_c * Q).ravel(order="C") + self.bbc
        if self.singular:
            rhs = rhs - (rhs.sum() / self.J.sum()) * self.J
            phi = self.lu.solve(np.concatenate([rhs, [0.0]]))[: rhs.size]
        else:
            phi = self.lu.solve(rhs)
        return phi.reshape(self.geom.Jc.shape)


def residual_norm(M, bbc, geom, Q, phi, bc):
    """Relative residual ||rhs - M phi|| / ||rhs|| (with the singular-case projection)."""
    rhs = (geom.omega_c * Q).ravel() + bbc
    if is_singular(bc, geom.dim):
        J = geom.Jc.ravel()
        rhs = rhs - (rhs.sum() / J.sum()) * J
    r = rhs - M @ phi.ravel()
    return float(np.linalg.norm(r) / max(np.linalg.norm(rhs), 1e-300))
