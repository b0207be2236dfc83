/*
 * FP64 hybrid mover and exact b2 deposit of the oracle, as plain C loops (test
 * infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use it).
 *
 * The definitions are those of mover.py::push64 and deposit.py::deposit_exact, written as a
 * loop over particles so that long oracle runs (the OML current check, whole-run
 * comparisons with the device, the CPU baseline) finish in seconds:
 *   push (Sec. II.B.4, eqs. (step1)-(step4)): b1 gather (eqs. (vvp), (Wvp), (b1))
 *     of k and of the logical field G at xi^n; E = -k^T G; v += dt (q/m) E (with a
 *     uniform B0: the Boris step); predictor
 *     xi' = xi^n + dt/2 k(xi^n) v (clamped into a non-periodic axis); k(xi') by b1
 *     gather; corrector xi^{n+1} = xi^n + dt k(xi') v; periodic wrap, absorption (a cell
 *     index < 0 or >= N on an absorbing axis removes the particle), specular reflection
 *     (mirror about the face in logical space, velocity reflected about row a of k(xi'));
 *   deposit (Sec. II.B.1, eqs. (pg), (Wpc), (b2) with the 1/2 of the outer branch
 *     restored): weight prod_a b2(t_a - 1/2 - m_a) on the 3^D cell centres around the
 *     particle, folded onto the boundary cell of a non-periodic axis, wrapped on a periodic
 *     one.
 * Same operation order as the numpy form where that form fixes one (corner order of the
 * gathers, left-to-right products), compiled with -ffp-contract=off.
 *
 * The particle loop may be split over OpenMP threads: static contiguous blocks; each thread
 * deposits into its own grid and the grids are added in thread order, so one thread count
 * always gives one result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { PBC_PERIODIC = 0, PBC_ABSORB = 1, PBC_REFLECT = 2 };

int oracle_openmp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* vertex linear index i + (N1 + 1) (j + (N2 + 1) k) */
static long vertex_index(int D, const int* n, const long* c) {
    long v = c[D - 1];
    for (int a = D - 2; a >= 0; --a) v = v * (n[a] + 1) + c[a];
    return v;
}

/* b1 interpolation of a vertex table with `comp` values per vertex at cell c, offsets t:
 * corners in the order of itertools.product((0, 1), repeat=D) (axis 0 the slowest), each
 * weighted by the product over axes of t_a (upper corner) or 1 - t_a (lower corner) */
static void gather(int D, const int* n, const double* tab, int comp, const long* c, const double* t, double* out) {
    for (int q = 0; q < comp; ++q) out[q] = 0.0;
    for (int k = 0; k < (1 << D); ++k) {
        long cv[3];
        double w = 1.0;
        for (int a = 0; a < D; ++a) {
            const int o = (k >> (D - 1 - a)) & 1;
            w = w * (o ? t[a] : 1.0 - t[a]);
            cv[a] = c[a] + o;
        }
        const double* val = tab + vertex_index(D, n, cv) * comp;
        for (int q = 0; q < comp; ++q) out[q] = out[q] + w * val[q];
    }
}

/* split renormalisation: c = floor(x), f = x - c, f = 1 -> (0, c + 1) */
static void renorm(double x, long* c, double* f) {
    double cf = floor(x);
    double fr = x - cf;
    if (fr >= 1.0) {
        fr = 0.0;
        cf = cf + 1.0;
    }
    *c = (long)cf;
    *f = fr;
}

static long wrap(long c, long n) {
    long r = c % n;
    return r < 0 ? r + n : r;
}

/* Boris step (FP64, the numpy form's order): v- = v + h E, v' = v- + v- x t,
 * v+ = v- + v' x s, v = v+ + h E, t = h B, s = 2 t / (1 + |t|^2), h = dt q/m / 2 */
static void boris64(double* v, const double* E, double h, const double* B) {
    double t[3], s[3], m[3], q[3];
    for (int a = 0; a < 3; ++a) t[a] = h * B[a];
    const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + tt);
    for (int a = 0; a < 3; ++a) m[a] = v[a] + h * E[a];
    q[0] = m[0] + (m[1] * t[2] - m[2] * t[1]);
    q[1] = m[1] + (m[2] * t[0] - m[0] * t[2]);
    q[2] = m[2] + (m[0] * t[1] - m[1] * t[0]);
    v[0] = m[0] + (q[1] * s[2] - q[2] * s[1]) + h * E[0];
    v[1] = m[1] + (q[2] * s[0] - q[0] * s[2]) + h * E[1];
    v[2] = m[2] + (q[0] * s[1] - q[1] * s[0]) + h * E[2];
}

/* The exact motion in the uniform field alone over dt (mover.py gyro_flow64, same order):
 * gy = (b0, b1, b2, cos th, sin th, f1, f2); u = v x b, par = (v . b) b, perp = v - par;
 * v' = (par + cos th perp) + sin th u, d = dt ((par + f1 perp) + f2 u). */
static void gyro_flow64(const double* v, double dt, const double* gy, double* d, double* vn) {
    const double* b = gy;
    const double vpar = v[0] * b[0] + v[1] * b[1] + v[2] * b[2];
    const double u[3] = {v[1] * b[2] - v[2] * b[1], v[2] * b[0] - v[0] * b[2], v[0] * b[1] - v[1] * b[0]};
    for (int a = 0; a < 3; ++a) {
        const double par = vpar * b[a], perp = v[a] - par;
        vn[a] = (par + gy[3] * perp) + gy[4] * u[a];
        d[a] = dt * ((par + gy[5] * perp) + gy[6] * u[a]);
    }
}

static void push_one(int D, const int* n, const int* pbc, const double* K, const double* G, double dt, double qm,
                     const double* B, const double* R, const double* gy, long* c, double* t, double* v,
                     int* face_out, double* vdot_out) {
    double kp[9], gp[3], E[3], vold[3];
    gather(D, n, K, D * D, c, t, kp);
    gather(D, n, G, D, c, t, gp);
    for (int b = 0; b < D; ++b) {
        double e = 0.0;
        for (int a = 0; a < D; ++a) e = e + gp[a] * kp[a * D + b];
        E[b] = -e;
    }
    for (int q = 0; q < 3; ++q) vold[q] = v[q];
    if (B) {
        double E3[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < D; ++b) E3[b] = E[b];
        boris64(v, E3, 0.5 * dt * qm, B);
    } else {
        const double dtqm = dt * qm;
        for (int b = 0; b < D; ++b) v[b] = v[b] + dtqm * E[b];
    }
    double vk[3] = {v[0], v[1], v[2]};
    /* axisymmetric run: the meridional displacement of straight 3D motion over the step and
     * the frame's turn (mover.py axisym_step); cyclotronic push: the gyration flow's
     * displacement and velocity, then (axisymmetric) the frame step (mover.py axisym_frame) */
    double disp[3] = {0.0, 0.0, 0.0}, vrot[3] = {v[0], v[1], v[2]};
    const int dform = gy != 0 || R != 0;
    if (gy) {
        double d3[3], vn[3];
        gyro_flow64(v, dt, gy, d3, vn);
        for (int q = 0; q < 3; ++q) vrot[q] = vn[q];
        if (R) {
            double rn;
            gather(D, n, R, 1, c, t, &rn);
            const double x = rn + d3[0], y = d3[2];
            const double r1 = sqrt(x * x + y * y);
            const double ca = r1 > 0.0 ? x / r1 : 1.0, sa = r1 > 0.0 ? y / r1 : 0.0;
            disp[0] = r1 - rn;
            disp[1] = d3[1];
            vrot[0] = ca * vn[0] + sa * vn[2];
            vrot[2] = ca * vn[2] - sa * vn[0];
        } else {
            for (int q = 0; q < D; ++q) disp[q] = d3[q];
        }
    } else if (R) {
        double rn;
        gather(D, n, R, 1, c, t, &rn);
        const double x = rn + dt * v[0], y = dt * v[2];
        const double r1 = sqrt(x * x + y * y);
        const double ca = r1 > 0.0 ? x / r1 : 1.0, sa = r1 > 0.0 ? y / r1 : 0.0;
        disp[0] = r1 - rn;
        disp[1] = dt * v[1];
        vrot[0] = ca * v[0] + sa * v[2];
        vrot[2] = ca * v[2] - sa * v[0];
    }
    /* predictor: in 2D only the in-plane velocity moves xi */
    long ip[3];
    double tp[3];
    for (int a = 0; a < D; ++a) {
        double d = 0.0;
        long dc;
        if (dform) {
            for (int b = 0; b < D; ++b) d = d + kp[a * D + b] * disp[b];
            renorm(t[a] + 0.5 * d, &dc, &tp[a]);
        } else {
            for (int b = 0; b < D; ++b) d = d + kp[a * D + b] * v[b];
            renorm(t[a] + (0.5 * dt) * d, &dc, &tp[a]);
        }
        ip[a] = c[a] + dc;
        if (pbc[2 * a] == PBC_PERIODIC) {
            ip[a] = wrap(ip[a], n[a]);
        } else if (ip[a] < 0) {
            ip[a] = 0;
            tp[a] = 0.0;
        } else if (ip[a] >= n[a]) {
            ip[a] = n[a] - 1;
            tp[a] = 1.0;
        }
    }
    double kq[9];
    gather(D, n, K, D * D, ip, tp, kq);
    long cn[3];
    double tn[3];
    for (int a = 0; a < D; ++a) {
        double d = 0.0;
        long dc;
        if (dform) {
            for (int b = 0; b < D; ++b) d = d + kq[a * D + b] * disp[b];
            renorm(t[a] + d, &dc, &tn[a]);
        } else {
            for (int b = 0; b < D; ++b) d = d + kq[a * D + b] * v[b];
            renorm(t[a] + dt * d, &dc, &tn[a]);
        }
        cn[a] = c[a] + dc;
    }
    if (dform)
        for (int q = 0; q < 3; ++q) v[q] = vrot[q];
    int face = -1;
    for (int a = 0; a < D; ++a) {
        if (pbc[2 * a] == PBC_PERIODIC) {
            cn[a] = wrap(cn[a], n[a]);
        } else if (pbc[2 * a] == PBC_ABSORB && face < 0) {
            if (cn[a] < 0) face = 2 * a;
            else if (cn[a] >= n[a]) face = 2 * a + 1;
        }
    }
    *vdot_out = vold[0] * vk[0] + vold[1] * vk[1] + vold[2] * vk[2];
    for (int a = 0; a < D; ++a) {
        if (pbc[2 * a] != PBC_REFLECT || face >= 0 || (cn[a] >= 0 && cn[a] < n[a])) continue;
        const int below = cn[a] < 0;
        long c2 = below ? -cn[a] - 1 : 2L * n[a] - 1 - cn[a];
        long add;
        double t2;
        renorm(1.0 - tn[a], &add, &t2);
        c2 += add;
        if (c2 < 0 || c2 >= n[a]) {
            face = 2 * a + (below ? 0 : 1);
            continue;
        }
        cn[a] = c2;
        tn[a] = t2;
        double nn = 0.0, dot = 0.0;
        for (int b = 0; b < D; ++b) {
            nn = nn + kq[a * D + b] * kq[a * D + b];
            dot = dot + v[b] * kq[a * D + b];
        }
        const double s = 2.0 * dot / nn;
        for (int b = 0; b < D; ++b) v[b] = v[b] - s * kq[a * D + b];
    }
    for (int a = 0; a < D; ++a) {
        c[a] = cn[a];
        t[a] = tn[a];
    }
    *face_out = face;
}

/* One FP64 push of np particles (arrays in the numpy layout: idx, t [D][np], v [3][np],
 * updated in place); K: vertex k table [vertex][a][alpha], G: [vertex][a]; face[p] = -1
 * (alive) or 2 a + side (removed there); vdot[p] = v^{n-1/2} . v^{n+1/2} (the kicked
 * velocity, before any reflection). B: the uniform field for the Boris step (component
 * basis) or NULL; gy: the cyclotronic push's gyro constants (mover.py gyro_constants64) or
 * NULL; R: the vertex radius table of an axisymmetric run or NULL. */
void oracle_push64(int D, const int* n, const int* pbc, long np, int64_t* idx, double* t, double* v,
                   const double* K, const double* G, double dt, double qm, int32_t* face, double* vdot,
                   int nthreads, const double* B, const double* R, const double* gy) {
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (long p = 0; p < np; ++p) {
        long c[3];
        double tt[3], vv[3];
        for (int a = 0; a < D; ++a) {
            c[a] = (long)idx[a * np + p];
            tt[a] = t[a * np + p];
        }
        for (int q = 0; q < 3; ++q) vv[q] = v[q * np + p];
        int f;
        push_one(D, n, pbc, K, G, dt, qm, B, R, gy, c, tt, vv, &f, &vdot[p]);
        for (int a = 0; a < D; ++a) {
            idx[a * np + p] = c[a];
            t[a * np + p] = tt[a];
        }
        for (int q = 0; q < 3; ++q) v[q * np + p] = vv[q];
        face[p] = f;
    }
}

/* eq. (b2) with the restored 1/2 */
static double b2(double x) {
    const double ax = fabs(x);
    if (ax < 0.5) return 0.75 - ax * ax;
    if (ax < 1.5) return 0.5 * ((1.5 - ax) * (1.5 - ax));
    return 0.0;
}

static void deposit_range(int D, const int* n, const int* periodic, long np, long p0, long p1, const int64_t* idx,
                          const double* t, double* C) {
    int nn = 1;
    for (int a = 0; a < D; ++a) nn *= 3;
    for (long p = p0; p < p1; ++p) {
        double d[3];
        for (int a = 0; a < D; ++a) d[a] = t[a * np + p] - 0.5;
        for (int k = 0; k < nn; ++k) {
            int m[3];
            int r = k;
            for (int a = D - 1; a >= 0; --a) {  /* itertools.product order: axis 0 slowest */
                m[a] = r % 3 - 1;
                r /= 3;
            }
            double w = 1.0;
            for (int a = 0; a < D; ++a) w = w * b2(d[a] - m[a]);
            long lin = 0;
            for (int a = D - 1; a >= 0; --a) {
                long c = (long)idx[a * np + p] + m[a];
                if (periodic[a]) c = wrap(c, n[a]);
                else c = c < 0 ? 0 : (c >= n[a] ? n[a] - 1 : c);
                lin = lin * n[a] + c;
            }
            C[lin] = C[lin] + w;
        }
    }
}

/* Exact FP64 b2 deposit (unit charge per particle) added into C (cells, i fastest). */
int oracle_deposit64(int D, const int* n, const int* periodic, long np, const int64_t* idx, const double* t,
                     double* C, int nthreads) {
    long ncell = 1;
    for (int a = 0; a < D; ++a) ncell *= n[a];
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1) {
        deposit_range(D, n, periodic, np, 0, np, idx, t, C);
        return 0;
    }
    double* part = (double*)calloc((size_t)nthreads * (size_t)ncell, sizeof(double));
    if (!part) return -1;
#pragma omp parallel num_threads(nthreads)
    {
#ifdef _OPENMP
        const int th = omp_get_thread_num(), nth = omp_get_num_threads();
#else
        const int th = 0, nth = 1;
#endif
        /* contiguous block per thread (the block count is the thread count asked for) */
        for (int b = th; b < nthreads; b += nth) {
            const long p0 = np * b / nthreads, p1 = np * (b + 1) / nthreads;
            deposit_range(D, n, periodic, np, p0, p1, idx, t, part + (size_t)b * ncell);
        }
    }
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (long i = 0; i < ncell; ++i) {
        double s = C[i];
        for (int b = 0; b < nthreads; ++b) s = s + part[(size_t)b * ncell + i];
        C[i] = s;
    }
    free(part);
    return 0;
}
