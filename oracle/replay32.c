/* FP32 replay of the hybrid mover's operation sequence (spec R). Test infrastructure: only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Sec. II.B.4, eqs. (hybridx), (step1)-(step4): full-step kick with the field gathered at
 * xi^n (eq. (step1); without a magnetic field a single fmaf per component, with a uniform
 * B0 the Boris step below), predictor
 * xi' = xi^n + dt/2 k(xi^n) v^{n+1/2} (eq. (step2)), k re-interpolated at xi' with b1
 * weights (eq. (step3)), corrector xi^{n+1} = xi^n + dt k(xi') v^{n+1/2} (eq. (step4)).
 * b1 weights and vertex interpolation: Sec. II.B.2 eqs. (vvp), (Wvp), (b1).
 *
 * Positions are split: integer cell per axis + float offset t in [0, 1), cell units.
 * Operation order (every rounding is part of the spec; compile with -ffp-contract=off):
 *   s_a = 1 - t_a; corner weight w_o = product over axes of (o_a ? t_a : s_a), multiplied
 *   from axis 0 upwards; corners in order o = 0 .. 2^D - 1 (bit a = offset along axis a);
 *   gather acc = w_0 * Q_0, then acc = fmaf(w_o, Q_o, acc) for o = 1 ...
 *   E^al = -(fmaf chain over a of K^{a al} G^a, starting with K^{0 al} * G^0)
 *   v^al = fmaf(dtqm, E^al, v^al) for al < D
 *   d_a = fmaf chain over al < D of K^{a al} v^al, starting with K^{a0} * v^0
 *   t'_a = fmaf(hdt, d_a, t_a); renormalise + clamp (below); K' = gather at (cell', t')
 *   t_a^{n+1} = fmaf(dt, d'_a, t_a) with d' from K'; renormalise + boundary.
 * Renormalisation of x on axis a: c = floorf(x), f = x - c, if f >= 1 then f = 0, c += 1;
 * c is clamped to [-2^24, 2^24] before conversion. Predictor point: periodic axes wrap,
 * other axes clamp to (0, 0) below and (N-1, 1) above (reading: the paper is silent on a
 * predictor point outside the domain). Final point: periodic wrap; a cell index below 0 or
 * at/above N on an absorbing axis removes the particle (Sec. II.B.4: a particle leaves the
 * domain when a logical coordinate becomes < 0 or > 1); the lowest such axis names the
 * face. A non-finite final offset also removes the particle (reported separately).
 */
#include <math.h>
#include <stdint.h>

#define PBC_PERIODIC 0
#define PBC_ABSORB 1
#define PBC_REFLECT 2

static int wrap(int c, int n) {
    int r = c % n;
    return r < 0 ? r + n : r;
}

static void renorm(float x, float* f, int* c) {
    float cf = floorf(x);
    float fr = x - cf;
    if (fr >= 1.0f) {
        fr = 0.0f;
        cf = cf + 1.0f;
    }
    if (cf < -16777216.0f) cf = -16777216.0f;
    if (cf > 16777216.0f) cf = 16777216.0f;
    *f = fr;
    *c = (int)cf;
}

/* Boris step with a uniform B0 (eq. (step1) with the magnetic term), FP32 in this order:
 * v- = v + h E; v' = v- + v- x t; v+ = v- + v' x s; v = v+ + h E, each cross-product
 * component computed as fmaf(a_y, b_z, -(a_z * b_y)) and added to the left vector's
 * component. bc = {h, t0, t1, t2, s0, s1, s2}; E has three components (E_z = 0 in 2D). */
static void boris32(float* v, const float* E, const float* bc) {
    const float h = bc[0];
    const float* t = bc + 1;
    const float* s = bc + 4;
    float m[3], q[3], w[3];
    for (int al = 0; al < 3; ++al) m[al] = fmaf(h, E[al], v[al]);
    q[0] = m[0] + fmaf(m[1], t[2], -(m[2] * t[1]));
    q[1] = m[1] + fmaf(m[2], t[0], -(m[0] * t[2]));
    q[2] = m[2] + fmaf(m[0], t[1], -(m[1] * t[0]));
    w[0] = m[0] + fmaf(q[1], s[2], -(q[2] * s[1]));
    w[1] = m[1] + fmaf(q[2], s[0], -(q[0] * s[2]));
    w[2] = m[2] + fmaf(q[0], s[1], -(q[1] * s[0]));
    for (int al = 0; al < 3; ++al) v[al] = fmaf(h, E[al], w[al]);
}

/* vertex table index of vertex (i, j[, k]) with N_a + 1 vertices per axis */
static long vtx(int D, const int* n, const int* c) {
    long v = c[D - 1];
    for (int a = D - 2; a >= 0; --a) v = v * (n[a] + 1) + c[a];
    return v;
}

/* gather nq components of table Q (nq floats per vertex) at (cell c, offsets t) */
static void gather(int D, const int* n, const float* Q, int nq, const int* c, const float* t,
                   float* out) {
    float s[3], w[8];
    int nc = 1 << D;
    for (int a = 0; a < D; ++a) s[a] = 1.0f - t[a];
    for (int o = 0; o < nc; ++o) {
        float ww = (o & 1) ? t[0] : s[0];
        for (int a = 1; a < D; ++a) ww = ww * (((o >> a) & 1) ? t[a] : s[a]);
        w[o] = ww;
    }
    for (int q = 0; q < nq; ++q) out[q] = 0.0f;
    for (int o = 0; o < nc; ++o) {
        int cc[3];
        for (int a = 0; a < D; ++a) cc[a] = c[a] + ((o >> a) & 1);
        const float* rec = Q + vtx(D, n, cc) * nq;
        for (int q = 0; q < nq; ++q) out[q] = (o == 0) ? (w[0] * rec[q]) : fmaf(w[o], rec[q], out[q]);
    }
}

/* One push of np particles. idx: (D, np) int32 per-axis cells; t: (D, np); v: (3, np);
 * K: vertex table of D*D floats [a][al]; G: vertex table of D floats.
 * pbc[2a+side]: particle boundary kinds. Outputs in place; face[p] = -1 alive, 2a+side
 * absorbed, 2*D non-finite. ke_fp[p] = llrintf(ke * 2^24) with the FP32 product
 * ke = fmaf(vo2, v2, fmaf(vo1, v1, vo0 * v0)) (spec D). */
void replay_push(int D, const int* n, const int* pbc, long np, int* idx, float* t, float* v,
                 const float* K, const float* G, float dtqm, float hdt, float dt, int* face,
                 long long* ke_fp, const float* boris, const float* R, const float* gyro) {
    for (long p = 0; p < np; ++p) {
        int c[3];
        float tt[3], vv[3], vo[3];
        for (int a = 0; a < D; ++a) {
            c[a] = idx[a * np + p];
            tt[a] = t[a * np + p];
        }
        for (int al = 0; al < 3; ++al) vo[al] = vv[al] = v[al * np + p];

        float kp[9], gp[3];
        gather(D, n, K, D * D, c, tt, kp);
        gather(D, n, G, D, c, tt, gp);
        float E[3] = {0.0f, 0.0f, 0.0f};
        for (int al = 0; al < D; ++al) {
            float e = kp[0 * D + al] * gp[0];
            for (int a = 1; a < D; ++a) e = fmaf(kp[a * D + al], gp[a], e);
            E[al] = -e;
        }
        if (boris)
            boris32(vv, E, boris);
        else
            for (int al = 0; al < D; ++al) vv[al] = fmaf(dtqm, E[al], vv[al]);
        float vk[3] = {vv[0], vv[1], vv[2]}; /* kicked velocity (kinetic-energy tally) */
        /* axisymmetric run (R: vertex cylindrical radius): straight 3D motion over the step,
         * x = fmaf(dt, v_r, r), y = dt * v_theta, r' = sqrtf(fmaf(x, x, y * y)); meridional
         * displacement (r' - r, dt * v_z); the frame turns by (x, y) / r' (cos, sin; (1, 0)
         * at r' = 0): v_r = fmaf(cos, v_r, sin * v_theta), v_theta = fmaf(cos, v_theta,
         * -(sin * v_r)); predictor t' = fmaf(0.5f, k . disp, t), corrector t + k' . disp */
        float disp[3] = {0.0f, 0.0f, 0.0f}, vrot[3] = {vv[0], vv[1], vv[2]};
        const int dform = gyro != 0 || R != 0;
        if (gyro) {
            /* cyclotronic push: exact gyration over dt after the plain kick, gyro = (b0, b1,
             * b2, cos th, sin th, f1, f2); vpar = fmaf chain of v . b, u = v x b (each
             * component fmaf(a_y, b_z, -(a_z * b_y))), par = vpar * b, perp = v - par,
             * v' = fmaf(sin, u, fmaf(cos, perp, par)), d = dt * fmaf(f2, u, fmaf(f1, perp, par));
             * axisymmetric: x = r + d_r, y = d_theta, disp = (sqrtf(fmaf(x, x, y * y)) - r,
             * d_z) and the frame turn of v' as above */
            const float* b = gyro;
            const float vpar = fmaf(vv[2], b[2], fmaf(vv[1], b[1], vv[0] * b[0]));
            const float u[3] = {fmaf(vv[1], b[2], -(vv[2] * b[1])), fmaf(vv[2], b[0], -(vv[0] * b[2])),
                                fmaf(vv[0], b[1], -(vv[1] * b[0]))};
            float d3[3], vn[3];
            for (int al = 0; al < 3; ++al) {
                const float par = vpar * b[al];
                const float perp = vv[al] - par;
                vn[al] = fmaf(gyro[4], u[al], fmaf(gyro[3], perp, par));
                d3[al] = dt * fmaf(gyro[6], u[al], fmaf(gyro[5], perp, par));
            }
            for (int al = 0; al < 3; ++al) vrot[al] = vn[al];
            if (R) {
                float rn;
                gather(D, n, R, 1, c, tt, &rn);
                const float x = rn + d3[0];
                const float y = d3[2];
                const float r1 = sqrtf(fmaf(x, x, y * y));
                float ca = 1.0f, sa = 0.0f;
                if (r1 > 0.0f) {
                    ca = x / r1;
                    sa = y / r1;
                }
                disp[0] = r1 - rn;
                disp[1] = d3[1];
                vrot[0] = fmaf(ca, vn[0], sa * vn[2]);
                vrot[2] = fmaf(ca, vn[2], -(sa * vn[0]));
            } else {
                for (int a = 0; a < D; ++a) disp[a] = d3[a];
            }
        } else if (R) {
            float rn;
            gather(D, n, R, 1, c, tt, &rn);
            const float x = fmaf(dt, vv[0], rn);
            const float y = dt * vv[2];
            const float r1 = sqrtf(fmaf(x, x, y * y));
            float ca = 1.0f, sa = 0.0f;
            if (r1 > 0.0f) {
                ca = x / r1;
                sa = y / r1;
            }
            disp[0] = r1 - rn;
            disp[1] = dt * vv[1];
            vrot[0] = fmaf(ca, vv[0], sa * vv[2]);
            vrot[2] = fmaf(ca, vv[2], -(sa * vv[0]));
        }
        /* predictor */
        int cp[3];
        float tp[3];
        for (int a = 0; a < D; ++a) {
            float x;
            if (dform) {
                float d = kp[a * D + 0] * disp[0];
                for (int b = 1; b < D; ++b) d = fmaf(kp[a * D + b], disp[b], d);
                x = fmaf(0.5f, d, tt[a]);
            } else {
                float d = kp[a * D + 0] * vv[0];
                for (int al = 1; al < D; ++al) d = fmaf(kp[a * D + al], vv[al], d);
                x = fmaf(hdt, d, tt[a]);
            }
            if (!isfinite(x)) {
                cp[a] = c[a];
                tp[a] = tt[a];
                continue;
            }
            int dc;
            renorm(x, &tp[a], &dc);
            int ci = c[a] + dc;
            if (pbc[2 * a] == PBC_PERIODIC) {
                ci = wrap(ci, n[a]);
            } else if (ci < 0) {
                ci = 0;
                tp[a] = 0.0f;
            } else if (ci >= n[a]) {
                ci = n[a] - 1;
                tp[a] = 1.0f;
            }
            cp[a] = ci;
        }
        float kq[9];
        gather(D, n, K, D * D, cp, tp, kq);
        /* corrector */
        int fc = -1;
        int cn[3];
        float tn[3];
        for (int a = 0; a < D; ++a) {
            float x;
            if (dform) {
                float d = kq[a * D + 0] * disp[0];
                for (int b = 1; b < D; ++b) d = fmaf(kq[a * D + b], disp[b], d);
                x = tt[a] + d;
            } else {
                float d = kq[a * D + 0] * vv[0];
                for (int al = 1; al < D; ++al) d = fmaf(kq[a * D + al], vv[al], d);
                x = fmaf(dt, d, tt[a]);
            }
            if (!isfinite(x)) {
                fc = 2 * D;
                cn[a] = c[a];
                tn[a] = tt[a];
                continue;
            }
            int dc;
            renorm(x, &tn[a], &dc);
            cn[a] = c[a] + dc;
        }
        if (fc < 0) {
            for (int a = 0; a < D; ++a) {
                if (pbc[2 * a] == PBC_PERIODIC) {
                    cn[a] = wrap(cn[a], n[a]);
                } else if (pbc[2 * a] == PBC_REFLECT) {
                    continue; /* mirrored after the kinetic-energy tally */
                } else if (cn[a] < 0) {
                    if (fc < 0) fc = 2 * a;
                } else if (cn[a] >= n[a]) {
                    if (fc < 0) fc = 2 * a + 1;
                }
            }
        }
        float ke = fmaf(vo[2], vk[2], fmaf(vo[1], vk[1], vo[0] * vk[0]));
        ke_fp[p] = llrintf(ldexpf(ke, 24));
        if (dform)
            for (int al = 0; al < 3; ++al) vv[al] = vrot[al];
        /* spec B: mirror about a reflecting face, reflect v about row a of k(xi') */
        if (fc < 0) {
            for (int a = 0; a < D && fc < 0; ++a) {
                if (pbc[2 * a] != PBC_REFLECT || (cn[a] >= 0 && cn[a] < n[a])) continue;
                int below = cn[a] < 0;
                int c2 = below ? (-cn[a] - 1) : (2 * n[a] - 1 - cn[a]);
                float t2 = 1.0f - tn[a];
                if (t2 >= 1.0f) {
                    t2 = 0.0f;
                    c2 += 1;
                }
                if (c2 < 0 || c2 >= n[a]) {
                    fc = 2 * a + (below ? 0 : 1);
                    break;
                }
                cn[a] = c2;
                tn[a] = t2;
                float nn = kq[a * D + 0] * kq[a * D + 0];
                float dot = vv[0] * kq[a * D + 0];
                for (int al = 1; al < D; ++al) {
                    nn = fmaf(kq[a * D + al], kq[a * D + al], nn);
                    dot = fmaf(vv[al], kq[a * D + al], dot);
                }
                float sf = (2.0f * dot) / nn;
                for (int al = 0; al < D; ++al) vv[al] = fmaf(-sf, kq[a * D + al], vv[al]);
            }
        }
        face[p] = fc;
        for (int a = 0; a < D; ++a) {
            idx[a * np + p] = cn[a]; /* removed particles keep their corrector cell */
            t[a * np + p] = tn[a];
        }
        for (int al = 0; al < 3; ++al) v[al * np + p] = vv[al];
    }
}

/* Half kick (leapfrog start-up, v^{-1/2} = v^0 - dt/2 q/m E(xi^0)): only the gather and
 * kick of the push, with the given (negative) coefficient. */
void replay_kick(int D, const int* n, long np, const int* idx, const float* t, float* v,
                 const float* K, const float* G, float coef, const float* boris) {
    for (long p = 0; p < np; ++p) {
        int c[3];
        float tt[3];
        for (int a = 0; a < D; ++a) {
            c[a] = idx[a * np + p];
            tt[a] = t[a * np + p];
        }
        float kp[9], gp[3];
        gather(D, n, K, D * D, c, tt, kp);
        gather(D, n, G, D, c, tt, gp);
        float E[3] = {0.0f, 0.0f, 0.0f};
        for (int al = 0; al < D; ++al) {
            float e = kp[0 * D + al] * gp[0];
            for (int a = 1; a < D; ++a) e = fmaf(kp[a * D + al], gp[a], e);
            E[al] = -e;
        }
        if (boris) {
            float vv[3];
            for (int al = 0; al < 3; ++al) vv[al] = v[al * np + p];
            boris32(vv, E, boris);
            for (int al = 0; al < 3; ++al) v[al * np + p] = vv[al];
        } else {
            for (int al = 0; al < D; ++al) v[al * np + p] = fmaf(coef, E[al], v[al * np + p]);
        }
    }
}
