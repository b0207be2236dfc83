// Row a0: metric coefficients from the vertex map (Sec. II.A: Jacobi matrix eq. (jcov), its
// inverse eq. (jcon), Jacobian eq. (jac), contravariant metric eq. (gcon) and the factor
// Omega J g^{ab} of eq. (poiscurv); metric by finite differences of the map known at
// vertices, last paragraph of Sec. II.A).
//
// FP64, cell units (logical coordinate u^a = N_a xi^a). Every floating-point operation is an
// explicit round-to-nearest intrinsic so that no multiply-add is contracted: the order of
// operations below is the one the finite-difference stencils are specified with, and the
// FP32 copy of k that the mover reads is reproducible bit for bit.
#include <math.h>

#include "internal.cuh"

namespace cpic {
namespace {

__device__ __forceinline__ double A_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double S_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double M_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double Q_(double a, double b) { return __ddiv_rn(a, b); }

// spec M: a cross coefficient no larger than this fraction of the face's diagonal one is
// the rounding residue of an orthogonal map and is zero
constexpr double kCrossRoundoff = 1e-12;

struct Grid {
    int D;
    int n[3];
    int nv[3];  // vertices per axis (n + 1)
    int per[3];
};

__device__ __forceinline__ long long vidx(const Grid& g, int i, int j, int k) {
    return (long long)i + (long long)g.nv[0] * ((long long)j + (long long)g.nv[1] * k);
}

// ---------------------------------------------------------------- analytic maps
__global__ void map_kernel(Grid g, int map_id, double p0, double p1, double p2, double* X) {
    long long nvt = (long long)g.nv[0] * g.nv[1] * (g.D == 3 ? g.nv[2] : 1);
    const double two_pi = 6.283185307179586476925286766559;
    const double pi = 3.141592653589793238462643383280;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvt;
         v += (long long)gridDim.x * blockDim.x) {
        int i = (int)(v % g.nv[0]);
        long long rest = v / g.nv[0];
        int j = (int)(rest % g.nv[1]);
        int k = (int)(rest / g.nv[1]);
        double xi = (double)i / g.n[0], eta = (double)j / g.n[1];
        double zeta = g.D == 3 ? (double)k / g.n[2] : 0.0;
        double* out = X + v * g.D;
        if (map_id == CPIC_MAP_SINE) {
            double s = p0 * sin(two_pi * xi) * sin(two_pi * eta);
            out[0] = xi + s;
            out[1] = eta + s;
        } else if (map_id == CPIC_MAP_ANNULUS) {
            double r = p0 * pow(p1 / p0, xi);
            double th = two_pi * eta;
            out[0] = r * cos(th);
            out[1] = r * sin(th);
        } else if (map_id == CPIC_MAP_SPHERE_AXISYM) {
            double rad = p0 + (p1 - p0) * xi;
            double ang = pi * (1.0 - eta);
            out[0] = rad * sin(ang);
            out[1] = rad * cos(ang);
        } else {  // CPIC_MAP_SHELL
            double r = p0 * pow(p1 / p0, xi);
            double th = p2 + (pi - 2.0 * p2) * eta;
            double ph = two_pi * zeta;
            out[0] = r * sin(th) * cos(ph);
            out[1] = r * sin(th) * sin(ph);
            out[2] = r * cos(th);
        }
    }
}

// exact periodic images / axis points, after map_kernel
__global__ void map_fix_kernel(Grid g, int map_id, double* X) {
    long long nvt = (long long)g.nv[0] * g.nv[1] * (g.D == 3 ? g.nv[2] : 1);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvt;
         v += (long long)gridDim.x * blockDim.x) {
        int i = (int)(v % g.nv[0]);
        long long rest = v / g.nv[0];
        int j = (int)(rest % g.nv[1]);
        int k = (int)(rest / g.nv[1]);
        double* out = X + v * g.D;
        if (map_id == CPIC_MAP_SINE) {
            // x(1, eta) = x(0, eta) + (1, 0); x(xi, 1) = x(xi, 0) + (0, 1)
            if (i == g.n[0] && j == g.n[1]) {
                out[0] = 1.0;
                out[1] = 1.0;
            } else if (i == g.n[0]) {
                double* o0 = X + vidx(g, 0, j, 0) * 2;
                out[0] = o0[0] + 1.0;
                out[1] = o0[1];
            } else if (j == g.n[1]) {
                double* o0 = X + vidx(g, i, 0, 0) * 2;
                out[0] = o0[0];
                out[1] = o0[1] + 1.0;
            }
        } else if (map_id == CPIC_MAP_ANNULUS) {
            if (j == g.n[1]) {
                double* o0 = X + vidx(g, i, 0, 0) * 2;
                out[0] = o0[0];
                out[1] = o0[1];
            }
        } else if (map_id == CPIC_MAP_SPHERE_AXISYM) {
            if (j == 0 || j == g.n[1]) out[0] = 0.0;
        } else if (map_id == CPIC_MAP_SHELL) {
            if (k == g.n[2]) {
                double* o0 = X + vidx(g, i, j, 0) * 3;
                out[0] = o0[0];
                out[1] = o0[1];
                out[2] = o0[2];
            }
        }
    }
}

// The map2 corner (n1, n2) is X(0,0) + (1,1) = (1,1) exactly because X(0,0) = (0,0);
// the general rule "image of the image" gives the same value.

// ---------------------------------------------------------------- vertex derivatives
// dv[a][v][alpha] = dX^alpha/du^a at vertex v (spec M stencils).
__global__ void vertex_derivative_kernel(Grid g, const double* __restrict__ X, double* dv) {
    long long nvt = (long long)g.nv[0] * g.nv[1] * (g.D == 3 ? g.nv[2] : 1);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvt;
         v += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = (int)(v % g.nv[0]);
        long long rest = v / g.nv[0];
        c[1] = (int)(rest % g.nv[1]);
        c[2] = (int)(rest / g.nv[1]);
        for (int a = 0; a < g.D; ++a) {
            int N = g.n[a];
            int x = c[a];
            long long stride = a == 0 ? 1 : (a == 1 ? g.nv[0] : (long long)g.nv[0] * g.nv[1]);
            const double* base = X + (v - (long long)x * stride) * g.D;  // vertex with x = 0
            double* out = dv + ((long long)a * nvt + v) * g.D;
            for (int al = 0; al < g.D; ++al) {
                auto at = [&](int xx) { return base[(long long)xx * stride * g.D + al]; };
                double r;
                if (g.per[a]) {
                    if (x == 0 || x == N) {
                        double shift = S_(at(N), at(0));
                        double prev0 = S_(at(N - 1), shift);
                        r = M_(S_(at(1), prev0), 0.5);
                    } else {
                        r = M_(S_(at(x + 1), at(x - 1)), 0.5);
                    }
                } else {
                    if (x == 0) {
                        r = M_(S_(S_(M_(4.0, at(1)), M_(3.0, at(0))), at(2)), 0.5);
                    } else if (x == N) {
                        r = M_(A_(S_(M_(3.0, at(N)), M_(4.0, at(N - 1))), at(N - 2)), 0.5);
                    } else {
                        r = M_(S_(at(x + 1), at(x - 1)), 0.5);
                    }
                }
                out[al] = r;
            }
        }
    }
}

__device__ __forceinline__ double det3(const double m[3][3]) {
    double c0 = S_(M_(m[1][1], m[2][2]), M_(m[1][2], m[2][1]));
    double c1 = S_(M_(m[1][0], m[2][2]), M_(m[1][2], m[2][0]));
    double c2 = S_(M_(m[1][0], m[2][1]), M_(m[1][1], m[2][0]));
    return A_(S_(M_(m[0][0], c0), M_(m[0][1], c1)), M_(m[0][2], c2));
}

// k = j^-1 at vertices (FP64) and the FP32 mover table.
__global__ void inverse_kernel(Grid g, const double* __restrict__ dv, double* k64, float* K32) {
    long long nvt = (long long)g.nv[0] * g.nv[1] * (g.D == 3 ? g.nv[2] : 1);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvt;
         v += (long long)gridDim.x * blockDim.x) {
        double j[3][3];  // j[alpha][a]
        for (int a = 0; a < g.D; ++a)
            for (int al = 0; al < g.D; ++al) j[al][a] = dv[((long long)a * nvt + v) * g.D + al];
        double k[3][3];  // k[a][alpha]
        if (g.D == 2) {
            double det = S_(M_(j[0][0], j[1][1]), M_(j[0][1], j[1][0]));
            k[0][0] = Q_(j[1][1], det);
            k[0][1] = Q_(-j[0][1], det);
            k[1][0] = Q_(-j[1][0], det);
            k[1][1] = Q_(j[0][0], det);
            double* o = k64 + v * 4;
            o[0] = k[0][0]; o[1] = k[0][1]; o[2] = k[1][0]; o[3] = k[1][1];
            float4 f = make_float4(__double2float_rn(k[0][0]), __double2float_rn(k[0][1]),
                                   __double2float_rn(k[1][0]), __double2float_rn(k[1][1]));
            reinterpret_cast<float4*>(K32)[v] = f;
        } else {
            double det = det3(j);
            for (int a = 0; a < 3; ++a)
                for (int al = 0; al < 3; ++al) {
                    int r0 = al == 0 ? 1 : 0, r1 = al == 2 ? 1 : 2;
                    int c0 = a == 0 ? 1 : 0, c1 = a == 2 ? 1 : 2;
                    double minor = S_(M_(j[r0][c0], j[r1][c1]), M_(j[r0][c1], j[r1][c0]));
                    double sm = ((al + a) % 2 == 0) ? minor : -minor;
                    k[a][al] = Q_(sm, det);
                }
            double* o = k64 + v * 9;
            float* f = K32 + v * 12;
            for (int a = 0; a < 3; ++a)
                for (int al = 0; al < 3; ++al) {
                    o[a * 3 + al] = k[a][al];
                    f[a * 3 + al] = __double2float_rn(k[a][al]);
                }
            f[9] = f[10] = f[11] = 0.0f;
        }
    }
}

// Cell Jacobian (det of the cell-averaged Jacobi matrix) and Omega at cells.
__global__ void cell_kernel(Grid g, int axisym, const double* __restrict__ X, double* Jc, double* om) {
    long long nc = (long long)g.n[0] * g.n[1] * (g.D == 3 ? g.n[2] : 1);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        int i = (int)(c % g.n[0]);
        long long rest = c / g.n[0];
        int j = (int)(rest % g.n[1]);
        int k = (int)(rest / g.n[1]);
        auto P = [&](int di, int dj, int dk) { return X + vidx(g, i + di, j + dj, k + dk) * g.D; };
        if (g.D == 2) {
            double d0[2], d1[2];
            for (int al = 0; al < 2; ++al) {
                double e0a = S_(P(1, 0, 0)[al], P(0, 0, 0)[al]);
                double e0b = S_(P(1, 1, 0)[al], P(0, 1, 0)[al]);
                double e1a = S_(P(0, 1, 0)[al], P(0, 0, 0)[al]);
                double e1b = S_(P(1, 1, 0)[al], P(1, 0, 0)[al]);
                d0[al] = M_(A_(e0a, e0b), 0.5);
                d1[al] = M_(A_(e1a, e1b), 0.5);
            }
            Jc[c] = S_(M_(d0[0], d1[1]), M_(d1[0], d0[1]));
            if (axisym) {
                double r = M_(A_(A_(A_(P(0, 0, 0)[0], P(1, 0, 0)[0]), P(0, 1, 0)[0]), P(1, 1, 0)[0]), 0.25);
                om[c] = r;
            } else {
                om[c] = 1.0;
            }
        } else {
            double m[3][3];  // m[alpha][a]
            for (int al = 0; al < 3; ++al) {
                double e0 = S_(P(1, 0, 0)[al], P(0, 0, 0)[al]);
                double e1 = S_(P(1, 1, 0)[al], P(0, 1, 0)[al]);
                double e2 = S_(P(1, 0, 1)[al], P(0, 0, 1)[al]);
                double e3 = S_(P(1, 1, 1)[al], P(0, 1, 1)[al]);
                m[al][0] = M_(A_(A_(A_(e0, e1), e2), e3), 0.25);
                e0 = S_(P(0, 1, 0)[al], P(0, 0, 0)[al]);
                e1 = S_(P(1, 1, 0)[al], P(1, 0, 0)[al]);
                e2 = S_(P(0, 1, 1)[al], P(0, 0, 1)[al]);
                e3 = S_(P(1, 1, 1)[al], P(1, 0, 1)[al]);
                m[al][1] = M_(A_(A_(A_(e0, e1), e2), e3), 0.25);
                e0 = S_(P(0, 0, 1)[al], P(0, 0, 0)[al]);
                e1 = S_(P(1, 0, 1)[al], P(1, 0, 0)[al]);
                e2 = S_(P(0, 1, 1)[al], P(0, 1, 0)[al]);
                e3 = S_(P(1, 1, 1)[al], P(1, 1, 0)[al]);
                m[al][2] = M_(A_(A_(A_(e0, e1), e2), e3), 0.25);
            }
            Jc[c] = det3(m);
            om[c] = 1.0;
        }
    }
}

__device__ __forceinline__ double dot2(const double* a, const double* b) {
    return A_(M_(a[0], b[0]), M_(a[1], b[1]));
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return A_(A_(M_(a[0], b[0]), M_(a[1], b[1])), M_(a[2], b[2]));
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
    o[0] = S_(M_(a[1], b[2]), M_(a[2], b[1]));
    o[1] = S_(M_(a[2], b[0]), M_(a[0], b[2]));
    o[2] = S_(M_(a[0], b[1]), M_(a[1], b[0]));
}

// Face coefficients a^{ab} = Omega J g^{ab} on the faces normal to axis `a`.
// face[b][f] for the face with index (i, j, k), vertex index along a, cell index otherwise.
__global__ void face_kernel(Grid g, int a, int axisym, const double* __restrict__ X,
                            const double* __restrict__ dv, double* face) {
    int fn[3] = {g.n[0], g.n[1], g.D == 3 ? g.n[2] : 1};
    fn[a] += 1;
    long long nf = (long long)fn[0] * fn[1] * fn[2];
    long long nvt = (long long)g.nv[0] * g.nv[1] * (g.D == 3 ? g.nv[2] : 1);
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
         f += (long long)gridDim.x * blockDim.x) {
        int i = (int)(f % fn[0]);
        long long rest = f / fn[0];
        int j = (int)(rest % fn[1]);
        int k = (int)(rest / fn[1]);
        auto P = [&](int di, int dj, int dk) { return X + vidx(g, i + di, j + dj, k + dk) * g.D; };
        auto DV = [&](int ax, int di, int dj, int dk) {
            return dv + ((long long)ax * nvt + vidx(g, i + di, j + dj, k + dk)) * g.D;
        };
        if (g.D == 2) {
            double xu[2], xv[2], om;
            if (a == 0) {  // xi-face between cells (i-1, j) and (i, j)
                for (int al = 0; al < 2; ++al) {
                    xv[al] = S_(P(0, 1, 0)[al], P(0, 0, 0)[al]);
                    xu[al] = M_(A_(DV(0, 0, 0, 0)[al], DV(0, 0, 1, 0)[al]), 0.5);
                }
                om = axisym ? M_(A_(P(0, 0, 0)[0], P(0, 1, 0)[0]), 0.5) : 1.0;
            } else {  // eta-face between cells (i, j-1) and (i, j)
                for (int al = 0; al < 2; ++al) {
                    xu[al] = S_(P(1, 0, 0)[al], P(0, 0, 0)[al]);
                    xv[al] = M_(A_(DV(1, 0, 0, 0)[al], DV(1, 1, 0, 0)[al]), 0.5);
                }
                om = axisym ? M_(A_(P(0, 0, 0)[0], P(1, 0, 0)[0]), 0.5) : 1.0;
            }
            double J = S_(M_(xu[0], xv[1]), M_(xv[0], xu[1]));
            double cross = -Q_(M_(om, dot2(xu, xv)), J);
            double diag = a == 0 ? Q_(M_(om, dot2(xv, xv)), J) : Q_(M_(om, dot2(xu, xu)), J);
            if (fabs(cross) <= M_(kCrossRoundoff, fabs(diag))) cross = 0.0;
            face[(long long)a * nf + f] = diag;
            face[(long long)(1 - a) * nf + f] = cross;
        } else {
            const double *q0, *q1, *q2, *q3, *d0, *d1, *d2, *d3;
            if (a == 0) {
                q0 = P(0, 0, 0); q1 = P(0, 1, 0); q2 = P(0, 0, 1); q3 = P(0, 1, 1);
                d0 = DV(0, 0, 0, 0); d1 = DV(0, 0, 1, 0); d2 = DV(0, 0, 0, 1); d3 = DV(0, 0, 1, 1);
            } else if (a == 1) {
                q0 = P(0, 0, 0); q1 = P(1, 0, 0); q2 = P(0, 0, 1); q3 = P(1, 0, 1);
                d0 = DV(1, 0, 0, 0); d1 = DV(1, 1, 0, 0); d2 = DV(1, 0, 0, 1); d3 = DV(1, 1, 0, 1);
            } else {
                q0 = P(0, 0, 0); q1 = P(1, 0, 0); q2 = P(0, 1, 0); q3 = P(1, 1, 0);
                d0 = DV(2, 0, 0, 0); d1 = DV(2, 1, 0, 0); d2 = DV(2, 0, 1, 0); d3 = DV(2, 1, 1, 0);
            }
            double xa[3], xb[3], xc[3];
            for (int al = 0; al < 3; ++al) {
                xa[al] = M_(A_(A_(A_(d0[al], d1[al]), d2[al]), d3[al]), 0.25);
                xb[al] = M_(A_(S_(q1[al], q0[al]), S_(q3[al], q2[al])), 0.5);
                xc[al] = M_(A_(S_(q2[al], q0[al]), S_(q3[al], q1[al])), 0.5);
            }
            double d[3][3];
            for (int al = 0; al < 3; ++al) {
                if (a == 0) { d[0][al] = xa[al]; d[1][al] = xb[al]; d[2][al] = xc[al]; }
                else if (a == 1) { d[0][al] = xb[al]; d[1][al] = xa[al]; d[2][al] = xc[al]; }
                else { d[0][al] = xb[al]; d[1][al] = xc[al]; d[2][al] = xa[al]; }
            }
            double Ab[3][3];
            cross3(d[1], d[2], Ab[0]);
            cross3(d[2], d[0], Ab[1]);
            cross3(d[0], d[1], Ab[2]);
            double J = dot3(d[0], Ab[0]);
            double coef[3];
            for (int b = 0; b < 3; ++b) coef[b] = Q_(dot3(Ab[a], Ab[b]), J);
            for (int b = 0; b < 3; ++b)
                if (b != a && fabs(coef[b]) <= M_(kCrossRoundoff, fabs(coef[a]))) coef[b] = 0.0;
            for (int b = 0; b < 3; ++b) face[(long long)b * nf + f] = coef[b];
        }
    }
}

// coarse vertex map: every other vertex of the finer level
__global__ void subsample_kernel(Grid gc, Grid gf, const double* __restrict__ Xf, double* Xc) {
    long long nvt = (long long)gc.nv[0] * gc.nv[1] * (gc.D == 3 ? gc.nv[2] : 1);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvt;
         v += (long long)gridDim.x * blockDim.x) {
        int i = (int)(v % gc.nv[0]);
        long long rest = v / gc.nv[0];
        int j = (int)(rest % gc.nv[1]);
        int k = (int)(rest / gc.nv[1]);
        const double* src = Xf + vidx(gf, 2 * i, 2 * j, 2 * k) * gc.D;
        for (int al = 0; al < gc.D; ++al) Xc[v * gc.D + al] = src[al];
    }
}

Grid make_grid(const cpic_run* r, const int* n) {
    Grid g;
    g.D = r->D;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < r->D ? n[a] : 1;
        g.nv[a] = a < r->D ? n[a] + 1 : 1;
        g.per[a] = a < r->D ? (r->cfg.field_bc[2 * a] == CPIC_BC_PERIODIC) : 0;
    }
    return g;
}

int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 16LL * device_sm_count()) b = 16LL * device_sm_count();
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int launch_map_analytic(cpic_run* r, int map_id, const double* params, int nparams) {
    Grid g = make_grid(r, r->n);
    double p[3] = {0, 0, 0};
    for (int i = 0; i < nparams && i < 3; ++i) p[i] = params[i];
    long long nvt = r->nvert;
    map_kernel<<<blocks_for(nvt, 256), 256, 0, r->stream>>>(g, map_id, p[0], p[1], p[2], r->lev[0].X);
    CPIC_CHECK_LAUNCH();
    map_fix_kernel<<<blocks_for(nvt, 256), 256, 0, r->stream>>>(g, map_id, r->lev[0].X);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

// Metric of every multigrid level (level 0 also fills the FP64/FP32 vertex k tables).
int launch_geometry(cpic_run* r) {
    for (int l = 0; l < r->nlevels; ++l) {
        Level& L = r->lev[l];
        Grid g = make_grid(r, L.n);
        long long nvt = (long long)g.nv[0] * g.nv[1] * (r->D == 3 ? g.nv[2] : 1);
        if (l > 0) {
            Grid gf = make_grid(r, r->lev[l - 1].n);
            subsample_kernel<<<blocks_for(nvt, 256), 256, 0, r->stream>>>(g, gf, r->lev[l - 1].X, L.X);
            CPIC_CHECK_LAUNCH();
        }
        vertex_derivative_kernel<<<blocks_for(nvt, 256), 256, 0, r->stream>>>(g, L.X, L.dv);
        CPIC_CHECK_LAUNCH();
        if (l == 0) {
            inverse_kernel<<<blocks_for(nvt, 256), 256, 0, r->stream>>>(g, L.dv, r->k64, r->K32);
            CPIC_CHECK_LAUNCH();
        }
        cell_kernel<<<blocks_for(L.ncell, 256), 256, 0, r->stream>>>(g, r->cfg.axisymmetric, L.X, L.Jc, L.omega);
        CPIC_CHECK_LAUNCH();
        for (int a = 0; a < r->D; ++a) {
            int fn[3] = {g.n[0], g.n[1], r->D == 3 ? g.n[2] : 1};
            fn[a] += 1;
            long long nf = (long long)fn[0] * fn[1] * fn[2];
            face_kernel<<<blocks_for(nf, 256), 256, 0, r->stream>>>(g, a, r->cfg.axisymmetric, L.X, L.dv, L.face[a]);
            CPIC_CHECK_LAUNCH();
        }
    }
    return CPIC_OK;
}

}  // namespace cpic
