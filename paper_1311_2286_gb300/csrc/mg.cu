// Row a9: the logical-space Poisson solve (Sec. II.B.3; eq. (poiscurv)), FP64, device
// resident.
//
// Discretisation (conservative finite volume with ghost cells): the flux through a face
// normal to axis a is a^{aa} (phi_R - phi_L) + sum_{b != a} a^{ab} / 4 [(phi_R(+b) + phi_L(+b))
// - (phi_R(-b) + phi_L(-b))], a^{ab} = Omega J g^{ab} from the geometry; Dirichlet ghosts
// 2 phi_b - phi_in (a Dirichlet face carries a^{aa} 2 (phi_in - phi_b)), Neumann ghosts
// phi_in (a Neumann face carries no flux), periodic wrap. The assembled row of cell c is
// M phi = Omega_c Q_c + (Dirichlet terms), M = -(divergence), stored as a 9-point (2D) or
// 19-point (3D) stencil, of which only the 5/7 face entries are used when the map is
// orthogonal.
//
// Solver: multigrid V-cycles, the method class the paper uses (Sec. II.B.3: coarse-grid
// correction plus Gauss-Seidel smoothing on each level). This implementation rediscretises
// each coarse level from the map sampled at every other vertex (BoxMG's variational coarse
// operators and operator-induced interpolation are not reproduced), restricts by summing
// the 2^D fine residuals (finite-volume conservation), prolongs (bi/tri)linearly with
// homogeneous ghost rules, and smooths with colour-ordered Gauss-Seidel (2 colours for
// 5/7-point stencils, 2^D colours when cross terms are present). Levels of at most
// COARSE_CELLS cells run inside one CTA; the coarsest level is solved with a dense inverse
// (bordered by the constant null vector when the problem is singular). A singular problem
// (no Dirichlet face) has its right-hand side projected by subtracting a uniform physical
// charge density and its solution gauged to sum_c J_c phi_c = 0.
//
// Convergence: ||b - M phi||_2 / ||b||_2 <= rtol (Sec. II.B.3 uses a relative tolerance of
// 1e-10). The residual kernel raises a device flag that makes the remaining cycles' kernels
// return at once, so a whole solve can be enqueued without a host round trip.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace cpic {
namespace {

constexpr int RED_BLOCKS = 256;

__constant__ int c_off2[9][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
__constant__ int c_off3[19][3] = {{0, 0, 0},  {-1, 0, 0},  {1, 0, 0},  {0, -1, 0}, {0, 1, 0},
                                  {0, 0, -1}, {0, 0, 1},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
                                  {1, 1, 0},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
                                  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

struct LV {
    int D;
    int n[3];
    long long ncell;
    int S;      // stored stencil entries (9 / 19)
    int used;   // entries used (5/7 without cross terms, else 9/19)
    int ncol;   // Gauss-Seidel colours (2 or 2^D)
    int per[3];
    int bc[6];
    const double* A;
    double* x;
    double* b;
};

struct LVSet {
    int nl;
    int first_cta;  // first level solved inside one CTA
    LV l[MAX_LEVELS];
    const double* dense_inv;
    int dense_m;   // unknowns of the coarsest level
    int singular;
};

__device__ __forceinline__ void cell_coords(const LV& L, long long c, int* q) {
    q[0] = (int)(c % L.n[0]);
    long long r = c / L.n[0];
    q[1] = (int)(r % L.n[1]);
    q[2] = (int)(r / L.n[1]);
}

__device__ __forceinline__ long long lin(const LV& L, const int* q) {
    return q[0] + (long long)L.n[0] * (q[1] + (long long)L.n[1] * q[2]);
}

__device__ __forceinline__ void offsets(int D, int k, int* o) {
    if (D == 2) {
        o[0] = c_off2[k][0];
        o[1] = c_off2[k][1];
        o[2] = 0;
    } else {
        o[0] = c_off3[k][0];
        o[1] = c_off3[k][1];
        o[2] = c_off3[k][2];
    }
}

// neighbour index with periodic wrap; non-periodic out-of-range entries have zero
// coefficients after assembly, their index is clamped
__device__ __forceinline__ long long nbr(const LV& L, const int* q, const int* o) {
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = q[a] + o[a];
        if (a < L.D) {
            if (v < 0) v = L.per[a] ? v + L.n[a] : 0;
            else if (v >= L.n[a]) v = L.per[a] ? v - L.n[a] : L.n[a] - 1;
        }
        c[a] = v;
    }
    return lin(L, c);
}

__device__ __forceinline__ double apply_row(const LV& L, long long c, const int* q, bool skip_centre) {
    double s = 0.0;
    for (int k = skip_centre ? 1 : 0; k < L.used; ++k) {
        int o[3];
        offsets(L.D, k, o);
        s += L.A[(long long)k * L.ncell + c] * L.x[nbr(L, q, o)];
    }
    return s;
}

// number of cells of one colour and the mapping colour-local index -> cell
__device__ __forceinline__ long long colour_cells(const LV& L) { return L.ncell / L.ncol; }

__device__ __forceinline__ void colour_cell(const LV& L, int colour, long long idx, int* q) {
    if (L.ncol == 2) {
        // parity colouring: (i + j + k) % 2 == colour; n[0] even
        int h = L.n[0] / 2;
        long long row = idx / h;
        int m = (int)(idx % h);
        int j = (int)(row % L.n[1]);
        int k = (int)(row / L.n[1]);
        q[1] = j;
        q[2] = k;
        q[0] = 2 * m + ((j + k + colour) & 1);
    } else {
        // one bit per axis
        int h[3] = {L.n[0] / 2, L.D > 1 ? L.n[1] / 2 : 1, L.D > 2 ? L.n[2] / 2 : 1};
        int m0 = (int)(idx % h[0]);
        long long r = idx / h[0];
        int m1 = (int)(r % h[1]);
        int m2 = (int)(r / h[1]);
        q[0] = 2 * m0 + (colour & 1);
        q[1] = 2 * m1 + ((colour >> 1) & 1);
        q[2] = L.D == 3 ? 2 * m2 + ((colour >> 2) & 1) : 0;
    }
}

__device__ __forceinline__ void smooth_cell(const LV& L, int colour, long long idx) {
    int q[3];
    colour_cell(L, colour, idx, q);
    long long c = lin(L, q);
    double s = L.b[c] - apply_row(L, c, q, true);
    L.x[c] = s / L.A[c];
}

// residual of the 2^D children of coarse cell C summed into the coarse right-hand side
__device__ __forceinline__ void restrict_cell(const LV& F, const LV& Cl, long long C) {
    int qc[3];
    cell_coords(Cl, C, qc);
    double acc = 0.0;
    int nch = F.D == 2 ? 4 : 8;
    for (int ch = 0; ch < nch; ++ch) {
        int q[3] = {2 * qc[0] + (ch & 1), 2 * qc[1] + ((ch >> 1) & 1), F.D == 3 ? 2 * qc[2] + ((ch >> 2) & 1) : 0};
        long long f = lin(F, q);
        acc += F.b[f] - apply_row(F, f, q, false);
    }
    Cl.b[C] = acc;
    Cl.x[C] = 0.0;
}

// coarse correction value at coarse coordinates q (possibly one outside per axis)
__device__ __forceinline__ double coarse_value(const LV& Cl, int* q) {
    double sign = 1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= Cl.D) break;
        if (q[a] < 0 || q[a] >= Cl.n[a]) {
            int side = q[a] < 0 ? 0 : 1;
            if (Cl.per[a]) {
                q[a] = q[a] < 0 ? q[a] + Cl.n[a] : q[a] - Cl.n[a];
            } else {
                q[a] = side == 0 ? 0 : Cl.n[a] - 1;
                if (Cl.bc[2 * a + side] == CPIC_BC_DIRICHLET) sign = -sign;
            }
        }
    }
    return sign * Cl.x[lin(Cl, q)];
}

__device__ __forceinline__ void prolong_cell(const LV& F, const LV& Cl, long long f) {
    int q[3];
    cell_coords(F, f, q);
    int p[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
    int s[3] = {(q[0] & 1) ? 1 : -1, (q[1] & 1) ? 1 : -1, (q[2] & 1) ? 1 : -1};
    double acc = 0.0;
    int nc = F.D == 2 ? 4 : 8;
    for (int o = 0; o < nc; ++o) {
        double w = 1.0;
        int qq[3] = {p[0], p[1], F.D == 3 ? p[2] : 0};
        for (int a = 0; a < F.D; ++a) {
            if ((o >> a) & 1) {
                qq[a] += s[a];
                w *= 0.25;
            } else {
                w *= 0.75;
            }
        }
        acc += w * coarse_value(Cl, qq);
    }
    F.x[f] += acc;
}

// ------------------------------------------------------------------ grid-wide kernels
__global__ void smooth_kernel(LV L, int colour, const int* done) {
    if (*done) return;
    long long m = colour_cells(L);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        smooth_cell(L, colour, i);
}

__global__ void restrict_kernel(LV F, LV Cl, const int* done) {
    if (*done) return;
    for (long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x; C < Cl.ncell; C += (long long)gridDim.x * blockDim.x)
        restrict_cell(F, Cl, C);
}

__global__ void prolong_kernel(LV F, LV Cl, const int* done) {
    if (*done) return;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < F.ncell; f += (long long)gridDim.x * blockDim.x)
        prolong_cell(F, Cl, f);
}

// the lower part of the V-cycle (levels first_cta .. nl-1) inside one CTA
__global__ void __launch_bounds__(1024) coarse_cycle_kernel(LVSet S, int nu1, int nu2, const int* done) {
    if (*done) return;
    __shared__ double sb[DENSE_MAX + 1];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int l = S.first_cta; l < S.nl - 1; ++l) {
        const LV& L = S.l[l];
        for (int it = 0; it < nu1; ++it)
            for (int col = 0; col < L.ncol; ++col) {
                long long m = colour_cells(L);
                for (long long i = tid; i < m; i += nt) smooth_cell(L, col, i);
                __syncthreads();
            }
        const LV& Cl = S.l[l + 1];
        for (long long C = tid; C < Cl.ncell; C += nt) restrict_cell(L, Cl, C);
        __syncthreads();
    }
    // coarsest: dense solve x = inv * [b; 0]
    {
        const LV& L = S.l[S.nl - 1];
        int m = S.dense_m;
        int mm = m + (S.singular ? 1 : 0);
        for (int i = tid; i < mm; i += nt) sb[i] = i < m ? L.b[i] : 0.0;
        __syncthreads();
        for (int i = tid; i < m; i += nt) {
            const double* row = S.dense_inv + (long long)i * mm;
            double acc = 0.0;
            for (int k = 0; k < mm; ++k) acc += row[k] * sb[k];
            L.x[i] = acc;
        }
        __syncthreads();
    }
    for (int l = S.nl - 2; l >= S.first_cta; --l) {
        const LV& L = S.l[l];
        const LV& Cl = S.l[l + 1];
        for (long long f = tid; f < L.ncell; f += nt) prolong_cell(L, Cl, f);
        __syncthreads();
        for (int it = 0; it < nu2; ++it)
            for (int col = L.ncol - 1; col >= 0; --col) {
                long long m = colour_cells(L);
                for (long long i = tid; i < m; i += nt) smooth_cell(L, col, i);
                __syncthreads();
            }
    }
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[2 * w] = a;
        sh[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            x += sh[2 * i];
            y += sh[2 * i + 1];
        }
        a = x;
        b = y;
    }
}

// mode 0: (||b - A x||^2, ||b||^2); mode 1: (sum b, 0); mode 2: (sum J x, 0)
__global__ void reduce_kernel(LV L, int mode, const double* Jc, double* part, const int* done) {
    if (done && *done) return;
    __shared__ double sh[64];
    double a = 0.0, b = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < L.ncell; c += (long long)gridDim.x * blockDim.x) {
        if (mode == 0) {
            int q[3];
            cell_coords(L, c, q);
            double r = L.b[c] - apply_row(L, c, q, false);
            a += r * r;
            b += L.b[c] * L.b[c];
        } else if (mode == 1) {
            a += L.b[c];
        } else {
            a += Jc[c] * L.x[c];
        }
    }
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// sums the block partials in a fixed order; mode 0 updates the convergence state
__global__ void norm_final_kernel(const double* part, int nb, double rtol, int count_cycle, DevCounters* ctr,
                                  int* done) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (*done) return;
    double rr = 0.0, bb = 0.0;
    for (int i = 0; i < nb; ++i) {
        rr += part[2 * i];
        bb += part[2 * i + 1];
    }
    double res = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
    if (count_cycle) ctr->mg_cycles += 1;
    ctr->mg_residual = res;
    ctr->mg_bnorm = sqrt(bb);
    if (res <= rtol) {
        *done = 1;
        ctr->mg_converged = 1;
    }
}

// b -= (sum b / sum J) J  (singular problems)
__global__ void project_kernel(LV L, const double* part, int nb, double sumJ, const double* Jc) {
    __shared__ double shift;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[2 * i];
        shift = s / sumJ;
    }
    __syncthreads();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < L.ncell; c += (long long)gridDim.x * blockDim.x)
        L.b[c] -= shift * Jc[c];
}

// x -= (sum J x / sum J)  (gauge of singular problems)
__global__ void gauge_kernel(LV L, const double* part, int nb, double sumJ) {
    __shared__ double shift;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[2 * i];
        shift = s / sumJ;
    }
    __syncthreads();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < L.ncell; c += (long long)gridDim.x * blockDim.x)
        L.x[c] -= shift;
}

__global__ void reset_solve_kernel(DevCounters* ctr, int* done) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *done = 0;
        ctr->mg_cycles = 0;
        ctr->mg_converged = 0;
    }
}

// ------------------------------------------------------------------ setup kernels
struct AsmParams {
    LV L;
    const double* face[3];
    int bc[6];
    double bcv[6];
    double* A;
    double* bbc;  // may be null (coarse levels: homogeneous)
    int* cross_flag;
};

__device__ __forceinline__ int slot_of(int D, const int* o) {
    if (D == 2) {
        const int tab[9] = {5, 3, 6, 1, 0, 2, 7, 4, 8};
        return tab[(o[0] + 1) + 3 * (o[1] + 1)];
    }
    for (int k = 0; k < 19; ++k)
        if (c_off3[k][0] == o[0] && c_off3[k][1] == o[1] && c_off3[k][2] == o[2]) return k;
    return -1;
}

__global__ void assemble_kernel(AsmParams P) {
    const LV& L = P.L;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < L.ncell; c += (long long)gridDim.x * blockDim.x) {
        int q[3];
        cell_coords(L, c, q);
        double a[19];
        for (int k = 0; k < 19; ++k) a[k] = 0.0;
        double rb = 0.0;
        auto add = [&](int* o, double val) {
            // fold ghost targets on non-periodic axes (Dirichlet: -phi_in + 2 phi_b)
            for (int ax = 0; ax < L.D; ++ax) {
                int tgt = q[ax] + o[ax];
                if (o[ax] != 0 && !L.per[ax] && (tgt < 0 || tgt >= L.n[ax])) {
                    int side = tgt < 0 ? 0 : 1;
                    o[ax] = 0;
                    if (P.bc[2 * ax + side] == CPIC_BC_DIRICHLET) {
                        rb -= 2.0 * val * P.bcv[2 * ax + side];
                        val = -val;
                    }
                }
            }
            int k = slot_of(L.D, o);
            a[k] += val;
        };
        for (int ax = 0; ax < L.D; ++ax) {
            int fn[3] = {L.n[0], L.n[1], L.D == 3 ? L.n[2] : 1};
            fn[ax] += 1;
            long long nf = (long long)fn[0] * fn[1] * fn[2];
            for (int side = 0; side < 2; ++side) {
                int fq[3] = {q[0], q[1], q[2]};
                fq[ax] += side;
                long long f = fq[0] + (long long)fn[0] * (fq[1] + (long long)fn[1] * fq[2]);
                double cf[3] = {0, 0, 0};
                for (int b = 0; b < L.D; ++b) cf[b] = P.face[ax][(long long)b * nf + f];
                bool boundary = !L.per[ax] && (fq[ax] == 0 || fq[ax] == L.n[ax]);
                if (boundary) {
                    if (P.bc[2 * ax + side] == CPIC_BC_DIRICHLET) {
                        a[0] += 2.0 * cf[ax];
                        rb += 2.0 * cf[ax] * P.bcv[2 * ax + side];
                    }
                    continue;
                }
                double sgn = side == 0 ? 1.0 : -1.0;
                int oR = side == 0 ? 0 : 1, oL = side == 0 ? -1 : 0;
                int o[3] = {0, 0, 0};
                o[ax] = oR;
                add(o, sgn * cf[ax]);
                o[0] = o[1] = o[2] = 0;
                o[ax] = oL;
                add(o, -sgn * cf[ax]);
                for (int b = 0; b < L.D; ++b) {
                    if (b == ax || cf[b] == 0.0) continue;
                    for (int sb = -1; sb <= 1; sb += 2) {
                        double val = sgn * sb * cf[b] * 0.25;
                        int o1[3] = {0, 0, 0};
                        o1[ax] = oR;
                        o1[b] = sb;
                        add(o1, val);
                        int o2[3] = {0, 0, 0};
                        o2[ax] = oL;
                        o2[b] = sb;
                        add(o2, val);
                    }
                }
            }
        }
        int faces = 2 * L.D + 1;
        bool cross = false;
        for (int k = 0; k < L.S; ++k) {
            P.A[(long long)k * L.ncell + c] = a[k];
            if (k >= faces && a[k] != 0.0) cross = true;
        }
        if (cross) atomicOr(P.cross_flag, 1);
        if (P.bbc) P.bbc[c] = rb;
    }
}

// dense matrix of the coarsest level (bordered with ones when singular), row-major mm x mm
__global__ void dense_matrix_kernel(LV L, int singular, double* M) {
    int m = (int)L.ncell, mm = m + (singular ? 1 : 0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)mm * mm; e += (long long)gridDim.x * blockDim.x)
        M[e] = 0.0;
    __syncthreads();
    if (blockIdx.x != 0) return;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        int q[3];
        cell_coords(L, c, q);
        for (int k = 0; k < L.used; ++k) {
            int o[3];
            offsets(L.D, k, o);
            long long nb = nbr(L, q, o);
            double v = L.A[(long long)k * L.ncell + c];
            if (v != 0.0) M[(long long)c * mm + nb] += v;
        }
        if (singular) {
            M[(long long)c * mm + m] = 1.0;
            M[(long long)m * mm + c] = 1.0;
        }
    }
}

// Gauss-Jordan inverse with partial pivoting, one block (setup only)
__global__ void gauss_jordan_kernel(double* M, double* Inv, int n, int* fail) {
    __shared__ int piv;
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) Inv[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int col = 0; col < n; ++col) {
        if (threadIdx.x == 0) {
            int best = col;
            double bv = fabs(M[(long long)col * n + col]);
            for (int r = col + 1; r < n; ++r) {
                double v = fabs(M[(long long)r * n + col]);
                if (v > bv) {
                    bv = v;
                    best = r;
                }
            }
            piv = best;
            if (bv == 0.0) *fail = 1;
        }
        __syncthreads();
        int p = piv;
        if (p != col)
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                double t = M[(long long)col * n + k];
                M[(long long)col * n + k] = M[(long long)p * n + k];
                M[(long long)p * n + k] = t;
                t = Inv[(long long)col * n + k];
                Inv[(long long)col * n + k] = Inv[(long long)p * n + k];
                Inv[(long long)p * n + k] = t;
            }
        __syncthreads();
        double d = M[(long long)col * n + col];
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            M[(long long)col * n + k] /= d;
            Inv[(long long)col * n + k] /= d;
        }
        __syncthreads();
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
            int r = (int)(e / n), k = (int)(e % n);
            if (r == col) continue;
            double f = M[(long long)r * n + col];
            if (k == col) continue;  // column col is cleared below
            M[e] -= f * M[(long long)col * n + k];
            Inv[e] -= f * Inv[(long long)col * n + k];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            if (r == col) continue;
            double f = M[(long long)r * n + col];
            Inv[(long long)r * n + col] -= f * Inv[(long long)col * n + col];
            M[(long long)r * n + col] = 0.0;
        }
        __syncthreads();
    }
}

LV make_lv(const cpic_run* r, int l) {
    const Level& Lv = r->lev[l];
    LV L;
    L.D = r->D;
    for (int a = 0; a < 3; ++a) {
        L.n[a] = a < r->D ? Lv.n[a] : 1;
        L.per[a] = a < r->D ? (r->cfg.field_bc[2 * a] == CPIC_BC_PERIODIC) : 0;
    }
    for (int f = 0; f < 6; ++f) L.bc[f] = r->cfg.field_bc[f];
    L.ncell = Lv.ncell;
    L.S = Lv.S;
    L.used = Lv.cross ? Lv.S : 2 * r->D + 1;
    L.ncol = Lv.cross ? (1 << r->D) : 2;
    L.A = Lv.A;
    L.x = Lv.x;
    L.b = Lv.b;
    return L;
}

int grid_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

LVSet make_set(const cpic_run* r) {
    LVSet S;
    S.nl = r->nlevels;
    S.first_cta = r->nlevels - 1;
    for (int l = 0; l < r->nlevels; ++l) {
        S.l[l] = make_lv(r, l);
        if (r->lev[l].ncell <= COARSE_CELLS && l < S.first_cta) S.first_cta = l;
    }
    S.dense_inv = r->dense_inv;
    S.dense_m = (int)r->lev[r->nlevels - 1].ncell;
    S.singular = r->singular ? 1 : 0;
    return S;
}

}  // namespace

int mg_setup(cpic_run* r) {
    int* flag = reinterpret_cast<int*>(r->red + 2 * RED_BLOCKS + 4);
    for (int l = 0; l < r->nlevels; ++l) {
        Level& Lv = r->lev[l];
        CPIC_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), r->stream));
        AsmParams P;
        Lv.cross = 1;  // make_lv stores all entries while assembling
        P.L = make_lv(r, l);
        for (int a = 0; a < 3; ++a) P.face[a] = Lv.face[a];
        for (int f = 0; f < 6; ++f) {
            P.bc[f] = r->cfg.field_bc[f];
            P.bcv[f] = l == 0 ? r->cfg.field_bc_value[f] : 0.0;
        }
        P.A = Lv.A;
        P.bbc = l == 0 ? r->rhs_bc : nullptr;
        P.cross_flag = flag;
        assemble_kernel<<<grid_blocks(Lv.ncell, 256), 256, 0, r->stream>>>(P);
        CPIC_CHECK_LAUNCH();
        int hflag = 0;
        CPIC_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
        Lv.cross = hflag;
    }
    // dense inverse of the coarsest level
    const Level& Lc = r->lev[r->nlevels - 1];
    int m = (int)Lc.ncell;
    int mm = m + (r->singular ? 1 : 0);
    r->dense_m = mm;
    double* M = r->dense_tmp;
    LV L = make_lv(r, r->nlevels - 1);
    dense_matrix_kernel<<<1, 256, 0, r->stream>>>(L, r->singular ? 1 : 0, M);
    CPIC_CHECK_LAUNCH();
    int* fail = flag;
    CPIC_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), r->stream));
    gauss_jordan_kernel<<<1, 1024, 0, r->stream>>>(M, r->dense_inv, mm, fail);
    CPIC_CHECK_LAUNCH();
    int hfail = 0;
    CPIC_CUDA(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    if (hfail) {
        set_error("coarsest multigrid operator is singular");
        return CPIC_ERR_INVALID;
    }
    return CPIC_OK;
}

static int vcycle_grid(cpic_run* r, const LVSet& S, int l, const int* done, int nu1, int nu2) {
    if (l >= S.first_cta) {
        coarse_cycle_kernel<<<1, 1024, 0, r->stream>>>(S, nu1, nu2, done);
        CPIC_CHECK_LAUNCH();
        return CPIC_OK;
    }
    const LV& L = S.l[l];
    const LV& C = S.l[l + 1];
    int tb = 256;
    for (int it = 0; it < nu1; ++it)
        for (int col = 0; col < L.ncol; ++col) {
            smooth_kernel<<<grid_blocks(L.ncell / L.ncol, tb), tb, 0, r->stream>>>(L, col, done);
            CPIC_CHECK_LAUNCH();
        }
    restrict_kernel<<<grid_blocks(C.ncell, tb), tb, 0, r->stream>>>(L, C, done);
    CPIC_CHECK_LAUNCH();
    int st = vcycle_grid(r, S, l + 1, done, nu1, nu2);
    if (st) return st;
    prolong_kernel<<<grid_blocks(L.ncell, tb), tb, 0, r->stream>>>(L, C, done);
    CPIC_CHECK_LAUNCH();
    for (int it = 0; it < nu2; ++it)
        for (int col = L.ncol - 1; col >= 0; --col) {
            smooth_kernel<<<grid_blocks(L.ncell / L.ncol, tb), tb, 0, r->stream>>>(L, col, done);
            CPIC_CHECK_LAUNCH();
        }
    return CPIC_OK;
}

int mg_solve(cpic_run* r, double rtol, int max_cycles, bool host_loop, int* cycles, double* res) {
    LVSet S = make_set(r);
    const LV& L0 = S.l[0];
    double* part = r->red;
    int* done = reinterpret_cast<int*>(r->red + 2 * RED_BLOCKS + 2);
    reset_solve_kernel<<<1, 32, 0, r->stream>>>(r->ctr, done);
    CPIC_CHECK_LAUNCH();
    int st = launch_rhs(r, r->lev[0].b);
    if (st) return st;
    if (r->singular) {
        reduce_kernel<<<RED_BLOCKS, 256, 0, r->stream>>>(L0, 1, r->lev[0].Jc, part, nullptr);
        CPIC_CHECK_LAUNCH();
        project_kernel<<<grid_blocks(L0.ncell, 256), 256, 0, r->stream>>>(L0, part, RED_BLOCKS, r->sumJ, r->lev[0].Jc);
        CPIC_CHECK_LAUNCH();
    }
    // initial residual (warm start from the previous phi)
    reduce_kernel<<<RED_BLOCKS, 256, 0, r->stream>>>(L0, 0, nullptr, part, done);
    CPIC_CHECK_LAUNCH();
    norm_final_kernel<<<1, 32, 0, r->stream>>>(part, RED_BLOCKS, rtol, 0, r->ctr, done);
    CPIC_CHECK_LAUNCH();
    const int nu1 = 2, nu2 = 2;
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        if (host_loop) {
            int hd = 0;
            CPIC_CUDA(cudaMemcpyAsync(&hd, done, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
            CPIC_CUDA(cudaStreamSynchronize(r->stream));
            if (hd) break;
        }
        st = vcycle_grid(r, S, 0, done, nu1, nu2);
        if (st) return st;
        reduce_kernel<<<RED_BLOCKS, 256, 0, r->stream>>>(L0, 0, nullptr, part, done);
        CPIC_CHECK_LAUNCH();
        norm_final_kernel<<<1, 32, 0, r->stream>>>(part, RED_BLOCKS, rtol, 1, r->ctr, done);
        CPIC_CHECK_LAUNCH();
    }
    if (r->singular) {
        reduce_kernel<<<RED_BLOCKS, 256, 0, r->stream>>>(L0, 2, r->lev[0].Jc, part, nullptr);
        CPIC_CHECK_LAUNCH();
        gauge_kernel<<<grid_blocks(L0.ncell, 256), 256, 0, r->stream>>>(L0, part, RED_BLOCKS, r->sumJ);
        CPIC_CHECK_LAUNCH();
    }
    st = launch_field_energy(r);
    if (st) return st;
    if (cycles || res) {
        DevCounters h;
        CPIC_CUDA(cudaMemcpyAsync(&h, r->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
        if (cycles) *cycles = h.mg_cycles;
        if (res) *res = h.mg_residual;
        if (!h.mg_converged) {
            set_error("multigrid: relative residual %.3e > %.3e after %d cycles", h.mg_residual, rtol, h.mg_cycles);
            return CPIC_ERR_NOT_CONVERGED;
        }
    }
    return CPIC_OK;
}

}  // namespace cpic
