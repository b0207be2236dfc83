// Row a9: the logical-space Poisson solve (Sec. II.B.3; eq. (poiscurv)), device resident.
//
// Discretisation (conservative finite volume with ghost cells): the flux through a face
// normal to axis a is a^{aa} (phi_R - phi_L) + sum_{b != a} a^{ab} / 4 [(phi_R(+b) + phi_L(+b))
// - (phi_R(-b) + phi_L(-b))], a^{ab} = Omega J g^{ab} from the geometry; Dirichlet ghosts
// 2 phi_b - phi_in (a Dirichlet face carries a^{aa} 2 (phi_in - phi_b)), Neumann ghosts
// phi_in (a Neumann face carries no flux), periodic wrap. The assembled row of cell c is
// M phi = Omega_c Q_c + (Dirichlet terms), M = -(divergence), stored as a 9-point (2D) or
// 19-point (3D) stencil of which only the 5/7 face entries are used when the map is
// orthogonal.
//
// Solver: multigrid, the method class the paper uses (Sec. II.B.3: coarse-grid correction
// plus Gauss-Seidel smoothing on each level), arranged for GB300, whose FP64 rate is ~1/64
// of its FP32 rate: the solution phi, the right-hand side and the residual are FP64, and
// each iteration solves for the correction with one FP32 V-cycle (mixed-precision
// iterative refinement):
//     r = b - M phi (FP64);  stop if ||r||_2 / ||b||_2 <= rtol;
//     e = V-cycle_FP32(M, float(r)) from e = 0;  phi += e (FP64).
// The FP32 cycle only has to reduce the error by its multigrid factor, so the iteration
// converges to FP64 accuracy at the rate of an FP64 multigrid.
// V-cycle: coarse levels rediscretised from the map sampled at every other vertex (BoxMG's
// variational coarse operators and operator-induced interpolation are not reproduced),
// restriction by summing the 2^D fine residuals (finite-volume conservation), (bi/tri)linear
// prolongation with homogeneous ghost rules, colour-ordered Gauss-Seidel (2 colours for
// 5/7-point stencils, 2^D colours with cross terms), levels of at most COARSE_CELLS cells
// inside one CTA, and a dense inverse on the coarsest level (bordered with the constant
// null vector when the problem is singular). A singular problem (no Dirichlet face) has its
// right-hand side projected by subtracting a uniform physical charge density and its
// solution gauged to sum_c J_c phi_c = 0.
//
// Optional outer Krylov iteration (cpic_set_solver): BiCGStab (van der Vorst 1992) on
// M phi = b, right-preconditioned by the same FP32 V-cycle, on the kernel-chain path. One
// iteration: p = r + beta (p - omega v); p^ = V(p); v = M p^, alpha = rho / (r^, v);
// s = r - alpha v; s^ = V(s); t = M s^, omega = (t, s) / (t, t); phi += alpha p^ + omega s^;
// then r = b - M phi is recomputed in FP64 (not updated), so the stopping test sees the true
// residual, and rho' = (r^, r), beta = (rho' / rho)(alpha / omega). A vanishing rho, alpha
// or omega restarts the recurrence with r^ = p = r. The direction vectors p, v, s and the
// products M p^ and M s^ only choose the search space and the step lengths alpha and omega:
// they are FP32 (the products with the FP32 copy of the full operator; FP64 on GB300 runs at
// 1/64 of the FP32 rate), while phi is only ever changed by FP64 additions of FP32 steps
// and the stopping test reads the FP64 residual, so the result's accuracy does not depend
// on them; the dot products accumulate in FP64.
//
// The residual kernel ends with a last-block reduction that decides whether to continue;
// it writes the decision into a CUDA graph conditional handle, so inside a captured step
// the cycle loop is a conditional WHILE node that runs on the device with no host round
// trip and no idle launches.
#include <stdlib.h>
#include <math.h>
#include <string.h>

#include <type_traits>

#include "internal.cuh"

namespace cpic {
namespace {

constexpr int RED_BLOCKS = 256;
// The V-cycle drops the cross entries of the stencil (face entries only: 2D+1 points, two
// colours) when no finest-level row's cross entries sum to more than this fraction of its
// diagonal, e.g. the shell map, orthogonal up to O(h^2) terms of a few 1e-3; the residual
// and the Krylov products keep the full operator, so only the preconditioner changes.
constexpr float PC_CROSS_DROP = 0.02f;

__constant__ int c_off2[9][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
// 3D slots: 19-point stencil, then the 8 corners that Galerkin coarse operators add
__constant__ int c_off3[27][3] = {{0, 0, 0},  {-1, 0, 0},  {1, 0, 0},  {0, -1, 0}, {0, 1, 0},
                                  {0, 0, -1}, {0, 0, 1},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
                                  {1, 1, 0},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
                                  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},
                                  {-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1},
                                  {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}, {1, 1, 1}};

template <typename R>
struct LV {
    int D;
    int n[3];
    int ncell;
    int S;      // stored stencil entries (9 / 27)
    int used;   // entries used (5/7 without cross terms, else 9 / 19, or 27 with Galerkin levels)
    int ncol;   // Gauss-Seidel colours (2 or 2^D)
    int per[3];
    int bc[6];
    const R* A;
    R* x;
    R* b;
    float* lw;  // 2D line relaxation: work [2][ncell] in global memory (FP32 levels)
    const R* pw;  // 2D operator-induced prolongation: own-parent weight per axis [2][ncell], or null
};

struct LVSet {
    int nl;
    int first_cta;  // first level solved inside one CTA
    int line;       // 1: alternating zebra line relaxation (2D) instead of point smoothing
    LV<float> l[MAX_LEVELS];
    const float* dense_inv;
    int dense_m;   // unknowns of the coarsest level
    int singular;
};

template <typename R>
__device__ __forceinline__ void cell_coords(const LV<R>& L, int c, int* q) {
    q[0] = c % L.n[0];
    int r = c / L.n[0];
    q[1] = r % L.n[1];
    q[2] = r / L.n[1];
}

template <typename R>
__device__ __forceinline__ int lin(const LV<R>& L, const int* q) {
    return q[0] + L.n[0] * (q[1] + L.n[1] * q[2]);
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
// coefficients after assembly, their index is clamped (setup kernels only)
template <typename R>
__device__ __forceinline__ int nbr(const LV<R>& L, const int* q, const int* o) {
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

// stencil offset of slot k along axis a (2D: 9 slots, 3D: 27 slots); called with
// unrolled constant arguments, so it folds away
__host__ __device__ constexpr int koff(int D, int k, int a) {
    constexpr int t2[9][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0},
                              {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}};
    constexpr int t3[27][3] = {{0, 0, 0},  {-1, 0, 0},  {1, 0, 0},  {0, -1, 0}, {0, 1, 0},  {0, 0, -1}, {0, 0, 1},
                               {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                               {1, 0, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},
                               {-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1},
                               {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}, {1, 1, 1}};
    return D == 2 ? t2[k][a] : t3[k][a];
}

// sum_{k >= K0} A_k x_{nb_k} for cell q with compile-time stencil shape <D, NPT>: the
// wrapped/clamped neighbour coordinates are computed once per axis, slot offsets fold to
// constants
template <int D, int NPT, int K0, typename R>
__device__ __forceinline__ R stencil_sum(const LV<R>& L, int c, const int* q) {
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = q[a] > 0 ? q[a] - 1 : (L.per[a] ? L.n[a] - 1 : 0);
        hi[a] = q[a] + 1 < L.n[a] ? q[a] + 1 : (L.per[a] ? 0 : L.n[a] - 1);
    }
    const int ix[3] = {lo[0], q[0], hi[0]};
    const int jy[3] = {L.n[0] * lo[1], L.n[0] * q[1], L.n[0] * hi[1]};
    int kz[3] = {0, 0, 0};
    if (D == 3) {
        const int pl = L.n[0] * L.n[1];
        kz[0] = pl * lo[2];
        kz[1] = pl * q[2];
        kz[2] = pl * hi[2];
    }
    R s = R(0);
#pragma unroll
    for (int k = K0; k < NPT; ++k) {
        const int idx = ix[koff(D, k, 0) + 1] + jy[koff(D, k, 1) + 1] + (D == 3 ? kz[koff(D, k, 2) + 1] : 0);
        s += L.A[k * L.ncell + c] * L.x[idx];
    }
    return s;
}

// sum_k A_k y_{nb_k} with the level's coefficients (type R) and values y of type TX,
// accumulated in R
template <int D, int NPT, typename R, typename TX>
__device__ __forceinline__ R stencil_apply(const LV<R>& L, const TX* __restrict__ y, int c, const int* q) {
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = q[a] > 0 ? q[a] - 1 : (L.per[a] ? L.n[a] - 1 : 0);
        hi[a] = q[a] + 1 < L.n[a] ? q[a] + 1 : (L.per[a] ? 0 : L.n[a] - 1);
    }
    const int ix[3] = {lo[0], q[0], hi[0]};
    const int jy[3] = {L.n[0] * lo[1], L.n[0] * q[1], L.n[0] * hi[1]};
    int kz[3] = {0, 0, 0};
    if (D == 3) {
        const int pl = L.n[0] * L.n[1];
        kz[0] = pl * lo[2];
        kz[1] = pl * q[2];
        kz[2] = pl * hi[2];
    }
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = ix[koff(D, k, 0) + 1] + jy[koff(D, k, 1) + 1] + (D == 3 ? kz[koff(D, k, 2) + 1] : 0);
        acc += L.A[k * L.ncell + c] * (R)y[idx];
    }
    return acc;
}

// cells of one colour: parity colouring (i + j + k) % 2 when ncol == 2 (n[0] even), one
// bit per axis otherwise (NPT > 2D + 1). The colour-local index space (m, j, k) has a
// half-length first axis.
template <int D, int NPT>
struct Col {
    static constexpr bool parity = NPT == 2 * D + 1;
    template <typename R>
    static __device__ __forceinline__ void dims(const LV<R>& L, int* d) {
        d[0] = L.n[0] / 2;
        d[1] = parity ? L.n[1] : L.n[1] / 2;
        d[2] = D == 3 ? (parity ? L.n[2] : L.n[2] / 2) : 1;
    }
    static __device__ __forceinline__ void cell(int colour, int m, int j, int k, int* q) {
        if (parity) {
            q[0] = 2 * m + ((j + k + colour) & 1);
            q[1] = j;
            q[2] = k;
        } else {
            q[0] = 2 * m + (colour & 1);
            q[1] = 2 * j + ((colour >> 1) & 1);
            q[2] = D == 3 ? 2 * k + ((colour >> 2) & 1) : 0;
        }
    }
};

template <int D, int NPT, typename R>
__device__ __forceinline__ void smooth_at(const LV<R>& L, const R* dinv, const int* q) {
    const int c = q[0] + L.n[0] * (q[1] + L.n[1] * q[2]);
    L.x[c] = (L.b[c] - stencil_sum<D, NPT, 1>(L, c, q)) * dinv[c];
}

template <int D, int NPT, typename R>
__device__ __forceinline__ void restrict_at(const LV<R>& F, const LV<R>& Cl, const int* qc) {
    R acc = R(0);
#pragma unroll
    for (int ch = 0; ch < (D == 2 ? 4 : 8); ++ch) {
        int q[3] = {2 * qc[0] + (ch & 1), 2 * qc[1] + ((ch >> 1) & 1), D == 3 ? 2 * qc[2] + ((ch >> 2) & 1) : 0};
        int f = q[0] + F.n[0] * (q[1] + F.n[1] * q[2]);
        acc += F.b[f] - stencil_sum<D, NPT, 0>(F, f, q);
    }
    int C = qc[0] + Cl.n[0] * (qc[1] + Cl.n[1] * qc[2]);
    Cl.b[C] = acc;
    Cl.x[C] = R(0);
}

// Prolongation x_f += sum over the 2^D parents of w * x_parent: per axis the fine cell's own
// parent (weight own, 3/4 when bilinear) and the parent on the fine cell's side (1 - own,
// with the correction's ghost rules: periodic wrap, or else the boundary parent itself, its
// sign flipped at a Dirichlet face). The per-axis offsets, signs
// and weights are set up once and combined per parent: w = ((1 w_0) w_1) w_2 and the signed
// parent value, accumulated over the parents in order.
template <int D, typename R>
__device__ __forceinline__ void prolong_at(const LV<R>& F, const LV<R>& Cl, const int* q) {
    const int f = q[0] + F.n[0] * (q[1] + F.n[1] * q[2]);
    R own[3] = {R(0.75), R(0.75), R(0.75)};  // weight of the own parent per axis (bilinear: 3/4)
    if (F.pw)
#pragma unroll
        for (int a = 0; a < D; ++a) own[a] = F.pw[a * F.ncell + f];
    int off[3][2];
    R sg[3][2], wt[3][2];
    int stride = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int pa = q[a] >> 1;
        int nb = pa + ((q[a] & 1) ? 1 : -1);
        R sign = R(1);
        if (nb < 0 || nb >= Cl.n[a]) {
            const int side = nb < 0 ? 0 : 1;
            if (Cl.per[a]) {
                nb = nb < 0 ? nb + Cl.n[a] : nb - Cl.n[a];
            } else {
                nb = side == 0 ? 0 : Cl.n[a] - 1;
                if (Cl.bc[2 * a + side] == CPIC_BC_DIRICHLET) sign = -sign;
            }
        }
        off[a][0] = pa * stride;
        off[a][1] = nb * stride;
        sg[a][0] = R(1);
        sg[a][1] = sign;
        wt[a][0] = own[a];
        wt[a][1] = R(1) - own[a];
        stride *= Cl.n[a];
    }
    R acc = R(0);
#pragma unroll
    for (int o = 0; o < (D == 2 ? 4 : 8); ++o) {
        R w = R(1), sign = R(1);
        int idx = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int bit = (o >> a) & 1;
            w *= wt[a][bit];
            sign *= sg[a][bit];
            idx += off[a][bit];
        }
        acc += w * (sign * Cl.x[idx]);
    }
    F.x[f] += acc;
}

// ------------------------------------------------------------------ line relaxation
// Zebra line Gauss-Seidel (robust for anisotropic cells, Sec. II.B.3): every line of cells
// along `axis` is solved exactly (a tridiagonal system, cyclic on a periodic axis) with the
// cells of the neighbouring lines at their current values. Lines are coloured by the parity
// of their transverse coordinates (a periodic transverse axis with an odd count gives its
// last index a third colour), so lines of one colour share no stencil entry and are
// independent. One sweep relaxes the lines along axis 0, then axis 1 (then axis 2).
template <int D, int NPT>
__device__ void line_solve(const LV<float>& L, int axis, int base) {
    const int n = L.n[axis];
    const int stride = axis == 0 ? 1 : (axis == 1 ? L.n[0] : L.n[0] * L.n[1]);
    const int km = 1 + 2 * axis, kp = 2 + 2 * axis;  // in-line -1 / +1 slots
    const bool per = L.per[axis] != 0;
    float* cp = L.lw;            // eliminated upper diagonal (cells of this line only)
    float* z = L.lw + L.ncell;   // second solve of the cyclic case
    const int nc = L.ncell;
    auto coeff = [&](int k, int c) { return L.A[k * nc + c]; };
    // right-hand side of cell c: b - (off-line stencil terms), neighbours as in stencil_sum
    auto rhs = [&](int c) {
        int q[3];
        cell_coords(L, c, q);
        int lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            lo[a] = q[a] > 0 ? q[a] - 1 : (L.per[a] ? L.n[a] - 1 : 0);
            hi[a] = q[a] + 1 < L.n[a] ? q[a] + 1 : (L.per[a] ? 0 : L.n[a] - 1);
        }
        const int ix[3] = {lo[0], q[0], hi[0]};
        const int jy[3] = {L.n[0] * lo[1], L.n[0] * q[1], L.n[0] * hi[1]};
        int kz[3] = {0, 0, 0};
        if (D == 3) {
            const int pl = L.n[0] * L.n[1];
            kz[0] = pl * lo[2];
            kz[1] = pl * q[2];
            kz[2] = pl * hi[2];
        }
        float sacc = L.b[c];
#pragma unroll
        for (int k = 1; k < NPT; ++k) {
            if (k == km || k == kp) continue;
            sacc -= coeff(k, c) * L.x[ix[koff(D, k, 0) + 1] + jy[koff(D, k, 1) + 1] + (D == 3 ? kz[koff(D, k, 2) + 1] : 0)];
        }
        return sacc;
    };
    if (n == 1) {
        const int c = base;
        const float d = coeff(0, c) + (per ? coeff(km, c) + coeff(kp, c) : 0.0f);
        L.x[c] = rhs(c) / d;
        return;
    }
    if (n == 2 && per) {  // both in-line neighbours are the other cell
        const int c0 = base, c1 = base + stride;
        const float a00 = coeff(0, c0), a01 = coeff(km, c0) + coeff(kp, c0);
        const float a10 = coeff(km, c1) + coeff(kp, c1), a11 = coeff(0, c1);
        const float r0 = rhs(c0), r1 = rhs(c1);
        const float det = a00 * a11 - a01 * a10;
        L.x[c0] = (r0 * a11 - a01 * r1) / det;
        L.x[c1] = (a00 * r1 - a10 * r0) / det;
        return;
    }
    // cyclic system: corners beta = A[0][n-1] (slot km of cell 0), alpha = A[n-1][0] (slot kp
    // of the last cell); Sherman-Morrison with gamma = -d_0: T' = A - v w^T, v = (gamma, 0, ..,
    // 0, alpha), w = (1, 0, .., 0, beta / gamma); x = y - z (w . y) / (1 + w . z) with T' y = r,
    // T' z = v
    const int cl = base + (n - 1) * stride;
    const float beta = per ? coeff(km, base) : 0.0f, alpha = per ? coeff(kp, cl) : 0.0f;
    const float gamma = -coeff(0, base);
    float prev_cp = 0.0f, prev_y = 0.0f, prev_z = 0.0f;
    for (int i = 0; i < n; ++i) {
        const int c = base + i * stride;
        float d = coeff(0, c);
        const float l = i == 0 ? 0.0f : coeff(km, c);
        const float u = i == n - 1 ? 0.0f : coeff(kp, c);
        if (per && i == 0) d -= gamma;
        if (per && i == n - 1) d -= alpha * beta / gamma;
        const float den = d - l * prev_cp;
        const float ci = u / den;
        const float yi = (rhs(c) - l * prev_y) / den;
        cp[c] = ci;
        L.x[c] = yi;
        prev_cp = ci;
        prev_y = yi;
        if (per) {
            const float v = i == 0 ? gamma : (i == n - 1 ? alpha : 0.0f);
            const float zi = (v - l * prev_z) / den;
            z[c] = zi;
            prev_z = zi;
        }
    }
    for (int i = n - 2; i >= 0; --i) {
        const int c = base + i * stride, cn = c + stride;
        L.x[c] -= cp[c] * L.x[cn];
        if (per) z[c] -= cp[c] * z[cn];
    }
    if (per) {
        const float fact = (L.x[base] + beta * L.x[cl] / gamma) / (1.0f + z[base] + beta * z[cl] / gamma);
        for (int i = 0; i < n; ++i) {
            const int c = base + i * stride;
            L.x[c] -= fact * z[c];
        }
    }
}

// colours per transverse axis (2, or 3 for a periodic axis of odd size) and of an index
__host__ __device__ inline int tcolours(int n, int per) { return per && (n & 1) ? 3 : 2; }
__host__ __device__ inline int tcolour(int x, int n, int per) { return tcolours(n, per) == 3 && x == n - 1 ? 2 : (x & 1); }

// the transverse axes of lines along `axis`, and the number of line colours
template <typename R>
__host__ __device__ inline void line_axes(const LV<R>& L, int D, int axis, int& b, int& c, int& ncol) {
    b = axis == 0 ? 1 : 0;
    c = D == 3 ? (axis == 2 ? 1 : 2) : -1;
    ncol = tcolours(L.n[b], L.per[b]) * (c >= 0 ? tcolours(L.n[c], L.per[c]) : 1);
}

// does line `idx` (transverse index, b fastest) have colour `col`? returns its first cell
template <typename R>
__host__ __device__ inline int line_start(const LV<R>& L, int D, int axis, int idx, int col) {
    int b, c, ncol;
    line_axes(L, D, axis, b, c, ncol);
    const int xb = idx % L.n[b], xc = c >= 0 ? idx / L.n[b] : 0;
    const int cb = tcolour(xb, L.n[b], L.per[b]);
    const int cc = c >= 0 ? tcolour(xc, L.n[c], L.per[c]) : 0;
    if (cb + tcolours(L.n[b], L.per[b]) * cc != col) return -1;
    int q[3] = {0, 0, 0};
    q[b] = xb;
    if (c >= 0) q[c] = xc;
    return q[0] + L.n[0] * (q[1] + L.n[1] * q[2]);
}

template <int D, int NPT>
__global__ void line_kernel(LV<float> L, int axis, int col, int lines) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= lines) return;
    const int start = line_start(L, D, axis, idx, col);
    if (start >= 0) line_solve<D, NPT>(L, axis, start);
}

// ------------------------------------------------------------------ Galerkin coarse operators
// A_C = R A P (BoxMG's variational coarse operator, Sec. II.B.3) with the V-cycle's own
// transfers: R sums the 2^D fine children, P is the prolongation of prolong_at (bilinear or
// operator-induced weights) with its homogeneous ghost rules (an out-of-range coarse source
// is the boundary cell, negated at a Dirichlet face; periodic axes wrap). Every source of
// P e_C' reached from a child of C lies within one coarse cell of C, so the coarse operator
// has the 3^D-point shape (9 in 2D, 27 in 3D). FP64, one thread per coarse cell, entries in
// stencil-slot order.
template <int D>
__global__ void galerkin_kernel(LV<double> F, LV<double> C, double* Ac) {
    constexpr int NS = D == 2 ? 9 : 27, NCH = 1 << D;
    for (int cc = blockIdx.x * blockDim.x + threadIdx.x; cc < C.ncell; cc += gridDim.x * blockDim.x) {
        int Q[3];
        cell_coords(C, cc, Q);
        double acc[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[k] = 0.0;
        for (int ch = 0; ch < NCH; ++ch) {
            int fq[3] = {2 * Q[0] + (ch & 1), 2 * Q[1] + ((ch >> 1) & 1), D == 3 ? 2 * Q[2] + ((ch >> 2) & 1) : 0};
            const int f = fq[0] + F.n[0] * (fq[1] + F.n[1] * fq[2]);
            for (int k = 0; k < NS; ++k) {
                const double a = F.A[k * F.ncell + f];
                if (a == 0.0) continue;
                int g[3], p[3], sdir[3];
                for (int ax = 0; ax < D; ++ax) {
                    g[ax] = fq[ax] + koff(D, k, ax);  // unwrapped
                    p[ax] = g[ax] >> 1;               // floor(g / 2), also for g = -1
                    sdir[ax] = (g[ax] & 1) ? 1 : -1;
                }
                double own[3] = {0.75, 0.75, 0.75};  // the prolongation row of fine cell g
                if (F.pw) {
                    int gw[3] = {0, 0, 0};
                    for (int ax = 0; ax < D; ++ax) gw[ax] = (g[ax] % F.n[ax] + F.n[ax]) % F.n[ax];
                    const int gi = gw[0] + F.n[0] * (gw[1] + F.n[1] * gw[2]);
                    for (int ax = 0; ax < D; ++ax) own[ax] = F.pw[ax * F.ncell + gi];
                }
                for (int o = 0; o < NCH; ++o) {
                    double w = 1.0;
                    int off[3] = {0, 0, 0};
                    for (int ax = 0; ax < D; ++ax) {
                        const int src = p[ax] + (((o >> ax) & 1) ? sdir[ax] : 0);
                        w *= ((o >> ax) & 1) ? 1.0 - own[ax] : own[ax];
                        off[ax] = src - Q[ax];
                        if (!C.per[ax] && (src < 0 || src >= C.n[ax])) {
                            off[ax] = 0;  // the ghost maps onto this boundary cell
                            const int side = src < 0 ? 0 : 1;
                            if (C.bc[2 * ax + side] == CPIC_BC_DIRICHLET) w = -w;
                        }
                    }
                    int slot = 0;
                    for (int k2 = 0; k2 < NS; ++k2)
                        if (koff(D, k2, 0) == off[0] && koff(D, k2, 1) == off[1] && (D == 2 || koff(D, k2, 2) == off[2]))
                            slot = k2;
                    acc[slot] += w * a;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) Ac[k * C.ncell + cc] = acc[k];
    }
}

// ------------------------------------------------------------------ operator-induced prolongation
// BoxMG takes its interpolation weights from the operator (Sec. II.B.3). Reading for this
// cell-centred 2:1 hierarchy: along each axis a fine cell is interpolated from its own
// coarse parent C and the parent's neighbour N on the fine cell's side, with the weights of
// the flux-continuous 1D solution between the two coarse centres: resistances from the fine
// operator's couplings across faces, collapsed over the transverse directions (the sum of
// the entries linking the two layers of cells, as BoxMG collapses its stencils),
//   R1 = 1 / (2 g(f_other -> f))   (C's centre is the face between its two children),
//   R2 = 1 / g(f -> n) + 1 / (2 g(n -> n_other))   (n, n_other: N's children, n next to f),
// own-parent weight R2 / (R1 + R2); uniform couplings give bilinear's 3/4. The weights of a
// cell are the product of its axes' weights. Cells whose neighbour parent is outside a
// non-periodic boundary, or whose couplings are not all positive, keep 3/4 (the ghost rule
// of prolong_at then applies).
template <int D>
__global__ void interp_weights_kernel(LV<double> F, double* pw, float* pw32) {
    constexpr int NS = D == 2 ? 9 : 27;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F.ncell; f += gridDim.x * blockDim.x) {
        int q[3];
        cell_coords(F, f, q);
        for (int ax = 0; ax < D; ++ax) {
            double w = 0.75;
            const int s = (q[ax] & 1) ? 1 : -1;  // side of the neighbour parent
            const int nc = F.n[ax] / 2;
            const int pn = (q[ax] >> 1) + s;      // neighbour parent (coarse index)
            const bool inside = F.per[ax] || (pn >= 0 && pn < nc);
            if (inside) {
                // fine cells along the axis: f_other, f, n, n_other at offsets -s, 0, s, 2s
                auto cell = [&](int d) {
                    int c[3] = {q[0], q[1], q[2]};
                    c[ax] = ((c[ax] + d) % F.n[ax] + F.n[ax]) % F.n[ax];
                    return c[0] + F.n[0] * (c[1] + F.n[1] * c[2]);
                };
                // collapsed coupling from cell c towards dir (+-1) along ax
                auto coupling = [&](int c, int dir) {
                    double gsum = 0.0;
                    for (int k = 1; k < NS; ++k)
                        if (koff(D, k, ax) == dir) gsum -= F.A[k * F.ncell + c];
                    return gsum;
                };
                const double g1 = coupling(cell(-s), s);  // f_other -> f
                const double g2 = coupling(f, s);          // f -> n
                const double g3 = coupling(cell(s), s);    // n -> n_other
                if (g1 > 0.0 && g2 > 0.0 && g3 > 0.0) {
                    const double R1 = 0.5 / g1, R2 = 1.0 / g2 + 0.5 / g3;
                    w = R2 / (R1 + R2);
                }
            }
            pw[ax * F.ncell + f] = w;
            pw32[ax * F.ncell + f] = (float)w;
        }
    }
}

// ------------------------------------------------------------------ FP32 cycle kernels
// 3D launch geometry: x covers the first (index) dimension, y the second, z the third.
template <int D, int NPT>
__global__ void smooth_kernel(LV<float> L, const float* __restrict__ dinv, int colour) {
    int d[3];
    Col<D, NPT>::dims(L, d);
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (m >= d[0] || j >= d[1] || k >= d[2]) return;
    int q[3];
    Col<D, NPT>::cell(colour, m, j, k, q);
    smooth_at<D, NPT>(L, dinv, q);
}

template <int D, int NPT>
__global__ void __launch_bounds__(256) restrict_kernel(LV<float> F, LV<float> Cl) {
    // one thread per fine cell (block RB_X x RB_Y x RB_Z fine cells): its residual goes to
    // shared memory, then one thread per coarse cell of the block sums its 2^D children in
    // restrict_at's order (children ch = 0 .. 2^D - 1, axis 0 fastest)
    constexpr int BX = 32, BY = D == 3 ? 4 : 8, BZ = D == 3 ? 2 : 1;
    __shared__ float rs[BX * BY * BZ];
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int t = tx + BX * (ty + BY * tz);
    int q[3] = {(int)blockIdx.x * BX + tx, (int)blockIdx.y * BY + ty, D == 3 ? (int)blockIdx.z * BZ + tz : 0};
    float r = 0.0f;
    if (q[0] < F.n[0] && q[1] < F.n[1] && q[2] < F.n[2]) {
        const int f = q[0] + F.n[0] * (q[1] + F.n[1] * q[2]);
        r = F.b[f] - stencil_sum<D, NPT, 0>(F, f, q);
    }
    rs[t] = r;
    __syncthreads();
    constexpr int CX = BX / 2, CY = BY / 2, CZ = D == 3 ? BZ / 2 : 1;
    if (t < CX * CY * CZ) {
        const int ci = t % CX, cj = (t / CX) % CY, ck = t / (CX * CY);
        const int qc[3] = {(int)blockIdx.x * CX + ci, (int)blockIdx.y * CY + cj, D == 3 ? (int)blockIdx.z * CZ + ck : 0};
        if (qc[0] < Cl.n[0] && qc[1] < Cl.n[1] && qc[2] < Cl.n[2]) {
            float acc = 0.0f;
#pragma unroll
            for (int ch = 0; ch < (D == 2 ? 4 : 8); ++ch)
                acc += rs[(2 * ci + (ch & 1)) + BX * ((2 * cj + ((ch >> 1) & 1)) + BY * (D == 3 ? 2 * ck + ((ch >> 2) & 1) : 0))];
            const int C = qc[0] + Cl.n[0] * (qc[1] + Cl.n[1] * qc[2]);
            Cl.b[C] = acc;
            Cl.x[C] = 0.0f;
        }
    }
}

template <int D>
__global__ void prolong_kernel(LV<float> F, LV<float> Cl) {
    int q[3] = {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(blockIdx.y * blockDim.y + threadIdx.y), (int)blockIdx.z};
    if (q[0] >= F.n[0] || q[1] >= F.n[1] || q[2] >= F.n[2]) return;
    prolong_at<D>(F, Cl, q);
}

// The lower part of the V-cycle (levels first_cta .. nl-1) inside one CTA, with every
// level's stencil, inverse diagonal, correction and right-hand side in shared memory (the
// top level's right-hand side comes from global memory, its correction goes back there).
// All levels of a run share one stencil shape <D, NPT>.
template <int D, int NPT>
__global__ void __launch_bounds__(512) coarse_cycle_kernel(LVSet S, int nu1, int nu2) {
    extern __shared__ float sm[];
    __shared__ float sb[DENSE_MAX + 1];
    __shared__ LV<float> V[MAX_LEVELS];
    __shared__ float* Dv[MAX_LEVELS];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        int off = 0;
        for (int l = S.first_cta; l < S.nl; ++l) {
            V[l] = S.l[l];
            V[l].A = sm + off;
            off += NPT * S.l[l].ncell;
            Dv[l] = sm + off;
            off += S.l[l].ncell;
            V[l].x = sm + off;
            off += S.l[l].ncell;
            V[l].b = sm + off;
            off += S.l[l].ncell;
        }
    }
    __syncthreads();
    for (int l = S.first_cta; l < S.nl; ++l) {
        const LV<float>& G = S.l[l];
        float* A = const_cast<float*>(V[l].A);
        for (int e = tid; e < NPT * G.ncell; e += nt) A[e] = G.A[e];
        for (int c = tid; c < G.ncell; c += nt) {
            Dv[l][c] = 1.0f / G.A[c];
            V[l].x[c] = 0.0f;
            if (l == S.first_cta) V[l].b[c] = G.b[c];
        }
    }
    __syncthreads();
    // alternating zebra line relaxation: lines along each axis in turn, each colour in turn
    // (reverse order after the coarse-grid correction)
    auto line_sweep = [&](int l, bool reverse) {
        const LV<float>& L = V[l];
        for (int st = 0; st < D; ++st) {
            const int axis = reverse ? D - 1 - st : st;
            int b, c, ncol;
            line_axes(L, D, axis, b, c, ncol);
            const int lines = L.ncell / L.n[axis];
            for (int cc = 0; cc < ncol; ++cc) {
                const int col = reverse ? ncol - 1 - cc : cc;
                for (int idx = tid; idx < lines; idx += nt) {
                    const int start = line_start(L, D, axis, idx, col);
                    if (start >= 0) line_solve<D, NPT>(L, axis, start);
                }
                __syncthreads();
            }
        }
    };
    auto sweep = [&](int l, int col) {
        const LV<float>& L = V[l];
        int d[3];
        Col<D, NPT>::dims(L, d);
        const int plane = d[0] * d[1];
        for (int idx = tid; idx < plane * d[2]; idx += nt) {
            int k = idx / plane, r = idx - k * plane;
            int j = r / d[0], m = r - j * d[0];
            int q[3];
            Col<D, NPT>::cell(col, m, j, k, q);
            smooth_at<D, NPT>(L, (const float*)Dv[l], q);
        }
        __syncthreads();
    };
    for (int l = S.first_cta; l < S.nl - 1; ++l) {
        for (int it = 0; it < nu1; ++it) {
            if (S.line) line_sweep(l, false);
            else
                for (int col = 0; col < V[l].ncol; ++col) sweep(l, col);
        }
        const LV<float>& C = V[l + 1];
        const int plane = C.n[0] * C.n[1];
        for (int idx = tid; idx < C.ncell; idx += nt) {
            int k = idx / plane, r = idx - k * plane;
            int j = r / C.n[0];
            int q[3] = {r - j * C.n[0], j, k};
            restrict_at<D, NPT>(V[l], C, q);
        }
        __syncthreads();
    }
    {
        const LV<float>& L = V[S.nl - 1];
        int m = S.dense_m;
        int mm = m + (S.singular ? 1 : 0);
        for (int i = tid; i < mm; i += nt) sb[i] = i < m ? L.b[i] : 0.0f;
        __syncthreads();
        for (int i = tid; i < m; i += nt) {
            const float* row = S.dense_inv + i * mm;
            float acc = 0.0f;
            for (int k = 0; k < mm; ++k) acc += row[k] * sb[k];
            L.x[i] = acc;
        }
        __syncthreads();
    }
    for (int l = S.nl - 2; l >= S.first_cta; --l) {
        const LV<float>& L = V[l];
        const int plane = L.n[0] * L.n[1];
        for (int idx = tid; idx < L.ncell; idx += nt) {
            int k = idx / plane, r = idx - k * plane;
            int j = r / L.n[0];
            int q[3] = {r - j * L.n[0], j, k};
            prolong_at<D>(L, V[l + 1], q);
        }
        __syncthreads();
        for (int it = 0; it < nu2; ++it) {
            if (S.line) line_sweep(l, true);
            else
                for (int col = V[l].ncol - 1; col >= 0; --col) sweep(l, col);
        }
    }
    const LV<float>& T = S.l[S.first_cta];
    for (int c = tid; c < T.ncell; c += nt) T.x[c] = V[S.first_cta].x[c];
}

// ------------------------------------------------------------------ FP64 outer iteration
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    int w = tid >> 5, l = tid & 31;
    if (l == 0) {
        sh[2 * w] = a;
        sh[2 * w + 1] = b;
    }
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x * blockDim.y) >> 5;
        a = l < nw ? sh[2 * l] : 0.0;
        b = l < nw ? sh[2 * l + 1] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    int w = tid >> 5, l = tid & 31;
    if (l == 0) {
        sh[3 * w] = a;
        sh[3 * w + 1] = b;
        sh[3 * w + 2] = c;
    }
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x * blockDim.y) >> 5;
        a = l < nw ? sh[3 * l] : 0.0;
        b = l < nw ? sh[3 * l + 1] : 0.0;
        c = l < nw ? sh[3 * l + 2] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
    }
    __syncthreads();
}

struct ResidualParams {
    LV<double> L;       // finest level, FP64 (x = phi, b = right-hand side)
    float* r32;         // FP32 residual (right-hand side of the correction cycle), or null
    double* r64;        // FP64 residual (Krylov iteration), or null
    const double* rh;   // shadow residual r^: (r^, r) is reduced when ks is set and !init
    KrylovState* ks;    // Krylov scalars to update, or null
    int init;           // first residual of a Krylov solve: start the recurrence
    double* part;       // [3 * gridDim.x]
    unsigned* ticket;
    DevCounters* ctr;
    int* done;
    double rtol;
    int max_cycles;
    int count_cycle;    // V-cycles since the previous residual
    int use_handle;
    cudaGraphConditionalHandle handle;
};

// r = b - M phi in FP64, its FP32 copy, and ||r||, ||b||; the last block to finish sums the
// block partials in a fixed tree, updates the counters and decides whether to continue.
// Blocks of 32 x 8 threads walk rows (j, k) of 32-cell segments.
template <int D, int NPT>
__global__ void __launch_bounds__(256) residual_kernel(ResidualParams P) {
    __shared__ double sh[96];
    __shared__ bool last;
    const LV<double>& L = P.L;
    const bool dot_rh = P.ks && !P.init;
    double rr = 0.0, bb = 0.0, hr = 0.0;
    const int nrows = L.n[1] * L.n[2];
    for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < nrows; row += gridDim.x * blockDim.y) {
        int j = row % L.n[1], k = row / L.n[1];
        for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
            int q[3] = {i, j, k};
            int c = i + L.n[0] * row;
            double r = L.b[c] - stencil_sum<D, NPT, 0>(L, c, q);
            if (P.r32) P.r32[c] = (float)r;
            if (P.r64) P.r64[c] = r;
            rr += r * r;
            bb += L.b[c] * L.b[c];
            if (dot_rh) hr += P.rh[c] * r;
        }
    }
    block_sum3(rr, bb, hr, sh);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid == 0) {
        P.part[3 * blockIdx.x] = rr;
        P.part[3 * blockIdx.x + 1] = bb;
        P.part[3 * blockIdx.x + 2] = hr;
        __threadfence();
        unsigned t = atomicAdd(P.ticket, 1u);
        last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0, h = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += blockDim.x * blockDim.y) {
        a += P.part[3 * i];
        b += P.part[3 * i + 1];
        h += P.part[3 * i + 2];
    }
    block_sum3(a, b, h, sh);
    if (tid == 0) {
        *P.ticket = 0;
        DevCounters* ctr = P.ctr;
        ctr->mg_cycles += P.count_cycle;
        if (KrylovState* ks = P.ks) {
            // (r^, r) of the new residual; a vanishing rho, alpha or omega restarts the
            // recurrence from r^ = p = r, whose rho is (r, r)
            const bool restart = P.init || !(ks->omega != 0.0) || !(ks->rho != 0.0) || !(ks->alpha != 0.0) ||
                                 !(fabs(h) > 1e-300) || !isfinite(h);
            if (restart) {
                ks->restart = 1;
                ks->rho = a;
                ks->beta = 0.0;
            } else {
                ks->restart = 0;
                ks->beta = (h / ks->rho) * (ks->alpha / ks->omega);
                ks->rho = h;
            }
        }
        double res = b > 0.0 ? sqrt(a) / sqrt(b) : 0.0;
        ctr->mg_residual = res;
        ctr->mg_bnorm = sqrt(b);
        bool converged = res <= P.rtol;
        if (converged) ctr->mg_converged = 1;
        bool cont = !converged && ctr->mg_cycles < P.max_cycles;
        *P.done = cont ? 0 : 1;
        if (P.use_handle) cudaGraphSetConditional(P.handle, cont ? 1u : 0u);
    }
}

// phi += e (FP64 update with the FP32 correction)
__global__ void update_kernel(double* phi, const float* e, int n) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) phi[c] += (double)e[c];
}

// ---- BiCGStab steps (the scalars live in KrylovState; see the header comment)

// p = r + beta (p - omega v), or p = r^ = r on a restart; p is also the V-cycle's right-hand
// side. The direction vectors p, v and s are FP32 (they only shape the Krylov space: the
// residual and phi stay FP64), which keeps these passes off GB300's FP64 units.
__global__ void bicg_direction_kernel(int n, const double* __restrict__ r, double* rh, float* p, const float* v,
                                      float* b32, const KrylovState* ks) {
    const float beta = (float)ks->beta, omega = (float)ks->omega;
    const bool restart = ks->restart != 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        float pc;
        if (restart) {
            rh[c] = r[c];
            pc = (float)r[c];
        } else {
            pc = (float)r[c] + beta * (p[c] - omega * v[c]);
        }
        p[c] = pc;
        b32[c] = pc;
    }
}

// y = M x32 over the finest level with the FP32 copy of the full operator (every stencil
// entry; on GB300 an FP64 product is bound by the FP64 rate, at about a third of the memory
// rate), reduced in FP64; mode 0: v = y, p^ = x32 kept, reduce (r^, v) ->
// alpha = rho / (r^, v); mode 1: reduce (y, s), (y, y) -> omega = (t, s) / (t, t)
template <int D, int NPT>
__global__ void __launch_bounds__(256) bicg_matvec_kernel(LV<float> L, const float* __restrict__ x32, int mode,
                                                           float* v, float* ph32, const double* __restrict__ wr,
                                                           const float* __restrict__ ws, KrylovState* ks) {
    __shared__ double sh[96];
    __shared__ bool last;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    const int nrows = L.n[1] * L.n[2];
    // one cell's product and its contributions to the reductions
    auto emit = [&](int c, float yf) {
        const double y = (double)yf;
        if (mode == 0) {
            v[c] = yf;
            ph32[c] = x32[c];
            d0 += wr[c] * y;  // r^
        } else {
            d0 += y * (double)ws[c];  // s
            d1 += y * y;
        }
    };
    if (L.n[0] % 4 == 0) {
        // four consecutive cells along axis 0 per thread: each stencil entry of the four is one
        // 16-byte load, and a neighbour row's four values one 16-byte load plus the value
        // beyond the end the shifted entries need; the per-cell sums are stencil_apply's
        const int n0 = L.n[0], q4 = n0 / 4;
        for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < nrows; row += gridDim.x * blockDim.y) {
            const int j = row % L.n[1], k = row / L.n[1];
            int lo[3], hi[3];
            const int qq[3] = {0, j, k};
#pragma unroll
            for (int a = 1; a < D; ++a) {
                lo[a] = qq[a] > 0 ? qq[a] - 1 : (L.per[a] ? L.n[a] - 1 : 0);
                hi[a] = qq[a] + 1 < L.n[a] ? qq[a] + 1 : (L.per[a] ? 0 : L.n[a] - 1);
            }
            const int jy[3] = {n0 * lo[1], n0 * j, n0 * hi[1]};
            int kz[3] = {0, 0, 0};
            if (D == 3) {
                const int pl = n0 * L.n[1];
                kz[0] = pl * lo[2];
                kz[1] = pl * k;
                kz[2] = pl * hi[2];
            }
            for (int g = threadIdx.x; g < q4; g += blockDim.x) {
                const int i0 = 4 * g;
                const int il = i0 > 0 ? i0 - 1 : (L.per[0] ? n0 - 1 : 0);
                const int ir = i0 + 4 < n0 ? i0 + 4 : (L.per[0] ? 0 : n0 - 1);
                const int c = i0 + n0 * row;
                float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int e = 0; e < NPT; ++e) {
                    const int dx = koff(D, e, 0);
                    const int rb = jy[koff(D, e, 1) + 1] + (D == 3 ? kz[koff(D, e, 2) + 1] : 0);
                    const float4 xm = *reinterpret_cast<const float4*>(x32 + rb + i0);
                    float xs[4];
                    if (dx == 0) {
                        xs[0] = xm.x, xs[1] = xm.y, xs[2] = xm.z, xs[3] = xm.w;
                    } else if (dx < 0) {
                        // cell i0's left neighbour: wrapped, or i0 itself at a closed face
                        xs[0] = i0 > 0 || L.per[0] ? x32[rb + il] : xm.x;
                        xs[1] = xm.x, xs[2] = xm.y, xs[3] = xm.z;
                    } else {
                        xs[0] = xm.y, xs[1] = xm.z, xs[2] = xm.w;
                        xs[3] = i0 + 4 < n0 || L.per[0] ? x32[rb + ir] : xm.w;
                    }
                    const float4 a4 = *reinterpret_cast<const float4*>(L.A + (size_t)e * L.ncell + c);
                    acc[0] += a4.x * xs[0];
                    acc[1] += a4.y * xs[1];
                    acc[2] += a4.z * xs[2];
                    acc[3] += a4.w * xs[3];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) emit(c + u, acc[u]);
            }
        }
    } else {
        for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < nrows; row += gridDim.x * blockDim.y) {
            int j = row % L.n[1], k = row / L.n[1];
            for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
                int q[3] = {i, j, k};
                int c = i + L.n[0] * row;
                emit(c, stencil_apply<D, NPT>(L, x32, c, q));
            }
        }
    }
    block_sum3(d0, d1, d2, sh);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid == 0) {
        ks->part[3 * blockIdx.x] = d0;
        ks->part[3 * blockIdx.x + 1] = d1;
        __threadfence();
        unsigned t = atomicAdd(&ks->ticket, 1u);
        last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0, z = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += blockDim.x * blockDim.y) {
        a += ks->part[3 * i];
        b += ks->part[3 * i + 1];
    }
    block_sum3(a, b, z, sh);
    if (tid == 0) {
        ks->ticket = 0;
        if (mode == 0) {
            const double al = ks->rho / a;
            ks->alpha = (a != 0.0 && isfinite(al)) ? al : 0.0;
            ks->restart = 0;
        } else {
            const double om = a / b;
            ks->omega = (b > 0.0 && isfinite(om)) ? om : 0.0;
        }
    }
}

// s = r - alpha v (FP32), also the V-cycle's right-hand side
__global__ void bicg_s_kernel(int n, const double* __restrict__ r, const float* __restrict__ v, float* s,
                              float* b32, const KrylovState* ks) {
    const float alpha = (float)ks->alpha;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const float sc = (float)r[c] - alpha * v[c];
        s[c] = sc;
        b32[c] = sc;
    }
}

// phi += alpha p^ + omega s^: the step formed in FP32, added to phi in FP64
__global__ void bicg_update_kernel(int n, double* phi, const float* __restrict__ ph32, const float* __restrict__ sh32,
                                   const KrylovState* ks) {
    const float alpha = (float)ks->alpha, omega = (float)ks->omega;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        phi[c] += (double)(alpha * ph32[c] + omega * sh32[c]);
}

// mode 1: (sum b, -); mode 2: (sum J phi, -)
__global__ void sum_kernel(LV<double> L, int mode, const double* Jc, double* part) {
    __shared__ double sh[64];
    double a = 0.0, b = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell; c += gridDim.x * blockDim.x)
        a += mode == 1 ? L.b[c] : Jc[c] * L.x[c];
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = a;
}

__device__ __forceinline__ double sum_parts(const double* part, int nb, double* sh) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[2 * i];
    block_sum2(a, b, sh);
    return a;  // valid in warp 0
}

// b -= (sum b / sum J) J  (singular problems)
__global__ void project_kernel(LV<double> L, const double* part, int nb, double sumJ, const double* Jc) {
    __shared__ double sh[64];
    __shared__ double shift;
    double s = sum_parts(part, nb, sh);
    if (threadIdx.x == 0) shift = s / sumJ;
    __syncthreads();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell; c += gridDim.x * blockDim.x) L.b[c] -= shift * Jc[c];
}

// phi -= (sum J phi / sum J)  (gauge of singular problems)
__global__ void gauge_kernel(LV<double> L, const double* part, int nb, double sumJ) {
    __shared__ double sh[64];
    __shared__ double shift;
    double s = sum_parts(part, nb, sh);
    if (threadIdx.x == 0) shift = s / sumJ;
    __syncthreads();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell; c += gridDim.x * blockDim.x) L.x[c] -= shift;
}

__global__ void reset_solve_kernel(DevCounters* ctr, int* done, unsigned* ticket) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *done = 0;
        *ticket = 0;
        ctr->mg_cycles = 0;
        ctr->mg_converged = 0;
    }
}

// ------------------------------------------------------------------ setup kernels
struct AsmParams {
    LV<double> L;
    const double* face[3];
    int bc[6];
    double bcv[6];
    double* A;
    double* bbc;  // may be null (coarse levels: homogeneous)
    int* cross_flag;
    unsigned* cross_max;  // largest (sum of |cross entries|) / diagonal of a row, as float bits
};

__device__ __forceinline__ int slot_of(int D, const int* o) {
    if (D == 2) {
        const int tab[9] = {5, 3, 6, 1, 0, 2, 7, 4, 8};
        return tab[(o[0] + 1) + 3 * (o[1] + 1)];
    }
    for (int k = 0; k < 27; ++k)
        if (c_off3[k][0] == o[0] && c_off3[k][1] == o[1] && c_off3[k][2] == o[2]) return k;
    return -1;
}

__global__ void assemble_kernel(AsmParams P) {
    const LV<double>& L = P.L;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell; c += gridDim.x * blockDim.x) {
        int q[3];
        cell_coords(L, c, q);
        double a[27];
        for (int k = 0; k < 27; ++k) a[k] = 0.0;
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
            P.A[(size_t)k * L.ncell + c] = a[k];
            if (k >= faces && a[k] != 0.0) cross = true;
        }
        if (cross) {
            atomicOr(P.cross_flag, 1);
            double off = 0.0;
            for (int k = faces; k < L.S; ++k) off += fabs(a[k]);
            const float ratio = a[0] != 0.0 ? (float)(off / fabs(a[0])) : 3.0e38f;
            atomicMax(P.cross_max, __float_as_uint(ratio));  // non-negative floats order as their bits
        }
        if (P.bbc) P.bbc[c] = rb;
    }
}

__global__ void inv_diag_kernel(const float* A, float* dinv, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dinv[i] = 1.0f / A[i];
}

__global__ void to_float_kernel(const double* src, float* dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// dense matrix of the coarsest level (bordered with ones when singular), row-major mm x mm
__global__ void dense_matrix_kernel(LV<double> L, int singular, double* M) {
    int m = (int)L.ncell, mm = m + (singular ? 1 : 0);
    for (long long e = threadIdx.x; e < (long long)mm * mm; e += blockDim.x) M[e] = 0.0;
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        int q[3];
        cell_coords(L, c, q);
        for (int k = 0; k < L.used; ++k) {
            int o[3];
            offsets(L.D, k, o);
            long long nb = nbr(L, q, o);
            double v = L.A[(size_t)k * L.ncell + c];
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
            if (r == col || k == col) continue;
            double f = M[(long long)r * n + col];
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

template <typename R>
LV<R> make_lv(const cpic_run* r, int l, bool fp32) {
    const Level& Lv = r->lev[l];
    LV<R> L;
    L.D = r->D;
    for (int a = 0; a < 3; ++a) {
        L.n[a] = a < r->D ? Lv.n[a] : 1;
        L.per[a] = a < r->D ? (r->cfg.field_bc[2 * a] == CPIC_BC_PERIODIC) : 0;
    }
    for (int f = 0; f < 6; ++f) L.bc[f] = r->cfg.field_bc[f];
    L.ncell = (int)Lv.ncell;
    L.S = Lv.S;
    const bool cross = Lv.cross && !(fp32 && r->pc_face_only);
    const int full = r->D == 2 ? 9 : (r->mg_coarse == CPIC_MG_COARSE_GALERKIN ? 27 : 19);
    L.used = cross ? full : 2 * r->D + 1;
    L.ncol = cross ? (1 << r->D) : 2;
    L.lw = Lv.lw;
    L.pw = nullptr;
    if (r->mg_interp == CPIC_MG_INTERP_OPERATOR && l + 1 < r->nlevels)
        L.pw = fp32 ? (const R*)(const void*)Lv.pw32 : (const R*)(const void*)Lv.pw;
    if (fp32) {
        L.A = (const R*)Lv.A32;
        L.x = (R*)Lv.x32;
        L.b = (R*)Lv.b32;
    } else {
        L.A = (const R*)Lv.A;
        L.x = (R*)Lv.x;
        L.b = (R*)Lv.b;
    }
    return L;
}

int grid_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 8LL * device_sm_count()) b = 8LL * device_sm_count();
    if (b < 1) b = 1;
    return (int)b;
}

constexpr size_t CTA_SMEM_MAX = 200 * 1024;  // shared memory of the one-CTA coarse cycle

LVSet make_set(const cpic_run* r) {
    LVSet S;
    S.nl = r->nlevels;
    S.line = r->mg_smoother == CPIC_MG_SMOOTH_LINE ? 1 : 0;
    for (int l = 0; l < r->nlevels; ++l) S.l[l] = make_lv<float>(r, l, true);
    // the one-CTA part starts at the first level of at most COARSE_CELLS cells from which
    // every coarser level fits the CTA's shared memory (stencil, inverse diagonal, x, b)
    S.first_cta = r->nlevels - 1;
    for (int l = r->nlevels - 1; l >= 0; --l) {
        if (r->lev[l].ncell > COARSE_CELLS) break;
        size_t f = 0;
        for (int k = l; k < r->nlevels; ++k) f += (size_t)(S.l[k].used + 3) * S.l[k].ncell;
        if (f * sizeof(float) > CTA_SMEM_MAX) break;
        S.first_cta = l;
    }
    S.dense_inv = r->dense_inv32;
    S.dense_m = (int)r->lev[r->nlevels - 1].ncell;
    S.singular = r->singular ? 1 : 0;
    return S;
}

size_t cta_smem_bytes(const LVSet& S) {
    size_t f = 0;
    for (int l = S.first_cta; l < S.nl; ++l) f += (size_t)(S.l[l].used + 3) * S.l[l].ncell;
    return f * sizeof(float);
}

int* done_flag(cpic_run* r) { return reinterpret_cast<int*>(r->red + 3 * KRY_BLOCKS + 2); }

// blocks of a pass over the finest level's rows of cells (kCellBlock: eight rows a block)
int row_blocks(const cpic_run* r) {
    const long long rows = (long long)r->lev[0].n[1] * (r->D == 3 ? r->lev[0].n[2] : 1);
    const long long b = (rows + 7) / 8;
    return (int)(b < 1 ? 1 : (b > KRY_BLOCKS ? KRY_BLOCKS : b));
}

const dim3 kCellBlock(32, 8, 1);

dim3 cell_grid(int n0, int n1, int n2) {
    return dim3((unsigned)((n0 + 31) / 32), (unsigned)((n1 + 7) / 8), (unsigned)n2);
}

// calls f(std::integral_constant<int, D>, std::integral_constant<int, NPT>) for the run's
// stencil shape (all levels share it: the finest level's cross-term flag decides)
template <class F>
int dispatch_shape(const cpic_run* r, F f) {
    const bool cross = r->lev[0].cross != 0;
    if (r->D == 2) return cross ? f(std::integral_constant<int, 2>(), std::integral_constant<int, 9>())
                                : f(std::integral_constant<int, 2>(), std::integral_constant<int, 5>());
    if (r->mg_coarse == CPIC_MG_COARSE_GALERKIN)  // 27-point coarse levels
        return f(std::integral_constant<int, 3>(), std::integral_constant<int, 27>());
    return cross ? f(std::integral_constant<int, 3>(), std::integral_constant<int, 19>())
                 : f(std::integral_constant<int, 3>(), std::integral_constant<int, 7>());
}

// stencil shape of the FP32 V-cycle: the operator's, or its face entries alone when the
// cross entries are small enough to leave to the outer iteration (pc_face_only)
template <class F>
int dispatch_vshape(const cpic_run* r, F f) {
    const bool cross = r->lev[0].cross != 0 && !r->pc_face_only;
    if (r->D == 2) return cross ? f(std::integral_constant<int, 2>(), std::integral_constant<int, 9>())
                                : f(std::integral_constant<int, 2>(), std::integral_constant<int, 5>());
    if (r->mg_coarse == CPIC_MG_COARSE_GALERKIN)
        return f(std::integral_constant<int, 3>(), std::integral_constant<int, 27>());
    return cross ? f(std::integral_constant<int, 3>(), std::integral_constant<int, 19>())
                 : f(std::integral_constant<int, 3>(), std::integral_constant<int, 7>());
}

// one FP32 V-cycle on the correction equation (e = 0 first): lev[0].x32 = V(lev[0].b32)
int enqueue_vcycle(cpic_run* r, const LVSet& S) {
    return dispatch_vshape(r, [&](auto Dc, auto Nc) -> int {
        constexpr int D = decltype(Dc)::value, NPT = decltype(Nc)::value;
        cudaStream_t st = r->stream;
        const int nu1 = 2, nu2 = 2;
        CPIC_CUDA(cudaMemsetAsync(r->lev[0].x32, 0, sizeof(float) * r->lev[0].ncell, st));
        const int top = S.first_cta;
        auto smooth = [&](int l, int col) -> int {
            const LV<float>& L = S.l[l];
            int d[3] = {L.n[0] / 2, Col<D, NPT>::parity ? L.n[1] : L.n[1] / 2,
                        D == 3 ? (Col<D, NPT>::parity ? L.n[2] : L.n[2] / 2) : 1};
            smooth_kernel<D, NPT><<<cell_grid(d[0], d[1], d[2]), kCellBlock, 0, st>>>(L, r->lev[l].dinv32, col);
            CPIC_CHECK_LAUNCH();
            return CPIC_OK;
        };
        // alternating zebra line relaxation: one thread per line (those of other colours
        // return at once)
        auto line_smooth = [&](int l, bool reverse) -> int {
            const LV<float>& L = S.l[l];
            for (int stp = 0; stp < D; ++stp) {
                const int axis = reverse ? D - 1 - stp : stp;
                int b, c, ncol;
                line_axes(L, D, axis, b, c, ncol);
                const int lines = L.ncell / L.n[axis];
                for (int cc = 0; cc < ncol; ++cc) {
                    const int col = reverse ? ncol - 1 - cc : cc;
                    line_kernel<D, NPT><<<(lines + 63) / 64, 64, 0, st>>>(L, axis, col, lines);
                    CPIC_CHECK_LAUNCH();
                }
            }
            return CPIC_OK;
        };
        for (int l = 0; l < top; ++l) {
            for (int it = 0; it < nu1; ++it) {
                if (S.line) {
                    if (int e = line_smooth(l, false)) return e;
                    continue;
                }
                for (int col = 0; col < S.l[l].ncol; ++col)
                    if (int e = smooth(l, col)) return e;
            }
            const LV<float>& C = S.l[l + 1];
            const LV<float>& Fl = S.l[l];
            const dim3 rb(32, D == 3 ? 4 : 8, D == 3 ? 2 : 1);
            const dim3 rg((unsigned)((Fl.n[0] + 31) / 32), (unsigned)((Fl.n[1] + rb.y - 1) / rb.y),
                          (unsigned)(D == 3 ? (Fl.n[2] + 1) / 2 : 1));
            restrict_kernel<D, NPT><<<rg, rb, 0, st>>>(Fl, C);
            CPIC_CHECK_LAUNCH();
        }
        size_t smem = cta_smem_bytes(S);
        if (smem > CTA_SMEM_MAX) {
            set_error("multigrid: coarse levels need %zu bytes of shared memory", smem);
            return CPIC_ERR_INVALID;
        }
        // per-function attribute shared by every run (and by graphs captured earlier): set it
        // to the bound checked above, not to this run's need
        CPIC_CUDA(cudaFuncSetAttribute(coarse_cycle_kernel<D, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CTA_SMEM_MAX));
        coarse_cycle_kernel<D, NPT><<<1, 512, smem, st>>>(S, nu1, nu2);
        CPIC_CHECK_LAUNCH();
        for (int l = top - 1; l >= 0; --l) {
            const LV<float>& L = S.l[l];
            prolong_kernel<D><<<cell_grid(L.n[0], L.n[1], L.n[2]), kCellBlock, 0, st>>>(L, S.l[l + 1]);
            CPIC_CHECK_LAUNCH();
            for (int it = 0; it < nu2; ++it) {
                if (S.line) {
                    if (int e = line_smooth(l, true)) return e;
                    continue;
                }
                for (int col = L.ncol - 1; col >= 0; --col)
                    if (int e = smooth(l, col)) return e;
            }
        }
        return CPIC_OK;
    });
}

// one V-cycle on the residual, then phi += e
int enqueue_correction(cpic_run* r, const LVSet& S) {
    int st = enqueue_vcycle(r, S);
    if (st) return st;
    update_kernel<<<grid_blocks(r->lev[0].ncell, 256), 256, 0, r->stream>>>(r->lev[0].x, r->lev[0].x32,
                                                                            (int)r->lev[0].ncell);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

// krylov: 0 plain iteration (FP32 residual for the next V-cycle); 1 first residual of a
// BiCGStab solve; 2 residual after a BiCGStab iteration
int enqueue_residual(cpic_run* r, double rtol, int max_cycles, int count_cycle, bool use_handle,
                     cudaGraphConditionalHandle h, int krylov = 0) {
    ResidualParams P;
    P.L = make_lv<double>(r, 0, false);
    P.r32 = krylov ? nullptr : r->lev[0].b32;
    P.r64 = krylov ? r->kv : nullptr;
    P.rh = krylov ? r->kv + r->ncell : nullptr;
    P.ks = krylov ? r->kry : nullptr;
    P.init = krylov == 1 ? 1 : 0;
    P.part = r->red;
    P.ticket = r->ticket;
    P.ctr = r->ctr;
    P.done = done_flag(r);
    P.rtol = rtol;
    P.max_cycles = max_cycles;
    P.count_cycle = count_cycle;
    P.use_handle = use_handle ? 1 : 0;
    P.handle = h;
    return dispatch_shape(r, [&](auto Dc, auto Nc) -> int {
        residual_kernel<decltype(Dc)::value, decltype(Nc)::value><<<row_blocks(r), kCellBlock, 0, r->stream>>>(P);
        CPIC_CHECK_LAUNCH();
        return CPIC_OK;
    });
}

// one BiCGStab iteration (two V-cycles) ending with the residual that decides whether to go on
int enqueue_bicg_iteration(cpic_run* r, const LVSet& S, double rtol, int max_cycles, bool use_handle,
                           cudaGraphConditionalHandle h) {
    const int n = (int)r->ncell;
    double* rv = r->kv;
    double* rh = r->kv + r->ncell;
    float* p = reinterpret_cast<float*>(r->kv + 2 * r->ncell);  // FP32 p, v, s after r, r^
    float* v = p + r->ncell;
    float* s = v + r->ncell;
    float* b32 = r->lev[0].b32;
    float* x32 = r->lev[0].x32;
    cudaStream_t st = r->stream;
    const int gb = grid_blocks(n, 256);
    bicg_direction_kernel<<<gb, 256, 0, st>>>(n, rv, rh, p, v, b32, r->kry);
    CPIC_CHECK_LAUNCH();
    int e = enqueue_vcycle(r, S);
    if (e) return e;
    LV<float> L0 = make_lv<float>(r, 0, true);  // A32 holds every entry of the operator
    e = dispatch_shape(r, [&](auto Dc, auto Nc) -> int {
        bicg_matvec_kernel<decltype(Dc)::value, decltype(Nc)::value>
            <<<row_blocks(r), kCellBlock, 0, st>>>(L0, x32, 0, v, r->ph32, rh, nullptr, r->kry);
        CPIC_CHECK_LAUNCH();
        return CPIC_OK;
    });
    if (e) return e;
    bicg_s_kernel<<<gb, 256, 0, st>>>(n, rv, v, s, b32, r->kry);
    CPIC_CHECK_LAUNCH();
    e = enqueue_vcycle(r, S);
    if (e) return e;
    e = dispatch_shape(r, [&](auto Dc, auto Nc) -> int {
        bicg_matvec_kernel<decltype(Dc)::value, decltype(Nc)::value>
            <<<row_blocks(r), kCellBlock, 0, st>>>(L0, x32, 1, nullptr, nullptr, nullptr, s, r->kry);
        CPIC_CHECK_LAUNCH();
        return CPIC_OK;
    });
    if (e) return e;
    bicg_update_kernel<<<gb, 256, 0, st>>>(n, r->lev[0].x, r->ph32, x32, r->kry);
    CPIC_CHECK_LAUNCH();
    return enqueue_residual(r, rtol, max_cycles, 2, use_handle, h, 2);
}

bool use_krylov(const cpic_run* r) { return r->solver == CPIC_SOLVER_BICGSTAB && !r->cluster_cs; }

// right-hand side (and its projection); resets the solve counters
int enqueue_prologue(cpic_run* r) {
    reset_solve_kernel<<<1, 32, 0, r->stream>>>(r->ctr, done_flag(r), r->ticket);
    CPIC_CHECK_LAUNCH();
    int st = launch_rhs(r, r->lev[0].b);
    if (st) return st;
    if (r->singular) {
        LV<double> L0 = make_lv<double>(r, 0, false);
        sum_kernel<<<RED_BLOCKS, 256, 0, r->stream>>>(L0, 1, r->lev[0].Jc, r->red);
        CPIC_CHECK_LAUNCH();
        project_kernel<<<grid_blocks(L0.ncell, 256), 256, 0, r->stream>>>(L0, r->red, RED_BLOCKS, r->sumJ, r->lev[0].Jc);
        CPIC_CHECK_LAUNCH();
    }
    return CPIC_OK;
}

int enqueue_epilogue(cpic_run* r) {
    if (r->singular) {
        LV<double> L0 = make_lv<double>(r, 0, false);
        sum_kernel<<<RED_BLOCKS, 256, 0, r->stream>>>(L0, 2, r->lev[0].Jc, r->red);
        CPIC_CHECK_LAUNCH();
        gauge_kernel<<<grid_blocks(L0.ncell, 256), 256, 0, r->stream>>>(L0, r->red, RED_BLOCKS, r->sumJ);
        CPIC_CHECK_LAUNCH();
    }
    int st = launch_floating(r);  // a floating conductor's potential from its charge
    if (st) return st;
    return launch_field_energy(r);
}

}  // namespace

int mg_setup(cpic_run* r) {
    int* flag = reinterpret_cast<int*>(r->red + 3 * KRY_BLOCKS + 4);
    unsigned* cmax = reinterpret_cast<unsigned*>(r->red + 3 * KRY_BLOCKS + 6);
    r->pc_face_only = 0;
    for (int l = 0; l < r->nlevels; ++l) {
        Level& Lv = r->lev[l];
        CPIC_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), r->stream));
        CPIC_CUDA(cudaMemsetAsync(cmax, 0, sizeof(unsigned), r->stream));
        AsmParams P;
        Lv.cross = 1;  // all entries while assembling
        P.L = make_lv<double>(r, l, false);
        for (int a = 0; a < 3; ++a) P.face[a] = Lv.face[a];
        for (int f = 0; f < 6; ++f) {
            P.bc[f] = r->cfg.field_bc[f];
            P.bcv[f] = l == 0 ? r->cfg.field_bc_value[f] : 0.0;
        }
        P.A = Lv.A;
        P.bbc = l == 0 ? r->rhs_bc : nullptr;
        P.cross_flag = flag;
        P.cross_max = cmax;
        const bool galerkin = r->mg_coarse == CPIC_MG_COARSE_GALERKIN;
        if (l > 0 && r->mg_interp == CPIC_MG_INTERP_OPERATOR) {
            // the prolongation weights of the level above, from its (finished) operator
            LV<double> F = make_lv<double>(r, l - 1, false);
            if (r->D == 2)
                interp_weights_kernel<2><<<grid_blocks(F.ncell, 256), 256, 0, r->stream>>>(F, r->lev[l - 1].pw,
                                                                                           r->lev[l - 1].pw32);
            else
                interp_weights_kernel<3><<<grid_blocks(F.ncell, 256), 256, 0, r->stream>>>(F, r->lev[l - 1].pw,
                                                                                           r->lev[l - 1].pw32);
            CPIC_CHECK_LAUNCH();
        }
        if (galerkin && l > 0) {
            // variational coarse operator from the level above (its full stencil)
            LV<double> F = make_lv<double>(r, l - 1, false);
            if (r->D == 2)
                galerkin_kernel<2><<<grid_blocks(Lv.ncell, 256), 256, 0, r->stream>>>(F, P.L, Lv.A);
            else
                galerkin_kernel<3><<<grid_blocks(Lv.ncell, 256), 256, 0, r->stream>>>(F, P.L, Lv.A);
        } else {
            assemble_kernel<<<grid_blocks(Lv.ncell, 256), 256, 0, r->stream>>>(P);
        }
        CPIC_CHECK_LAUNCH();
        to_float_kernel<<<grid_blocks((long long)Lv.S * Lv.ncell, 256), 256, 0, r->stream>>>(Lv.A, Lv.A32,
                                                                                              (long long)Lv.S * Lv.ncell);
        CPIC_CHECK_LAUNCH();
        inv_diag_kernel<<<grid_blocks(Lv.ncell, 256), 256, 0, r->stream>>>(Lv.A32, Lv.dinv32, (int)Lv.ncell);
        CPIC_CHECK_LAUNCH();
        int hflag = 0;
        unsigned hmax = 0;
        CPIC_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
        CPIC_CUDA(cudaMemcpyAsync(&hmax, cmax, sizeof(unsigned), cudaMemcpyDeviceToHost, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
        Lv.cross = hflag;
        // Galerkin coarse operators are 9/27-point: the V-cycle keeps every entry on every level
        if (r->mg_coarse == CPIC_MG_COARSE_GALERKIN) Lv.cross = 1;
        if (l == 0) {
            float ratio;
            memcpy(&ratio, &hmax, sizeof(ratio));
            // CPIC_PC_FULL_STENCIL in the environment keeps the full stencil in the V-cycle
            // (the face-only form is a cost choice; both meet the same stopping test)
            r->pc_face_only = hflag && ratio <= PC_CROSS_DROP && !getenv("CPIC_PC_FULL_STENCIL") &&
                                      r->mg_coarse != CPIC_MG_COARSE_GALERKIN
                                  ? 1
                                  : 0;
        }
    }
    const Level& Lc = r->lev[r->nlevels - 1];
    int m = (int)Lc.ncell;
    int mm = m + (r->singular ? 1 : 0);
    r->dense_m = mm;
    LV<double> L = make_lv<double>(r, r->nlevels - 1, false);
    if (r->pc_face_only) L.used = 2 * r->D + 1;  // the coarsest solve of the V-cycle's operator
    dense_matrix_kernel<<<1, 256, 0, r->stream>>>(L, r->singular ? 1 : 0, r->dense_tmp);
    CPIC_CHECK_LAUNCH();
    int* fail = flag;
    CPIC_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), r->stream));
    gauss_jordan_kernel<<<1, 1024, 0, r->stream>>>(r->dense_tmp, r->dense_inv, mm, fail);
    CPIC_CHECK_LAUNCH();
    to_float_kernel<<<grid_blocks((long long)mm * mm, 256), 256, 0, r->stream>>>(r->dense_inv, r->dense_inv32,
                                                                                  (long long)mm * mm);
    CPIC_CHECK_LAUNCH();
    CPIC_CUDA(cudaMemsetAsync(r->ticket, 0, sizeof(unsigned) * 4, r->stream));
    CPIC_CUDA(cudaMemsetAsync(r->kry, 0, sizeof(KrylovState), r->stream));
    int hfail = 0;
    CPIC_CUDA(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    if (hfail) {
        set_error("coarsest multigrid operator is singular");
        return CPIC_ERR_INVALID;
    }
    return CPIC_OK;
}

// Stream-ordered solve; the host reads the device decision after every cycle
// (cpic_solve_field and the steps of an uncaptured cpic_step).
int mg_solve(cpic_run* r, double rtol, int max_cycles, bool host_loop, int* cycles, double* res) {
    (void)host_loop;
    LVSet S = make_set(r);
    int st = enqueue_prologue(r);
    if (st) return st;
    if (r->cluster_cs) {
        st = mg_cluster_solve(r, rtol, max_cycles);
        if (st) return st;
        max_cycles = 0;  // the loop ran inside the cluster kernel
    } else {
        st = enqueue_residual(r, rtol, max_cycles, 0, false, 0, use_krylov(r) ? 1 : 0);
        if (st) return st;
    }
    int* done = done_flag(r);
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        int hd = 0;
        CPIC_CUDA(cudaMemcpyAsync(&hd, done, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
        if (hd) break;
        if (use_krylov(r)) {
            st = enqueue_bicg_iteration(r, S, rtol, max_cycles, false, 0);
        } else {
            st = enqueue_correction(r, S);
            if (!st) st = enqueue_residual(r, rtol, max_cycles, 1, false, 0);
        }
        if (st) return st;
    }
    st = enqueue_epilogue(r);
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

// The solve as part of a graph being captured on r->stream (capture target `g`): the
// prologue and first residual are captured in place, the cycles go into the body of a
// conditional WHILE node the residual kernel drives, the epilogue follows the node.
int mg_capture_solve(cpic_run* r, cudaGraph_t g, double rtol, int max_cycles) {
    LVSet S = make_set(r);
    if (r->cluster_cs) {
        int st = enqueue_prologue(r);
        if (st) return st;
        st = mg_cluster_solve(r, rtol, max_cycles);
        if (st) return st;
        return enqueue_epilogue(r);
    }
    cudaGraphConditionalHandle h;
    CPIC_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    int st = enqueue_prologue(r);
    if (st) return st;
    st = enqueue_residual(r, rtol, max_cycles, 0, true, h, use_krylov(r) ? 1 : 0);
    if (st) return st;
    // splice the WHILE node after the current capture frontier
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CPIC_CUDA(cudaStreamGetCaptureInfo(r->stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    // the parameter struct has a union member without a default constructor: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = h;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    cudaGraphNode_t wnode;
    CPIC_CUDA(cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, np));
    cudaGraph_t body = np->conditional.phGraph_out[0];
    // the rest of the outer capture depends on the WHILE node
    CPIC_CUDA(cudaStreamUpdateCaptureDependencies(r->stream, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    // body: capture on a side stream into the body graph
    cudaStream_t side;
    CPIC_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    cudaStream_t saved = r->stream;
    r->stream = side;
    st = CPIC_OK;
    cudaError_t e = cudaStreamBeginCaptureToGraph(side, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        if (use_krylov(r)) {
            st = enqueue_bicg_iteration(r, S, rtol, max_cycles, true, h);
        } else {
            st = enqueue_correction(r, S);
            if (!st) st = enqueue_residual(r, rtol, max_cycles, 1, true, h);
        }
        cudaGraph_t out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(side, &out);
        if (!st && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture(body)", __FILE__, __LINE__);
    } else {
        st = cuda_fail(e, "cudaStreamBeginCaptureToGraph(body)", __FILE__, __LINE__);
    }
    r->stream = saved;
    cudaStreamDestroy(side);
    if (st) return st;
    return enqueue_epilogue(r);
}

}  // namespace cpic
