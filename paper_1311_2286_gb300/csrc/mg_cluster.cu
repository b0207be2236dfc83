// Row a9 on a thread-block cluster: the whole mixed-precision multigrid solve of a 2D
// 5-point problem in one kernel launch.
//
// Same method as mg.cu (FP64 residual and solution, FP32 V(2,2)-cycles on the correction,
// colour-ordered Gauss-Seidel, residual-sum restriction, bilinear prolongation, dense
// coarsest solve, stop at ||r||/||b|| <= rtol), laid out for GB300: the cluster's CTAs
// (16, or 8 where 16 cannot be co-scheduled) each own a slab of rows of every "distributed"
// level in shared memory; a cell's neighbours in the next/previous slab are read from the
// neighbouring CTA's shared memory (distributed shared memory); phases are separated by
// hardware cluster barriers instead of kernel boundaries; the coarse levels (fewer than four
// rows per CTA) are gathered into CTA 0 and solved there with block barriers only. The
// convergence decision is taken identically by every CTA from the per-CTA partial norms,
// summed in rank order, so the loop needs no host round trip and is deterministic.
// Used for 2D runs without cross terms whose finest row count is a multiple of the
// cluster size and whose levels fit shared memory; other runs use mg.cu's kernels.
#include <cooperative_groups.h>
#include <math.h>
#include <stdlib.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace cpic {
namespace {

constexpr int CL_MAX_LEVELS = 16;
constexpr int CL_THREADS = 1024;

struct ClLevel {
    int n0, n1;          // global cells
    int rows;            // rows per CTA (distributed levels); n1 for CTA-0 levels
    int distributed;     // 1: slab per CTA, 0: whole level in CTA 0
    const float* A;      // global FP32 stencil [5][ncell]
    const float* dinv;   // global FP32 inverse diagonal
    // shared-memory offsets (floats) of x, b, dinv, A[5] in the owning CTA
    int ox, ob, od, oa;
};

struct ClParams {
    int nl;              // levels
    int nd;              // distributed levels (0 .. nd-1)
    int cs;              // cluster size
    int per0, per1;      // periodic axes
    int bc[4];           // field bc kinds per face (ghost rules of the prolongation)
    ClLevel L[CL_MAX_LEVELS];
    const double* A64;   // finest FP64 stencil [5][ncell]
    const double* b64;   // finest right-hand side
    double* phi;         // finest solution (in/out)
    const float* dense_inv;
    int dense_m;         // coarsest unknowns
    int singular;
    int ophi;            // shared offset (in doubles) of the FP64 slab of phi
    int opart;           // shared offset (in doubles) of the partial norms
    double rtol;
    int max_cycles;
    DevCounters* ctr;
};

// value of x at global cell (i, j) of level l with ghost rules for out-of-range cells
// (homogeneous: the correction equation), reading the owning CTA's shared memory
__device__ __forceinline__ float xval(const ClParams& P, cg::cluster_group& cl, int l, float* sm, int i, int j) {
    const ClLevel& L = P.L[l];
    float sign = 1.0f;
    if (i < 0 || i >= L.n0) {
        int side = i < 0 ? 0 : 1;
        if (P.per0) i = i < 0 ? i + L.n0 : i - L.n0;
        else {
            i = side == 0 ? 0 : L.n0 - 1;
            if (P.bc[side] == CPIC_BC_DIRICHLET) sign = -sign;
        }
    }
    if (j < 0 || j >= L.n1) {
        int side = j < 0 ? 0 : 1;
        if (P.per1) j = j < 0 ? j + L.n1 : j - L.n1;
        else {
            j = side == 0 ? 0 : L.n1 - 1;
            if (P.bc[2 + side] == CPIC_BC_DIRICHLET) sign = -sign;
        }
    }
    if (!L.distributed) return sign * cl.map_shared_rank(sm, 0)[L.ox + i + L.n0 * j];  // held by CTA 0
    int owner = j / L.rows, jj = j - owner * L.rows;
    float* base = cl.map_shared_rank(sm, owner);
    return sign * base[L.ox + i + L.n0 * jj];
}

// neighbour rows of local row jj of a distributed level: local index or remote pointer
struct RowNb {
    const float* lo;  // row j-1 (x array base of that row)
    const float* hi;  // row j+1
};

__device__ __forceinline__ RowNb row_nb(const ClParams& P, cg::cluster_group& cl, int l, float* sm, int rank, int jj) {
    const ClLevel& L = P.L[l];
    const int j = rank * L.rows + jj;
    RowNb r;
    // row j-1
    if (jj > 0) r.lo = sm + L.ox + L.n0 * (jj - 1);
    else if (j > 0 || P.per1) {
        int o = (rank + P.cs - 1) % P.cs;
        r.lo = cl.map_shared_rank(sm, o) + L.ox + L.n0 * (L.rows - 1);
    } else
        r.lo = sm + L.ox;  // non-periodic bottom: coefficient is zero, any value
    if (jj < L.rows - 1) r.hi = sm + L.ox + L.n0 * (jj + 1);
    else if (j < L.n1 - 1 || P.per1) {
        int o = (rank + 1) % P.cs;
        r.hi = cl.map_shared_rank(sm, o) + L.ox;
    } else
        r.hi = sm + L.ox + L.n0 * jj;
    return r;
}

// one colour sweep of a distributed level (parity colouring)
__device__ void cl_sweep(const ClParams& P, cg::cluster_group& cl, int l, float* sm, int rank, int colour) {
    const ClLevel& L = P.L[l];
    const int half = L.n0 >> 1;
    const int tot = half * L.rows;
    const float* A = sm + L.oa;
    const int nc = L.n0 * L.rows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        int jj = idx / half, m = idx - jj * half;
        int j = rank * L.rows + jj;
        int i = 2 * m + ((j + colour) & 1);
        int c = i + L.n0 * jj;
        float* x = sm + L.ox;
        int im = i > 0 ? i - 1 : (P.per0 ? L.n0 - 1 : 0);
        int ip = i + 1 < L.n0 ? i + 1 : (P.per0 ? 0 : L.n0 - 1);
        RowNb rn = row_nb(P, cl, l, sm, rank, jj);
        float s = sm[L.ob + c];
        s -= A[1 * nc + c] * x[im + L.n0 * jj];
        s -= A[2 * nc + c] * x[ip + L.n0 * jj];
        s -= A[3 * nc + c] * rn.lo[i];
        s -= A[4 * nc + c] * rn.hi[i];
        x[c] = s * sm[L.od + c];
    }
}

// one colour sweep of a level held whole in CTA 0
__device__ void c0_sweep(const ClParams& P, int l, float* sm, int colour) {
    const ClLevel& L = P.L[l];
    const int half = L.n0 >> 1;
    const int tot = half * L.n1;
    const int nc = L.n0 * L.n1;
    const float* A = sm + L.oa;
    float* x = sm + L.ox;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        int j = idx / half, m = idx - j * half;
        int i = 2 * m + ((j + colour) & 1);
        int c = i + L.n0 * j;
        int im = i > 0 ? i - 1 : (P.per0 ? L.n0 - 1 : 0);
        int ip = i + 1 < L.n0 ? i + 1 : (P.per0 ? 0 : L.n0 - 1);
        int jm = j > 0 ? j - 1 : (P.per1 ? L.n1 - 1 : 0);
        int jp = j + 1 < L.n1 ? j + 1 : (P.per1 ? 0 : L.n1 - 1);
        float s = sm[L.ob + c];
        s -= A[1 * nc + c] * x[im + L.n0 * j];
        s -= A[2 * nc + c] * x[ip + L.n0 * j];
        s -= A[3 * nc + c] * x[i + L.n0 * jm];
        s -= A[4 * nc + c] * x[i + L.n0 * jp];
        x[c] = s * sm[L.od + c];
    }
}

// residual of fine cell (i, jj) of a distributed level (local row)
__device__ __forceinline__ float cl_residual(const ClParams& P, const ClLevel& L, float* sm, const RowNb& rn, int i,
                                             int jj) {
    const int nc = L.n0 * L.rows;
    const int c = i + L.n0 * jj;
    const float* A = sm + L.oa;
    const float* x = sm + L.ox;
    int im = i > 0 ? i - 1 : (P.per0 ? L.n0 - 1 : 0);
    int ip = i + 1 < L.n0 ? i + 1 : (P.per0 ? 0 : L.n0 - 1);
    float Ax = A[c] * x[c] + A[1 * nc + c] * x[im + L.n0 * jj] + A[2 * nc + c] * x[ip + L.n0 * jj] +
               A[3 * nc + c] * rn.lo[i] + A[4 * nc + c] * rn.hi[i];
    return sm[L.ob + c] - Ax;
}

__device__ __forceinline__ float c0_residual(const ClParams& P, const ClLevel& L, float* sm, int i, int j) {
    const int nc = L.n0 * L.n1;
    const int c = i + L.n0 * j;
    const float* A = sm + L.oa;
    const float* x = sm + L.ox;
    int im = i > 0 ? i - 1 : (P.per0 ? L.n0 - 1 : 0);
    int ip = i + 1 < L.n0 ? i + 1 : (P.per0 ? 0 : L.n0 - 1);
    int jm = j > 0 ? j - 1 : (P.per1 ? L.n1 - 1 : 0);
    int jp = j + 1 < L.n1 ? j + 1 : (P.per1 ? 0 : L.n1 - 1);
    float Ax = A[c] * x[c] + A[1 * nc + c] * x[im + L.n0 * j] + A[2 * nc + c] * x[ip + L.n0 * j] +
               A[3 * nc + c] * x[i + L.n0 * jm] + A[4 * nc + c] * x[i + L.n0 * jp];
    return sm[L.ob + c] - Ax;
}

__global__ void __launch_bounds__(CL_THREADS) mg_cluster_kernel(ClParams P) {
    extern __shared__ __align__(16) float sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x;
    double* smd = reinterpret_cast<double*>(sm);
    __shared__ double red[2 * 32];
    __shared__ int s_cont;

    // ---- stage this CTA's slabs (stencil, inverse diagonal) and phi
    for (int l = 0; l < P.nl; ++l) {
        const ClLevel& L = P.L[l];
        if (!L.distributed && rank != 0) continue;
        const int nc = L.n0 * L.rows;
        const int g0 = L.distributed ? rank * L.rows * L.n0 : 0;
        const int gn = L.n0 * L.n1;
        for (int e = tid; e < nc; e += nt) {
            for (int k = 0; k < 5; ++k) sm[L.oa + k * nc + e] = L.A[k * gn + g0 + e];
            sm[L.od + e] = L.dinv[g0 + e];
        }
    }
    const ClLevel& L0 = P.L[0];
    const int nc0 = L0.n0 * L0.rows, g00 = rank * nc0, gn0 = L0.n0 * L0.n1;
    for (int e = tid; e < nc0; e += nt) smd[P.ophi + e] = P.phi[g00 + e];
    cl.sync();

    double bb_total = -1.0;
    int cycles = 0;
    double res = 0.0;
    for (;;) {
        // ---- FP64 residual of the finest level, FP32 copy into the level-0 right-hand side
        double rr = 0.0, bb = 0.0;
        for (int e = tid; e < nc0; e += nt) {
            int jj = e / L0.n0, i = e - jj * L0.n0;
            int j = rank * L0.rows + jj;
            int im = i > 0 ? i - 1 : (P.per0 ? L0.n0 - 1 : 0);
            int ip = i + 1 < L0.n0 ? i + 1 : (P.per0 ? 0 : L0.n0 - 1);
            const double* ph = smd + P.ophi;
            double plo, phi_hi;
            if (jj > 0) plo = ph[i + L0.n0 * (jj - 1)];
            else if (j > 0 || P.per1) plo = cl.map_shared_rank(smd, (rank + P.cs - 1) % P.cs)[P.ophi + i + L0.n0 * (L0.rows - 1)];
            else plo = ph[e];
            if (jj < L0.rows - 1) phi_hi = ph[i + L0.n0 * (jj + 1)];
            else if (j < L0.n1 - 1 || P.per1) phi_hi = cl.map_shared_rank(smd, (rank + 1) % P.cs)[P.ophi + i];
            else phi_hi = ph[e];
            const int g = g00 + e;
            double Ax = P.A64[g] * ph[e] + P.A64[gn0 + g] * ph[im + L0.n0 * jj] + P.A64[2 * gn0 + g] * ph[ip + L0.n0 * jj] +
                        P.A64[3 * gn0 + g] * plo + P.A64[4 * gn0 + g] * phi_hi;
            double b = P.b64[g];
            double r = b - Ax;
            sm[L0.ob + e] = (float)r;
            rr += r * r;
            bb += b * b;
        }
        // block reduction in a fixed tree, then every CTA sums the CTA partials in rank order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
        }
        if ((tid & 31) == 0) {
            red[2 * (tid >> 5)] = rr;
            red[2 * (tid >> 5) + 1] = bb;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < nt / 32; ++w) {
                a += red[2 * w];
                b += red[2 * w + 1];
            }
            smd[P.opart] = a;
            smd[P.opart + 1] = b;
        }
        cl.sync();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < P.cs; ++q) {
                const double* pq = cl.map_shared_rank(smd, q);
                a += pq[P.opart];
                b += pq[P.opart + 1];
            }
            if (bb_total < 0.0) bb_total = b;
            res = bb_total > 0.0 ? sqrt(a) / sqrt(bb_total) : 0.0;
            bool conv = res <= P.rtol;
            s_cont = (!conv && cycles < P.max_cycles) ? 1 : 0;
            if (rank == 0) {
                P.ctr->mg_cycles = cycles;
                P.ctr->mg_residual = res;
                P.ctr->mg_bnorm = sqrt(bb_total);
                if (conv) P.ctr->mg_converged = 1;
            }
        }
        __syncthreads();
        if (!s_cont) break;  // identical decision in every CTA
        ++cycles;
        // the partial norms are rewritten next iteration: every CTA has read them
        cl.sync();

        // ---- FP32 V(2,2) cycle on the correction
        for (int l = 0; l < P.nd; ++l) {
            const ClLevel& L = P.L[l];
            const int nc = L.n0 * L.rows;
            for (int e = tid; e < nc; e += nt) sm[L.ox + e] = 0.0f;
            cl.sync();
            for (int it = 0; it < 2; ++it)
                for (int col = 0; col < 2; ++col) {
                    cl_sweep(P, cl, l, sm, rank, col);
                    cl.sync();
                }
            // restriction to level l + 1: the children of my coarse rows are my fine rows
            const ClLevel& C = P.L[l + 1];
            const int crows = L.rows / 2;
            for (int e = tid; e < C.n0 * crows; e += nt) {
                int jc = e / C.n0, ic = e - jc * C.n0;
                float acc = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    int i = 2 * ic + (ch & 1), jj = 2 * jc + (ch >> 1);
                    RowNb rn = row_nb(P, cl, l, sm, rank, jj);
                    acc += cl_residual(P, L, sm, rn, i, jj);
                }
                if (C.distributed) {
                    sm[C.ob + ic + C.n0 * jc] = acc;
                } else {
                    float* c0 = cl.map_shared_rank(sm, 0);
                    c0[C.ob + ic + C.n0 * (rank * crows + jc)] = acc;
                }
            }
            cl.sync();
        }
        // ---- coarse levels in CTA 0
        if (rank == 0) {
            for (int l = P.nd; l < P.nl; ++l)
                for (int e = tid; e < P.L[l].n0 * P.L[l].n1; e += nt) sm[P.L[l].ox + e] = 0.0f;
            __syncthreads();
            for (int l = P.nd; l < P.nl - 1; ++l) {
                for (int it = 0; it < 2; ++it)
                    for (int col = 0; col < 2; ++col) {
                        c0_sweep(P, l, sm, col);
                        __syncthreads();
                    }
                const ClLevel& L = P.L[l];
                const ClLevel& C = P.L[l + 1];
                for (int e = tid; e < C.n0 * C.n1; e += nt) {
                    int jc = e / C.n0, ic = e - jc * C.n0;
                    float acc = 0.0f;
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) acc += c0_residual(P, L, sm, 2 * ic + (ch & 1), 2 * jc + (ch >> 1));
                    sm[C.ob + e] = acc;
                }
                __syncthreads();
            }
            {
                const ClLevel& L = P.L[P.nl - 1];
                const int m = P.dense_m, mm = m + (P.singular ? 1 : 0);
                float* xs = sm + L.ox;
                const float* bs = sm + L.ob;
                for (int i = tid; i < m; i += nt) {
                    const float* row = P.dense_inv + i * mm;
                    float acc = 0.0f;
                    for (int k = 0; k < m; ++k) acc += row[k] * bs[k];
                    xs[i] = acc;
                }
                __syncthreads();
            }
            for (int l = P.nl - 2; l >= P.nd; --l) {
                const ClLevel& L = P.L[l];
                for (int e = tid; e < L.n0 * L.n1; e += nt) {
                    int j = e / L.n0, i = e - j * L.n0;
                    int I = i >> 1, J = j >> 1;
                    int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1;
                    float v = 0.5625f * xval(P, cl, l + 1, sm, I, J) + 0.1875f * xval(P, cl, l + 1, sm, I + si, J) +
                              0.1875f * xval(P, cl, l + 1, sm, I, J + sj) + 0.0625f * xval(P, cl, l + 1, sm, I + si, J + sj);
                    sm[L.ox + e] += v;
                }
                __syncthreads();
                for (int it = 0; it < 2; ++it)
                    for (int col = 1; col >= 0; --col) {
                        c0_sweep(P, l, sm, col);
                        __syncthreads();
                    }
            }
        }
        cl.sync();
        for (int l = P.nd - 1; l >= 0; --l) {
            const ClLevel& L = P.L[l];
            const int nc = L.n0 * L.rows;
            for (int e = tid; e < nc; e += nt) {
                int jj = e / L.n0, i = e - jj * L.n0;
                int j = rank * L.rows + jj;
                int I = i >> 1, J = j >> 1;
                int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1;
                float v = 0.5625f * xval(P, cl, l + 1, sm, I, J) + 0.1875f * xval(P, cl, l + 1, sm, I + si, J) +
                          0.1875f * xval(P, cl, l + 1, sm, I, J + sj) + 0.0625f * xval(P, cl, l + 1, sm, I + si, J + sj);
                sm[L.ox + e] += v;
            }
            cl.sync();
            for (int it = 0; it < 2; ++it)
                for (int col = 1; col >= 0; --col) {
                    cl_sweep(P, cl, l, sm, rank, col);
                    cl.sync();
                }
        }
        // ---- phi += e (FP64)
        for (int e = tid; e < nc0; e += nt) smd[P.ophi + e] += (double)sm[L0.ox + e];
        cl.sync();
    }
    // no CTA may leave while another can still read its shared memory
    cl.sync();
    for (int e = tid; e < nc0; e += nt) P.phi[g00 + e] = smd[P.ophi + e];
}

}  // namespace

// Layout and launch data of the cluster solver, or a reason it does not apply.
struct ClusterPlan {
    bool ok;
    int cs;
    size_t smem;
    ClParams P;
};

static bool plan_cluster(const cpic_run* r, int cs, ClusterPlan* out) {
    if (r->D != 2 || r->lev[0].cross || r->nlevels < 2 || r->nlevels > CL_MAX_LEVELS) return false;
    if (r->mg_coarse != CPIC_MG_COARSE_REDISCRETIZED || r->mg_smoother != CPIC_MG_SMOOTH_POINT ||
        r->mg_interp != CPIC_MG_INTERP_BILINEAR)
        return false;
    ClParams& P = out->P;
    P.nl = r->nlevels;
    P.cs = cs;
    P.per0 = r->cfg.field_bc[0] == CPIC_BC_PERIODIC;
    P.per1 = r->cfg.field_bc[2] == CPIC_BC_PERIODIC;
    for (int f = 0; f < 4; ++f) P.bc[f] = r->cfg.field_bc[f];
    // distributed levels: at least 4 rows per CTA and rows divisible by the cluster size
    int nd = 0;
    for (int l = 0; l < r->nlevels - 1; ++l) {
        int n1 = r->lev[l].n[1];
        if (n1 % cs == 0 && n1 / cs >= 4 && (n1 / cs) % 2 == 0 && nd == l) ++nd;
    }
    if (nd == 0) return false;
    P.nd = nd;
    // shared-memory layout: identical offsets in every CTA; CTA 0 also holds the coarse levels
    size_t off = 0;  // floats
    for (int l = 0; l < P.nl; ++l) {
        ClLevel& L = P.L[l];
        L.n0 = r->lev[l].n[0];
        L.n1 = r->lev[l].n[1];
        L.distributed = l < nd ? 1 : 0;
        L.rows = L.distributed ? L.n1 / cs : L.n1;
        if (L.n0 % 2) return false;
        L.A = r->lev[l].A32;
        L.dinv = r->lev[l].dinv32;
        int nc = L.n0 * L.rows;
        L.ox = (int)off;
        off += nc;
        L.ob = (int)off;
        off += nc;
        L.od = (int)off;
        off += nc;
        L.oa = (int)off;
        off += 5 * (size_t)nc;
    }
    off = (off + 3) & ~size_t(3);
    P.ophi = (int)(off / 2);
    off += 2 * (size_t)r->lev[0].n[0] * (r->lev[0].n[1] / cs);
    P.opart = (int)(off / 2);
    off += 4;
    out->smem = off * sizeof(float);
    if (out->smem > 200 * 1024) return false;
    P.A64 = r->lev[0].A;
    P.b64 = r->lev[0].b;
    P.phi = r->lev[0].x;
    P.dense_inv = r->dense_inv32;
    P.dense_m = (int)r->lev[r->nlevels - 1].ncell;
    P.singular = r->singular ? 1 : 0;
    P.ctr = r->ctr;
    out->cs = cs;
    return true;
}

// Decide once per run whether the cluster solver applies (and with which cluster size).
int mg_cluster_prepare(cpic_run* r) {
    r->cluster_cs = 0;
    if (getenv("CPIC_NO_CLUSTER_SOLVER")) return CPIC_OK;
    for (int cs : {16, 8}) {
        ClusterPlan plan;
        if (!plan_cluster(r, cs, &plan)) continue;
        if (cs > 8) {
            if (cudaFuncSetAttribute(mg_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
        }
        // the attribute is per function, shared by every run of the process: raise it to the
        // device's opt-in maximum once (it bounds launches, it does not change occupancy)
        {
            int dev = 0, optin = 0;
            CPIC_CUDA(cudaGetDevice(&dev));
            CPIC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            cudaFuncAttributes fa;
            CPIC_CUDA(cudaFuncGetAttributes(&fa, mg_cluster_kernel));
            const int dyn_max = optin - (int)fa.sharedSizeBytes;
            if ((int)plan.smem > dyn_max) continue;
            CPIC_CUDA(cudaFuncSetAttribute(mg_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(CL_THREADS, 1, 1);
        cfg.dynamicSmemBytes = plan.smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, mg_cluster_kernel, &cfg);
        if (e != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        r->cluster_cs = cs;
        return CPIC_OK;
    }
    return CPIC_OK;
}

// The solve loop on the cluster (right-hand side already assembled and projected).
int mg_cluster_solve(cpic_run* r, double rtol, int max_cycles) {
    ClusterPlan plan;
    if (!r->cluster_cs || !plan_cluster(r, r->cluster_cs, &plan)) {
        set_error("cluster solver not applicable");
        return CPIC_ERR_STATE;
    }
    plan.P.rtol = rtol;
    plan.P.max_cycles = max_cycles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.cs, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = r->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CPIC_CUDA(cudaLaunchKernelEx(&cfg, mg_cluster_kernel, plan.P));
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace cpic
