// Row a1 (logical field at vertices), the charge -> right-hand side map of row a9, and the
// field-energy diagnostic of row a10.
//
// Staggering (Sec. II.B): phi and rho at cell centres, the field at vertices. The vertex
// field in cell units is G^a = mean over the 2^(D-1) cell pairs straddling the vertex along
// a of the cell difference (the paper gives no formula; this is the implementation's
// reading), with ghost cells from the boundary conditions (Sec. II.B.3): Dirichlet
// 2 phi_b - phi_in, Neumann phi_in, periodic wrap; the ghost of a ghost applies the rules
// from axis 0 upwards. FP64 arithmetic in a fixed order (explicit intrinsics), rounded once
// to FP32 for the mover's table.
#include "internal.cuh"

namespace cpic {
namespace {

struct FieldGrid {
    int D;
    int n[3];
    int bc[6];
    double bcv[6];
    int fface;             // floating conductor's face (-1: none): its Dirichlet value is
    const double* fphi;    // the conductor potential of the last solve, read on the device
};

__device__ __forceinline__ double phi_ext(const FieldGrid& g, const double* __restrict__ phi, int i, int j, int k) {
    int c[3] = {i, j, k};
    int side[3] = {-1, -1, -1};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= g.D) break;
        if (c[a] < 0 || c[a] >= g.n[a]) {
            int sd = c[a] < 0 ? 0 : 1;
            if (g.bc[2 * a] == CPIC_BC_PERIODIC) {
                c[a] = c[a] < 0 ? c[a] + g.n[a] : c[a] - g.n[a];
            } else {
                side[a] = sd;
                c[a] = sd == 0 ? 0 : g.n[a] - 1;
            }
        }
    }
    double val = phi[c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2])];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= g.D) break;
        if (side[a] >= 0 && g.bc[2 * a + side[a]] == CPIC_BC_DIRICHLET)
            val = __dsub_rn(__dmul_rn(2.0, g.bcv[2 * a + side[a]]), val);
    }
    return val;
}

// 3D: G is also written into the three padding words of each vertex's k record (K[12 v + 9 ..
// 11]), so that the mover's first gather reads k and G in three 16-byte loads per corner.
__global__ void vertex_field_kernel(FieldGrid g, const double* __restrict__ phi, float* G, float* K) {
    if (g.fface >= 0) g.bcv[g.fface] = *g.fphi;
    long long nv0 = g.n[0] + 1, nv1 = g.n[1] + 1, nv2 = g.D == 3 ? g.n[2] + 1 : 1;
    long long nvt = nv0 * nv1 * nv2;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvt;
         v += (long long)gridDim.x * blockDim.x) {
        int i = (int)(v % nv0);
        long long rest = v / nv0;
        int j = (int)(rest % nv1);
        int k = (int)(rest / nv1);
        if (g.D == 2) {
            double p00 = phi_ext(g, phi, i - 1, j - 1, 0);
            double p01 = phi_ext(g, phi, i, j - 1, 0);
            double p10 = phi_ext(g, phi, i - 1, j, 0);
            double p11 = phi_ext(g, phi, i, j, 0);
            double g0 = __dmul_rn(__dadd_rn(__dsub_rn(p01, p00), __dsub_rn(p11, p10)), 0.5);
            double g1 = __dmul_rn(__dadd_rn(__dsub_rn(p10, p00), __dsub_rn(p11, p01)), 0.5);
            reinterpret_cast<float2*>(G)[v] = make_float2(__double2float_rn(g0), __double2float_rn(g1));
        } else {
            double c8[8];  // c8[di + 2 dj + 4 dk] = phi_ext(i-1+di, j-1+dj, k-1+dk)
#pragma unroll
            for (int o = 0; o < 8; ++o) c8[o] = phi_ext(g, phi, i - 1 + (o & 1), j - 1 + ((o >> 1) & 1), k - 1 + ((o >> 2) & 1));
            float out[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int o0 = a == 0 ? 1 : 0, o1 = a == 2 ? 1 : 2;  // the other axes, increasing
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int oa = q & 1, ob = q >> 1;  // first other axis fastest
                    int lo = (oa << o0) | (ob << o1);
                    int hi = lo | (1 << a);
                    double d = __dsub_rn(c8[hi], c8[lo]);
                    acc = q == 0 ? d : __dadd_rn(acc, d);
                }
                out[a] = __double2float_rn(__dmul_rn(acc, 0.25));
            }
            reinterpret_cast<float4*>(G)[v] = make_float4(out[0], out[1], out[2], 0.0f);
            float* kr = K + 12 * v;
            kr[9] = out[0];
            kr[10] = out[1];
            kr[11] = out[2];
        }
    }
}

struct RhsParams {
    long long ncell;
    int nsp;
    double qw[CPIC_MAX_SPECIES];
    double background;
    const double* Jc;
    const double* omega;
    const double* bbc;
    const unsigned long long* charge;
    int axisym;  // Omega = r: macro-particles are rings
};

// Q_c = background J_c + sum_s q_s w_s C_{s,c} 2^-24 (eq. (pg) with J_c cancelled against
// the cell volume); b_c = Omega_c Q_c + Dirichlet terms. In an axisymmetric run a
// macro-particle is a ring of charge q w around the axis, spread over the ring volume
// 2 pi r J_c: its term is divided by 2 pi Omega_c.
__device__ __forceinline__ double charge_of(const RhsParams& p, long long c) {
    double Q = __dmul_rn(p.background, p.Jc[c]);
    const double ring = p.axisym ? __ddiv_rn(1.0, __dmul_rn(2.0 * M_PI, p.omega[c])) : 1.0;
    for (int s = 0; s < p.nsp; ++s) {
        double C = (double)(long long)p.charge[(long long)s * p.ncell + c];
        double t = __dmul_rn(p.qw[s], ldexp(C, -QF));
        if (p.axisym) t = __dmul_rn(t, ring);
        Q = __dadd_rn(Q, t);
    }
    return Q;
}

__global__ void rhs_kernel(RhsParams p, double* b) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double Q = charge_of(p, c);
        b[c] = __dadd_rn(__dmul_rn(p.omega[c], Q), p.bbc[c]);
    }
}

// deterministic block reduction (fixed shuffle tree, fixed block count)
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;
}

__global__ void field_energy_partial(RhsParams p, const double* __restrict__ phi, double* part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.ncell;
         c += (long long)gridDim.x * blockDim.x)
        acc += phi[c] * charge_of(p, c);
    double r = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void field_energy_final(const double* part, int nb, DevCounters* ctr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[i];
        ctr->field_energy = 0.5 * s;
    }
}

FieldGrid make_field_grid(const cpic_run* r) {
    FieldGrid g;
    g.D = r->D;
    for (int a = 0; a < 3; ++a) g.n[a] = a < r->D ? r->n[a] : 1;
    for (int f = 0; f < 6; ++f) {
        g.bc[f] = r->cfg.field_bc[f];
        g.bcv[f] = r->cfg.field_bc_value[f];
    }
    g.fface = r->floating_face;
    g.fphi = &r->ctr->object_potential;
    return g;
}

// Floating conductor on the face normal to axis 0 at side `side` (Sec. III.A-B: an object
// that collects the particles reaching it and floats to the potential its charge gives).
// Gauss's law for the conductor: its charge is minus the outward flux of grad phi through
// its surface, which in the finite-volume scheme is the Dirichlet face flux
// 2 a^{00}_f (phi_c - phi_b) summed over the face's cells (a^{00} = Omega J g^{00} of the
// face, cell units). With phi = phi_0 + V psi (phi_0: the solve with the conductor at 0;
// psi: charge-free, conductor at 1, other Dirichlet values 0), the charge condition
// Q = -sum 2 a (phi_0 + V psi - V) fixes V = -(Q + G0) / Cpsi, G0 = sum 2 a phi_0,
// Cpsi = sum 2 a (psi - 1). Sums run in a fixed order (one block).
struct FloatParams {
    int n0, n1, n2, side, face, nsp;
    long long nf;           // faces normal to axis 0
    const double* a00;      // face coefficient a^{00} of those faces
    const double* phi;      // cell potential
    const double* psi;
    double q0;              // charge before any collection
    double qw[CPIC_MAX_SPECIES];
    int axisym;             // Omega = r: Gauss's law on the ring-charge scale (Q / 2 pi)
};

__device__ double face_flux_sum(const FloatParams& p, const double* u, double ub) {
    __shared__ double part[256];
    const int i = p.side == 0 ? 0 : p.n0 - 1, fi = p.side == 0 ? 0 : p.n0;
    const long long m = (long long)p.n1 * p.n2;
    double acc = 0.0;
    for (long long jk = threadIdx.x; jk < m; jk += blockDim.x) {
        const long long c = i + (long long)p.n0 * jk;
        const long long f = fi + (long long)(p.n0 + 1) * jk;
        acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(2.0, p.a00[f]), __dsub_rn(u[c], ub)));
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + w]);
        __syncthreads();
    }
    return part[0];
}

__global__ void floating_kernel(FloatParams p, DevCounters* ctr) {
    const double g0 = face_flux_sum(p, p.phi, 0.0);
    if (threadIdx.x == 0) {
        double q = p.q0;
        for (int s = 0; s < p.nsp; ++s) q = __dadd_rn(q, __dmul_rn(p.qw[s], (double)ctr->absorbed[s][p.face]));
        ctr->object_charge = q;
        const double qr = p.axisym ? q / (2.0 * M_PI) : q;
        ctr->object_potential = -(qr + g0) / ctr->float_cpsi;
    }
}

__global__ void floating_capacity_kernel(FloatParams p, DevCounters* ctr) {
    const double c = face_flux_sum(p, p.psi, 1.0);
    if (threadIdx.x == 0) ctr->float_cpsi = c;
}

__global__ void floating_axpy_kernel(double* phi, const double* psi, long long n, const DevCounters* ctr) {
    const double v = ctr->object_potential;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        phi[c] = __fma_rn(v, psi[c], phi[c]);
}

FloatParams make_float_params(const cpic_run* r) {
    FloatParams p;
    p.n0 = r->n[0];
    p.n1 = r->n[1];
    p.n2 = r->D == 3 ? r->n[2] : 1;
    p.face = r->floating_face;
    p.side = r->floating_face & 1;
    p.nsp = r->cfg.n_species;
    p.nf = (long long)(p.n0 + 1) * p.n1 * p.n2;
    p.a00 = r->lev[0].face[0];
    p.phi = r->lev[0].x;
    p.psi = r->psi;
    p.q0 = r->float_q0;
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) p.qw[s] = s < p.nsp ? r->cfg.q[s] * r->cfg.w[s] : 0.0;
    p.axisym = r->cfg.axisymmetric;
    return p;
}

}  // namespace

RhsParams make_rhs_params(const cpic_run* r) {
    RhsParams p;
    p.ncell = r->ncell;
    p.nsp = r->cfg.n_species;
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) p.qw[s] = s < p.nsp ? r->cfg.q[s] * r->cfg.w[s] : 0.0;
    p.background = r->cfg.background;
    p.Jc = r->lev[0].Jc;
    p.omega = r->lev[0].omega;
    p.bbc = r->rhs_bc;
    p.charge = r->charge;
    p.axisym = r->cfg.axisymmetric;
    return p;
}

int launch_vertex_field(cpic_run* r) {
    FieldGrid g = make_field_grid(r);
    long long b = (r->nvert + 255) / 256;
    if (b > 8LL * device_sm_count()) b = 8LL * device_sm_count();
    vertex_field_kernel<<<(int)b, 256, 0, r->stream>>>(g, r->lev[0].x, r->G32, r->K32);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_rhs(cpic_run* r, double* b) {
    RhsParams p = make_rhs_params(r);
    long long nb = (r->ncell + 255) / 256;
    if (nb > 8LL * device_sm_count()) nb = 8LL * device_sm_count();
    rhs_kernel<<<(int)nb, 256, 0, r->stream>>>(p, b);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_floating(cpic_run* r) {
    if (r->floating_face < 0) return CPIC_OK;
    FloatParams p = make_float_params(r);
    floating_kernel<<<1, 256, 0, r->stream>>>(p, r->ctr);
    CPIC_CHECK_LAUNCH();
    long long nb = (r->ncell + 255) / 256;
    if (nb > 8LL * device_sm_count()) nb = 8LL * device_sm_count();
    floating_axpy_kernel<<<(int)nb, 256, 0, r->stream>>>(r->lev[0].x, r->psi, r->ncell, r->ctr);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_floating_capacity(cpic_run* r) {
    FloatParams p = make_float_params(r);
    floating_capacity_kernel<<<1, 256, 0, r->stream>>>(p, r->ctr);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_field_energy(cpic_run* r) {
    RhsParams p = make_rhs_params(r);
    const int nb = 256;
    field_energy_partial<<<nb, 256, 0, r->stream>>>(p, r->lev[0].x, r->red);
    CPIC_CHECK_LAUNCH();
    field_energy_final<<<1, 32, 0, r->stream>>>(r->red, nb, r->ctr);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace cpic
