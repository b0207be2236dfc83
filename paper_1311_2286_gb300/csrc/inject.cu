// Row a8: Maxwellian flux injection at a boundary face (Sec. III.A-B: plasma particles are
// injected from the outer boundary every step with fluxes of a (drifting) Maxwellian).
//
// The paper gives no formulas; this implementation's reading:
//  * particles per step: rate r = n vth / sqrt(2 pi) * A * dt / w (one-sided Maxwellian
//    flux through the face's physical length A), step n injects floor((n+1) r) - floor(n r);
//  * draws: Philox4x32-10 (Salmon et al., SC'11) with key (seed low, seed high) and counter
//    (p, n, species, word), u -> (u + 1/2) 2^-32;
//  * position uniform in the face's logical coordinate (axisymmetric runs: the segment by
//    its surface of revolution 2 pi r_mid |dX|, the offset along it uniform); inward normal speed
//    vth sqrt(-2 ln U1), tangential/z components vth sqrt(-2 ln U2) (cos, sin)(2 pi U3),
//    plus the drift; the normal is -+ k^{0.}/|k^{0.}| from k interpolated along the face;
//  * partial first push u = u_face + U4 dt (k v) for a uniform entry time within the step,
//    then the split (cell, FP32 offset); a particle whose partial push leaves the domain is
//    written as a dead slot.
// New particles are appended to their species in draw order and deposited at once.
// The arithmetic after the draws is FP32 (u rounded to FP32, the face k from the FP32 vertex
// table, FP32 Box-Muller, the partial push on the split position), so it agrees with the
// FP64 reading to FP32 rounding; FP64 on this part runs at a small fraction of the FP32 rate
// and would make the injection a long serial chain.
#include <math.h>

#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;


// u -> (u + 1/2) 2^-32 in (0, 1], in FP32
__device__ __forceinline__ float u01f(unsigned u) {
    return __fmaf_rn(__uint2float_rn(u), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

struct InjectOne {
    int s, side;
    double rate;
    float vth, drift[3];
    unsigned long long seed;
    int blocks;  // blocks covering this species' draws
    int drifting;          // 2D drifting Maxwellian: segment by dcdf, bisected normal speed
    const double* dcdf;    // its segment prefixes of Gamma(u_j) A_j
    double dtot, vthd, dr[3];
};

// drifting Maxwellian: CDF on v > 0 of the flux-weighted normal speed density
// v exp(-(v - u)^2 / 2 vth^2), and its inverse by 64 bisections of [0, max(u, 0) + 12 vth]
// (FP64, the same steps as the reading's definition)
__device__ double drift_normal_cdf(double v, double u, double vth) {
    const double s2 = vth * vth;
    const double a = sqrt(0.5 * M_PI) * u * vth;
    const double e0 = exp(-u * u / (2.0 * s2));
    const double erf0 = erf(u / (sqrt(2.0) * vth));
    const double z = s2 * e0 + a * (1.0 + erf0);
    const double f = s2 * (e0 - exp(-(v - u) * (v - u) / (2.0 * s2))) + a * (erf((v - u) / (sqrt(2.0) * vth)) + erf0);
    return f / z;
}

__device__ double drift_normal_speed(double q, double u, double vth) {
    double lo = 0.0, hi = (u > 0.0 ? u : 0.0) + 12.0 * vth;
    for (int it = 0; it < 64; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (drift_normal_cdf(mid, u, vth) < q) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

struct InjectParams {
    PushParams p;
    float dt;
    int nsp;  // injecting species in this launch (blockIdx.y)
    InjectOne sp[CPIC_MAX_SPECIES];
    const double* fcdf;  // 3D: face-cell area prefixes of faces 0 and 1; axisymmetric 2D: the
                         // face segments' surface-of-revolution prefixes
    double farea[2];     // face areas (the prefixes' last entries)
    int axisym;          // 2D, Omega = r
};

__device__ __forceinline__ long long inject_count(double rate, long long step) {
    return (long long)(floor((double)(step + 1) * rate) - floor((double)step * rate));
}

// split renormalisation of a small FP32 displacement from the start of cell c
__device__ __forceinline__ void split(float x, int c0, int& c, float& t) {
    float cf = floorf(x);
    float f = __fsub_rn(x, cf);
    if (f >= 1.0f) {
        f = 0.0f;
        cf = __fadd_rn(cf, 1.0f);
    }
    cf = fminf(fmaxf(cf, -16777216.0f), 16777216.0f);
    c = c0 + (int)cf;
    t = f;
}

// Counts the kept particles and, in the last block of the species to finish, appends the
// new slots to the species (so later kernels of the step see them).
__device__ __forceinline__ void commit_injection(const PushParams& p, int s, int kept_lane, long long start,
                                                 long long nslots) {
    int k = kept_lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(FULL, k, o);
    if ((threadIdx.x & 31) == 0 && k) {
        atomicAdd((unsigned long long*)&p.ctr->injected[s], (unsigned long long)k);
        atomicAdd((unsigned long long*)&p.ctr->alive[s], (unsigned long long)k);
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&p.ctr->inject_ticket[s], 1u);
        last = t == (unsigned)gridDim.x - 1u;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        p.ctr->count[s] = start + nslots;
        p.ctr->inject_ticket[s] = 0u;
    }
}

// One launch injects every species (blockIdx.y); the last block of a species to finish
// commits its new particle count (so later kernels of the step see the particles).
__global__ void inject_kernel(InjectParams ip) {
    const PushParams& p = ip.p;
    const InjectOne& sp = ip.sp[blockIdx.y];
    const int s = sp.s;
    const long long step = p.ctr->step - 1;
    const long long count = inject_count(sp.rate, step);
    const long long start = p.ctr->count[s];
    const long long room = p.pb.capacity[s] - start;
    const long long nslots = count < room ? count : (room > 0 ? room : 0);
    if (blockIdx.x == 0 && threadIdx.x == 0 && count > nslots)
        atomicAdd((unsigned long long*)&p.ctr->dropped[s], (unsigned long long)(count - nslots));
    const int cur = p.ctr->cur;
    const long long T = p.pb.total;
    const int n1 = p.n[0], n2 = p.n[1];
    const int nv0 = n1 + 1;
    const float4* K4 = reinterpret_cast<const float4*>(p.K);
    const uint2 key = make_uint2((unsigned)(sp.seed & 0xffffffffull), (unsigned)(sp.seed >> 32));
    int kept_lane = 0;
    // warp-uniform loop bound
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nslots; base += (long long)sp.blocks * blockDim.x) {
        long long pi = base + threadIdx.x;
        bool act = pi < nslots;
        int c[3] = {0, 0, 0};
        float tt[3] = {0.f, 0.f, 0.f};
        bool alive = false;
        if (act) {
            uint4 r0 = philox4x32_10(make_uint4((unsigned)pi, (unsigned)step, (unsigned)s, 0u), key);
            uint4 r1 = philox4x32_10(make_uint4((unsigned)pi, (unsigned)step, (unsigned)s, 1u), key);
            const float U0 = u01f(r0.x), U1 = u01f(r0.y), U2 = u01f(r0.z), U3 = u01f(r0.w), U4 = u01f(r1.x);
            int j;
            float sfr;
            if (sp.drifting) {
                // drifting Maxwellian: the segment by inverse CDF of Gamma(u_j) A_j (FP64),
                // the offset along it from U5
                const double* cdf = sp.dcdf;
                const double target = (((double)r0.x + 0.5) * 2.3283064365386962890625e-10) * sp.dtot;
                int lo = 0, hi = n2 - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cdf[mid] > target) hi = mid;
                    else lo = mid + 1;
                }
                j = lo;
                sfr = u01f(r1.y);
            } else if (ip.axisym) {
                // axisymmetric: the segment by inverse CDF of the surfaces of revolution (FP64,
                // as for the 3D face cells), the offset along it from U5
                const double* cdf = ip.fcdf + (sp.side ? n2 : 0);
                const double target = (((double)r0.x + 0.5) * 2.3283064365386962890625e-10) * ip.farea[sp.side];
                int lo = 0, hi = n2 - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cdf[mid] > target) hi = mid;
                    else lo = mid + 1;
                }
                j = lo;
                sfr = u01f(r1.y);
            } else {
                const float u1 = __fmul_rn(U0, (float)n2);
                j = (int)floorf(u1);
                if (j > n2 - 1) j = n2 - 1;
                sfr = __fsub_rn(u1, (float)j);
            }
            const int col = sp.side == 0 ? 0 : n1;
            // k interpolated along the face (FP32 vertex table)
            const float4 ka = __ldg(K4 + col + nv0 * j), kb_ = __ldg(K4 + col + nv0 * (j + 1));
            const float oms = __fsub_rn(1.0f, sfr);
            const float kb[4] = {__fmaf_rn(sfr, kb_.x, __fmul_rn(oms, ka.x)), __fmaf_rn(sfr, kb_.y, __fmul_rn(oms, ka.y)),
                                 __fmaf_rn(sfr, kb_.z, __fmul_rn(oms, ka.z)), __fmaf_rn(sfr, kb_.w, __fmul_rn(oms, ka.w))};
            // inward unit normal along grad xi^0 (row 0 of k) and the tangent
            const float gn = sqrtf(__fmaf_rn(kb[0], kb[0], __fmul_rn(kb[1], kb[1])));
            const float sgn = sp.side == 1 ? -1.0f : 1.0f;
            const float nin0 = __fdiv_rn(sgn * kb[0], gn), nin1 = __fdiv_rn(sgn * kb[1], gn);
            const float tau0 = -nin1, tau1 = nin0;
            // flux-weighted normal speed, Gaussian tangential and z components (Box-Muller)
            const float rho = sp.vth * sqrtf(-2.0f * logf(U2));
            float sn, cs;
            sincospif(2.0f * U3, &sn, &cs);
            const float vz = rho * sn;
            float v0, v1;
            if (sp.drifting) {
                // the normal speed of the drifting flux (inverse CDF at 1 - U1, FP64) and the
                // drift's tangential part on the Gaussian tangential speed
                const double un = sp.dr[0] * (double)nin0 + sp.dr[1] * (double)nin1;
                const double ut = sp.dr[0] * (double)tau0 + sp.dr[1] * (double)tau1;
                const double q = 1.0 - ((double)r0.y + 0.5) * 2.3283064365386962890625e-10;
                const float vn = (float)drift_normal_speed(q, un, sp.vthd);
                const float vt = __fadd_rn(rho * cs, (float)ut);
                v0 = __fmaf_rn(vn, nin0, __fmul_rn(vt, tau0));
                v1 = __fmaf_rn(vn, nin1, __fmul_rn(vt, tau1));
            } else {
                const float vn = sp.vth * sqrtf(-2.0f * logf(U1));
                const float vt = rho * cs;
                v0 = __fadd_rn(__fmaf_rn(vn, nin0, __fmul_rn(vt, tau0)), sp.drift[0]);
                v1 = __fadd_rn(__fmaf_rn(vn, nin1, __fmul_rn(vt, tau1)), sp.drift[1]);
            }
            const float v2 = __fadd_rn(vz, sp.drift[2]);
            // partial first push over a uniform fraction U4 of the step, on the split position
            const float fdt = __fmul_rn(U4, ip.dt);
            const float du0 = __fmul_rn(fdt, __fmaf_rn(kb[0], v0, __fmul_rn(kb[1], v1)));
            const float du1 = __fmul_rn(fdt, __fmaf_rn(kb[2], v0, __fmul_rn(kb[3], v1)));
            split(du0, col, c[0], tt[0]);
            split(__fadd_rn(sfr, du1), j, c[1], tt[1]);
            if (ip.axisym) {  // axis 1 ends on the symmetry axis: not periodic
                alive = c[0] >= 0 && c[0] < n1 && c[1] >= 0 && c[1] < n2;
            } else {
                c[1] = ((c[1] % n2) + n2) % n2;
                alive = c[0] >= 0 && c[0] < n1;
            }
            long long slot = p.pb.base[s] + start + pi;
            p.pb.cell[cur][slot] = alive ? encode<2>(c) : -1;
            if (p.hist && alive)  // the push builds this step's sort histogram: add the newcomers
                atomicAdd(p.hist + (size_t)s * n1 * n2 + c[0] + (size_t)n1 * c[1], 1);
            p.pb.t[cur][slot] = tt[0];
            p.pb.t[cur][T + slot] = tt[1];
            p.pb.v[cur][slot] = v0;
            p.pb.v[cur][T + slot] = v1;
            p.pb.v[cur][2 * T + slot] = v2;
            kept_lane += alive ? 1 : 0;
        }
        deposit_warp<2>(p, s, alive, c, tt);
    }
    commit_injection(p, s, kept_lane, start, nslots);
}

// 3D faces normal to axis 0 (the outer shell of the sphere runs): the face cell is drawn
// by inverse CDF of the face-cell areas (FP64, as the count of the draw decides a cell),
// offsets along axes 1 and 2 from U5 and U6, the inward normal from row 0 of k bilinear in
// the face cell, a tangent basis from the coordinate axis least aligned with the normal,
// and the partial first push on the split position; a particle that leaves axis 0 or
// axis 1 in its partial push is a dead slot; axis 2 (periodic) wraps.
__global__ void inject3d_kernel(InjectParams ip) {
    const PushParams& p = ip.p;
    const InjectOne& sp = ip.sp[blockIdx.y];
    const int s = sp.s;
    const long long step = p.ctr->step - 1;
    const long long count = inject_count(sp.rate, step);
    const long long start = p.ctr->count[s];
    const long long room = p.pb.capacity[s] - start;
    const long long nslots = count < room ? count : (room > 0 ? room : 0);
    if (blockIdx.x == 0 && threadIdx.x == 0 && count > nslots)
        atomicAdd((unsigned long long*)&p.ctr->dropped[s], (unsigned long long)(count - nslots));
    const int cur = p.ctr->cur;
    const long long T = p.pb.total;
    const int n1 = p.n[0], n2 = p.n[1], n3 = p.n[2];
    const int nv0 = n1 + 1, nv1 = n2 + 1;
    const long long nf = (long long)n2 * n3;
    const double* cdf = ip.fcdf + (sp.side ? nf : 0);
    const double total = ip.farea[sp.side];
    const float4* K4 = reinterpret_cast<const float4*>(p.K);
    const uint2 key = make_uint2((unsigned)(sp.seed & 0xffffffffull), (unsigned)(sp.seed >> 32));
    int kept_lane = 0;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nslots; base += (long long)sp.blocks * blockDim.x) {
        long long pi = base + threadIdx.x;
        bool act = pi < nslots;
        int c[3] = {0, 0, 0};
        float tt[3] = {0.f, 0.f, 0.f};
        bool alive = false;
        if (act) {
            const uint4 r0 = philox4x32_10(make_uint4((unsigned)pi, (unsigned)step, (unsigned)s, 0u), key);
            const uint4 r1 = philox4x32_10(make_uint4((unsigned)pi, (unsigned)step, (unsigned)s, 1u), key);
            const double target = (((double)r0.x + 0.5) * 2.3283064365386962890625e-10) * total;
            long long lo = 0, hi = nf - 1;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (cdf[mid] > target) hi = mid;
                else lo = mid + 1;
            }
            const int j = (int)(lo % n2), k = (int)(lo / n2);
            const float U1 = u01f(r0.y), U2 = u01f(r0.z), U3 = u01f(r0.w), U4 = u01f(r1.x);
            const float t1 = u01f(r1.y), t2 = u01f(r1.z);
            const int col = sp.side == 0 ? 0 : n1;
            // k at the face point: bilinear in (t1, t2) over the face cell's four vertices
            const float w00 = __fmul_rn(__fsub_rn(1.0f, t1), __fsub_rn(1.0f, t2)), w10 = __fmul_rn(t1, __fsub_rn(1.0f, t2));
            const float w01 = __fmul_rn(__fsub_rn(1.0f, t1), t2), w11 = __fmul_rn(t1, t2);
            const int vv[4] = {col + nv0 * (j + nv1 * k), col + nv0 * (j + 1 + nv1 * k), col + nv0 * (j + nv1 * (k + 1)),
                               col + nv0 * (j + 1 + nv1 * (k + 1))};
            const float wv[4] = {w00, w10, w01, w11};
            float kf[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) kf[q] = 0.0f;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const float4 a = __ldg(K4 + 3 * vv[o]), b = __ldg(K4 + 3 * vv[o] + 1), cc = __ldg(K4 + 3 * vv[o] + 2);
                const float kv[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, cc.x};
#pragma unroll
                for (int q = 0; q < 9; ++q) kf[q] = __fmaf_rn(wv[o], kv[q], kf[q]);
            }
            // inward unit normal and tangent basis
            const float gn = sqrtf(__fmaf_rn(kf[2], kf[2], __fmaf_rn(kf[1], kf[1], __fmul_rn(kf[0], kf[0]))));
            const float sgn = sp.side == 1 ? -1.0f : 1.0f;
            const float nin[3] = {__fdiv_rn(sgn * kf[0], gn), __fdiv_rn(sgn * kf[1], gn), __fdiv_rn(sgn * kf[2], gn)};
            int ax = 0;
            if (fabsf(nin[1]) < fabsf(nin[ax])) ax = 1;
            if (fabsf(nin[2]) < fabsf(nin[ax])) ax = 2;
            float ta[3] = {-nin[ax] * nin[0], -nin[ax] * nin[1], -nin[ax] * nin[2]};
            ta[ax] = __fadd_rn(ta[ax], 1.0f);
            const float tn = sqrtf(__fmaf_rn(ta[2], ta[2], __fmaf_rn(ta[1], ta[1], __fmul_rn(ta[0], ta[0]))));
            ta[0] = __fdiv_rn(ta[0], tn);
            ta[1] = __fdiv_rn(ta[1], tn);
            ta[2] = __fdiv_rn(ta[2], tn);
            const float tb[3] = {__fsub_rn(__fmul_rn(nin[1], ta[2]), __fmul_rn(nin[2], ta[1])),
                                 __fsub_rn(__fmul_rn(nin[2], ta[0]), __fmul_rn(nin[0], ta[2])),
                                 __fsub_rn(__fmul_rn(nin[0], ta[1]), __fmul_rn(nin[1], ta[0]))};
            const float vn = sp.vth * sqrtf(-2.0f * logf(U1));
            const float rho = sp.vth * sqrtf(-2.0f * logf(U2));
            float sn, cs;
            sincospif(2.0f * U3, &sn, &cs);
            const float va = rho * cs, vb = rho * sn;
            float v[3];
#pragma unroll
            for (int al = 0; al < 3; ++al)
                v[al] = __fadd_rn(__fmaf_rn(vn, nin[al], __fmaf_rn(va, ta[al], __fmul_rn(vb, tb[al]))), sp.drift[al]);
            // partial first push over a uniform fraction U4 of the step
            const float fdt = __fmul_rn(U4, ip.dt);
            float du[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                du[a] = __fmul_rn(fdt, __fmaf_rn(kf[3 * a + 2], v[2], __fmaf_rn(kf[3 * a + 1], v[1], __fmul_rn(kf[3 * a], v[0]))));
            split(du[0], col, c[0], tt[0]);
            split(__fadd_rn(t1, du[1]), j, c[1], tt[1]);
            split(__fadd_rn(t2, du[2]), k, c[2], tt[2]);
            c[2] = ((c[2] % n3) + n3) % n3;
            alive = c[0] >= 0 && c[0] < n1 && c[1] >= 0 && c[1] < n2;
            const long long slot = p.pb.base[s] + start + pi;
            p.pb.cell[cur][slot] = alive ? encode<3>(c) : -1;
            if (p.hist && alive)  // the push builds this step's sort histogram: add the newcomers
                atomicAdd(p.hist + (size_t)s * n1 * n2 * n3 + c[0] + (size_t)n1 * (c[1] + (size_t)n2 * c[2]), 1);
#pragma unroll
            for (int a = 0; a < 3; ++a) p.pb.t[cur][a * T + slot] = tt[a];
#pragma unroll
            for (int al = 0; al < 3; ++al) p.pb.v[cur][al * T + slot] = v[al];
            kept_lane += alive ? 1 : 0;
        }
        deposit_warp<3>(p, s, alive, c, tt);
    }
    commit_injection(p, s, kept_lane, start, nslots);
}

}  // namespace

int launch_inject(cpic_run* r) {
    InjectParams ip;
    ip.p = make_push_params(r);
    ip.dt = (float)r->cfg.dt;
    ip.nsp = 0;
    long long maxb = 1;
    for (int s = 0; s < r->cfg.n_species; ++s) {
        const InjectSpec& sp = r->inj[s];
        if (!sp.enabled) continue;
        InjectOne& o = ip.sp[ip.nsp++];
        o.s = s;
        o.side = sp.face & 1;
        o.rate = sp.rate;
        o.vth = (float)sp.vth;
        for (int a = 0; a < 3; ++a) o.drift[a] = (float)sp.drift[a];
        o.seed = sp.seed;
        o.drifting = sp.drifting;
        o.dcdf = r->dcdf ? r->dcdf + (size_t)s * r->n[1] : nullptr;
        o.dtot = sp.dtot;
        o.vthd = sp.vth;
        for (int a = 0; a < 3; ++a) o.dr[a] = sp.drift[a];
        long long maxc = (long long)ceil(sp.rate) + 1;
        long long b = (maxc + 255) / 256;
        if (b > 4LL * device_sm_count()) b = 4LL * device_sm_count();
        if (b > maxb) maxb = b;
    }
    if (!ip.nsp) return CPIC_OK;
    for (int k = 0; k < ip.nsp; ++k) ip.sp[k].blocks = (int)maxb;
    ip.fcdf = r->fcdf;
    ip.farea[0] = r->face_len[0];
    ip.farea[1] = r->face_len[1];
    ip.axisym = r->D == 2 && r->cfg.axisymmetric;
    if (r->D == 2)
        inject_kernel<<<dim3((unsigned)maxb, (unsigned)ip.nsp), 256, 0, r->stream>>>(ip);
    else
        inject3d_kernel<<<dim3((unsigned)maxb, (unsigned)ip.nsp), 256, 0, r->stream>>>(ip);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace cpic
