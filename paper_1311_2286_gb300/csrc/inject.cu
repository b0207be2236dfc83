// Row a8: Maxwellian flux injection at a boundary face (Sec. III.A-B: plasma particles are
// injected from the outer boundary every step with fluxes of a (drifting) Maxwellian).
//
// The paper gives no formulas; this implementation's reading:
//  * particles per step: rate r = n vth / sqrt(2 pi) * A * dt / w (one-sided Maxwellian
//    flux through the face's physical length A), step n injects floor((n+1) r) - floor(n r);
//  * draws: Philox4x32-10 (Salmon et al., SC'11) with key (seed low, seed high) and counter
//    (p, n, species, word), u -> (u + 1/2) 2^-32;
//  * position uniform in the face's logical coordinate; inward normal speed
//    vth sqrt(-2 ln U1), tangential/z components vth sqrt(-2 ln U2) (cos, sin)(2 pi U3),
//    plus the drift; the normal is -+ k^{0.}/|k^{0.}| from k interpolated along the face;
//  * partial first push u = u_face + U4 dt (k v) for a uniform entry time within the step,
//    then the split (cell, FP32 offset); a particle whose partial push leaves the domain is
//    written as a dead slot.
// New particles are appended to their species in draw order and deposited at once.
#include <math.h>

#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const unsigned W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double u01(unsigned u) { return __dmul_rn(__dadd_rn((double)u, 0.5), 2.3283064365386962890625e-10); }

struct InjectParams {
    PushParams p;
    int sp;
    int side;
    double rate;
    double vth;
    double drift[3];
    unsigned long long seed;
    double dt;
    const double* k64;
};

__device__ __forceinline__ long long inject_count(double rate, long long step) {
    return (long long)(floor((double)(step + 1) * rate) - floor((double)step * rate));
}

__global__ void inject_kernel(InjectParams ip) {
    const PushParams& p = ip.p;
    const int s = ip.sp;
    const long long step = p.ctr->step - 1;
    const long long count = inject_count(ip.rate, step);
    const long long start = p.ctr->count[s];
    const long long room = p.pb.capacity[s] - start;
    const long long nslots = count < room ? count : (room > 0 ? room : 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.ctr->pending_inject[s] = (int)nslots;
        if (count > nslots) atomicAdd((unsigned long long*)&p.ctr->dropped[s], (unsigned long long)(count - nslots));
    }
    const int cur = p.ctr->cur;
    const long long T = p.pb.total;
    const int n1 = p.n[0], n2 = p.n[1];
    const int nv0 = n1 + 1;
    const uint2 key = make_uint2((unsigned)(ip.seed & 0xffffffffull), (unsigned)(ip.seed >> 32));
    int kept_lane = 0;
    // warp-uniform loop bound
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nslots; base += (long long)gridDim.x * blockDim.x) {
        long long pi = base + threadIdx.x;
        bool act = pi < nslots;
        int c[3] = {0, 0, 0};
        float tt[3] = {0.f, 0.f, 0.f};
        bool alive = false;
        if (act) {
            uint4 r0 = philox4x32_10(make_uint4((unsigned)pi, (unsigned)step, (unsigned)s, 0u), key);
            uint4 r1 = philox4x32_10(make_uint4((unsigned)pi, (unsigned)step, (unsigned)s, 1u), key);
            double U0 = u01(r0.x), U1 = u01(r0.y), U2 = u01(r0.z), U3 = u01(r0.w), U4 = u01(r1.x);
            double u1 = __dmul_rn(U0, (double)n2);
            int j = (int)floor(u1);
            if (j > n2 - 1) j = n2 - 1;
            double sfr = __dsub_rn(u1, (double)j);
            int col = ip.side == 0 ? 0 : n1;
            const double* ka = ip.k64 + ((long long)col + (long long)nv0 * j) * 4;
            const double* kb_ = ip.k64 + ((long long)col + (long long)nv0 * (j + 1)) * 4;
            double oms = __dsub_rn(1.0, sfr);
            double kb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) kb[q] = __dadd_rn(__dmul_rn(oms, ka[q]), __dmul_rn(sfr, kb_[q]));
            double ga0 = kb[0], ga1 = kb[1];
            double gn = __dsqrt_rn(__dadd_rn(__dmul_rn(ga0, ga0), __dmul_rn(ga1, ga1)));
            double sgn = ip.side == 1 ? -1.0 : 1.0;
            double nin0 = __ddiv_rn(__dmul_rn(sgn, ga0), gn), nin1 = __ddiv_rn(__dmul_rn(sgn, ga1), gn);
            double tau0 = -nin1, tau1 = nin0;
            double vn = __dmul_rn(ip.vth, __dsqrt_rn(__dmul_rn(-2.0, log(U1))));
            double rho = __dmul_rn(ip.vth, __dsqrt_rn(__dmul_rn(-2.0, log(U2))));
            const double two_pi = 6.283185307179586;
            double vt = __dmul_rn(rho, cos(__dmul_rn(two_pi, U3)));
            double vz = __dmul_rn(rho, sin(__dmul_rn(two_pi, U3)));
            float v0 = __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(vn, nin0), __dmul_rn(vt, tau0)), ip.drift[0]));
            float v1 = __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(vn, nin1), __dmul_rn(vt, tau1)), ip.drift[1]));
            float v2 = __double2float_rn(__dadd_rn(vz, ip.drift[2]));
            double vd0 = v0, vd1 = v1;
            double fdt = __dmul_rn(U4, ip.dt);
            double du0 = __dmul_rn(fdt, __dadd_rn(__dmul_rn(kb[0], vd0), __dmul_rn(kb[1], vd1)));
            double du1 = __dmul_rn(fdt, __dadd_rn(__dmul_rn(kb[2], vd0), __dmul_rn(kb[3], vd1)));
            double uu[2] = {__dadd_rn(ip.side == 0 ? 0.0 : (double)n1, du0), __dadd_rn(__dadd_rn((double)j, sfr), du1)};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                double cf = floor(uu[a]);
                float f = __double2float_rn(__dsub_rn(uu[a], cf));
                if (f >= 1.0f) {
                    f = 0.0f;
                    cf = cf + 1.0;
                }
                c[a] = (int)cf;
                tt[a] = f;
            }
            c[1] = ((c[1] % n2) + n2) % n2;
            alive = c[0] >= 0 && c[0] < n1;
            long long slot = p.pb.base[s] + start + pi;
            p.pb.cell[cur][slot] = alive ? encode<2>(c) : -1;
            p.pb.t[cur][slot] = tt[0];
            p.pb.t[cur][T + slot] = tt[1];
            p.pb.v[cur][slot] = v0;
            p.pb.v[cur][T + slot] = v1;
            p.pb.v[cur][2 * T + slot] = v2;
            kept_lane += alive ? 1 : 0;
        }
        deposit_warp<2>(p, s, alive, c, tt);
    }
    int k = kept_lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(FULL, k, o);
    if ((threadIdx.x & 31) == 0 && k) {
        atomicAdd((unsigned long long*)&p.ctr->injected[s], (unsigned long long)k);
        atomicAdd((unsigned long long*)&p.ctr->alive[s], (unsigned long long)k);
    }
}

__global__ void inject_commit_kernel(DevCounters* ctr, int sp) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctr->count[sp] += ctr->pending_inject[sp];
        ctr->pending_inject[sp] = 0;
    }
}

}  // namespace

PushParams make_push_params(cpic_run* r);

int launch_inject(cpic_run* r) {
    for (int s = 0; s < r->cfg.n_species; ++s) {
        const InjectSpec& sp = r->inj[s];
        if (!sp.enabled) continue;
        InjectParams ip;
        ip.p = make_push_params(r);
        ip.sp = s;
        ip.side = sp.face & 1;
        ip.rate = sp.rate;
        ip.vth = sp.vth;
        for (int a = 0; a < 3; ++a) ip.drift[a] = sp.drift[a];
        ip.seed = sp.seed;
        ip.dt = r->cfg.dt;
        ip.k64 = r->k64;
        long long maxc = (long long)ceil(sp.rate) + 1;
        long long blocks = (maxc + 255) / 256;
        if (blocks > 152 * 4) blocks = 152 * 4;
        if (blocks < 1) blocks = 1;
        inject_kernel<<<(int)blocks, 256, 0, r->stream>>>(ip);
        CPIC_CHECK_LAUNCH();
        inject_commit_kernel<<<1, 32, 0, r->stream>>>(r->ctr, s);
        CPIC_CHECK_LAUNCH();
    }
    return CPIC_OK;
}

}  // namespace cpic
