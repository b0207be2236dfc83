// Device-side initial loading of a species: a Maxwellian plasma of uniform physical density
// (the paper's runs start from a uniform Maxwellian plasma, Sec. III.A-B).
//
// Particle i of the load draws Philox4x32-10 words with counter (i, 0x10AD, species, word)
// under the key `seed`:
//   cell: the first cell whose inclusive prefix of cell Jacobians exceeds U0 * sum J_c, so
//         a cell is picked with probability J_c / sum J_c (J_c is the cell's physical volume
//         in logical units, so the density is uniform in physical space, piecewise constant
//         per cell); in an axisymmetric run the weights are Omega_c J_c (the ring volume
//         over 2 pi), uniform in the 3D volume;
//   offsets: uniform in [0, 1) per axis (24-bit draws, exact in FP32);
//   velocity: vth times standard normals from Box-Muller pairs, plus the drift.
// The species' previous particles are replaced.
#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

struct LoadParams {
    int D, n[3], sp;
    long long count, ncell;
    double total;
    const double* cdf;
    int* cell;
    float* t;
    float* v;
    long long T;
    float vth, drift[3];
    unsigned long long seed;
};

__device__ __forceinline__ float u24(unsigned u) { return (float)(u >> 8) * 5.9604644775390625e-8f; }  // [0, 1)
__device__ __forceinline__ float u01o(unsigned u) {  // (0, 1]
    return __fmaf_rn(__uint2float_rn(u), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

__global__ void maxwellian_kernel(LoadParams lp) {
    const uint2 key = make_uint2((unsigned)(lp.seed & 0xffffffffull), (unsigned)(lp.seed >> 32));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < lp.count;
         i += (long long)gridDim.x * blockDim.x) {
        const uint4 a = philox4x32_10(make_uint4((unsigned)i, 0x10ADu, (unsigned)lp.sp, 0u), key);
        const uint4 b = philox4x32_10(make_uint4((unsigned)i, 0x10ADu, (unsigned)lp.sp, 1u), key);
        // cell by inverse CDF of the cell Jacobians
        const double target = (((double)a.x + 0.5) * 2.3283064365386962890625e-10) * lp.total;
        long long lo = 0, hi = lp.ncell - 1;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (lp.cdf[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        const long long c = lo;
        int ci[3];
        ci[0] = (int)(c % lp.n[0]);
        ci[1] = (int)((c / lp.n[0]) % lp.n[1]);
        ci[2] = (int)(c / ((long long)lp.n[0] * lp.n[1]));
        const float t0 = u24(a.y), t1 = u24(a.z), t2 = u24(a.w);
        float n0, n1, n2, n3;
        {
            const float r0 = sqrtf(-2.0f * logf(u01o(b.x))), r1 = sqrtf(-2.0f * logf(u01o(b.z)));
            float s0, c0, s1, c1;
            sincospif(2.0f * u01o(b.y), &s0, &c0);
            sincospif(2.0f * u01o(b.w), &s1, &c1);
            n0 = r0 * c0;
            n1 = r0 * s0;
            n2 = r1 * c1;
            n3 = r1 * s1;
        }
        (void)n3;
        lp.cell[i] = lp.D == 2 ? (ci[0] | (ci[1] << 16)) : (ci[0] | (ci[1] << 10) | (ci[2] << 20));
        lp.t[i] = t0;
        lp.t[lp.T + i] = t1;
        if (lp.D == 3) lp.t[2 * lp.T + i] = t2;
        lp.v[i] = __fmaf_rn(lp.vth, n0, lp.drift[0]);
        lp.v[lp.T + i] = __fmaf_rn(lp.vth, n1, lp.drift[1]);
        lp.v[2 * lp.T + i] = __fmaf_rn(lp.vth, n2, lp.drift[2]);
    }
}

__global__ void set_species_count_kernel(DevCounters* ctr, int sp, long long n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctr->count[sp] = n;
        ctr->alive[sp] = n;
    }
}

}  // namespace

int launch_load_maxwellian(cpic_run* r, int sp, long long n, double vth, const double* drift, unsigned long long seed) {
    LoadParams lp;
    lp.D = r->D;
    for (int a = 0; a < 3; ++a) lp.n[a] = r->n[a];
    lp.sp = sp;
    lp.count = n;
    lp.ncell = r->ncell;
    lp.total = r->load_total;
    lp.cdf = r->jcdf;
    const int b = r->cur_host;
    const long long base = r->pb.base[sp];
    lp.T = r->pb.total;
    lp.cell = r->pb.cell[b] + base;
    lp.t = r->pb.t[b] + base;
    lp.v = r->pb.v[b] + base;
    lp.vth = (float)vth;
    for (int a = 0; a < 3; ++a) lp.drift[a] = drift ? (float)drift[a] : 0.0f;
    lp.seed = seed;
    if (n > 0) {
        long long blocks = (n + 255) / 256;
        if (blocks > 16LL * device_sm_count()) blocks = 16LL * device_sm_count();
        maxwellian_kernel<<<(int)blocks, 256, 0, r->stream>>>(lp);
        CPIC_CHECK_LAUNCH();
    }
    set_species_count_kernel<<<1, 32, 0, r->stream>>>(r->ctr, sp, n);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace cpic
