// Device helpers shared by the particle kernels (push, deposit, kick, injection):
// split-position renormalisation, the spec Q integer b2 weights, the b1 vertex gathers of
// the mover's FP32 tables, and the warp-aggregated fixed-point deposit.
#pragma once

#include "internal.cuh"

namespace cpic {
namespace pk {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int wrapi(int c, int n) {
    int r = c % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void renorm(float x, float& f, int& c) {
    float cf = floorf(x);
    float fr = __fsub_rn(x, cf);
    if (fr >= 1.0f) {
        fr = 0.0f;
        cf = __fadd_rn(cf, 1.0f);
    }
    cf = fminf(fmaxf(cf, -16777216.0f), 16777216.0f);
    f = fr;
    c = (int)cf;
}

// per-axis integer b2 weights (spec Q), W[m+1] for m = -1, 0, +1
__device__ __forceinline__ void axis_weights(float t, unsigned W[3]) {
    int u = (int)floorf(__fmul_rn(t, 4096.0f));
    int s = 2 * u + 1 - 4096;
    W[0] = (unsigned)((4096 - s) * (4096 - s));
    W[1] = (unsigned)(2 * (3 * 4096 * 4096 - s * s));
    W[2] = (unsigned)((4096 + s) * (4096 + s));
}

template <int D>
struct Tab;

template <>
struct Tab<2> {
    // gather K (4) and optionally G (2) at vertex v0 of the cell, offsets t
    static __device__ __forceinline__ void gather(const PushParams& p, long long v0, const float* t,
                                                  float* kp, float* gp) {
        const float4* K4 = reinterpret_cast<const float4*>(p.K);
        const int nv0 = p.n[0] + 1;
        float s0 = __fsub_rn(1.0f, t[0]), s1 = __fsub_rn(1.0f, t[1]);
        float w0 = __fmul_rn(s0, s1), w1 = __fmul_rn(t[0], s1);
        float w2 = __fmul_rn(s0, t[1]), w3 = __fmul_rn(t[0], t[1]);
        float4 a = __ldg(K4 + v0), b = __ldg(K4 + v0 + 1);
        float4 c = __ldg(K4 + v0 + nv0), d = __ldg(K4 + v0 + nv0 + 1);
        kp[0] = __fmaf_rn(w3, d.x, __fmaf_rn(w2, c.x, __fmaf_rn(w1, b.x, __fmul_rn(w0, a.x))));
        kp[1] = __fmaf_rn(w3, d.y, __fmaf_rn(w2, c.y, __fmaf_rn(w1, b.y, __fmul_rn(w0, a.y))));
        kp[2] = __fmaf_rn(w3, d.z, __fmaf_rn(w2, c.z, __fmaf_rn(w1, b.z, __fmul_rn(w0, a.z))));
        kp[3] = __fmaf_rn(w3, d.w, __fmaf_rn(w2, c.w, __fmaf_rn(w1, b.w, __fmul_rn(w0, a.w))));
        if (gp) {
            const float2* G2 = reinterpret_cast<const float2*>(p.G);
            float2 ga = __ldg(G2 + v0), gb = __ldg(G2 + v0 + 1);
            float2 gc = __ldg(G2 + v0 + nv0), gd = __ldg(G2 + v0 + nv0 + 1);
            gp[0] = __fmaf_rn(w3, gd.x, __fmaf_rn(w2, gc.x, __fmaf_rn(w1, gb.x, __fmul_rn(w0, ga.x))));
            gp[1] = __fmaf_rn(w3, gd.y, __fmaf_rn(w2, gc.y, __fmaf_rn(w1, gb.y, __fmul_rn(w0, ga.y))));
        }
    }
};

template <>
struct Tab<3> {
    static __device__ __forceinline__ void gather(const PushParams& p, long long v0, const float* t,
                                                  float* kp, float* gp) {
        const float4* K4 = reinterpret_cast<const float4*>(p.K);
        const float4* G4 = reinterpret_cast<const float4*>(p.G);
        const long long nv0 = p.n[0] + 1, nv01 = nv0 * (p.n[1] + 1);
        float s[3] = {__fsub_rn(1.0f, t[0]), __fsub_rn(1.0f, t[1]), __fsub_rn(1.0f, t[2])};
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            float w = __fmul_rn(__fmul_rn((o & 1) ? t[0] : s[0], (o & 2) ? t[1] : s[1]), (o & 4) ? t[2] : s[2]);
            long long v = v0 + ((o & 1) ? 1 : 0) + ((o & 2) ? nv0 : 0) + ((o & 4) ? nv01 : 0);
            float4 k0 = __ldg(K4 + 3 * v), k1 = __ldg(K4 + 3 * v + 1), k2 = __ldg(K4 + 3 * v + 2);
            float kv[9] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w, k2.x};
#pragma unroll
            for (int q = 0; q < 9; ++q) kp[q] = o == 0 ? __fmul_rn(w, kv[q]) : __fmaf_rn(w, kv[q], kp[q]);
            if (gp) {
                float4 g = __ldg(G4 + v);
                gp[0] = o == 0 ? __fmul_rn(w, g.x) : __fmaf_rn(w, g.x, gp[0]);
                gp[1] = o == 0 ? __fmul_rn(w, g.y) : __fmaf_rn(w, g.y, gp[1]);
                gp[2] = o == 0 ? __fmul_rn(w, g.z) : __fmaf_rn(w, g.z, gp[2]);
            }
        }
    }
};

template <int D>
__device__ __forceinline__ void decode(int w, int* c) {
    if (D == 2) {
        c[0] = w & 0xFFFF;
        c[1] = w >> 16;
    } else {
        c[0] = w & 1023;
        c[1] = (w >> 10) & 1023;
        c[2] = w >> 20;
    }
}
template <int D>
__device__ __forceinline__ int encode(const int* c) {
    return D == 2 ? (c[0] | (c[1] << 16)) : (c[0] | (c[1] << 10) | (c[2] << 20));
}
template <int D>
__device__ __forceinline__ long long vertex_of(const PushParams& p, const int* c) {
    long long v = c[D - 1];
#pragma unroll
    for (int a = D - 2; a >= 0; --a) v = v * (p.n[a] + 1) + c[a];
    return v;
}

// Warp-aggregated fixed-point deposit of one particle per lane (alive lanes only; every
// lane of the warp must call it). centre: per-axis cell; t: offsets.
template <int D>
__device__ __forceinline__ void deposit_warp(const PushParams& p, int s, bool alive, const int* c,
                                             const float* t) {
    constexpr int NN = D == 2 ? 9 : 27;
    unsigned W[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) axis_weights(alive ? t[a] : 0.0f, W[a]);
    long long key = -1;
    if (alive) {
        key = c[D - 1];
#pragma unroll
        for (int a = D - 2; a >= 0; --a) key = key * p.n[a] + c[a];
    }
    unsigned peers = __match_any_sync(FULL, (unsigned long long)key);
    int lane = threadIdx.x & 31;
    bool leader = alive && (__ffs(peers) - 1) == lane;
    // neighbour indices per axis (wrap or fold)
    int nb[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int n = p.n[a];
        bool per = p.pbc[2 * a] == CPIC_PBC_PERIODIC;
        int cm = c[a] - 1, cp = c[a] + 1;
        nb[a][0] = per ? (cm < 0 ? cm + n : cm) : (cm < 0 ? 0 : cm);
        nb[a][1] = c[a];
        nb[a][2] = per ? (cp >= n ? cp - n : cp) : (cp >= n ? n - 1 : cp);
    }
    unsigned long long* grid = p.charge + (long long)s * p.ncell;
    unsigned qsum_off = 0;
    unsigned qc = 0;
#pragma unroll
    for (int node = 0; node < NN; ++node) {
        int m0 = node % 3, m1 = (node / 3) % 3, m2 = node / 9;
        bool centre = (m0 == 1) && (m1 == 1) && (D == 2 || m2 == 1);
        unsigned q = 0;
        if (alive && !centre) {
            unsigned long long pr = (unsigned long long)W[0][m0] * W[1][m1];
            unsigned long long q01 = (pr + (1ull << 29)) >> 30;
            if (D == 3) q01 = (q01 * W[2][m2] + (1ull << 26)) >> 27;
            q = (unsigned)q01;
            qsum_off += q;
        }
        if (centre) continue;
        unsigned tot = __reduce_add_sync(peers, q);
        if (leader && tot) {
            long long idx = nb[0][m0] + (long long)p.n[0] * (nb[1][m1] + (D == 3 ? (long long)p.n[1] * nb[2][m2] : 0));
            atomicAdd(grid + idx, (unsigned long long)tot);
        }
    }
    qc = alive ? ((1u << QF) - qsum_off) : 0u;
    unsigned totc = __reduce_add_sync(peers, qc);
    if (leader) {
        long long idx = c[0] + (long long)p.n[0] * (c[1] + (D == 3 ? (long long)p.n[1] * c[2] : 0));
        atomicAdd(grid + idx, (unsigned long long)totc);
    }
}

struct SpeciesRanges {
    long long cnt[CPIC_MAX_SPECIES];
    long long voff[CPIC_MAX_SPECIES + 1];
};

__device__ __forceinline__ SpeciesRanges species_ranges(const PushParams& p) {
    SpeciesRanges r;
    r.voff[0] = 0;
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        long long c = s < p.nsp ? p.ctr->count[s] : 0;
        r.cnt[s] = c;
        r.voff[s + 1] = r.voff[s] + ((c + 31) & ~31ll);
    }
    return r;
}

__device__ __forceinline__ int species_of(const SpeciesRanges& r, int nsp, long long vi) {
    int s = 0;
#pragma unroll
    for (int x = 1; x < CPIC_MAX_SPECIES; ++x)
        if (x < nsp && vi >= r.voff[x]) s = x;
    return s;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}


}  // namespace pk
}  // namespace cpic
