// Device helpers shared by the particle kernels (push, deposit, kick, injection):
// split-position renormalisation, the spec Q integer b2 weights, the b1 vertex gathers of
// the mover's FP32 tables, and the warp-aggregated fixed-point deposit.
#pragma once

#include "internal.cuh"

namespace cpic {
namespace pk {

constexpr unsigned FULL = 0xffffffffu;

// c mod n for a periodic axis; displacements are almost always within one period, so the
// integer remainder is only taken for the rare larger ones
__device__ __forceinline__ int wrapi(int c, int n) {
    if (c < 0) c += n;
    else if (c >= n) c -= n;
    if ((unsigned)c >= (unsigned)n) {
        c %= n;
        if (c < 0) c += n;
    }
    return c;
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

// Per-axis fixed-point b2 weights (spec Q), w[m+1] for m = -1, 0, +1, at QB = 16 bits: the
// offset is quantised to u = floor(t 2^16) (exact for an FP32 offset in [0, 1)); the exact
// integer b2 values of the sub-cell centre, scaled by 2^35, are (2^16 -+ s)^2 for the outer
// nodes, s = 2u + 1 - 2^16 (up to 2^34, so 64-bit); those are rounded to 16 bits (halves up)
// and the centre takes the remainder, so the three sum to 2^16. Every weight is below 2^16.
__device__ __forceinline__ void axis_weights(float t, unsigned w[3]) {
    constexpr int H = 2 * QK + 3 - QB;
    const int u = (int)floorf(__fmul_rn(t, 65536.0f));
    const int s = 2 * u + 1 - 65536;
    const unsigned lo = (unsigned)(65536 - s), hi = (unsigned)(65536 + s);
    w[0] = (unsigned)(((unsigned long long)lo * lo + (1ull << (H - 1))) >> H);
    w[2] = (unsigned)(((unsigned long long)hi * hi + (1ull << (H - 1))) >> H);
    w[1] = (1u << QB) - w[0] - w[2];
}

// Node weights (spec Q) of every node but the centre: the exact product of the per-axis
// weights rounded to QF = 24 bits (halves up). 2D: a b < 2^32; 3D: a (b c) < 2^48. The
// centre node takes 2^24 minus the others, so a particle deposits exactly 2^24 units and
// every node weight is below 2^24.
__device__ __forceinline__ unsigned node_weight2(unsigned a, unsigned b) {
    return (a * b + (1u << (2 * QB - QF - 1))) >> (2 * QB - QF);
}
__device__ __forceinline__ unsigned node_weight3(unsigned a, unsigned bc) {
    return (unsigned)(((unsigned long long)a * bc + (1ull << (3 * QB - QF - 1))) >> (3 * QB - QF));
}

// all 3^D node weights of one particle in node order (m0 fastest), centre included
template <int D>
__device__ __forceinline__ void node_weights(const float* t, unsigned* q) {
    constexpr int NN = D == 2 ? 9 : 27;
    constexpr int CENTRE = NN / 2;
    unsigned w[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) axis_weights(t[a], w[a]);
    unsigned rest = 0;
#pragma unroll
    for (int node = 0; node < NN; ++node) {
        if (node == CENTRE) continue;
        const int m0 = node % 3, m1 = (node / 3) % 3, m2 = node / 9;
        q[node] = D == 2 ? node_weight2(w[0][m0], w[1][m1]) : node_weight3(w[0][m0], w[1][m1] * w[2][m2]);
        rest += q[node];
    }
    q[CENTRE] = (1u << QF) - rest;
}

// Boris step for a uniform B0 (eq. (step1) with the magnetic term; Boris split): with the
// half kick h, t = h B0 (q/m folded into h) and s = 2 t / (1 + |t|^2),
//   v- = v + h E;  v' = v- + v- x t;  v+ = v- + v' x s;  v = v+ + h E,
// FP32 in this order, each cross-product component as fmaf(a_y, b_z, -(a_z b_y)) added to
// the left vector's component. E has three components (E_z = 0 in 2D).
__device__ __forceinline__ void boris_kick(float* v, const float* E, float h, const float* t, const float* s) {
    const float m0 = __fmaf_rn(h, E[0], v[0]), m1 = __fmaf_rn(h, E[1], v[1]), m2 = __fmaf_rn(h, E[2], v[2]);
    const float p0 = __fadd_rn(m0, __fmaf_rn(m1, t[2], -__fmul_rn(m2, t[1])));
    const float p1 = __fadd_rn(m1, __fmaf_rn(m2, t[0], -__fmul_rn(m0, t[2])));
    const float p2 = __fadd_rn(m2, __fmaf_rn(m0, t[1], -__fmul_rn(m1, t[0])));
    const float q0 = __fadd_rn(m0, __fmaf_rn(p1, s[2], -__fmul_rn(p2, s[1])));
    const float q1 = __fadd_rn(m1, __fmaf_rn(p2, s[0], -__fmul_rn(p0, s[2])));
    const float q2 = __fadd_rn(m2, __fmaf_rn(p0, s[1], -__fmul_rn(p1, s[0])));
    v[0] = __fmaf_rn(h, E[0], q0);
    v[1] = __fmaf_rn(h, E[1], q1);
    v[2] = __fmaf_rn(h, E[2], q2);
}

template <int D>
struct Tab;

template <>
struct Tab<2> {
    // gather K (4) and optionally G (2) at vertex v0 of the cell, offsets t
    static __device__ __forceinline__ void gather(const PushParams& p, int v0, const float* t,
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

// b1 interpolation of a scalar 2D vertex table (the axisymmetric radius), with the corner
// weights and summation order of Tab<2>
__device__ __forceinline__ float gather_scalar2(const PushParams& p, int v0, const float* t) {
    const int nv0 = p.n[0] + 1;
    const float s0 = __fsub_rn(1.0f, t[0]), s1 = __fsub_rn(1.0f, t[1]);
    const float w0 = __fmul_rn(s0, s1), w1 = __fmul_rn(t[0], s1);
    const float w2 = __fmul_rn(s0, t[1]), w3 = __fmul_rn(t[0], t[1]);
    const float a = __ldg(p.R + v0), b = __ldg(p.R + v0 + 1), c = __ldg(p.R + v0 + nv0), d = __ldg(p.R + v0 + nv0 + 1);
    return __fmaf_rn(w3, d, __fmaf_rn(w2, c, __fmaf_rn(w1, b, __fmul_rn(w0, a))));
}

// Collection tally (which part of the object collects the particles, Fig. 7): a particle
// removed at a face normal to axis 0 counts in that face's cell at its corrector point,
// the transverse indices clamped into the face (a particle that left through an edge).
template <int D>
__device__ __forceinline__ void collect_face(const PushParams& p, int s, int face, const int* cn) {
    if (face != 0 && face != 1) return;
    int idx = min(max(cn[1], 0), p.n[1] - 1);
    if (D == 3) idx += p.n[1] * min(max(cn[2], 0), p.n[2] - 1);
    atomicAdd(p.collect + ((long long)(2 * s + face)) * p.ncollect + idx, 1ull);
}

template <>
struct Tab<3> {
    static __device__ __forceinline__ void gather(const PushParams& p, int v0, const float* t,
                                                  float* kp, float* gp) {
        const float4* K4 = reinterpret_cast<const float4*>(p.K);
        const float4* G4 = reinterpret_cast<const float4*>(p.G);
        const int nv0 = p.n[0] + 1, nv01 = nv0 * (p.n[1] + 1);
        float s[3] = {__fsub_rn(1.0f, t[0]), __fsub_rn(1.0f, t[1]), __fsub_rn(1.0f, t[2])};
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            float w = __fmul_rn(__fmul_rn((o & 1) ? t[0] : s[0], (o & 2) ? t[1] : s[1]), (o & 4) ? t[2] : s[2]);
            int v = v0 + ((o & 1) ? 1 : 0) + ((o & 2) ? nv0 : 0) + ((o & 4) ? nv01 : 0);
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
__device__ __forceinline__ int vertex_of(const PushParams& p, const int* c) {
    int v = c[D - 1];
#pragma unroll
    for (int a = D - 2; a >= 0; --a) v = v * (p.n[a] + 1) + c[a];
    return v;
}

// Warp-aggregated fixed-point deposit of one particle per lane into the padded grid (one
// halo layer per side, folded into the cell grid afterwards, so node addresses are the
// cell's address plus fixed offsets and need no wrap or fold). Every lane of the warp must
// call it (alive lanes deposit). c: per-axis cell; t: offsets.
// The node weights are exact integer products of the per-axis weights. Particles are kept
// in cell order, so many lanes of a warp share one cell: the largest group of lanes with a
// common cell (__match_any_sync) is summed with full-warp __reduce_add_sync (a node weight
// is below 2^24, so 32 of them fit 32 bits) and its leader deposits the sums; the other
// lanes deposit their own weights. Integer sums are exact, so the grouping does not change
// the result.
template <int D>
__device__ __forceinline__ void deposit_warp(const PushParams& p, int s, bool alive, const int* c,
                                             const float* t) {
    constexpr int NN = D == 2 ? 9 : 27;
    const int lane = threadIdx.x & 31;
    const unsigned live = __ballot_sync(FULL, alive);
    if (!live) return;
    unsigned q[NN];
    {
        float tz[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < D; ++a) tz[a] = alive ? t[a] : 0.0f;
        node_weights<D>(tz, q);
    }
    if (!alive) {  // dead lanes carry zero weight
#pragma unroll
        for (int node = 0; node < NN; ++node) q[node] = 0u;
    }
    // padded offset of this lane's cell (dead lanes: keys of their own); every group of lanes
    // that share a cell is summed over its lanes and deposited by its lowest lane
    const int off = alive ? c[0] + c[1] * p.hs1 + (D == 3 ? c[2] * p.hs2 : 0) : -1 - lane;
    const unsigned peers = __match_any_sync(FULL, off);
    const int my_leader = __ffs(peers) - 1;
    const bool issue = alive && lane == my_leader;
    for (unsigned g = __ballot_sync(FULL, issue && (peers & (peers - 1u)) != 0u); g; g &= g - 1u) {
        if (my_leader == __ffs(g) - 1) {
#pragma unroll
            for (int node = 0; node < NN; ++node) q[node] = __reduce_add_sync(peers, q[node]);
        }
    }
    if (issue) {  // every node, without a per-node test (a zero weight adds nothing)
        unsigned long long* g = p.charge + (long long)s * p.ncell_h + p.origin + off;
#pragma unroll
        for (int m12 = 0; m12 < NN / 3; ++m12) {
            unsigned long long* row = g + ((m12 % 3) - 1) * p.hs1 + (D == 3 ? (m12 / 3 - 1) * p.hs2 : 0);
            atomicAdd(row - 1, (unsigned long long)q[3 * m12]);
            atomicAdd(row, (unsigned long long)q[3 * m12 + 1]);
            atomicAdd(row + 1, (unsigned long long)q[3 * m12 + 2]);
        }
    }
}

// Philox4x32-10 counter-based generator (Salmon et al., SC'11): 10 rounds of the two
// 32x32 -> 64-bit multiplies with the published multipliers and Weyl key increments.
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

// Live-slot ranges of the species in one particle kernel. The virtual index space
// concatenates the species, each padded to a multiple of 32, so every warp holds one
// species. Kept in named registers (no indexed local arrays).
struct SpeciesRanges {
    long long c0, c1, c2, c3;      // slots in use per species
    long long v1, v2, v3, total;   // start of species 1, 2, 3 and the end
};

__device__ __forceinline__ SpeciesRanges species_ranges(const PushParams& p) {
    SpeciesRanges r;
    const DevCounters* ctr = p.ctr;
    r.c0 = ctr->count[0];
    r.c1 = p.nsp > 1 ? ctr->count[1] : 0;
    r.c2 = p.nsp > 2 ? ctr->count[2] : 0;
    r.c3 = p.nsp > 3 ? ctr->count[3] : 0;
    r.v1 = (r.c0 + 31) & ~31ll;
    r.v2 = r.v1 + ((r.c1 + 31) & ~31ll);
    r.v3 = r.v2 + ((r.c2 + 31) & ~31ll);
    r.total = r.v3 + ((r.c3 + 31) & ~31ll);
    return r;
}

// species of virtual index vi, its local index and whether it is an occupied slot
__device__ __forceinline__ int species_of(const SpeciesRanges& r, int vi, long long& local, bool& occupied) {
    int s = (vi >= r.v1) + (vi >= r.v2) + (vi >= r.v3);
    long long start = s == 0 ? 0 : s == 1 ? r.v1 : s == 2 ? r.v2 : r.v3;
    long long cnt = s == 0 ? r.c0 : s == 1 ? r.c1 : s == 2 ? r.c2 : r.c3;
    local = vi - start;
    occupied = vi < r.total && local < cnt;
    return s;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

}  // namespace pk
}  // namespace cpic
