// Rows a2-a6 for three-dimensional runs: the fused hybrid-mover kernel (Sec. II.B.4) with its
// grid coupling, specialised for the hot path. Same arithmetic as the generic particle kernel
// (push.cu) — b1 gathers, kick, predictor / k re-gather / corrector, boundaries (periodic,
// absorbing, spec B reflection), b2 fixed-point deposit — organised like the 2D kernel:
//   - blocks walk chunks of one species (at most CHUNK particles, so that a chunk of the
//     cell-sorted particles covers a few rows of one plane);
//   - the boundary kind of each axis is a template parameter;
//   - the next particle's state is loaded before the current one is processed;
//   - the deposit goes into a shared-memory tile of the chunk's sampled planes and rows (with
//     the stencil's neighbours), in the padded layout,
//     flushed once per chunk; lanes whose 3x3x3 stencil leaves the tile
//     deposit straight into the padded global grid. With ~30 particles per cell, most lanes
//     of a warp hold a few neighbouring cells, and sending each lane's 27 node weights to L2
//     as 64-bit atomics would bind the kernel on L2 atomic throughput;
//   - instruction economy as in the 2D kernel: component pairs of the gathers in packed
//     FP32x2 arithmetic (each lane rounds as the scalar form), the tile atomics' carries
//     collected in a bit mask, predicated state stores, the iteration loop specialised on
//     whether the chunk's tile is in use.
#include <atomic>
#include <type_traits>

#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

constexpr int P3_THREADS = 256;
constexpr int P3_CHUNK = 4096;        // particles per chunk (a few rows of one plane)
constexpr int P3_TILE_CELLS = 8192;   // 64 KB of shared memory (two 32-bit words per cell):
                                      // three blocks per SM (80 registers a thread)

enum { K_PER = CPIC_PBC_PERIODIC, K_ABS = CPIC_PBC_ABSORB, K_REF = CPIC_PBC_REFLECT };

struct Tile3 {
    unsigned lo;          // shared-memory address of the low words
    unsigned* hi_ptr;     // the high words
    int i0, j0, k0;       // cell of the tile's corner (tile coordinates are taken modulo the
                          // axis length on periodic axes)
    int W, R, P;          // columns, rows, planes
    bool on;
};

// tile coordinate of cell index c on an axis: c - origin, wrapped into [0, n) when periodic
template <int KIND>
__device__ __forceinline__ int tile_coord(int c, int origin, int n) {
    int d = c - origin;
    if (KIND == CPIC_PBC_PERIODIC) {
        if (d < 0) d += n;
        if (d >= n) d -= n;
    }
    return d;
}

#define CPIC_TILE3_ADD(OFF, ARG)                        \
    "atom.shared.add.u32 o, [%1+" OFF "], " ARG ";\n\t" \
    "add.cc.u32 s, o, " ARG ";\n\t"                      \
    "addc.u32 %0, %0, %0;\n\t"

// adds q0, q1, q2 to three consecutive low words from shared address a (32-bit atomics); m is
// shifted left by one bit per word and takes the word's carry out in its lowest bit
__device__ __forceinline__ void tile3_add_row(unsigned& m, unsigned a, unsigned q0, unsigned q1, unsigned q2) {
    asm volatile("{\n\t.reg .u32 o, s;\n\t" CPIC_TILE3_ADD("0", "%2") CPIC_TILE3_ADD("4", "%3")
                     CPIC_TILE3_ADD("8", "%4") "}"
                 : "+r"(m)
                 : "r"(a), "r"(q0), "r"(q1), "r"(q2)
                 : "memory");
}

// Deposit of one particle per lane into the chunk's tile; lanes whose stencil leaves the
// tile deposit into the padded global grid (deposit_warp). Lanes that share a cell are summed
// first (__reduce_add_sync over each such group) and deposited by one lane of the group.
// Node weights are produced and deposited one row of three at a time (nine rows).
template <int K0, int K1, int K2>
__device__ __forceinline__ void deposit_tile3(const PushParams& p, const Tile3& tl, int s, bool alive, const int* c,
                                              const float* t) {
    const int lane = threadIdx.x & 31;
    const int px = tile_coord<K0>(c[0], tl.i0, p.n[0]);
    const int ry = tile_coord<K1>(c[1], tl.j0, p.n[1]);
    const int pz = tile_coord<K2>(c[2], tl.k0, p.n[2]);
    const bool in = alive && px >= 1 && px + 1 < tl.W && pz >= 1 && pz + 1 < tl.P && ry >= 1 && ry + 1 < tl.R;
    const bool out = alive && !in;
    if (__any_sync(FULL, out)) deposit_warp<3>(p, s, out, c, t);
    if (!__any_sync(FULL, in)) return;
    unsigned w[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) axis_weights(t[a], w[a]);
    // lanes that do not deposit here get keys of their own; every group of lanes that share a
    // cell is summed over its lanes (__reduce_add_sync) and deposited by its lowest lane, so
    // no two lanes of one atomic instruction add to the same word
    const int off = in ? (pz * tl.R + ry) * tl.W + px : -1 - lane;
    const unsigned peers = __match_any_sync(FULL, off);
    const int my_leader = __ffs(peers) - 1;
    const bool issue = in && lane == my_leader;
    const unsigned groups = __ballot_sync(FULL, issue && (peers & (peers - 1u)) != 0u);  // leaders of shared cells
    const int plane = tl.R * tl.W;
    const unsigned base = tl.lo + 4u * (unsigned)(off - 1 - tl.W - plane);
    // rows of three nodes (m1, m2) in the order below, the centre row (1, 1) last, so that the
    // centre node can take 2^24 minus the other 26 node weights of the lane
    constexpr int ROW[9] = {0, 1, 2, 3, 5, 6, 7, 8, 4};
    unsigned rest = 0;
    unsigned m = 0;  // carry out of the k-th node added (k = 3 i + m0 for the i-th row) in bit 26 - k
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int m1 = ROW[i] % 3, m2 = ROW[i] / 3;
        const unsigned w12 = w[1][m1] * w[2][m2];
        unsigned q0 = node_weight3(w[0][0], w12), q2 = node_weight3(w[0][2], w12), q1;
        if (ROW[i] == 4) {
            q1 = (1u << QF) - rest - q0 - q2;
        } else {
            q1 = node_weight3(w[0][1], w12);
            rest += q0 + q1 + q2;
        }
        for (unsigned g = groups; g; g &= g - 1u) {  // warp-uniform: one pass per shared cell
            if (my_leader == __ffs(g) - 1) {
                q0 = __reduce_add_sync(peers, q0);
                q1 = __reduce_add_sync(peers, q1);
                q2 = __reduce_add_sync(peers, q2);
            }
        }
        if (issue) tile3_add_row(m, base + 4u * (unsigned)(m1 * tl.W + m2 * plane), q0, q1, q2);
    }
    if (issue && m) {  // rare: carries into the high words
        unsigned* hi = tl.hi_ptr + (off - 1 - tl.W - plane);
#pragma unroll
        for (int k = 0; k < 27; ++k) {
            const int r = ROW[k / 3];
            if ((m >> (26 - k)) & 1u) atomicAdd(hi + (k % 3) + (r % 3) * tl.W + (r / 3) * plane, 1u);
        }
    }
}

// the seven state words of one particle, stored when p holds (predicated, no branch)
__device__ __forceinline__ void store_state3(bool p, int* c, int cv, float* t0, float* t1, float* t2, const float* t,
                                             float* v0, float* v1, float* v2, const float* v) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
        "@q st.global.b32 [%1], %2;\n\t@q st.global.f32 [%3], %4;\n\t@q st.global.f32 [%5], %6;\n\t"
        "@q st.global.f32 [%7], %8;\n\t@q st.global.f32 [%9], %10;\n\t@q st.global.f32 [%11], %12;\n\t"
        "@q st.global.f32 [%13], %14;\n\t}" ::"r"((unsigned)p),
        "l"(c), "r"(cv), "l"(t0), "f"(t[0]), "l"(t1), "f"(t[1]), "l"(t2), "f"(t[2]), "l"(v0), "f"(v[0]), "l"(v1),
        "f"(v[1]), "l"(v2), "f"(v[2])
        : "memory");
}

// b1 gather of the vertex k table (and G when gp is given) at vertex v0 of the cell, offsets
// t: the same products and accumulation order as the scalar form, component pairs in packed
// FP32x2 arithmetic. A vertex record holds k (9 words) and G (3 words, written there by the
// vertex-field pass), so both come in three 16-byte loads.
__device__ __forceinline__ void gather3(const PushParams& p, int v0, const float* t, float* kp, float* gp) {
    const float4* K4 = reinterpret_cast<const float4*>(p.K);
    const int nv0 = p.n[0] + 1, nv01 = nv0 * (p.n[1] + 1);
    const float s[3] = {__fsub_rn(1.0f, t[0]), __fsub_rn(1.0f, t[1]), __fsub_rn(1.0f, t[2])};
    float2 k01, k23, k45, k67, g01;
    float k8, g2;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const float w = __fmul_rn(__fmul_rn((o & 1) ? t[0] : s[0], (o & 2) ? t[1] : s[1]), (o & 4) ? t[2] : s[2]);
        const int v = v0 + ((o & 1) ? 1 : 0) + ((o & 2) ? nv0 : 0) + ((o & 4) ? nv01 : 0);
        const float4 a = __ldg(K4 + 3 * v), b = __ldg(K4 + 3 * v + 1);
        float4 g;  // (k22, G0, G1, G2)
        if (gp)
            g = __ldg(K4 + 3 * v + 2);
        else
            g.x = __ldg(reinterpret_cast<const float*>(K4 + 3 * v + 2));
        const float c = g.x;
        const float2 ww = make_float2(w, w);
        if (o == 0) {
            k01 = __fmul2_rn(ww, make_float2(a.x, a.y));
            k23 = __fmul2_rn(ww, make_float2(a.z, a.w));
            k45 = __fmul2_rn(ww, make_float2(b.x, b.y));
            k67 = __fmul2_rn(ww, make_float2(b.z, b.w));
            k8 = __fmul_rn(w, c);
        } else {
            k01 = __ffma2_rn(ww, make_float2(a.x, a.y), k01);
            k23 = __ffma2_rn(ww, make_float2(a.z, a.w), k23);
            k45 = __ffma2_rn(ww, make_float2(b.x, b.y), k45);
            k67 = __ffma2_rn(ww, make_float2(b.z, b.w), k67);
            k8 = __fmaf_rn(w, c, k8);
        }
        if (gp) {
            if (o == 0) {
                g01 = __fmul2_rn(ww, make_float2(g.y, g.z));
                g2 = __fmul_rn(w, g.w);
            } else {
                g01 = __ffma2_rn(ww, make_float2(g.y, g.z), g01);
                g2 = __fmaf_rn(w, g.w, g2);
            }
        }
    }
    kp[0] = k01.x;
    kp[1] = k01.y;
    kp[2] = k23.x;
    kp[3] = k23.y;
    kp[4] = k45.x;
    kp[5] = k45.y;
    kp[6] = k67.x;
    kp[7] = k67.y;
    kp[8] = k8;
    if (gp) {
        gp[0] = g01.x;
        gp[1] = g01.y;
        gp[2] = g2;
    }
}

template <int KIND>
__device__ __forceinline__ void predict_axis3(float x, int c, int n, int& cp, float& tp) {
    int dc;
    renorm(x, tp, dc);
    int ci = c + dc;
    if (KIND == K_PER) {
        ci = wrapi(ci, n);
    } else {
        if (ci < 0) {
            ci = 0;
            tp = 0.0f;
        }
        if (ci >= n) {
            ci = n - 1;
            tp = 1.0f;
        }
    }
    cp = ci;
}

// Rows a2-a5 for one particle (per lane): b1 gather of k and G at xi^n, kick, predictor, k
// re-gather, corrector, boundaries (periodic wrap, absorption, spec B reflection). cw: the
// packed cell (-1: empty slot); t, v: offsets and velocity in, new velocity out; cn, tn: the
// new cell and offsets; face: -1 (kept) or the face it left by (6: non-finite); ke32: the
// FP32 product v_old . v_new of the kinetic-energy tally (0 for empty slots).
template <int K0, int K1, int K2>
__device__ __forceinline__ void mover3(const PushParams& p, float dtqm, int cw, float* t, float* v, int* cn,
                                       float* tn, int& face, float& ke32) {
    constexpr int KIND[3] = {K0, K1, K2};
    const float hdt = p.hdt, dt = p.dt;
    const bool active = cw >= 0;
    int c[3] = {active ? (cw & 1023) : 0, active ? ((cw >> 10) & 1023) : 0, active ? (cw >> 20) : 0};
    if (!active) t[0] = t[1] = t[2] = v[0] = v[1] = v[2] = 0.0f;

    // a2: b1 gather of k and G at xi^n
    float kp[9], gp[3];
    gather3(p, vertex_of<3>(p, c), t, kp, gp);
    // a3: E^al = -sum_a G^a k^{a al}, kick
    const float vo0 = v[0], vo1 = v[1], vo2 = v[2];
#pragma unroll
    for (int al = 0; al < 3; ++al) {
        float e = __fmul_rn(kp[al], gp[0]);
        e = __fmaf_rn(kp[3 + al], gp[1], e);
        e = __fmaf_rn(kp[6 + al], gp[2], e);
        v[al] = __fmaf_rn(dtqm, -e, v[al]);
    }
    // a4: predictor
    int cpred[3];
    float tpred[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float d = __fmul_rn(kp[3 * a], v[0]);
        d = __fmaf_rn(kp[3 * a + 1], v[1], d);
        d = __fmaf_rn(kp[3 * a + 2], v[2], d);
        float x = __fmaf_rn(hdt, d, t[a]);
        if (!isfinite(x)) x = t[a];
        if (KIND[a] == K_PER)
            predict_axis3<K_PER>(x, c[a], p.n[a], cpred[a], tpred[a]);
        else
            predict_axis3<K_ABS>(x, c[a], p.n[a], cpred[a], tpred[a]);
    }
    float kq[9];
    gather3(p, vertex_of<3>(p, cpred), tpred, kq, nullptr);
    // corrector
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float d = __fmul_rn(kq[3 * a], v[0]);
        d = __fmaf_rn(kq[3 * a + 1], v[1], d);
        d = __fmaf_rn(kq[3 * a + 2], v[2], d);
        float x = __fmaf_rn(dt, d, t[a]);
        if (!isfinite(x)) {
            bad = true;
            x = t[a];
        }
        int dc;
        renorm(x, tn[a], dc);
        cn[a] = c[a] + dc;
    }
    // a5: boundaries (periodic wrap, absorption), then spec B after the tally
    face = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (KIND[a] == K_PER) {
            cn[a] = wrapi(cn[a], p.n[a]);
        } else if (KIND[a] == K_ABS && face < 0) {
            if (cn[a] < 0) face = 2 * a;
            else if (cn[a] >= p.n[a]) face = 2 * a + 1;
        }
    }
    if (bad) face = 6;
    ke32 = active ? __fmaf_rn(vo2, v[2], __fmaf_rn(vo1, v[1], __fmul_rn(vo0, v[0]))) : 0.0f;
    if (face < 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (KIND[a] != K_REF || face >= 0 || (cn[a] >= 0 && cn[a] < p.n[a])) continue;
            const bool below = cn[a] < 0;
            int c2 = below ? (-cn[a] - 1) : (2 * p.n[a] - 1 - cn[a]);
            float t2 = __fsub_rn(1.0f, tn[a]);
            if (t2 >= 1.0f) {
                t2 = 0.0f;
                c2 += 1;
            }
            if (c2 < 0 || c2 >= p.n[a]) {
                face = 2 * a + (below ? 0 : 1);
                continue;
            }
            cn[a] = c2;
            tn[a] = t2;
            float nn = __fmul_rn(kq[3 * a], kq[3 * a]);
            float dot = __fmul_rn(v[0], kq[3 * a]);
            nn = __fmaf_rn(kq[3 * a + 1], kq[3 * a + 1], nn);
            dot = __fmaf_rn(v[1], kq[3 * a + 1], dot);
            nn = __fmaf_rn(kq[3 * a + 2], kq[3 * a + 2], nn);
            dot = __fmaf_rn(v[2], kq[3 * a + 2], dot);
            const float sf = __fdiv_rn(__fmul_rn(2.0f, dot), nn);
#pragma unroll
            for (int al = 0; al < 3; ++al) v[al] = __fmaf_rn(-sf, kq[3 * a + al], v[al]);
        }
    }
    if (!active) face = -2;
}

template <int K0, int K1, int K2>
__global__ void __launch_bounds__(P3_THREADS, 3) push3d_kernel(PushParams p) {
    extern __shared__ unsigned tile_dyn[];  // [P3_TILE_CELLS] low words, then high words
    unsigned* tile_lo = tile_dyn;
    unsigned* tile_hi = tile_dyn + P3_TILE_CELLS;
    __shared__ int red[6][P3_THREADS / 32];
    __shared__ int sh_gone[8];  // removed particles of the chunk per face (6: non-finite)
    const DevCounters* ctr = p.ctr;
    const int cur = ctr->cur;
    const int nsp = p.nsp;
    int cnt[CPIC_MAX_SPECIES];
    int total = 0;
#pragma unroll
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        cnt[s] = s < nsp ? (int)ctr->count[s] : 0;
        total += cnt[s];
    }
    if (total == 0) return;
    int C = ((total + (int)gridDim.x - 1) / (int)gridDim.x + P3_THREADS - 1) / P3_THREADS * P3_THREADS;
    if (C > P3_CHUNK) C = P3_CHUNK;
    if (p.chunk > 0) C = p.chunk;
    const int n0 = p.n[0], n1 = p.n[1], n2 = p.n[2];
    const long long T = p.pb.total;
    const float hdt = p.hdt, dt = p.dt;
    constexpr int KIND[3] = {K0, K1, K2};

    for (int ch = blockIdx.x;; ch += gridDim.x) {
        int s = 0, local = ch;
        while (s < nsp) {
            const int nch = (cnt[s] + C - 1) / C;
            if (local < nch) break;
            local -= nch;
            ++s;
        }
        if (s >= nsp) break;
        const int lo = local * C;
        const int hi = min(lo + C, cnt[s]);
        const long long b0 = p.pb.base[s];
        int* __restrict__ cellp = p.pb.cell[cur] + b0;
        float* __restrict__ tq0 = p.pb.t[cur] + b0;
        float* __restrict__ vq0 = p.pb.v[cur] + b0;
        const float dtqm = p.dtqm[s];

        // tile: planes and rows of the chunk's (sampled) particles, one plane and one row
        // of margin each side for the stencil
        Tile3 tl;
        tl.lo = (unsigned)__cvta_generic_to_shared(tile_lo);
        tl.hi_ptr = tile_hi;
        {
            // The tile: the cells around the chunk's middle particle that its sampled
            // particles occupy, plus two cells on every side (the stencil's neighbour and one
            // cell of motion since the last sort). Samples more than two planes or eight rows
            // from the middle one (particles near the polar caps cross the small azimuthal
            // cells quickly, a chunk may end in the next plane) are left out of the bounds:
            // the few particles outside the tile deposit through the global path.
            const int si = lo + (int)(((long long)(hi - lo - 1) * threadIdx.x) / (P3_THREADS - 1));
            const int sc = cellp[si];
            __syncthreads();  // the previous chunk's flush is done with the tile and red[]
            if (threadIdx.x == 0) red[0][0] = 0x7fffffff;
            __syncthreads();
            const int dist = threadIdx.x > P3_THREADS / 2 ? threadIdx.x - P3_THREADS / 2 : P3_THREADS / 2 - threadIdx.x;
            if (sc >= 0) atomicMin(&red[0][0], dist * 1024 + (int)threadIdx.x);
            __syncthreads();
            const int pick = red[0][0];
            int cc[3] = {0, 0, 0};
            bool have = pick != 0x7fffffff;
            if (have) {
                const int cw = cellp[lo + (int)(((long long)(hi - lo - 1) * (pick & 1023)) / (P3_THREADS - 1))];
                cc[0] = cw & 1023;
                cc[1] = (cw >> 10) & 1023;
                cc[2] = cw >> 20;
            }
            int dmin[3] = {0, 0, 0}, dmax[3] = {0, 0, 0};
            if (have && sc >= 0) {
                const int sx[3] = {sc & 1023, (sc >> 10) & 1023, sc >> 20};
                int d[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    d[a] = sx[a] - cc[a];
                    if (KIND[a] == K_PER) {  // nearest image
                        if (2 * d[a] > p.n[a]) d[a] -= p.n[a];
                        if (2 * d[a] < -p.n[a]) d[a] += p.n[a];
                    }
                }
                if (d[2] >= -2 && d[2] <= 2 && d[1] >= -8 && d[1] <= 8) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) dmin[a] = dmax[a] = d[a];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    dmin[a] = min(dmin[a], __shfl_xor_sync(FULL, dmin[a], o));
                    dmax[a] = max(dmax[a], __shfl_xor_sync(FULL, dmax[a], o));
                }
            }
            __syncthreads();  // everyone has read red[0][0]
            if ((threadIdx.x & 31) == 0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    red[a][threadIdx.x >> 5] = dmin[a];
                    red[3 + a][threadIdx.x >> 5] = dmax[a];
                }
            }
            if (threadIdx.x < 8) sh_gone[threadIdx.x] = 0;
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dmin[a] = red[a][0];
                dmax[a] = red[3 + a][0];
            }
#pragma unroll
            for (int w = 1; w < P3_THREADS / 32; ++w) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    dmin[a] = min(dmin[a], red[a][w]);
                    dmax[a] = max(dmax[a], red[3 + a][w]);
                }
            }
            tl.i0 = cc[0] + dmin[0] - 2;
            tl.j0 = cc[1] + dmin[1] - 2;
            tl.k0 = cc[2] + dmin[2] - 2;
            tl.W = dmax[0] - dmin[0] + 5;
            tl.R = dmax[1] - dmin[1] + 5;
            tl.P = dmax[2] - dmin[2] + 5;
            // a spread-out chunk (few particles per cell): narrow the columns, then the rows,
            // to a window around the middle particle that fits the shared memory
            if (tl.P * tl.R * tl.W > P3_TILE_CELLS) {
                const int wmax = max(5, P3_TILE_CELLS / (tl.P * tl.R));
                if (tl.W > wmax) {
                    tl.W = wmax;
                    tl.i0 = cc[0] - wmax / 2;
                }
                const int rmax = max(5, P3_TILE_CELLS / (tl.P * tl.W));
                if (tl.R > rmax) {
                    tl.R = rmax;
                    tl.j0 = cc[1] - rmax / 2;
                }
            }
            tl.on = p.tile && have && tl.P * tl.R * tl.W <= P3_TILE_CELLS;
            if (tl.on)
                for (int k = threadIdx.x; k < tl.P * tl.R * tl.W; k += P3_THREADS) tile_lo[k] = tile_hi[k] = 0u;
            __syncthreads();
        }

        long long ke = 0;

        int i = lo + (int)threadIdx.x;
        int ncw = -1;
        float nt[3] = {0.f, 0.f, 0.f}, nv[3] = {0.f, 0.f, 0.f};
        if (i < hi) {
            ncw = cellp[i];
#pragma unroll
            for (int a = 0; a < 3; ++a) nt[a] = tq0[a * T + i];
#pragma unroll
            for (int a = 0; a < 3; ++a) nv[a] = vq0[a * T + i];
        }
        // the iteration loop, specialised on whether the chunk's tile is in use
        auto iterate = [&](auto tile_tag) {
            constexpr bool TILE = decltype(tile_tag)::value;
            for (int base = lo; base < hi; base += P3_THREADS) {
                const int slot = i;
                const int cw = ncw;
                float t[3] = {nt[0], nt[1], nt[2]};
                float v[3] = {nv[0], nv[1], nv[2]};
                i += P3_THREADS;
                ncw = -1;
                if (i < hi) {
                    ncw = cellp[i];
    #pragma unroll
                    for (int a = 0; a < 3; ++a) nt[a] = tq0[a * T + i];
    #pragma unroll
                    for (int a = 0; a < 3; ++a) nv[a] = vq0[a * T + i];
                }
                int cn[3], face;
                float tn[3], ke32;
                const bool active = cw >= 0;
                mover3<K0, K1, K2>(p, dtqm, cw, t, v, cn, tn, face, ke32);
                ke += __float2ll_rn(__fmul_rn(ke32, 16777216.0f));
                const bool alive = active && face < 0;
                if (active && face >= 0) {  // rare
                    atomicAdd(&sh_gone[face], 1);
                    collect_face<3>(p, s, face, cn);
                }
                store_state3(active, cellp + slot, alive ? (cn[0] | (cn[1] << 10) | (cn[2] << 20)) : -1, tq0 + slot,
                             tq0 + T + slot, tq0 + 2 * T + slot, tn, vq0 + slot, vq0 + T + slot, vq0 + 2 * T + slot, v);
                // a6: deposit
                if constexpr (TILE)
                    deposit_tile3<K0, K1, K2>(p, tl, s, alive, cn, tn);
                else
                    deposit_warp<3>(p, s, alive, cn, tn);
            }
        };
        if (tl.on)
            iterate(std::true_type{});
        else
            iterate(std::false_type{});
        // flush the tile into the padded grid (one halo layer per side; a periodic axis wraps
        // tile cells beyond its halo, a non-periodic one holds nothing there)
        if (tl.on) {
            __syncthreads();
            unsigned long long* g = p.charge + (long long)s * p.ncell_h;
            const int plane = tl.R * tl.W;
            for (int k = threadIdx.x; k < tl.P * plane; k += P3_THREADS) {
                const unsigned long long val = ((unsigned long long)tile_hi[k] << 32) | tile_lo[k];
                if (!val) continue;
                const int pk_ = k / plane, rem = k - pk_ * plane;
                const int rr = rem / tl.W;
                int gx = tl.i0 + (rem - rr * tl.W), gy = tl.j0 + rr, gz = tl.k0 + pk_;
                if (K0 == K_PER) gx = gx < -1 ? gx + n0 : (gx > n0 ? gx - n0 : gx);
                if (K1 == K_PER) gy = gy < -1 ? gy + n1 : (gy > n1 ? gy - n1 : gy);
                if (K2 == K_PER) gz = gz < -1 ? gz + n2 : (gz > n2 ? gz - n2 : gz);
                if (gx < -1 || gx > n0 || gy < -1 || gy > n1 || gz < -1 || gz > n2) continue;
                atomicAdd(g + ((long long)(gz + 1) * (n1 + 2) + (gy + 1)) * (n0 + 2) + (gx + 1), val);
            }
        }
        // tallies of this chunk
        ke = warp_sum_ll(ke);
        if ((threadIdx.x & 31) == 0 && ke) atomicAdd((unsigned long long*)&p.ctr->ke_fp[s], (unsigned long long)ke);
        __syncthreads();  // every absorption of the chunk is in sh_gone
        if (threadIdx.x == 0) {
            DevCounters* cw = p.ctr;
            long long removed = 0;
            for (int f = 0; f < 7; ++f) {
                const int g = sh_gone[f];
                removed += g;
                if (!g) continue;
                if (f < 6)
                    atomicAdd((unsigned long long*)&cw->absorbed[s][f], (unsigned long long)g);
                else
                    atomicAdd((unsigned long long*)&cw->nonfinite, (unsigned long long)g);
            }
            if (removed) atomicAdd((unsigned long long*)&cw->alive[s], (unsigned long long)(-removed));
        }
    }
}

// ---------------------------------------------------------------- direct-deposit kernel
// The same mover, with the b2 deposit going straight into the padded global grid through a
// per-warp transposition: every lane writes its 27 node weights (spec Q) into its row of the
// warp's shared buffer; then lane j (j < 27) walks the 32 rows, summing node j over each
// run of consecutive lanes whose particles share a cell (particles are kept in cell order),
// and adds the run's sum for node j with one 64-bit atomic when the run ends. A warp whose
// 32 particles lie in one cell thus issues a single 27-lane atomic instruction; no lane
// reduction instructions are needed, and the order of integer additions does not change
// the result. No deposit tile: the kernel needs 28 KB of shared memory per block and runs
// four blocks per SM.
constexpr int PD_THREADS = 256;
constexpr int PD_STRIDE = 28;  // words per lane row: 27 node weights and one zero

__device__ __forceinline__ void deposit_runs3(const PushParams& p, int s, bool alive, const int* c, const float* t,
                                              unsigned* wq) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(FULL, alive)) return;
    unsigned w[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) axis_weights(alive ? t[a] : 0.0f, w[a]);
    // node weights in node order (m0 fastest), four to a 16-byte store; the centre (node 13)
    // is written last, as 2^24 minus the other 26
    unsigned* row = wq + lane * PD_STRIDE;
    unsigned rest = 0, q4[4];
#pragma unroll
    for (int node = 0; node < 28; ++node) {
        unsigned q = 0;
        if (node < 27 && node != 13) {
            q = node_weight3(w[0][node % 3], w[1][(node / 3) % 3] * w[2][node / 9]);
            rest += q;
        }
        q4[node & 3] = alive ? q : 0u;
        if ((node & 3) == 3) reinterpret_cast<uint4*>(row)[node >> 2] = make_uint4(q4[0], q4[1], q4[2], q4[3]);
    }
    row[13] = alive ? (1u << QF) - rest : 0u;
    const int off = alive ? c[0] + c[1] * p.hs1 + c[2] * p.hs2 : -1;
    const int next = __shfl_down_sync(FULL, off, 1);  // every lane takes part (lane 31 gets its own)
    const unsigned ends = __ballot_sync(FULL, lane == 31 || next != off);
    __syncwarp();
    const int j = lane < 27 ? lane : 27;  // lanes 27-31 read the zero word
    const int dj = (j % 3 - 1) + ((j / 3) % 3 - 1) * p.hs1 + (j / 9 - 1) * p.hs2;
    unsigned long long* g = p.charge + (long long)s * p.ncell_h + p.origin + dj;
    unsigned acc = 0;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        acc += wq[r * PD_STRIDE + j];
        if ((ends >> r) & 1u) {  // warp-uniform
            const int o = __shfl_sync(FULL, off, r);
            if (o >= 0 && lane < 27) atomicAdd(g + o, (unsigned long long)acc);
            acc = 0;
        }
    }
    __syncwarp();  // the rows are read before the next particle's weights overwrite them
}

template <int K0, int K1, int K2>
__global__ void __launch_bounds__(PD_THREADS, 4) push3d_direct_kernel(PushParams p) {
    __shared__ __align__(16) unsigned qbuf[PD_THREADS / 32][32 * PD_STRIDE];
    __shared__ int sh_gone[8];  // removed particles of the chunk per face (6: non-finite)
    const DevCounters* ctr = p.ctr;
    const int cur = ctr->cur;
    // a fused sort left its order pending: slot i of the other buffer's cell array holds the
    // current-buffer index of the particle that belongs in slot i; read it from there and
    // write the pushed state to slot i of the other buffer (the step's finalisation flips)
    const bool perm = ctr->perm != 0;
    const int dst = perm ? 1 - cur : cur;
    const int nsp = p.nsp;
    int cnt[CPIC_MAX_SPECIES];
    int total = 0;
#pragma unroll
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        cnt[s] = s < nsp ? (int)ctr->count[s] : 0;
        total += cnt[s];
    }
    if (total == 0) return;
    int C = ((total + (int)gridDim.x - 1) / (int)gridDim.x + PD_THREADS - 1) / PD_THREADS * PD_THREADS;
    if (C > P3_CHUNK) C = P3_CHUNK;
    if (p.chunk > 0) C = p.chunk;
    const long long T = p.pb.total;
    unsigned* wq = qbuf[threadIdx.x >> 5];

    for (int ch = blockIdx.x;; ch += gridDim.x) {
        int s = 0, local = ch;
        while (s < nsp) {
            const int nch = (cnt[s] + C - 1) / C;
            if (local < nch) break;
            local -= nch;
            ++s;
        }
        if (s >= nsp) break;
        const int lo = local * C;
        const int hi = min(lo + C, cnt[s]);
        const long long b0 = p.pb.base[s];
        const int* cellp = p.pb.cell[cur] + b0;
        const float* tq0 = p.pb.t[cur] + b0;
        const float* vq0 = p.pb.v[cur] + b0;
        int* cellq = p.pb.cell[dst] + b0;
        float* tq1 = p.pb.t[dst] + b0;
        float* vq1 = p.pb.v[dst] + b0;
        const float dtqm = p.dtqm[s];
        __syncthreads();  // the previous chunk's tallies are read
        if (threadIdx.x < 8) sh_gone[threadIdx.x] = 0;
        __syncthreads();

        long long ke = 0;
        int i = lo + (int)threadIdx.x;
        int ncw = -1;
        float nt[3] = {0.f, 0.f, 0.f}, nv[3] = {0.f, 0.f, 0.f};
        if (i < hi) {
            const int src = perm ? cellq[i] : i;
            ncw = cellp[src];
#pragma unroll
            for (int a = 0; a < 3; ++a) nt[a] = tq0[a * T + src];
#pragma unroll
            for (int a = 0; a < 3; ++a) nv[a] = vq0[a * T + src];
        }
        for (int base = lo; base < hi; base += PD_THREADS) {
            const int slot = i;
            const int cw = ncw;
            float t[3] = {nt[0], nt[1], nt[2]};
            float v[3] = {nv[0], nv[1], nv[2]};
            i += PD_THREADS;
            ncw = -1;
            if (i < hi) {
                const int src = perm ? cellq[i] : i;
                ncw = cellp[src];
#pragma unroll
                for (int a = 0; a < 3; ++a) nt[a] = tq0[a * T + src];
#pragma unroll
                for (int a = 0; a < 3; ++a) nv[a] = vq0[a * T + src];
            }
            int cn[3], face;
            float tn[3], ke32;
            const bool active = cw >= 0;
            mover3<K0, K1, K2>(p, dtqm, cw, t, v, cn, tn, face, ke32);
            ke += __float2ll_rn(__fmul_rn(ke32, 16777216.0f));
            const bool alive = active && face < 0;
            if (active && face >= 0) {  // rare
                atomicAdd(&sh_gone[face], 1);
                collect_face<3>(p, s, face, cn);
            }
            if (p.hist) {  // the next sort's histogram: one atomic per run of equal cells
                const int key = alive ? cn[0] + p.n[0] * (cn[1] + p.n[1] * cn[2]) : -1;
                const unsigned peers = __match_any_sync(FULL, key);
                if (key >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
                    atomicAdd(p.hist + (size_t)s * p.n[0] * p.n[1] * p.n[2] + key, (int)__popc(peers));
            }
            store_state3(active, cellq + slot, alive ? (cn[0] | (cn[1] << 10) | (cn[2] << 20)) : -1, tq1 + slot,
                         tq1 + T + slot, tq1 + 2 * T + slot, tn, vq1 + slot, vq1 + T + slot, vq1 + 2 * T + slot, v);
            deposit_runs3(p, s, alive, cn, tn, wq);  // a6
        }
        ke = warp_sum_ll(ke);
        if ((threadIdx.x & 31) == 0 && ke) atomicAdd((unsigned long long*)&p.ctr->ke_fp[s], (unsigned long long)ke);
        __syncthreads();
        if (threadIdx.x == 0) {
            DevCounters* cw = p.ctr;
            long long removed = 0;
            for (int f = 0; f < 7; ++f) {
                const int g = sh_gone[f];
                removed += g;
                if (!g) continue;
                if (f < 6)
                    atomicAdd((unsigned long long*)&cw->absorbed[s][f], (unsigned long long)g);
                else
                    atomicAdd((unsigned long long*)&cw->nonfinite, (unsigned long long)g);
            }
            if (removed) atomicAdd((unsigned long long*)&cw->alive[s], (unsigned long long)(-removed));
        }
    }
}

template <int K0, int K1, int K2>
int launch_push3d_direct_t(cpic_run* r, const PushParams& p) {
    static std::atomic<int> per_sm[64];
    int dev = 0;
    CPIC_CUDA(cudaGetDevice(&dev));
    std::atomic<int>& cache = per_sm[dev & 63];
    int b = cache.load(std::memory_order_acquire);
    if (b <= 0) {
        CPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, push3d_direct_kernel<K0, K1, K2>, PD_THREADS, 0));
        if (b < 1) b = 1;
        cache.store(b, std::memory_order_release);
    }
    const long long occ = (long long)b * device_sm_count();
    long long tot = 0;
    for (int s = 0; s < r->cfg.n_species; ++s) tot += r->pb.capacity[s];
    long long blocks = (tot + PD_THREADS - 1) / PD_THREADS;
    if (blocks > occ) blocks = occ;
    if (blocks < 1) blocks = 1;
    push3d_direct_kernel<K0, K1, K2><<<(int)blocks, PD_THREADS, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

template <int K0, int K1, int K2>
int launch_push3d_t(cpic_run* r, const PushParams& p) {
    constexpr size_t smem = sizeof(unsigned) * 2 * P3_TILE_CELLS;
    static std::atomic<int> per_sm[64];  // resident blocks per SM, per device (after the
                                         // shared-memory attribute is set on that device)
    int dev = 0;
    CPIC_CUDA(cudaGetDevice(&dev));
    std::atomic<int>& cache = per_sm[dev & 63];
    int b = cache.load(std::memory_order_acquire);
    if (b <= 0) {
        CPIC_CUDA(cudaFuncSetAttribute(push3d_kernel<K0, K1, K2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, push3d_kernel<K0, K1, K2>, P3_THREADS, smem));
        if (b < 1) b = 1;
        cache.store(b, std::memory_order_release);
    }
    const long long occ = (long long)b * device_sm_count();  // one wave
    long long tot = 0;
    for (int s = 0; s < r->cfg.n_species; ++s) tot += r->pb.capacity[s];
    long long blocks = (tot + P3_THREADS - 1) / P3_THREADS;
    if (blocks > occ) blocks = occ;
    if (blocks < 1) blocks = 1;
    push3d_kernel<K0, K1, K2><<<(int)blocks, P3_THREADS, smem, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace

// whether the 3D push the run takes is the direct kernel (see push_fused_ok)
bool push3d_direct_taken(const cpic_run* r) {
    if (r->D != 3 || r->magnetized || r->push_tile) return false;
    const int k0 = r->cfg.particle_bc[0], k1 = r->cfg.particle_bc[2], k2 = r->cfg.particle_bc[4];
    return (k0 == K_ABS && k1 == K_REF && k2 == K_PER) || (k0 == K_PER && k1 == K_PER && k2 == K_PER);
}

// the specialised 3D kernel for the axis kinds it is instantiated for; CPIC_ERR_NOT_BUILT
// for others (the caller then takes the generic kernel)
int launch_push3d(cpic_run* r, const PushParams& p) {
    if (p.magnetized) return CPIC_ERR_NOT_BUILT;
    const int k0 = p.pbc[0], k1 = p.pbc[2], k2 = p.pbc[4];
    if (k0 == K_ABS && k1 == K_REF && k2 == K_PER)
        return p.tile ? launch_push3d_t<K_ABS, K_REF, K_PER>(r, p) : launch_push3d_direct_t<K_ABS, K_REF, K_PER>(r, p);
    if (k0 == K_PER && k1 == K_PER && k2 == K_PER)
        return p.tile ? launch_push3d_t<K_PER, K_PER, K_PER>(r, p) : launch_push3d_direct_t<K_PER, K_PER, K_PER>(r, p);
    return CPIC_ERR_NOT_BUILT;
}

}  // namespace cpic
