// Rows a2-a6 for two-dimensional runs: the fused hybrid-mover kernel (Sec. II.B.4) with its
// grid coupling, specialised for the hot path.
//
// Same arithmetic as the generic particle kernel (push.cu), which stays in use for three
// dimensions and for the deposit-only and kick-only passes; this one is organised for
// instruction economy:
//   - each block walks chunks of one species (a species' particles are split into chunks
//     of equal size, a multiple of the block), so q/m and the tallies are block-uniform;
//   - the boundary kind of each axis is a template parameter (periodic wrap, or clamp of
//     the predictor and absorption at the corrector);
//   - 32-bit slot indices, branch-free handling of empty lanes (they gather at vertex 0 and
//     store nothing) and of non-finite positions (the particle keeps its old cell/offset);
//   - absorbed counts and the kinetic-energy tally stay in registers until the chunk ends;
//   - the particle state of the next iteration is loaded before the current one is
//     processed, so its HBM latency overlaps the arithmetic;
//   - component pairs of the gathers and the kick use packed FP32x2 arithmetic (each lane
//     rounds exactly as the scalar operation, so results are unchanged);
//   - the deposit tile's 32-bit atomics collect their carries in a bit mask (one rare branch
//     per deposit instead of one per node), and the state stores are predicated;
//   - the iteration loop is specialised on whether the chunk's tile is in use.
//
// Per particle: b1 gather of G and k at xi^n (eqs. (vvp), (Wvp), (b1)); E = -k^T G and the
// leapfrog kick (eq. (step1)); predictor xi' = xi^n + dt/2 k(xi^n) v (eq. (step2)); k
// re-gathered at xi' (eq. (step3)); corrector xi^{n+1} = xi^n + dt k(xi') v (eq. (step4));
// boundaries (Sec. II.B.4); b2 deposit in 64-bit fixed point (eqs. (pg), (Wpc), (b2)).
#include <atomic>
#include <type_traits>

#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

constexpr int P2_THREADS = 256;

// predictor component on axis a: renormalise; periodic axes wrap, others clamp to the
// domain (offset 0 below, 1 above)
template <bool PER>
__device__ __forceinline__ void predict_axis(float x, int c, int n, int& cp, float& tp) {
    int dc;
    renorm(x, tp, dc);
    int ci = c + dc;
    if (PER) {
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

// Shared-memory charge tile of one chunk: rows [r0, r0 + R) of the padded grid's layout
// (W = n0 + 2 columns, column 0 and W - 1 the halo), 64-bit counts kept as 32-bit low words
// with carries into high words (shared 32-bit atomics; a group's node weight is below 2^32,
// so one add carries at most once).
constexpr int TILE_CELLS = 2048;  // 16 KB of shared memory per block

struct Tile {
    unsigned lo;      // shared-memory address of the low words
    unsigned* hi_ptr; // the high words
    int r0, R, W;
    bool on;
};

#define CPIC_TILE_ADD(OFF, ARG)                         \
    "atom.shared.add.u32 o, [%1+" OFF "], " ARG ";\n\t" \
    "add.cc.u32 s, o, " ARG ";\n\t"                      \
    "addc.u32 %0, %0, %0;\n\t"

// adds q0, q1, q2 to three consecutive low words starting at shared address a (32-bit
// atomics); m is shifted left by one bit per word and takes the word's carry out in its
// lowest bit
__device__ __forceinline__ void tile_add_row(unsigned& m, unsigned a, unsigned q0, unsigned q1, unsigned q2) {
    asm volatile("{\n\t.reg .u32 o, s;\n\t" CPIC_TILE_ADD("0", "%2") CPIC_TILE_ADD("4", "%3") CPIC_TILE_ADD("8", "%4") "}"
                 : "+r"(m)
                 : "r"(a), "r"(q0), "r"(q1), "r"(q2)
                 : "memory");
}

// Deposit of one particle per lane into the chunk's tile; lanes whose 3x3 stencil leaves the
// tile rows deposit straight into the padded global grid. Lanes that share a cell are summed
// first (__reduce_add_sync over each such group) and deposited by one lane of the group.
__device__ __forceinline__ void deposit_tile(const PushParams& p, const Tile& tl, int s, bool alive,
                                             const int* c, const float* t) {
    const int lane = threadIdx.x & 31;
    const int rr = c[1] - tl.r0;  // tile row of the cell
    const bool in = alive && rr >= 1 && rr + 1 < tl.R;
    const bool out = alive && !in;
    if (__any_sync(FULL, out)) deposit_warp<2>(p, s, out, c, t);
    if (!__any_sync(FULL, in)) return;
    unsigned q[9];
    node_weights<2>(t, q);
    // lanes that do not deposit here get keys of their own; every group of lanes that share a
    // cell is summed over its lanes and deposited by its lowest lane
    const int off = in ? rr * tl.W + c[0] + 1 : -1 - lane;
    const unsigned peers = __match_any_sync(FULL, off);
    const int my_leader = __ffs(peers) - 1;
    const bool issue = in && lane == my_leader;
    for (unsigned g = __ballot_sync(FULL, issue && (peers & (peers - 1u)) != 0u); g; g &= g - 1u) {
        if (my_leader == __ffs(g) - 1) {
#pragma unroll
            for (int node = 0; node < 9; ++node) q[node] = __reduce_add_sync(peers, q[node]);
        }
    }
    if (issue) {
        const unsigned mid = tl.lo + 4u * (unsigned)(off - 1), dw = 4u * (unsigned)tl.W;
        unsigned m = 0;  // carry out of node k's low word in bit 8 - k
        tile_add_row(m, mid - dw, q[0], q[1], q[2]);
        tile_add_row(m, mid, q[3], q[4], q[5]);
        tile_add_row(m, mid + dw, q[6], q[7], q[8]);
        if (m) {  // rare: carries into the high words
            unsigned* hi = tl.hi_ptr + (off - 1);
#pragma unroll
            for (int node = 0; node < 9; ++node)
                if ((m >> (8 - node)) & 1u) atomicAdd(hi + (node % 3) + (node / 3 - 1) * tl.W, 1u);
        }
    }
}

// the six state words of one particle, stored when p holds (predicated, no branch)
__device__ __forceinline__ void store_state(bool p, int* c, int cv, float* a, float av, float* b, float bv, float* d,
                                            float dv, float* e, float ev, float* f, float fv) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
        "@q st.global.b32 [%1], %2;\n\t@q st.global.f32 [%3], %4;\n\t@q st.global.f32 [%5], %6;\n\t"
        "@q st.global.f32 [%7], %8;\n\t@q st.global.f32 [%9], %10;\n\t@q st.global.f32 [%11], %12;\n\t}" ::"r"(
            (unsigned)p),
        "l"(c), "r"(cv), "l"(a), "f"(av), "l"(b), "f"(bv), "l"(d), "f"(dv), "l"(e), "f"(ev), "l"(f), "f"(fv)
        : "memory");
}

// One run's particle step on a virtual grid of nb blocks of which this block is bid: the
// body of the single-run kernel and of the batched kernel (a run's blocks are a slice of
// the batched launch).
template <bool PER0, bool PER1>
__device__ __forceinline__ void push2d_run(const PushParams& p, int bid, int nb, unsigned* tile_lo, unsigned* tile_hi,
                                           int* red_min, int* red_max) {
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
    // chunk size: a multiple of the block, about one chunk per block unless set
    const int C = p.chunk > 0 ? p.chunk
                              : ((total + nb - 1) / nb + P2_THREADS - 1) / P2_THREADS * P2_THREADS;
    const int n0 = p.n[0], n1 = p.n[1], nv0 = n0 + 1;
    const float4* __restrict__ K4 = reinterpret_cast<const float4*>(p.K);
    const float2* __restrict__ G2 = reinterpret_cast<const float2*>(p.G);
    const long long T = p.pb.total;
    const float hdt = p.hdt, dt = p.dt;

    for (int ch = bid;; ch += nb) {
        // species and range of chunk ch (block-uniform)
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
        const int* cellp = p.pb.cell[cur] + b0;  // read (through cellq's indices when perm)
        const float* tp = p.pb.t[cur] + b0;
        const float* vp = p.pb.v[cur] + b0;
        int* cellq = p.pb.cell[dst] + b0;  // written
        float* tq = p.pb.t[dst] + b0;
        float* vq = p.pb.v[dst] + b0;
        const float dtqm = p.dtqm[s];

        // tile rows: the rows of the chunk's particles (sampled; the chunk is in cell order
        // since the last sort) with two rows of margin for motion and the stencil
        Tile tl;
        tl.lo = (unsigned)__cvta_generic_to_shared(tile_lo);
        tl.hi_ptr = tile_hi;
        tl.W = n0 + 2;
        {
            const int si = lo + (int)(((long long)(hi - lo - 1) * threadIdx.x) / (P2_THREADS - 1));
            const int sc = cellp[perm ? cellq[si] : si];
            int rmin = sc >= 0 ? (sc >> 16) : 0x7fffffff, rmax = sc >= 0 ? (sc >> 16) : -1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rmin = min(rmin, __shfl_xor_sync(FULL, rmin, o));
                rmax = max(rmax, __shfl_xor_sync(FULL, rmax, o));
            }
            __syncthreads();  // the previous chunk's flush is done with the tile
            if ((threadIdx.x & 31) == 0) {
                red_min[threadIdx.x >> 5] = rmin;
                red_max[threadIdx.x >> 5] = rmax;
            }
            __syncthreads();
            rmin = red_min[0];
            rmax = red_max[0];
#pragma unroll
            for (int k = 1; k < P2_THREADS / 32; ++k) {
                rmin = min(rmin, red_min[k]);
                rmax = max(rmax, red_max[k]);
            }
            tl.r0 = rmin - 2;
            tl.R = rmax - rmin + 5;
            tl.on = p.tile && rmax >= rmin && tl.R * tl.W <= TILE_CELLS;
            if (tl.on)
                for (int k = threadIdx.x; k < tl.R * tl.W; k += P2_THREADS) tile_lo[k] = tile_hi[k] = 0u;
            __syncthreads();
        }

        long long ke = 0;
        int g0 = 0, g1 = 0, g2 = 0, g3 = 0, gbad = 0;

        int i = lo + (int)threadIdx.x;
        int ncw = -1;
        float nt0 = 0.f, nt1 = 0.f, nv0_ = 0.f, nv1_ = 0.f, nv2_ = 0.f;
        if (i < hi) {
            const int j = perm ? cellq[i] : i;
            ncw = cellp[j];
            nt0 = tp[j];
            nt1 = tp[T + j];
            nv0_ = vp[j];
            nv1_ = vp[T + j];
            nv2_ = vp[2 * T + j];
        }
        // the iteration loop, specialised on whether the chunk's tile is in use
        auto iterate = [&](auto tile_tag) {
            constexpr bool TILE = decltype(tile_tag)::value;
            for (int base = lo; base < hi; base += P2_THREADS) {
                const int slot = i;
                const int cw = ncw;
                float t[2] = {nt0, nt1};
                float v[3] = {nv0_, nv1_, nv2_};
                i += P2_THREADS;
                ncw = -1;
                if (i < hi) {
                    const int j = perm ? cellq[i] : i;
                    ncw = cellp[j];
                    nt0 = tp[j];
                    nt1 = tp[T + j];
                    nv0_ = vp[j];
                    nv1_ = vp[T + j];
                    nv2_ = vp[2 * T + j];
                }
                const bool active = cw >= 0;
                int c[2] = {active ? (cw & 0xFFFF) : 0, active ? (cw >> 16) : 0};
                if (!active) t[0] = t[1] = v[0] = v[1] = v[2] = 0.0f;

                // a2: b1 gather of k and G at xi^n (pairs of components in packed FP32x2
                // arithmetic: each lane rounds exactly as the scalar form)
                float2 k01, k23, gp;
                {
                    const int v00 = c[0] + c[1] * nv0;
                    const float s0 = __fsub_rn(1.0f, t[0]), s1 = __fsub_rn(1.0f, t[1]);
                    const float2 wa = __fmul2_rn(make_float2(s0, t[0]), make_float2(s1, s1));
                    const float2 wb = __fmul2_rn(make_float2(s0, t[0]), make_float2(t[1], t[1]));
                    const float2 W0 = make_float2(wa.x, wa.x), W1 = make_float2(wa.y, wa.y);
                    const float2 W2 = make_float2(wb.x, wb.x), W3 = make_float2(wb.y, wb.y);
                    const float4 a = __ldg(K4 + v00), b = __ldg(K4 + v00 + 1);
                    const float4 cc = __ldg(K4 + v00 + nv0), d = __ldg(K4 + v00 + nv0 + 1);
                    const float2 ga = __ldg(G2 + v00), gb = __ldg(G2 + v00 + 1);
                    const float2 gc = __ldg(G2 + v00 + nv0), gd = __ldg(G2 + v00 + nv0 + 1);
                    k01 = __fmul2_rn(W0, make_float2(a.x, a.y));
                    k23 = __fmul2_rn(W0, make_float2(a.z, a.w));
                    gp = __fmul2_rn(W0, ga);
                    k01 = __ffma2_rn(W1, make_float2(b.x, b.y), k01);
                    k23 = __ffma2_rn(W1, make_float2(b.z, b.w), k23);
                    gp = __ffma2_rn(W1, gb, gp);
                    k01 = __ffma2_rn(W2, make_float2(cc.x, cc.y), k01);
                    k23 = __ffma2_rn(W2, make_float2(cc.z, cc.w), k23);
                    gp = __ffma2_rn(W2, gc, gp);
                    k01 = __ffma2_rn(W3, make_float2(d.x, d.y), k01);
                    k23 = __ffma2_rn(W3, make_float2(d.z, d.w), k23);
                    gp = __ffma2_rn(W3, gd, gp);
                }
                const float kp[4] = {k01.x, k01.y, k23.x, k23.y};
                // a3: E^al = -sum_a G^a k^{a al}, kick
                const float vo0 = v[0], vo1 = v[1], vo2 = v[2];
                {
                    float2 e = __fmul2_rn(k01, make_float2(gp.x, gp.x));
                    e = __ffma2_rn(k23, make_float2(gp.y, gp.y), e);
                    const float2 vv = __ffma2_rn(make_float2(-dtqm, -dtqm), e, make_float2(v[0], v[1]));
                    v[0] = vv.x;
                    v[1] = vv.y;
                }
                // a4: predictor (a non-finite component keeps the particle where it is)
                int cpred[2];
                float tpred[2];
    #pragma unroll
                for (int a = 0; a < 2; ++a) {
                    float d = __fmul_rn(kp[2 * a], v[0]);
                    d = __fmaf_rn(kp[2 * a + 1], v[1], d);
                    float x = __fmaf_rn(hdt, d, t[a]);
                    if (!isfinite(x)) x = t[a];
                    if (a == 0)
                        predict_axis<PER0>(x, c[0], n0, cpred[0], tpred[0]);
                    else
                        predict_axis<PER1>(x, c[1], n1, cpred[1], tpred[1]);
                }
                // k re-gathered at xi'
                float kq[4];
                {
                    const int v00 = cpred[0] + cpred[1] * nv0;
                    const float s0 = __fsub_rn(1.0f, tpred[0]), s1 = __fsub_rn(1.0f, tpred[1]);
                    const float2 wa = __fmul2_rn(make_float2(s0, tpred[0]), make_float2(s1, s1));
                    const float2 wb = __fmul2_rn(make_float2(s0, tpred[0]), make_float2(tpred[1], tpred[1]));
                    const float4 a = __ldg(K4 + v00), b = __ldg(K4 + v00 + 1);
                    const float4 cc = __ldg(K4 + v00 + nv0), d = __ldg(K4 + v00 + nv0 + 1);
                    float2 q01 = __fmul2_rn(make_float2(wa.x, wa.x), make_float2(a.x, a.y));
                    float2 q23 = __fmul2_rn(make_float2(wa.x, wa.x), make_float2(a.z, a.w));
                    q01 = __ffma2_rn(make_float2(wa.y, wa.y), make_float2(b.x, b.y), q01);
                    q23 = __ffma2_rn(make_float2(wa.y, wa.y), make_float2(b.z, b.w), q23);
                    q01 = __ffma2_rn(make_float2(wb.x, wb.x), make_float2(cc.x, cc.y), q01);
                    q23 = __ffma2_rn(make_float2(wb.x, wb.x), make_float2(cc.z, cc.w), q23);
                    q01 = __ffma2_rn(make_float2(wb.y, wb.y), make_float2(d.x, d.y), q01);
                    q23 = __ffma2_rn(make_float2(wb.y, wb.y), make_float2(d.z, d.w), q23);
                    kq[0] = q01.x;
                    kq[1] = q01.y;
                    kq[2] = q23.x;
                    kq[3] = q23.y;
                }
                // corrector
                bool bad = false;
                int cn[2];
                float tn[2];
    #pragma unroll
                for (int a = 0; a < 2; ++a) {
                    float d = __fmul_rn(kq[2 * a], v[0]);
                    d = __fmaf_rn(kq[2 * a + 1], v[1], d);
                    float x = __fmaf_rn(dt, d, t[a]);
                    if (!isfinite(x)) {
                        bad = true;
                        x = t[a];
                    }
                    int dc;
                    renorm(x, tn[a], dc);
                    cn[a] = c[a] + dc;
                }
                // a5: boundaries
                int face = -1;
                if (PER0) {
                    cn[0] = wrapi(cn[0], n0);
                } else {
                    if (cn[0] < 0) face = 0;
                    else if (cn[0] >= n0) face = 1;
                }
                if (PER1) {
                    cn[1] = wrapi(cn[1], n1);
                } else if (face < 0) {
                    if (cn[1] < 0) face = 2;
                    else if (cn[1] >= n1) face = 3;
                }
                if (bad) face = 6;
                const bool alive = active && face < 0;
                if (__any_sync(FULL, active && face >= 0)) {
                    g0 += active && face == 0;
                    g1 += active && face == 1;
                    g2 += active && face == 2;
                    g3 += active && face == 3;
                    gbad += active && face == 6;
                    if (active) collect_face<2>(p, s, face, cn);
                }
                // spec D: v_old . v_new as an FP32 fma chain, then round(x 2^24) to int64
                const float ke32 = __fmaf_rn(vo2, v[2], __fmaf_rn(vo1, v[1], __fmul_rn(vo0, v[0])));
                if (active) ke += __float2ll_rn(__fmul_rn(ke32, 16777216.0f));
                if (p.hist) {  // the next sort's histogram: one atomic per run of equal cells
                    const int key = alive ? cn[0] + n0 * cn[1] : -1;
                    const unsigned peers = __match_any_sync(FULL, key);
                    if (key >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
                        atomicAdd(p.hist + (size_t)s * n0 * n1 + key, (int)__popc(peers));
                }
                store_state(active, cellq + slot, alive ? (cn[0] | (cn[1] << 16)) : -1, tq + slot, tn[0],
                            tq + T + slot, tn[1], vq + slot, v[0], vq + T + slot, v[1], vq + 2 * T + slot, v[2]);
                // a6: deposit
                if constexpr (TILE)
                    deposit_tile(p, tl, s, alive, cn, tn);
                else
                    deposit_warp<2>(p, s, alive, cn, tn);
            }
        };
        if (tl.on)
            iterate(std::true_type{});
        else
            iterate(std::false_type{});
        // flush the tile into the padded grid (rows -1 .. n1 exist there; the others hold
        // nothing)
        if (tl.on) {
            __syncthreads();
            unsigned long long* g = p.charge + (long long)s * p.ncell_h;
            for (int k = threadIdx.x; k < tl.R * tl.W; k += P2_THREADS) {
                const unsigned long long v = ((unsigned long long)tile_hi[k] << 32) | tile_lo[k];
                if (!v) continue;
                const int row = tl.r0 + k / tl.W;
                if (row < -1 || row > n1) continue;
                atomicAdd(g + (long long)(row + 1) * tl.W + k % tl.W, v);
            }
        }
        // tallies of this chunk
        ke = warp_sum_ll(ke);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g0 += __shfl_xor_sync(FULL, g0, o);
            g1 += __shfl_xor_sync(FULL, g1, o);
            g2 += __shfl_xor_sync(FULL, g2, o);
            g3 += __shfl_xor_sync(FULL, g3, o);
            gbad += __shfl_xor_sync(FULL, gbad, o);
        }
        if ((threadIdx.x & 31) == 0) {
            DevCounters* cw = p.ctr;
            if (ke) atomicAdd((unsigned long long*)&cw->ke_fp[s], (unsigned long long)ke);
            const int gf[4] = {g0, g1, g2, g3};
#pragma unroll
            for (int f = 0; f < 4; ++f)
                if (gf[f]) atomicAdd((unsigned long long*)&cw->absorbed[s][f], (unsigned long long)gf[f]);
            if (gbad) atomicAdd((unsigned long long*)&cw->nonfinite, (unsigned long long)gbad);
            const long long removed = (long long)g0 + g1 + g2 + g3 + gbad;
            if (removed) atomicAdd((unsigned long long*)&cw->alive[s], (unsigned long long)(-removed));
        }
    }
}

template <bool PER0, bool PER1>
__global__ void __launch_bounds__(P2_THREADS, 4) push2d_kernel(PushParams p) {
    __shared__ unsigned tile_lo[TILE_CELLS], tile_hi[TILE_CELLS];
    __shared__ int red_min[P2_THREADS / 32], red_max[P2_THREADS / 32];
    push2d_run<PER0, PER1>(p, (int)blockIdx.x, (int)gridDim.x, tile_lo, tile_hi, red_min, red_max);
}

// Row a11: the particle step of many runs in one persistent launch. Run r owns virtual
// blocks [vbase[r], vbase[r + 1]) (in proportion to its particle capacity); the resident
// blocks walk the virtual blocks of all runs, each taking its run's parameters from the
// device table, so runs of uneven size share one wave of the GPU.
template <bool PER0, bool PER1>
__global__ void __launch_bounds__(P2_THREADS, 4) push2d_batch_kernel(const PushParams* __restrict__ runs,
                                                                      const int* __restrict__ vbase, int nruns) {
    __shared__ unsigned tile_lo[TILE_CELLS], tile_hi[TILE_CELLS];
    __shared__ int red_min[P2_THREADS / 32], red_max[P2_THREADS / 32];
    const int total = vbase[nruns];
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int a = 0, b = nruns;  // the run of virtual block vb: vbase[a] <= vb < vbase[a + 1]
        while (b - a > 1) {
            const int m = (a + b) >> 1;
            if (vbase[m] <= vb) a = m;
            else b = m;
        }
        push2d_run<PER0, PER1>(runs[a], vb - vbase[a], vbase[a + 1] - vbase[a], tile_lo, tile_hi, red_min, red_max);
        __syncthreads();  // the next virtual block reuses the tile
    }
}

template <bool PER0, bool PER1>
int launch_push2d_t(cpic_run* r, const PushParams& p) {
    static std::atomic<int> per_sm[64];  // resident blocks per SM, per device
    int dev = 0;
    CPIC_CUDA(cudaGetDevice(&dev));
    std::atomic<int>& cache = per_sm[dev & 63];
    int b = cache.load(std::memory_order_acquire);
    if (b <= 0) {
        CPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, push2d_kernel<PER0, PER1>, P2_THREADS, 0));
        if (b < 1) b = 1;
        cache.store(b, std::memory_order_release);
    }
    const long long occ = (long long)b * device_sm_count();  // one wave
    long long tot = 0;
    for (int s = 0; s < r->cfg.n_species; ++s) tot += r->pb.capacity[s];
    long long blocks = (tot + P2_THREADS - 1) / P2_THREADS;
    if (blocks > occ) blocks = occ;
    if (blocks < 1) blocks = 1;
    push2d_kernel<PER0, PER1><<<(int)blocks, P2_THREADS, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace

int push2d_batch_blocks() {
    static std::atomic<int> per_sm[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return device_sm_count();
    std::atomic<int>& cache = per_sm[dev & 63];
    int b = cache.load(std::memory_order_acquire);
    if (b <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, push2d_batch_kernel<false, true>, P2_THREADS, 0) !=
            cudaSuccess)
            b = 1;
        if (b < 1) b = 1;
        cache.store(b, std::memory_order_release);
    }
    return b * device_sm_count();
}

int launch_push2d_batch(const PushParams* runs, const int* vbase, int nruns, int per0, int per1, int blocks,
                        cudaStream_t stream) {
    if (per0 && per1) push2d_batch_kernel<true, true><<<blocks, P2_THREADS, 0, stream>>>(runs, vbase, nruns);
    else if (per0) push2d_batch_kernel<true, false><<<blocks, P2_THREADS, 0, stream>>>(runs, vbase, nruns);
    else if (per1) push2d_batch_kernel<false, true><<<blocks, P2_THREADS, 0, stream>>>(runs, vbase, nruns);
    else push2d_batch_kernel<false, false><<<blocks, P2_THREADS, 0, stream>>>(runs, vbase, nruns);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_push2d(cpic_run* r, const PushParams& p) {
    const bool per0 = p.pbc[0] == CPIC_PBC_PERIODIC, per1 = p.pbc[2] == CPIC_PBC_PERIODIC;
    if (p.pbc[0] == CPIC_PBC_REFLECT || p.pbc[2] == CPIC_PBC_REFLECT) return CPIC_ERR_NOT_BUILT;
    if (per0) return per1 ? launch_push2d_t<true, true>(r, p) : launch_push2d_t<true, false>(r, p);
    return per1 ? launch_push2d_t<false, true>(r, p) : launch_push2d_t<false, false>(r, p);
}

}  // namespace cpic
