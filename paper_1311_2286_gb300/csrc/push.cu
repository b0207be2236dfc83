// Rows a2-a6: the fused hybrid-mover kernel (Sec. II.B.4) with its grid coupling.
//
// Per particle (one thread, structure-of-arrays, coalesced):
//   a2  b1 gather of the logical field G and of k at xi^n (Sec. II.B.2, eqs. (vvp), (Wvp),
//       (b1)) - both vertex tables are read through the read-only path;
//   a3  E^alpha = -sum_a G^a k^{a alpha}, v^{n+1/2} = v^{n-1/2} + dt (q/m) E (eq. (step1);
//       unmagnetised, so the Boris rotation is the identity);
//   a4  predictor xi' = xi^n + dt/2 k(xi^n) v (eq. (step2)), k re-gathered at xi'
//       (eq. (step3)), corrector xi^{n+1} = xi^n + dt k(xi') v (eq. (step4)), on the split
//       (cell, offset) representation in cell units;
//   a5  boundaries: periodic wrap; absorption when a logical coordinate leaves [0, 1)
//       (Sec. II.B.4), tallied per face and species;
//   a6  b2 deposit (eqs. (pg), (Wpc), (b2)) in 64-bit fixed point: integer node weights
//       from the offset quantised to 2^-12 of a cell, 2^24 units per particle. Lanes of a
//       warp whose particles share a cell are found with __match_any_sync, their node
//       weights summed with __reduce_add_sync (each < 2^24, so a warp's sum fits 32 bits),
//       and one lane per group issues the 3^D global 64-bit reductions.
//
// The FP32 operation sequence (explicit __fmaf_rn / __fmul_rn / __fsub_rn, never
// contracted) is the one the mover is specified with: s = 1 - t; corner weights multiplied
// from axis 0 upwards; gathers as a fused multiply-add chain over corners in the order
// 0 .. 2^D - 1 (bit a = +1 along axis a); renormalisation c = floor(x), f = x - c, f == 1
// -> (0, c + 1); the predictor point is clamped on non-periodic axes.
#include <atomic>
#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

// Per-warp tallies of the current species (the species is warp-uniform, so the flush is
// taken by whole warps): kinetic-energy products (per lane), removed particles per face
// and non-finite (counted with ballots, so the counts are warp-uniform registers).
struct Tally {
    long long ke = 0;
    int gone[7] = {0, 0, 0, 0, 0, 0, 0};  // faces 0..5, 6 = non-finite
    __device__ __forceinline__ void add(int face) {
        if (__any_sync(FULL, face >= 0)) {
#pragma unroll
            for (int f = 0; f < 7; ++f) gone[f] += __popc(__ballot_sync(FULL, face == f));
        }
    }
    __device__ __forceinline__ void flush(DevCounters* ctr, int s) {
        long long k = warp_sum_ll(ke);
        bool lane0 = (threadIdx.x & 31) == 0;
        if (lane0 && k != 0) atomicAdd((unsigned long long*)&ctr->ke_fp[s], (unsigned long long)k);
        long long removed = 0;
#pragma unroll
        for (int f = 0; f < 7; ++f) {
            removed += gone[f];
            if (lane0 && gone[f]) {
                if (f < 6)
                    atomicAdd((unsigned long long*)&ctr->absorbed[s][f], (unsigned long long)gone[f]);
                else
                    atomicAdd((unsigned long long*)&ctr->nonfinite, (unsigned long long)gone[f]);
            }
            gone[f] = 0;
        }
        if (lane0 && removed) atomicAdd((unsigned long long*)&ctr->alive[s], (unsigned long long)(-removed));
        ke = 0;
    }
};

// MODE 0: full push + deposit; MODE 1: deposit only; MODE 2: gather + kick only
template <int D, int MODE>
__global__ void __launch_bounds__(256, D == 2 ? 4 : 2) particle_kernel(PushParams p, float kick_coef0, float kick_coef1,
                                                       float kick_coef2, float kick_coef3) {
    const SpeciesRanges R = species_ranges(p);
    const long long total = R.total;
    const int cur = p.ctr->cur;
    int* __restrict__ cellp = p.pb.cell[cur];
    const long long T = p.pb.total;
    // per-component base pointers: slots are 32-bit offsets from these
    float* __restrict__ tq[3] = {p.pb.t[cur], p.pb.t[cur] + T, p.pb.t[cur] + (D == 3 ? 2 * T : T)};
    float* __restrict__ vq[3] = {p.pb.v[cur], p.pb.v[cur] + T, p.pb.v[cur] + 2 * T};
    Tally tally;
    int s_acc = -1;
    // blocked distribution: each block walks one contiguous chunk of the (cell-sorted)
    // particles, so consecutive iterations gather nearby vertex records (L1 reuse)
    const int total32 = (int)total;
    const int bd = blockDim.x;
    const int chunk = ((total32 + (int)gridDim.x - 1) / (int)gridDim.x + bd - 1) / bd * bd;
    const int lo = (int)blockIdx.x * chunk;
    const int hi = lo + chunk < total32 ? lo + chunk : total32;

    // software pipelining: the particle state of the next iteration is loaded before the
    // current particle is processed, so its HBM latency overlaps the arithmetic
    struct Raw {
        int s, slot, cw;
        bool active;
        float t[3], v[3];
    };
    auto fetch = [&](int base) {
        Raw r;
        const int vi = base + (int)threadIdx.x;
        long long local;
        r.s = species_of(R, vi, local, r.active);
        r.active = r.active && base < hi;
        r.slot = (int)(p.pb.base[r.s] + local);
        r.cw = r.active ? cellp[r.slot] : -1;
#pragma unroll
        for (int a = 0; a < 3; ++a) r.t[a] = 0.0f, r.v[a] = 0.0f;
        if (r.active) {
#pragma unroll
            for (int a = 0; a < D; ++a) r.t[a] = tq[a][r.slot];
            if (MODE != 1) {
#pragma unroll
                for (int al = 0; al < 3; ++al) r.v[al] = vq[al][r.slot];
            }
        }
        return r;
    };
    Raw nxt = fetch(lo);
    for (int base = lo; base < hi; base += bd) {
        const Raw cur = nxt;
        nxt = fetch(base + bd);
        const int s = cur.s;
        if (MODE == 0 && s != s_acc) {  // warp-uniform
            if (s_acc >= 0) tally.flush(p.ctr, s_acc);
            s_acc = s;
        }
        const int slot = cur.slot;
        const int cw = cur.cw;
        bool active = cur.active && cw >= 0;
        int c[3] = {0, 0, 0};
        float t[3] = {cur.t[0], cur.t[1], cur.t[2]};
        float v[3] = {cur.v[0], cur.v[1], cur.v[2]};
        if (active) decode<D>(cw, c);
        if (MODE == 1) {
            deposit_warp<D>(p, s, active, c, t);
            continue;
        }
        float kp[9], gp[3];
        if (active) {
            Tab<D>::gather(p, vertex_of<D>(p, c), t, kp, gp);
        }
        if (MODE == 2) {
            if (active && p.magnetized && !p.gyro) {  // Boris step over the kick's fraction of dt
                float E[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    float e = __fmul_rn(kp[0 * D + al], gp[0]);
#pragma unroll
                    for (int a = 1; a < D; ++a) e = __fmaf_rn(kp[a * D + al], gp[a], e);
                    E[al] = -e;
                }
                boris_kick(v, E, p.bh[s], p.bt[s], p.bs[s]);
#pragma unroll
                for (int al = 0; al < 3; ++al) vq[al][slot] = v[al];
            } else if (active) {
                float coef = s == 0 ? kick_coef0 : s == 1 ? kick_coef1 : s == 2 ? kick_coef2 : kick_coef3;
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    float e = __fmul_rn(kp[0 * D + al], gp[0]);
#pragma unroll
                    for (int a = 1; a < D; ++a) e = __fmaf_rn(kp[a * D + al], gp[a], e);
                    e = -e;
                    vq[al][slot] = __fmaf_rn(coef, e, v[al]);
                }
            }
            continue;
        }
        // ---- MODE 0: full push
        bool alive = active;
        int face = -1;
        int cn[3] = {0, 0, 0};
        float tn[3] = {0.f, 0.f, 0.f};
        if (active) {
            const float vo0 = v[0], vo1 = v[1], vo2 = v[2];
            const float dtqm = p.dtqm[s];
            if (p.magnetized && !p.gyro) {  // warp-uniform
                float E[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    float e = __fmul_rn(kp[0 * D + al], gp[0]);
#pragma unroll
                    for (int a = 1; a < D; ++a) e = __fmaf_rn(kp[a * D + al], gp[a], e);
                    E[al] = -e;
                }
                boris_kick(v, E, p.bh[s], p.bt[s], p.bs[s]);
            } else {
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    float e = __fmul_rn(kp[0 * D + al], gp[0]);
#pragma unroll
                    for (int a = 1; a < D; ++a) e = __fmaf_rn(kp[a * D + al], gp[a], e);
                    e = -e;
                    v[al] = __fmaf_rn(dtqm, e, v[al]);
                }
            }
            // axisymmetric run (2D, Omega = r): the particle moves on a straight line in 3D
            // over the step, x = r + dt v_r, y = dt v_theta, r' = |(x, y)|; the meridional
            // displacement is (r' - r, dt v_z) and (v_r, v_theta) turns with the frame by the
            // azimuth of (x, y), keeping r v_theta (the inertial forces of the cylindrical
            // frame); the kinetic-energy tally takes the velocity before the turn
            const bool axi = D == 2 && p.R != nullptr;  // warp-uniform
            const bool dform = axi || p.gyro;           // the position moves by disp
            float disp[3] = {0.0f, 0.0f, 0.0f}, vrot[3] = {v[0], v[1], v[2]};
            if (p.gyro) {
                // cyclotronic integrator: after the plain kick, the exact motion in the
                // uniform field alone over dt, b = B0 / |B0| (velocity components' basis),
                // th = (q/m) |B0| dt: u = v x b, par = (v . b) b, perp = v - par,
                // v' = par + cos th perp + sin th u, d = dt (par + f1 perp + f2 u) with
                // f1 = sin th / th, f2 = (1 - cos th) / th
                const float* b = p.gb;
                const float cs = p.gy[s][0], sn = p.gy[s][1], f1 = p.gy[s][2], f2 = p.gy[s][3];
                const float vpar = __fmaf_rn(v[2], b[2], __fmaf_rn(v[1], b[1], __fmul_rn(v[0], b[0])));
                const float u[3] = {__fmaf_rn(v[1], b[2], -__fmul_rn(v[2], b[1])),
                                    __fmaf_rn(v[2], b[0], -__fmul_rn(v[0], b[2])),
                                    __fmaf_rn(v[0], b[1], -__fmul_rn(v[1], b[0]))};
                float d3[3];
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const float par = __fmul_rn(vpar, b[al]);
                    const float perp = __fsub_rn(v[al], par);
                    vrot[al] = __fmaf_rn(sn, u[al], __fmaf_rn(cs, perp, par));
                    d3[al] = __fmul_rn(p.dt, __fmaf_rn(f2, u[al], __fmaf_rn(f1, perp, par)));
                }
                if (axi) {  // the displacement starts at the particle's point in 3D
                    const float rn = gather_scalar2(p, vertex_of<D>(p, c), t);
                    const float x = __fadd_rn(rn, d3[0]);
                    const float y = d3[2];
                    const float r1 = __fsqrt_rn(__fmaf_rn(x, x, __fmul_rn(y, y)));
                    float ca = 1.0f, sa = 0.0f;
                    if (r1 > 0.0f) {
                        ca = __fdiv_rn(x, r1);
                        sa = __fdiv_rn(y, r1);
                    }
                    disp[0] = __fsub_rn(r1, rn);
                    disp[1] = d3[1];
                    const float w0 = vrot[0], w2 = vrot[2];
                    vrot[0] = __fmaf_rn(ca, w0, __fmul_rn(sa, w2));
                    vrot[2] = __fmaf_rn(ca, w2, -__fmul_rn(sa, w0));
                } else {
#pragma unroll
                    for (int a = 0; a < D; ++a) disp[a] = d3[a];
                }
            } else if (axi) {
                const float rn = gather_scalar2(p, vertex_of<D>(p, c), t);
                const float x = __fmaf_rn(p.dt, v[0], rn);
                const float y = __fmul_rn(p.dt, v[2]);
                const float r1 = __fsqrt_rn(__fmaf_rn(x, x, __fmul_rn(y, y)));
                float ca = 1.0f, sa = 0.0f;
                if (r1 > 0.0f) {
                    ca = __fdiv_rn(x, r1);
                    sa = __fdiv_rn(y, r1);
                }
                disp[0] = __fsub_rn(r1, rn);
                disp[1] = __fmul_rn(p.dt, v[1]);
                vrot[0] = __fmaf_rn(ca, v[0], __fmul_rn(sa, v[2]));
                vrot[2] = __fmaf_rn(ca, v[2], -__fmul_rn(sa, v[0]));
            }
            // predictor
            int cpred[3];
            float tpred[3];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                float x;
                if (dform) {
                    float d = __fmul_rn(kp[a * D + 0], disp[0]);
#pragma unroll
                    for (int b = 1; b < D; ++b) d = __fmaf_rn(kp[a * D + b], disp[b], d);
                    x = __fmaf_rn(0.5f, d, t[a]);
                } else {
                    float d = __fmul_rn(kp[a * D + 0], v[0]);
#pragma unroll
                    for (int al = 1; al < D; ++al) d = __fmaf_rn(kp[a * D + al], v[al], d);
                    x = __fmaf_rn(p.hdt, d, t[a]);
                }
                if (!isfinite(x)) {
                    cpred[a] = c[a];
                    tpred[a] = t[a];
                    continue;
                }
                int dc;
                renorm(x, tpred[a], dc);
                int ci = c[a] + dc;
                if (p.pbc[2 * a] == CPIC_PBC_PERIODIC) {
                    ci = wrapi(ci, p.n[a]);
                } else if (ci < 0) {
                    ci = 0;
                    tpred[a] = 0.0f;
                } else if (ci >= p.n[a]) {
                    ci = p.n[a] - 1;
                    tpred[a] = 1.0f;
                }
                cpred[a] = ci;
            }
            float kq[9];
            Tab<D>::gather(p, vertex_of<D>(p, cpred), tpred, kq, nullptr);
            // corrector
            bool bad = false;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                float x;
                if (dform) {
                    float d = __fmul_rn(kq[a * D + 0], disp[0]);
#pragma unroll
                    for (int b = 1; b < D; ++b) d = __fmaf_rn(kq[a * D + b], disp[b], d);
                    x = __fadd_rn(t[a], d);
                } else {
                    float d = __fmul_rn(kq[a * D + 0], v[0]);
#pragma unroll
                    for (int al = 1; al < D; ++al) d = __fmaf_rn(kq[a * D + al], v[al], d);
                    x = __fmaf_rn(p.dt, d, t[a]);
                }
                if (!isfinite(x)) {
                    bad = true;
                    cn[a] = c[a];
                    tn[a] = t[a];
                    continue;
                }
                int dc;
                renorm(x, tn[a], dc);
                cn[a] = c[a] + dc;
            }
            if (bad) {
                face = 6;
            } else {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    if (p.pbc[2 * a] == CPIC_PBC_PERIODIC) {
                        cn[a] = wrapi(cn[a], p.n[a]);
                    } else if (p.pbc[2 * a] == CPIC_PBC_REFLECT) {
                        continue;  // mirrored below, after the kinetic-energy tally
                    } else if (cn[a] < 0) {
                        if (face < 0) face = 2 * a;
                    } else if (cn[a] >= p.n[a]) {
                        if (face < 0) face = 2 * a + 1;
                    }
                }
            }
            // spec D: v_old . v_new as an FP32 fma chain, then round(x 2^24) to int64 (FP64
            // throughput on this part is ~1/64 of FP32, so the product stays in FP32)
            float ke32 = __fmaf_rn(vo2, v[2], __fmaf_rn(vo1, v[1], __fmul_rn(vo0, v[0])));
            tally.ke += __float2ll_rn(__fmul_rn(ke32, 16777216.0f));
            if (dform) {
#pragma unroll
                for (int al = 0; al < 3; ++al) v[al] = vrot[al];
            }
            // spec B: a reflecting face mirrors the position in logical space (u -> -u below,
            // u -> 2N - u above) and reflects v about row a of k(xi'); still outside after one
            // mirror: removed at that face
            if (face < 0) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    if (face >= 0 || p.pbc[2 * a] != CPIC_PBC_REFLECT || (cn[a] >= 0 && cn[a] < p.n[a])) continue;
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
                    float nn = __fmul_rn(kq[a * D], kq[a * D]);
                    float dot = __fmul_rn(v[0], kq[a * D]);
#pragma unroll
                    for (int al = 1; al < D; ++al) {
                        nn = __fmaf_rn(kq[a * D + al], kq[a * D + al], nn);
                        dot = __fmaf_rn(v[al], kq[a * D + al], dot);
                    }
                    const float sf = __fdiv_rn(__fmul_rn(2.0f, dot), nn);
#pragma unroll
                    for (int al = 0; al < D; ++al) v[al] = __fmaf_rn(-sf, kq[a * D + al], v[al]);
                }
            }
            alive = face < 0;
            // store
            cellp[slot] = alive ? encode<D>(cn) : -1;
#pragma unroll
            for (int a = 0; a < D; ++a) tq[a][slot] = tn[a];
#pragma unroll
            for (int al = 0; al < 3; ++al) vq[al][slot] = v[al];
        }
        tally.add(face);
        if (active && face >= 0) collect_face<D>(p, s, face, cn);
        deposit_warp<D>(p, s, alive, cn, tn);
    }
    if (MODE == 0 && s_acc >= 0) tally.flush(p.ctr, s_acc);
}

// Folds the padded deposit grid into the cell grid the field solve reads: every cell takes
// its own padded entry plus, on each axis where it is an edge cell, the halo entry that maps
// onto it (periodic axes wrap: halo -1 -> n-1, halo n -> 0; other axes fold the halo onto
// the adjacent boundary cell, so charge deposited outside is kept). Gather form: each cell
// is written by one thread, no atomics.
struct FoldParams {
    int D, n[3], per[3], hs1, hs2, nsp;
    long long ncell, ncell_h;
    const unsigned long long* src;
    unsigned long long* dst;
};

__global__ void fold_kernel(FoldParams f) {
    const long long total = f.ncell * f.nsp;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(x / f.ncell);
        const long long c = x - (long long)s * f.ncell;
        int ci[3] = {(int)(c % f.n[0]), (int)((c / f.n[0]) % f.n[1]), (int)(c / ((long long)f.n[0] * f.n[1]))};
        // padded source coordinates per axis: the cell itself and at most one halo
        int src[3][2], ns[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            src[a][0] = ci[a] + 1;
            ns[a] = 1;
            if (a < f.D) {
                const int n = f.n[a];
                const int lo = f.per[a] ? n - 1 : 0;   // cell receiving halo -1
                const int hi = f.per[a] ? 0 : n - 1;   // cell receiving halo n
                if (ci[a] == lo) src[a][ns[a]++] = 0;
                if (ci[a] == hi) src[a][ns[a]++] = n + 1;
            }
        }
        const unsigned long long* g = f.src + (long long)s * f.ncell_h;
        unsigned long long acc = 0;
        for (int k = 0; k < (f.D == 3 ? ns[2] : 1); ++k)
            for (int j = 0; j < ns[1]; ++j)
                for (int i = 0; i < ns[0]; ++i) {
                    long long idx = src[0][i] + (long long)src[1][j] * f.hs1;
                    if (f.D == 3) idx += (long long)src[2][k] * f.hs2;
                    acc += g[idx];
                }
        f.dst[x] = acc;
    }
}

// step count; a push that read through a pending sort order wrote the other buffer: flip
__global__ void finalize_step_kernel(DevCounters* ctr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctr->step += 1;
        if (ctr->perm) {
            ctr->cur = 1 - ctr->cur;
            ctr->perm = 0;
        }
    }
}

}  // namespace

PushParams make_push_params(cpic_run* r) {
    PushParams p;
    p.D = r->D;
    for (int a = 0; a < 3; ++a) p.n[a] = a < r->D ? r->n[a] : 1;
    for (int f = 0; f < 6; ++f) p.pbc[f] = r->cfg.particle_bc[f];
    p.nsp = r->cfg.n_species;
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s)
        p.dtqm[s] = s < p.nsp ? (float)(r->cfg.dt * r->cfg.q[s] / r->cfg.m[s]) : 0.0f;
    p.hdt = (float)(0.5 * r->cfg.dt);
    p.dt = (float)r->cfg.dt;
    p.K = r->K32;
    p.G = r->G32;
    p.collect = r->collect;
    p.ncollect = r->ncollect;
    p.R = r->D == 2 ? r->R32 : nullptr;
    p.pb = r->pb;
    p.charge = r->charge_h;
    p.ncell_h = r->ncell_h;
    p.hs1 = r->n[0] + 2;
    p.hs2 = r->D == 3 ? (r->n[0] + 2) * (r->n[1] + 2) : 0;
    p.origin = 1 + p.hs1 + p.hs2;
    p.ctr = r->ctr;
    p.chunk = r->push_chunk;
    p.hist = r->count_hist ? r->hist : nullptr;
    p.tile = r->push_tile;
    set_boris_constants(r, &p, 1.0);
    return p;
}

// Boris constants of the species for a kick over `fraction` of dt (1: the push; -1/2: the
// start-up half step backwards), computed in FP64 and rounded once
void set_boris_constants(const cpic_run* r, PushParams* p, double fraction) {
    p->magnetized = r->magnetized;
    // the field in the velocity components' basis: an axisymmetric run's (v_r, v_z,
    // v_theta) is left-handed, so the component cross product with -B0 is the physical v x B0
    double Bc[3];
    for (int a = 0; a < 3; ++a) Bc[a] = r->cfg.axisymmetric ? -r->B0[a] : r->B0[a];
    // cyclotronic integrator: b = Bc / |Bc| and per species cos th, sin th, sin th / th,
    // (1 - cos th) / th with th = (q/m) |B0| dt (FP64, rounded once)
    p->gyro = r->magnetized && r->gyro_kind == CPIC_GYRO_CYCLOTRONIC;
    const double bm = sqrt(Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2]);
    for (int a = 0; a < 3; ++a) p->gb[a] = bm > 0.0 ? (float)(Bc[a] / bm) : 0.0f;
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        double g4[4] = {1.0, 0.0, 1.0, 0.0};
        if (s < r->cfg.n_species) {
            const double th = r->cfg.q[s] / r->cfg.m[s] * bm * r->cfg.dt;
            if (th != 0.0) {
                const double sh = sin(0.5 * th);
                g4[0] = cos(th);
                g4[1] = sin(th);
                g4[2] = sin(th) / th;
                g4[3] = 2.0 * sh * sh / th;
            }
        }
        for (int k = 0; k < 4; ++k) p->gy[s][k] = (float)g4[k];
    }
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        double h = 0.0, t[3] = {0.0, 0.0, 0.0};
        if (s < r->cfg.n_species) {
            h = 0.5 * fraction * r->cfg.dt * r->cfg.q[s] / r->cfg.m[s];
            for (int a = 0; a < 3; ++a) t[a] = h * Bc[a];
        }
        const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        p->bh[s] = (float)h;
        for (int a = 0; a < 3; ++a) {
            p->bt[s][a] = (float)t[a];
            p->bs[s][a] = (float)(2.0 * t[a] / (1.0 + tt));
        }
    }
}

// one wave of resident blocks over all SMs (the kernel walks its chunk in a loop)
template <int D, int MODE>
static int particle_grid(cpic_run* r) {
    static std::atomic<int> per_sm[64];  // resident blocks per SM, per device
    int dev = 0;
    CPIC_CUDA(cudaGetDevice(&dev));
    std::atomic<int>& cache = per_sm[dev & 63];
    int bs = cache.load(std::memory_order_acquire);
    if (bs <= 0) {
        CPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, particle_kernel<D, MODE>, 256, 0));
        if (bs < 1) bs = 1;
        cache.store(bs, std::memory_order_release);
    }
    const long long occ = (long long)bs * device_sm_count();
    long long tot = 0;
    for (int s = 0; s < r->cfg.n_species; ++s) tot += r->pb.capacity[s] + 32;
    long long b = (tot + 255) / 256;
    if (b > occ) b = occ;
    if (b < 1) b = 1;
    return (int)b;
}

template <int MODE>
static int launch_particles(cpic_run* r, float c0, float c1, float c2, float c3) {
    PushParams p = make_push_params(r);
    if (MODE == 2) set_boris_constants(r, &p, r->kick_fraction);
    if (r->D == 2) {
        int blocks = particle_grid<2, MODE>(r);
        if (blocks < 0) return blocks;
        particle_kernel<2, MODE><<<blocks, 256, 0, r->stream>>>(p, c0, c1, c2, c3);
    } else {
        int blocks = particle_grid<3, MODE>(r);
        if (blocks < 0) return blocks;
        particle_kernel<3, MODE><<<blocks, 256, 0, r->stream>>>(p, c0, c1, c2, c3);
    }
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_push_prep(cpic_run* r) {
    CPIC_CUDA(cudaMemsetAsync(r->charge_h, 0, sizeof(unsigned long long) * r->ncell_h * r->cfg.n_species, r->stream));
    CPIC_CUDA(cudaMemsetAsync(&r->ctr->ke_fp[0], 0, sizeof(long long) * CPIC_MAX_SPECIES, r->stream));
    return CPIC_OK;
}

// whether the run's push kernel can read through a pending sort order and count the next
// sort's histogram (so that the sort may leave its histogram and gather to the push): the
// direct 3D kernel and the 2D kernel (periodic and absorbing axes, no field, Omega = 1)
bool push_fused_ok(const cpic_run* r) {
    if (r->magnetized) return false;
    if (r->D == 3) return push3d_direct_taken(r);
    if (r->cfg.axisymmetric) return false;
    for (int f = 0; f < 4; ++f)
        if (r->cfg.particle_bc[f] == CPIC_PBC_REFLECT) return false;
    return true;
}

int launch_push_kernel(cpic_run* r) {
    // a pending sort order: the direct 3D kernel and the 2D kernel read through it (the step's
    // finalisation flips the buffers); any other kernel needs the particles gathered first
    if (r->order_pending) {
        if (push_fused_ok(r)) {
            r->order_pending = false;
        } else if (int e = resolve_order(r)) {
            return e;
        }
    }
    // the specialised 2D kernel covers periodic and absorbing axes; reflecting ones take the
    // generic kernel
    bool reflect = false;
    for (int f = 0; f < 2 * r->D; ++f) reflect = reflect || r->cfg.particle_bc[f] == CPIC_PBC_REFLECT;
    // Boris kick and the axisymmetric mover: the generic kernel
    if (r->magnetized || (r->D == 2 && r->cfg.axisymmetric)) return launch_particles<0>(r, 0, 0, 0, 0);
    if (r->D == 2 && !reflect) return launch_push2d(r, make_push_params(r));
    if (r->D == 3) {
        const int st = launch_push3d(r, make_push_params(r));
        if (st != CPIC_ERR_NOT_BUILT) return st;
    }
    return launch_particles<0>(r, 0, 0, 0, 0);
}

int launch_push(cpic_run* r) {
    int st = launch_push_prep(r);
    if (!st) st = launch_push_kernel(r);
    if (st) return st;
    return launch_finalize_step(r);
}

int launch_deposit(cpic_run* r) {
    CPIC_CUDA(cudaMemsetAsync(r->charge_h, 0, sizeof(unsigned long long) * r->ncell_h * r->cfg.n_species, r->stream));
    return launch_particles<1>(r, 0, 0, 0, 0);
}

int launch_kick(cpic_run* r, double fraction) {
    float c[4] = {0, 0, 0, 0};
    for (int s = 0; s < r->cfg.n_species; ++s) c[s] = (float)(fraction * r->cfg.dt * r->cfg.q[s] / r->cfg.m[s]);
    r->kick_fraction = fraction;  // the Boris constants of this kick (magnetised runs)
    const int st = launch_particles<2>(r, c[0], c[1], c[2], c[3]);
    r->kick_fraction = 1.0;
    return st;
}

int launch_fold(cpic_run* r) {
    FoldParams f;
    f.D = r->D;
    for (int a = 0; a < 3; ++a) {
        f.n[a] = r->n[a];
        f.per[a] = a < r->D && r->cfg.particle_bc[2 * a] == CPIC_PBC_PERIODIC;
    }
    f.hs1 = r->n[0] + 2;
    f.hs2 = (r->n[0] + 2) * (r->n[1] + 2);
    f.nsp = r->cfg.n_species;
    f.ncell = r->ncell;
    f.ncell_h = r->ncell_h;
    f.src = r->charge_h;
    f.dst = r->charge;
    long long b = (r->ncell * f.nsp + 255) / 256;
    if (b > 8LL * device_sm_count()) b = 8LL * device_sm_count();
    fold_kernel<<<(int)b, 256, 0, r->stream>>>(f);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

int launch_finalize_step(cpic_run* r) {
    finalize_step_kernel<<<1, 32, 0, r->stream>>>(r->ctr);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace cpic
