// Row a7: periodic cell sort for locality (not in the paper: the particle order is free in
// the method, and sorting by cell makes a warp's gathers hit the same vertex records and
// its deposits aggregate into one group per cell).
//
// Counting sort of every species by its row-major cell index i + N1 (j + N2 k), compacting
// dead slots away: histogram (warp-aggregated atomics) -> exclusive scan over
// [species][cell] -> scatter into the other particle buffer (one atomic per cell group per
// warp reserves consecutive slots; the order inside a cell is unspecified) -> live counts.
#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

struct SortParams {
    int D;
    int n[3];
    int nsp;
    long long ncell;
    ParticleBuffers pb;
    DevCounters* ctr;
    int* hist;         // [nsp][ncell]
    long long* scan;   // [nsp * ncell + 1]
};

__device__ __forceinline__ long long cell_key(const SortParams& p, int cw) {
    if (cw < 0) return -1;
    if (p.D == 2) return (long long)(cw & 0xFFFF) + (long long)p.n[0] * (cw >> 16);
    return (long long)(cw & 1023) + (long long)p.n[0] * (((cw >> 10) & 1023) + (long long)p.n[1] * (cw >> 20));
}

struct Ranges {
    long long cnt[CPIC_MAX_SPECIES];
    long long voff[CPIC_MAX_SPECIES + 1];
};

__device__ __forceinline__ Ranges ranges(const SortParams& p) {
    Ranges r;
    r.voff[0] = 0;
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        long long c = s < p.nsp ? p.ctr->count[s] : 0;
        r.cnt[s] = c;
        r.voff[s + 1] = r.voff[s] + ((c + 31) & ~31ll);
    }
    return r;
}

__device__ __forceinline__ int species_at(const Ranges& r, int nsp, long long vi) {
    int s = 0;
#pragma unroll
    for (int x = 1; x < CPIC_MAX_SPECIES; ++x)
        if (x < nsp && vi >= r.voff[x]) s = x;
    return s;
}

__global__ void hist_kernel(SortParams p) {
    const Ranges R = ranges(p);
    const long long total = R.voff[p.nsp];
    const int cur = p.ctr->cur;
    const int* cellp = p.pb.cell[cur];
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += (long long)gridDim.x * blockDim.x) {
        long long vi = base + threadIdx.x;
        int s = species_at(R, p.nsp, vi);
        long long local = vi - R.voff[s];
        bool act = vi < total && local < R.cnt[s];
        long long key = act ? cell_key(p, cellp[p.pb.base[s] + local]) : -1;
        unsigned peers = __match_any_sync(FULL, (unsigned long long)key);
        if (key >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(p.hist + (long long)s * p.ncell + key, __popc(peers));
    }
}

// ---- exclusive scan of hist (int) into scan (long long), three phases
constexpr int SCAN_THREADS = 1024;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long* total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        long long y = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        long long z = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long q = __shfl_up_sync(FULL, z, o);
            if (lane >= o) z += q;
        }
        sh[lane] = z - y;  // exclusive warp offsets
        if (lane == 31) sh[32] = z;
    }
    __syncthreads();
    long long res = x - v + sh[w];
    *total = sh[32];
    __syncthreads();
    return res;
}

__global__ void scan_partial_kernel(const int* hist, long long N, long long chunk, long long* blocksum) {
    __shared__ long long sh[33];
    long long lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
    long long acc = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += hist[i];
    long long tot;
    block_exclusive_scan(acc, sh, &tot);
    if (threadIdx.x == 0) blocksum[blockIdx.x] = tot;
}

__global__ void scan_blocks_kernel(long long* blocksum, int nb) {
    __shared__ long long sh[33];
    // single block; nb <= blockDim.x
    long long v = (int)threadIdx.x < nb ? blocksum[threadIdx.x] : 0;
    long long tot;
    long long ex = block_exclusive_scan(v, sh, &tot);
    if ((int)threadIdx.x < nb) blocksum[threadIdx.x] = ex;
    if (threadIdx.x == 0) blocksum[nb] = tot;
}

__global__ void scan_final_kernel(const int* hist, long long N, long long chunk, const long long* blocksum, long long* scan) {
    __shared__ long long sh[33];
    long long lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
    long long carry = blocksum[blockIdx.x];
    for (long long t0 = lo; t0 < hi; t0 += blockDim.x) {
        long long i = t0 + threadIdx.x;
        long long v = i < hi ? hist[i] : 0;
        long long tot;
        long long ex = block_exclusive_scan(v, sh, &tot);
        if (i < hi) scan[i] = carry + ex;
        carry += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) scan[N] = carry;
}

// Scatter: blocks walk chunks of one species (block-uniform species, 32-bit slot indices);
// every thread loads its particle's whole state before reserving its destination, so the
// loads overlap the cursor atomics; lanes with the same cell reserve consecutive slots with
// one atomic per group.
template <int D>
__global__ void __launch_bounds__(256) scatter_kernel(SortParams p) {
    const int nsp = p.nsp;
    int cnt[CPIC_MAX_SPECIES];
    int total = 0;
#pragma unroll
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        cnt[s] = s < nsp ? (int)p.ctr->count[s] : 0;
        total += cnt[s];
    }
    if (total == 0) return;
    const int C = ((total + (int)gridDim.x - 1) / (int)gridDim.x + 255) / 256 * 256;
    const int cur = p.ctr->cur, nxt = 1 - cur;
    const long long T = p.pb.total;
    const int lane = threadIdx.x & 31;
    const int n0 = p.n[0], n1 = p.n[1];
    for (int ch = blockIdx.x;; ch += gridDim.x) {
        int s = 0, local = ch;
        while (s < nsp) {
            const int nch = (cnt[s] + C - 1) / C;
            if (local < nch) break;
            local -= nch;
            ++s;
        }
        if (s >= nsp) break;
        const int lo = local * C, hi = min(lo + C, cnt[s]);
        const long long b0 = p.pb.base[s];
        const int* __restrict__ cin = p.pb.cell[cur] + b0;
        const float* __restrict__ tin = p.pb.t[cur] + b0;
        const float* __restrict__ vin = p.pb.v[cur] + b0;
        int* __restrict__ cout = p.pb.cell[nxt] + b0;
        float* __restrict__ tout = p.pb.t[nxt] + b0;
        float* __restrict__ vout = p.pb.v[nxt] + b0;
        const long long* __restrict__ scan_s = p.scan + (long long)s * p.ncell;
        int* __restrict__ cursor = p.hist + (long long)s * p.ncell;
        const long long sbase = scan_s[0];
        for (int i = lo + (int)threadIdx.x; i - (int)threadIdx.x < hi; i += 256) {
            const bool act = i < hi;
            const int cw = act ? cin[i] : -1;
            float t[3], v[3];
#pragma unroll
            for (int a = 0; a < D; ++a) t[a] = act ? tin[a * T + i] : 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = act ? vin[a * T + i] : 0.f;
            int key = -1;
            if (cw >= 0)
                key = D == 2 ? (cw & 0xFFFF) + n0 * (cw >> 16)
                             : (cw & 1023) + n0 * (((cw >> 10) & 1023) + n1 * (cw >> 20));
            const unsigned peers = __match_any_sync(FULL, key);
            const int leader = __ffs(peers) - 1;
            int start = 0;
            if (key >= 0 && leader == lane) start = atomicAdd(cursor + key, __popc(peers));
            start = __shfl_sync(FULL, start, leader);
            if (key >= 0) {
                const int dst = (int)(scan_s[key] - sbase) + start + __popc(peers & ((1u << lane) - 1u));
                cout[dst] = cw;
#pragma unroll
                for (int a = 0; a < D; ++a) tout[a * T + dst] = t[a];
#pragma unroll
                for (int a = 0; a < 3; ++a) vout[a * T + dst] = v[a];
            }
        }
    }
}

__global__ void sort_finalize_kernel(SortParams p) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int s = 0; s < p.nsp; ++s) {
            long long n = p.scan[(long long)(s + 1) * p.ncell] - p.scan[(long long)s * p.ncell];
            p.ctr->count[s] = n;
            p.ctr->alive[s] = n;
        }
        p.ctr->cur = 1 - p.ctr->cur;
    }
}

}  // namespace

int launch_sort(cpic_run* r) {
    SortParams p;
    p.D = r->D;
    for (int a = 0; a < 3; ++a) p.n[a] = a < r->D ? r->n[a] : 1;
    p.nsp = r->cfg.n_species;
    p.ncell = r->ncell;
    p.pb = r->pb;
    p.ctr = r->ctr;
    p.hist = r->hist;
    p.scan = r->scan;
    long long N = (long long)p.nsp * r->ncell;
    long long tot = 0;
    for (int s = 0; s < p.nsp; ++s) tot += r->pb.capacity[s] + 32;
    long long pblocks = (tot + 255) / 256;
    if (pblocks > 152 * 8) pblocks = 152 * 8;
    if (pblocks < 1) pblocks = 1;
    CPIC_CUDA(cudaMemsetAsync(r->hist, 0, sizeof(int) * N, r->stream));
    hist_kernel<<<(int)pblocks, 256, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    long long chunk = 4096;
    while ((N + chunk - 1) / chunk > SCAN_THREADS) chunk *= 2;
    int nb = (int)((N + chunk - 1) / chunk);
    scan_partial_kernel<<<nb, SCAN_THREADS, 0, r->stream>>>(r->hist, N, chunk, r->scan_blocks);
    CPIC_CHECK_LAUNCH();
    scan_blocks_kernel<<<1, SCAN_THREADS, 0, r->stream>>>(r->scan_blocks, nb);
    CPIC_CHECK_LAUNCH();
    scan_final_kernel<<<nb, SCAN_THREADS, 0, r->stream>>>(r->hist, N, chunk, r->scan_blocks, r->scan);
    CPIC_CHECK_LAUNCH();
    CPIC_CUDA(cudaMemsetAsync(r->hist, 0, sizeof(int) * N, r->stream));
    if (p.D == 2)
        scatter_kernel<2><<<(int)pblocks, 256, 0, r->stream>>>(p);
    else
        scatter_kernel<3><<<(int)pblocks, 256, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    sort_finalize_kernel<<<1, 32, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace cpic
