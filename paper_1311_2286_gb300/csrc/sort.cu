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

// Histogram of cells per species: chunks of SC_CHUNK particles of one species count their
// keys in a shared histogram over the chunk's key range (warp-aggregated shared atomics) and
// add each non-zero count to the global histogram once; chunks with wide key ranges add
// per warp and cell.
__global__ void __launch_bounds__(256) hist_kernel(SortParams p) {
    constexpr int CHUNK = 256 * 8, RANGE = 4096;
    __shared__ int h[RANGE];
    __shared__ int red[2][8];
    const int nsp = p.nsp;
    int cnt[CPIC_MAX_SPECIES];
    int total = 0;
#pragma unroll
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        cnt[s] = s < nsp ? (int)p.ctr->count[s] : 0;
        total += cnt[s];
    }
    if (total == 0) return;
    const int cur = p.ctr->cur;
    const int lane = threadIdx.x & 31;
    for (int ch = blockIdx.x;; ch += gridDim.x) {
        int s = 0, local = ch;
        while (s < nsp) {
            const int nch = (cnt[s] + CHUNK - 1) / CHUNK;
            if (local < nch) break;
            local -= nch;
            ++s;
        }
        if (s >= nsp) break;
        const int lo = local * CHUNK, hi = min(lo + CHUNK, cnt[s]);
        const int* __restrict__ cin = p.pb.cell[cur] + p.pb.base[s];
        int* __restrict__ hist_s = p.hist + (long long)s * p.ncell;
        int key[8];
        int kmin = 0x7fffffff, kmax = -1;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = lo + (int)threadIdx.x + e * 256;
            const long long k = i < hi ? cell_key(p, cin[i]) : -1;
            key[e] = (int)k;
            if (k >= 0) {
                kmin = min(kmin, (int)k);
                kmax = max(kmax, (int)k);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(FULL, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
        }
        __syncthreads();
        if (lane == 0) {
            red[0][threadIdx.x >> 5] = kmin;
            red[1][threadIdx.x >> 5] = kmax;
        }
        __syncthreads();
        kmin = red[0][0];
        kmax = red[1][0];
#pragma unroll
        for (int w = 1; w < 8; ++w) {
            kmin = min(kmin, red[0][w]);
            kmax = max(kmax, red[1][w]);
        }
        if (kmax < kmin) continue;
        if (kmax - kmin < RANGE) {
            const int range = kmax - kmin + 1;
            for (int k = threadIdx.x; k < range; k += 256) h[k] = 0;
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = key[e];
                const unsigned peers = __match_any_sync(FULL, k);
                if (k >= 0 && (__ffs(peers) - 1) == lane) atomicAdd(&h[k - kmin], __popc(peers));
            }
            __syncthreads();
            for (int k = threadIdx.x; k < range; k += 256)
                if (h[k]) atomicAdd(hist_s + kmin + k, h[k]);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = key[e];
                const unsigned peers = __match_any_sync(FULL, k);
                if (k >= 0 && (__ffs(peers) - 1) == lane) atomicAdd(hist_s + k, __popc(peers));
            }
        }
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

// Scatter. Blocks walk chunks of SC_CHUNK particles of one species (block-uniform species,
// 32-bit slot indices). Between sorts the particles are nearly in cell order, so a chunk's
// keys span a narrow range: the chunk counts its keys in a shared histogram over that range
// (warp-aggregated), reserves each cell's slots with one global cursor atomic per cell and
// chunk, and ranks its particles with shared atomics, so the long chain global atomic ->
// store runs once per cell and chunk instead of once per warp and cell. Chunks whose keys
// span more than SC_RANGE cells (unsorted loads, injected particles) reserve per warp and
// cell. Lanes with the same cell get consecutive slots either way.
constexpr int SC_THREADS = 256;
constexpr int SC_PER_THREAD = 8;
constexpr int SC_CHUNK = SC_THREADS * SC_PER_THREAD;
constexpr int SC_RANGE = 4096;

template <int D>
__global__ void __launch_bounds__(SC_THREADS) scatter_kernel(SortParams p) {
    __shared__ int hcount[SC_RANGE];  // counts, then reserved global starts
    __shared__ int hrank[SC_RANGE];   // running ranks
    __shared__ int red[2][SC_THREADS / 32];
    const int nsp = p.nsp;
    int cnt[CPIC_MAX_SPECIES];
    int total = 0;
#pragma unroll
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s) {
        cnt[s] = s < nsp ? (int)p.ctr->count[s] : 0;
        total += cnt[s];
    }
    if (total == 0) return;
    const int cur = p.ctr->cur, nxt = 1 - cur;
    const long long T = p.pb.total;
    const int lane = threadIdx.x & 31;
    const int n0 = p.n[0], n1 = p.n[1];
    for (int ch = blockIdx.x;; ch += gridDim.x) {
        int s = 0, local = ch;
        while (s < nsp) {
            const int nch = (cnt[s] + SC_CHUNK - 1) / SC_CHUNK;
            if (local < nch) break;
            local -= nch;
            ++s;
        }
        if (s >= nsp) break;
        const int lo = local * SC_CHUNK, hi = min(lo + SC_CHUNK, cnt[s]);
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
        // keys of this thread's particles (element e: slot lo + threadIdx.x + e * SC_THREADS)
        int key[SC_PER_THREAD];
        int kmin = 0x7fffffff, kmax = -1;
#pragma unroll
        for (int e = 0; e < SC_PER_THREAD; ++e) {
            const int i = lo + (int)threadIdx.x + e * SC_THREADS;
            const int cw = i < hi ? cin[i] : -1;
            int k = -1;
            if (cw >= 0)
                k = D == 2 ? (cw & 0xFFFF) + n0 * (cw >> 16) : (cw & 1023) + n0 * (((cw >> 10) & 1023) + n1 * (cw >> 20));
            key[e] = k;
            if (k >= 0) {
                kmin = min(kmin, k);
                kmax = max(kmax, k);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(FULL, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
        }
        __syncthreads();  // previous chunk done with the shared arrays
        if (lane == 0) {
            red[0][threadIdx.x >> 5] = kmin;
            red[1][threadIdx.x >> 5] = kmax;
        }
        __syncthreads();
        kmin = red[0][0];
        kmax = red[1][0];
#pragma unroll
        for (int w = 1; w < SC_THREADS / 32; ++w) {
            kmin = min(kmin, red[0][w]);
            kmax = max(kmax, red[1][w]);
        }
        if (kmax < kmin) continue;  // no live particle in the chunk (block-uniform)
        const bool local_path = kmax - kmin < SC_RANGE;
        if (local_path) {
            const int range = kmax - kmin + 1;
            for (int k = threadIdx.x; k < range; k += SC_THREADS) hcount[k] = hrank[k] = 0;
            __syncthreads();
#pragma unroll
            for (int e = 0; e < SC_PER_THREAD; ++e) {
                const int k = key[e];
                const unsigned peers = __match_any_sync(FULL, k);
                if (k >= 0 && (__ffs(peers) - 1) == lane) atomicAdd(&hcount[k - kmin], __popc(peers));
            }
            __syncthreads();
            // one global reservation per cell of the chunk: hcount becomes the cell's first slot
            for (int k = threadIdx.x; k < range; k += SC_THREADS) {
                const int c = hcount[k];
                if (c) hcount[k] = (int)(scan_s[kmin + k] - sbase) + atomicAdd(cursor + kmin + k, c);
            }
            __syncthreads();
        }
#pragma unroll
        for (int e = 0; e < SC_PER_THREAD; ++e) {
            const int i = lo + (int)threadIdx.x + e * SC_THREADS;
            const int k = key[e];
            const bool act = k >= 0;
            float t[3], v[3];
#pragma unroll
            for (int a = 0; a < D; ++a) t[a] = act ? tin[a * T + i] : 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = act ? vin[a * T + i] : 0.f;
            const unsigned peers = __match_any_sync(FULL, k);
            const int leader = __ffs(peers) - 1;
            int start = 0;
            if (act && leader == lane) {
                if (local_path)
                    start = hcount[k - kmin] + atomicAdd(&hrank[k - kmin], __popc(peers));
                else
                    start = (int)(scan_s[k] - sbase) + atomicAdd(cursor + k, __popc(peers));
            }
            start = __shfl_sync(FULL, start, leader);
            if (act) {
                const int dst = start + __popc(peers & ((1u << lane) - 1u));
                cout[dst] = cin[i];
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
