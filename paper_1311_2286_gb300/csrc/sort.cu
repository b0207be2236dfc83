// Row a7: periodic cell sort for locality (not in the paper: the particle order is free in
// the method, and sorting by cell makes a warp's gathers hit the same vertex records and
// its deposits aggregate into one group per cell).
//
// Counting sort of every species by its row-major cell index i + N1 (j + N2 k), compacting
// dead slots away: histogram (warp-aggregated atomics) -> exclusive scan over
// [species][cell] -> rank (each live particle's slot in the other buffer; one atomic per cell
// group reserves consecutive slots; the order inside a cell is unspecified) -> gather of the
// particle data into the other buffer in slot order -> live counts.
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
    unsigned* ticket;  // last-block counter of the gather (zero between sorts)
    int flush;         // gather only if an order is pending (DevCounters::perm)
};

__device__ __forceinline__ long long cell_key(const SortParams& p, int cw) {
    if (cw < 0) return -1;
    if (p.D == 2) return (long long)(cw & 0xFFFF) + (long long)p.n[0] * (cw >> 16);
    return (long long)(cw & 1023) + (long long)p.n[0] * (((cw >> 10) & 1023) + (long long)p.n[1] * (cw >> 20));
}

// Block-wide key window of a chunk for the shared-memory path: [wlo, whi] with
// whi - wlo < RANGE. When all live keys fit, it is their [min, max]; otherwise (3D chunks whose
// particles have moved to other planes since the last sort: a plane is n0 n1 keys away) it is
// the [min, max] of the keys within RANGE / 2 of the key at the chunk's middle slot, and the
// keys outside take the global path. wlo > whi: no key in a window (all global or no live key).
// Every thread of the block must call it; red is [2][8] shared ints.
template <int PER, int RANGE>
__device__ __forceinline__ void chunk_window(const int (&key)[PER], int kmid, int (*red)[8], int& wlo, int& whi) {
    const int lane = threadIdx.x & 31;
    auto block_minmax = [&](int lo_bound, int hi_bound, int& mn, int& mx) {
        mn = 0x7fffffff;
        mx = -1;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int k = key[e];
            if (k >= lo_bound && k <= hi_bound) {
                mn = min(mn, k);
                mx = max(mx, k);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(FULL, mn, o));
            mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        }
        __syncthreads();  // the previous use of red (and of the chunk's shared arrays) is done
        if (lane == 0) {
            red[0][threadIdx.x >> 5] = mn;
            red[1][threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        mn = red[0][0];
        mx = red[1][0];
#pragma unroll
        for (int w = 1; w < 8; ++w) {
            mn = min(mn, red[0][w]);
            mx = max(mx, red[1][w]);
        }
    };
    int mn, mx;
    block_minmax(0, 0x7fffffff, mn, mx);
    if (mx < mn || mx - mn < RANGE) {
        wlo = mn;
        whi = mx;
        return;
    }
    const int c = kmid >= 0 ? kmid : mn;
    block_minmax(max(c - RANGE / 2, 0), c + RANGE / 2 - 1, mn, mx);
    wlo = mn;
    whi = mx;
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
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = lo + (int)threadIdx.x + e * 256;
            key[e] = i < hi ? (int)cell_key(p, cin[i]) : -1;
        }
        int kmin, kmax;
        chunk_window<8, RANGE>(key, (int)cell_key(p, cin[lo + (hi - lo) / 2]), red, kmin, kmax);
        const bool win = kmax >= kmin;  // block-uniform
        if (win) {
            const int range = kmax - kmin + 1;
            for (int k = threadIdx.x; k < range; k += 256) h[k] = 0;
            __syncthreads();
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = key[e];
            const unsigned peers = __match_any_sync(FULL, k);
            if (k >= 0 && (__ffs(peers) - 1) == lane) {
                if (win && k >= kmin && k <= kmax)
                    atomicAdd(&h[k - kmin], __popc(peers));
                else
                    atomicAdd(hist_s + k, __popc(peers));
            }
        }
        if (win) {
            __syncthreads();
            for (int k = threadIdx.x; k < kmax - kmin + 1; k += 256)
                if (h[k]) atomicAdd(hist_s + kmin + k, h[k]);
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

// Rank. Blocks walk chunks of SC_CHUNK particles of one species (block-uniform species,
// 32-bit slot indices) and give every live particle its slot in the sorted order; the slot
// receives the particle's source index (in the other buffer's cell array, which the gather
// below then overwrites), so the particle data itself moves once, in the gather, with
// coalesced writes. Between sorts the particles are nearly in cell order, so a chunk's keys
// span a narrow range: the chunk counts its keys in a shared histogram over that range
// (warp-aggregated), reserves each cell's slots with one global cursor atomic per cell and
// chunk, and ranks its particles with shared atomics, so the long chain global atomic ->
// store runs once per cell and chunk instead of once per warp and cell. Chunks whose keys
// span more than SC_RANGE cells (unsorted loads, injected particles) reserve per warp and
// cell; in chunks whose particles have partly moved to other planes (3D), the keys near the
// chunk's middle key take the shared path and the others the per-warp one. Lanes with the
// same cell get consecutive slots either way.
constexpr int SC_THREADS = 256;
constexpr int SC_PER_THREAD = 8;
constexpr int SC_CHUNK = SC_THREADS * SC_PER_THREAD;
constexpr int SC_RANGE = 4096;

template <int D>
__global__ void __launch_bounds__(SC_THREADS) rank_kernel(SortParams p) {
    __shared__ int hcount[SC_RANGE];  // the chunk's count per cell
    __shared__ int hstart[SC_RANGE];  // the chunk's first slot per cell
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
        int* __restrict__ cout = p.pb.cell[nxt] + b0;  // receives source indices
        const long long* __restrict__ scan_s = p.scan + (long long)s * p.ncell;
        int* __restrict__ cursor = p.hist + (long long)s * p.ncell;
        const long long sbase = scan_s[0];
        // keys of this thread's particles (element e: slot lo + threadIdx.x + e * SC_THREADS)
        auto key_of = [&](int cw) {
            if (cw < 0) return -1;
            return D == 2 ? (cw & 0xFFFF) + n0 * (cw >> 16) : (cw & 1023) + n0 * (((cw >> 10) & 1023) + n1 * (cw >> 20));
        };
        int key[SC_PER_THREAD];
#pragma unroll
        for (int e = 0; e < SC_PER_THREAD; ++e) {
            const int i = lo + (int)threadIdx.x + e * SC_THREADS;
            key[e] = key_of(i < hi ? cin[i] : -1);
        }
        int kmin, kmax;
        chunk_window<SC_PER_THREAD, SC_RANGE>(key, key_of(cin[lo + (hi - lo) / 2]), red, kmin, kmax);
        const bool local_path = kmax >= kmin;  // block-uniform: keys in [kmin, kmax] go through shared memory
        // one pass groups the lanes of a warp by key; a group's leader adds the group to its
        // cell's chunk count (shared) and gets the group's offset in the chunk's share of the
        // cell back, or (keys outside the window) reserves slots in the global cursor
        int gpos[SC_PER_THREAD];  // offset in the chunk's share of the cell, or global slot
        if (local_path) {
            for (int k = threadIdx.x; k < kmax - kmin + 1; k += SC_THREADS) hcount[k] = 0;
            __syncthreads();
        }
#pragma unroll
        for (int e = 0; e < SC_PER_THREAD; ++e) {
            const int k = key[e];
            const unsigned peers = __match_any_sync(FULL, k);
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (k >= 0 && leader == lane) {
                if (local_path && k >= kmin && k <= kmax)
                    base = atomicAdd(&hcount[k - kmin], __popc(peers));
                else
                    base = (int)(scan_s[k] - sbase) + atomicAdd(cursor + k, __popc(peers));
            }
            gpos[e] = __shfl_sync(FULL, base, leader) + __popc(peers & ((1u << lane) - 1u));
        }
        if (local_path) {
            __syncthreads();
            // one global reservation per cell of the chunk: hstart is the chunk's first slot
            for (int k = threadIdx.x; k < kmax - kmin + 1; k += SC_THREADS) {
                const int c = hcount[k];
                if (c) hstart[k] = (int)(scan_s[kmin + k] - sbase) + atomicAdd(cursor + kmin + k, c);
            }
            __syncthreads();
        }
#pragma unroll
        for (int e = 0; e < SC_PER_THREAD; ++e) {
            const int k = key[e];
            if (k < 0) continue;
            const int dst = (local_path && k >= kmin && k <= kmax) ? hstart[k - kmin] + gpos[e] : gpos[e];
            cout[dst] = lo + (int)threadIdx.x + e * SC_THREADS;
        }
    }
}

// Gather: slot d of species s in the other buffer takes the particle whose source index the
// rank pass stored there; reads follow the source order (mostly ascending: the particles
// were nearly sorted), writes are coalesced. blockIdx.y is the species. The last block to
// finish sets the live counts from the scan and flips the current buffer.
template <int D>
__global__ void __launch_bounds__(256) gather_kernel(SortParams p) {
    __shared__ bool last;
    if (p.flush && !p.ctr->perm) return;  // nothing pending (the same for every block)
    const int s = blockIdx.y;
    const long long n = p.scan[(long long)(s + 1) * p.ncell] - p.scan[(long long)s * p.ncell];
    const int cur = p.ctr->cur, nxt = 1 - cur;
    const long long T = p.pb.total, b0 = p.pb.base[s];
    const int* __restrict__ cin = p.pb.cell[cur] + b0;
    const float* __restrict__ tin = p.pb.t[cur] + b0;
    const float* __restrict__ vin = p.pb.v[cur] + b0;
    int* __restrict__ cout = p.pb.cell[nxt] + b0;
    float* __restrict__ tout = p.pb.t[nxt] + b0;
    float* __restrict__ vout = p.pb.v[nxt] + b0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < (int)n; d += gridDim.x * blockDim.x) {
        const int i = cout[d];
        const int cw = cin[i];
        float t[3], v[3];
#pragma unroll
        for (int a = 0; a < D; ++a) t[a] = tin[a * T + i];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = vin[a * T + i];
        cout[d] = cw;
#pragma unroll
        for (int a = 0; a < D; ++a) tout[a * T + d] = t[a];
#pragma unroll
        for (int a = 0; a < 3; ++a) vout[a * T + d] = v[a];
    }
    __syncthreads();  // every thread of the block has read ctr->cur
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(p.ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    *p.ticket = 0;
    for (int sp = 0; sp < p.nsp; ++sp) {
        const long long cnt = p.scan[(long long)(sp + 1) * p.ncell] - p.scan[(long long)sp * p.ncell];
        p.ctr->count[sp] = cnt;
        p.ctr->alive[sp] = cnt;
    }
    p.ctr->cur = 1 - p.ctr->cur;
    p.ctr->perm = 0;
}

// Fused sort: the live counts become the sorted ones and the order is left pending; the next
// push reads slot i's particle from the index the rank pass stored in the other buffer, writes
// it to slot i there, and the step's finalisation flips the buffers.
__global__ void sort_fused_finish_kernel(SortParams p) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int sp = 0; sp < p.nsp; ++sp) {
        const long long cnt = p.scan[(long long)(sp + 1) * p.ncell] - p.scan[(long long)sp * p.ncell];
        p.ctr->count[sp] = cnt;
        p.ctr->alive[sp] = cnt;
    }
    p.ctr->perm = 1;
}

SortParams sort_params(cpic_run* r) {
    SortParams p;
    p.D = r->D;
    for (int a = 0; a < 3; ++a) p.n[a] = a < r->D ? r->n[a] : 1;
    p.nsp = r->cfg.n_species;
    p.ncell = r->ncell;
    p.pb = r->pb;
    p.ctr = r->ctr;
    p.hist = r->hist;
    p.scan = r->scan;
    p.ticket = r->ticket + 2;
    p.flush = 0;
    return p;
}

int launch_gather(cpic_run* r, const SortParams& p) {
    int dev = 0, nsm = 0;
    CPIC_CUDA(cudaGetDevice(&dev));
    CPIC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const dim3 ggrid((unsigned)(nsm * 8 / p.nsp > 0 ? nsm * 8 / p.nsp : 1), (unsigned)p.nsp);
    if (p.D == 2)
        gather_kernel<2><<<ggrid, 256, 0, r->stream>>>(p);
    else
        gather_kernel<3><<<ggrid, 256, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}

}  // namespace

int resolve_order(cpic_run* r) {
    if (!r->order_pending) return CPIC_OK;
    r->order_pending = false;
    SortParams p = sort_params(r);
    p.flush = 1;
    return launch_gather(r, p);
}

int launch_sort(cpic_run* r, bool fused) {
    if (int e = resolve_order(r)) return e;
    SortParams p = sort_params(r);
    long long N = (long long)p.nsp * r->ncell;
    long long tot = 0;
    for (int s = 0; s < p.nsp; ++s) tot += r->pb.capacity[s] + 32;
    long long pblocks = (tot + 255) / 256;
    if (pblocks > 8LL * device_sm_count()) pblocks = 8LL * device_sm_count();
    if (pblocks < 1) pblocks = 1;
    if (r->count_hist) {
        r->count_hist = false;  // the step's push and injection counted the cells
    } else {
        CPIC_CUDA(cudaMemsetAsync(r->hist, 0, sizeof(int) * N, r->stream));
        hist_kernel<<<(int)pblocks, 256, 0, r->stream>>>(p);
        CPIC_CHECK_LAUNCH();
    }
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
        rank_kernel<2><<<(int)pblocks, 256, 0, r->stream>>>(p);
    else
        rank_kernel<3><<<(int)pblocks, 256, 0, r->stream>>>(p);
    CPIC_CHECK_LAUNCH();
    if (fused) {
        sort_fused_finish_kernel<<<1, 32, 0, r->stream>>>(p);
        CPIC_CHECK_LAUNCH();
        r->order_pending = true;
        return CPIC_OK;
    }
    return launch_gather(r, p);
}

}  // namespace cpic
