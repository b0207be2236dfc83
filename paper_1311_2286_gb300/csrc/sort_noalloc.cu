// Cell sort for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being captured
// (allocation is not a capturable operation), host frameworks whose memory manager owns all
// device memory and forbids side allocations, and latency-bound loops that must not pay an
// allocation. cpic_sort_cells_noalloc sorts one set of particles by cell like cpic_sort
// does for a run, but takes its input and output arrays from the caller and keeps its
// per-cell histogram and prefix sums in a scratch array that lives in this file as a
// static device variable: the library allocates nothing, before or during the call.
//
// The scratch (CPIC_NOALLOC_MAX_CELLS cells of histogram plus prefix sums, 8 MiB) exists
// on every GPU that loads the library, until the process exits. Host code may not use the
// array's name as a device pointer; its device address is looked up with
// cudaGetSymbolAddress on every call made on a stream that is not capturing (the first call
// on a device is always one: make it before any stream capture), and cached per device. Every call uses the same scratch and
// leaves its contents behind, so the histogram is cleared at the start of each call, and
// two calls whose work overlaps on the GPU (different streams, or graph branches without
// an ordering between them) race on it.
#include <mutex>

#include "particles.cuh"

namespace cpic {
namespace {

using namespace pk;

constexpr long long NOALLOC_SCAN_CHUNK_MAX_BLOCKS = 1024;

// [hist: MAX_CELLS int32][scan: MAX_CELLS + 1 int32][block sums: 1025 int32]
constexpr size_t kScratchInts = 2 * (size_t)CPIC_NOALLOC_MAX_CELLS + 1 + (NOALLOC_SCAN_CHUNK_MAX_BLOCKS + 1);
static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

struct NSort {
    int D;
    int n[3];
    long long ncell;
    long long count;
    const int* cell_in;
    const float* t_in;
    const float* v_in;
    int* cell_out;
    float* t_out;
    float* v_out;
    long long* live_out;
    int* hist;
    int* scan;
    int* blocks;
};

__device__ __forceinline__ long long key_of(const NSort& p, int cw) {
    if (cw < 0) return -1;
    int c0, c1, c2 = 0;
    if (p.D == 2) {
        c0 = cw & 0xFFFF;
        c1 = cw >> 16;
    } else {
        c0 = cw & 1023;
        c1 = (cw >> 10) & 1023;
        c2 = cw >> 20;
    }
    if (c0 >= p.n[0] || c1 >= p.n[1] || (p.D == 3 && c2 >= p.n[2])) return -1;  // outside: dropped
    return c0 + (long long)p.n[0] * (c1 + (long long)p.n[1] * c2);
}

__global__ void ns_hist(NSort p) {
    for (long long base = (long long)blockIdx.x * blockDim.x; base < p.count; base += (long long)gridDim.x * blockDim.x) {
        long long i = base + threadIdx.x;
        long long key = i < p.count ? key_of(p, p.cell_in[i]) : -1;
        unsigned peers = __match_any_sync(FULL, (unsigned long long)key);
        if (key >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(p.hist + key, __popc(peers));
    }
}

__device__ __forceinline__ int block_excl_scan(int v, int* sh, int* total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int y = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        int z = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int q = __shfl_up_sync(FULL, z, o);
            if (lane >= o) z += q;
        }
        sh[lane] = z - y;
        if (lane == 31) sh[32] = z;
    }
    __syncthreads();
    int res = x - v + sh[w];
    *total = sh[32];
    __syncthreads();
    return res;
}

__global__ void ns_scan_partial(NSort p, long long chunk) {
    __shared__ int sh[33];
    long long lo = blockIdx.x * chunk, hi = lo + chunk < p.ncell ? lo + chunk : p.ncell;
    int acc = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += p.hist[i];
    int tot;
    block_excl_scan(acc, sh, &tot);
    if (threadIdx.x == 0) p.blocks[blockIdx.x] = tot;
}

__global__ void ns_scan_blocks(NSort p, int nb) {
    __shared__ int sh[33];
    int v = (int)threadIdx.x < nb ? p.blocks[threadIdx.x] : 0;
    int tot;
    int ex = block_excl_scan(v, sh, &tot);
    if ((int)threadIdx.x < nb) p.blocks[threadIdx.x] = ex;
    if (threadIdx.x == 0) p.blocks[nb] = tot;
}

__global__ void ns_scan_final(NSort p, long long chunk) {
    __shared__ int sh[33];
    long long lo = blockIdx.x * chunk, hi = lo + chunk < p.ncell ? lo + chunk : p.ncell;
    int carry = p.blocks[blockIdx.x];
    for (long long t0 = lo; t0 < hi; t0 += blockDim.x) {
        long long i = t0 + threadIdx.x;
        int v = i < hi ? p.hist[i] : 0;
        int tot;
        int ex = block_excl_scan(v, sh, &tot);
        if (i < hi) p.scan[i] = carry + ex;
        carry += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        p.scan[p.ncell] = carry;
        *p.live_out = carry;
    }
}

__global__ void ns_scatter(NSort p) {
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < p.count; base += (long long)gridDim.x * blockDim.x) {
        long long i = base + threadIdx.x;
        int cw = i < p.count ? p.cell_in[i] : -1;
        long long key = key_of(p, cw);
        unsigned peers = __match_any_sync(FULL, (unsigned long long)key);
        int leader = __ffs(peers) - 1;
        int start = 0;
        if (key >= 0 && leader == lane) start = atomicAdd(p.hist + key, __popc(peers));
        start = __shfl_sync(peers, start, leader);
        if (key >= 0) {
            long long dst = (long long)p.scan[key] + start + __popc(peers & ((1u << lane) - 1u));
            p.cell_out[dst] = cw;
            for (int a = 0; a < p.D; ++a) p.t_out[a * p.count + dst] = p.t_in[a * p.count + i];
            for (int a = 0; a < 3; ++a) p.v_out[a * p.count + dst] = p.v_in[a * p.count + i];
        }
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device. A call on a stream that is not
// capturing looks the address up again (after a device reset the library's module is loaded
// anew, possibly elsewhere); a call on a capturing stream uses the address cached by the
// device's last call outside capture.
int scratch_for_current_device(cudaStream_t stream, int** out) {
    int dev = -1;
    CPIC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("sort_cells_noalloc: device ordinal %d outside [0, %d)", dev, kMaxDevices);
        return CPIC_ERR_INVALID;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;  // not decidable here: take the cached address
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_scratch_ptr[dev] = static_cast<int*>(p);
    }
    *out = g_scratch_ptr[dev];
    return CPIC_OK;
}

}  // namespace
}  // namespace cpic

using namespace cpic;

extern "C" int cpic_sort_cells_noalloc(int dim, const int32_t* n, int64_t count, const int32_t* cell_in,
                                       const float* t_in, const float* v_in, int32_t* cell_out, float* t_out,
                                       float* v_out, int64_t* live_out, void* stream) {
    if ((dim != 2 && dim != 3) || !n) {
        set_error("sort_cells_noalloc: dim must be 2 or 3 and n non-NULL");
        return CPIC_ERR_INVALID;
    }
    long long ncell = 1;
    for (int a = 0; a < dim; ++a) {
        int lim = dim == 2 ? (a == 0 ? 65535 : 32767) : 1023;
        if (n[a] < 1 || n[a] > lim) {
            set_error("sort_cells_noalloc: n[%d] = %d outside [1, %d]", a, n[a], lim);
            return CPIC_ERR_INVALID;
        }
        ncell *= n[a];
    }
    if (ncell > CPIC_NOALLOC_MAX_CELLS) {
        set_error("sort_cells_noalloc: %lld cells exceed the fixed scratch of %d cells", ncell, CPIC_NOALLOC_MAX_CELLS);
        return CPIC_ERR_INVALID;
    }
    if (count < 0 || count > (1ll << 31) - 1) {
        set_error("sort_cells_noalloc: count %lld outside [0, 2^31)", (long long)count);
        return CPIC_ERR_INVALID;
    }
    if (!live_out || (count > 0 && (!cell_in || !t_in || !v_in || !cell_out || !t_out || !v_out))) {
        set_error("sort_cells_noalloc: NULL array");
        return CPIC_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int* scratch = nullptr;
    int st = scratch_for_current_device(s, &scratch);
    if (st) return st;
    NSort p;
    p.D = dim;
    for (int a = 0; a < 3; ++a) p.n[a] = a < dim ? n[a] : 1;
    p.ncell = ncell;
    p.count = count;
    p.cell_in = cell_in;
    p.t_in = t_in;
    p.v_in = v_in;
    p.cell_out = cell_out;
    p.t_out = t_out;
    p.v_out = v_out;
    p.live_out = reinterpret_cast<long long*>(live_out);
    p.hist = scratch;
    p.scan = scratch + CPIC_NOALLOC_MAX_CELLS;
    p.blocks = scratch + 2 * (size_t)CPIC_NOALLOC_MAX_CELLS + 1;
    // the scratch keeps the previous call's contents: clear the histogram first
    CPIC_CUDA(cudaMemsetAsync(p.hist, 0, sizeof(int) * ncell, s));
    long long pblocks = (count + 255) / 256;
    if (pblocks > 8LL * device_sm_count()) pblocks = 8LL * device_sm_count();
    if (pblocks < 1) pblocks = 1;
    ns_hist<<<(int)pblocks, 256, 0, s>>>(p);
    CPIC_CHECK_LAUNCH();
    long long chunk = 1024;
    while ((ncell + chunk - 1) / chunk > NOALLOC_SCAN_CHUNK_MAX_BLOCKS) chunk *= 2;
    int nb = (int)((ncell + chunk - 1) / chunk);
    ns_scan_partial<<<nb, 1024, 0, s>>>(p, chunk);
    CPIC_CHECK_LAUNCH();
    ns_scan_blocks<<<1, 1024, 0, s>>>(p, nb);
    CPIC_CHECK_LAUNCH();
    ns_scan_final<<<nb, 1024, 0, s>>>(p, chunk);
    CPIC_CHECK_LAUNCH();
    CPIC_CUDA(cudaMemsetAsync(p.hist, 0, sizeof(int) * ncell, s));  // cursors
    ns_scatter<<<(int)pblocks, 256, 0, s>>>(p);
    CPIC_CHECK_LAUNCH();
    return CPIC_OK;
}
