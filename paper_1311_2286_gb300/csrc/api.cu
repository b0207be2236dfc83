// C ABI of include/cpic.h: validation, device-memory planning (one arena per run), the PIC
// cycle's orchestration on the run's stream, and data transfer. All arithmetic of the
// method runs in the kernels of geometry.cu, fields.cu, push.cu, inject.cu, sort.cu, mg.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "internal.cuh"

namespace cpic {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int device_sm_count() {
    constexpr int MAXDEV = 64;
    static std::atomic<int> cache[MAXDEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    if (dev >= MAXDEV) dev = MAXDEV - 1;
    int v = cache[dev].load(std::memory_order_acquire);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cache[dev].store(v, std::memory_order_release);
    }
    return v;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? CPIC_ERR_OOM : CPIC_ERR_CUDA;
}

namespace {

// ------------------------------------------------------------------ memory planning
struct Planner {
    char* base = nullptr;  // null: dry run
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T*>(base + off) : nullptr;
    }
};

int validate(const cpic_config* c) {
    if (!c) {
        set_error("config is NULL");
        return CPIC_ERR_INVALID;
    }
    if (c->dim != 2 && c->dim != 3) {
        set_error("dim must be 2 or 3 (got %d)", c->dim);
        return CPIC_ERR_INVALID;
    }
    for (int a = 0; a < c->dim; ++a) {
        int lim = c->dim == 2 ? (a == 0 ? 65535 : 32767) : 1023;
        if (c->n[a] < 2 || c->n[a] > lim) {
            set_error("n[%d] = %d outside [2, %d]", a, c->n[a], lim);
            return CPIC_ERR_INVALID;
        }
        bool p0 = c->field_bc[2 * a] == CPIC_BC_PERIODIC, p1 = c->field_bc[2 * a + 1] == CPIC_BC_PERIODIC;
        if (p0 != p1) {
            set_error("axis %d: a periodic axis needs both faces periodic", a);
            return CPIC_ERR_INVALID;
        }
        for (int s = 0; s < 2; ++s) {
            int fb = c->field_bc[2 * a + s], pb = c->particle_bc[2 * a + s];
            if (fb < 0 || fb > 2 || pb < 0 || pb > 2) {
                set_error("face %d: unknown boundary kind", 2 * a + s);
                return CPIC_ERR_INVALID;
            }
            if ((fb == CPIC_BC_PERIODIC) != (pb == CPIC_PBC_PERIODIC)) {
                set_error("face %d: particle boundary must be periodic exactly when the field is", 2 * a + s);
                return CPIC_ERR_INVALID;
            }
        }
        if (c->particle_bc[2 * a] != c->particle_bc[2 * a + 1]) {
            set_error("axis %d: different particle boundary kinds on its two faces are not built", a);
            return CPIC_ERR_NOT_BUILT;
        }
        if (p0 && (c->n[a] & 1)) {
            set_error("axis %d: a periodic axis needs an even cell count", a);
            return CPIC_ERR_INVALID;
        }
    }
    if (!(c->dt > 0.0) || !isfinite(c->dt)) {
        set_error("dt must be positive and finite");
        return CPIC_ERR_INVALID;
    }
    if (c->n_species < 1 || c->n_species > CPIC_MAX_SPECIES) {
        set_error("n_species must be in [1, %d]", CPIC_MAX_SPECIES);
        return CPIC_ERR_INVALID;
    }
    for (int s = 0; s < c->n_species; ++s) {
        if (!(c->m[s] > 0.0) || !(c->w[s] > 0.0) || c->capacity[s] < 0 || c->capacity[s] > (1ll << 31) - 64) {
            set_error("species %d: need m > 0, w > 0, 0 <= capacity < 2^31", s);
            return CPIC_ERR_INVALID;
        }
    }
    long long tot = 0;
    for (int s = 0; s < c->n_species; ++s) tot += (c->capacity[s] + 31) & ~31ll;
    // the particle kernels index slots with 32-bit integers and look up to three blocks of
    // 256 past the last slot: keep 4096 slots of headroom below 2^31
    if (tot > (1ll << 31) - 4096) {
        set_error("total particle capacity %lld exceeds 2^31 - 4096 slots", tot);
        return CPIC_ERR_INVALID;
    }
    if (c->axisymmetric && c->dim != 2) {
        set_error("axisymmetric (Omega = r) geometry is 2D only");
        return CPIC_ERR_INVALID;
    }
    return CPIC_OK;
}

// multigrid levels: halve every axis while all are even, at least 4, and the level has
// more than 64 cells
int plan_levels(const cpic_config* c, int lev_n[MAX_LEVELS][3], int* nl) {
    int n[3] = {c->n[0], c->n[1], c->dim == 3 ? c->n[2] : 1};
    int l = 0;
    for (;;) {
        for (int a = 0; a < 3; ++a) lev_n[l][a] = n[a];
        long long cells = (long long)n[0] * n[1] * n[2];
        bool can = cells > 64 && l + 1 < MAX_LEVELS;
        // a periodic axis keeps at least four cells: with two, a cell spans half the period
        // and a curved map (azimuth) makes it degenerate (vertices on opposite sides)
        for (int a = 0; a < c->dim; ++a)
            can = can && (n[a] % 2 == 0) && n[a] >= (c->field_bc[2 * a] == CPIC_BC_PERIODIC ? 8 : 4);
        ++l;
        if (!can) break;
        for (int a = 0; a < c->dim; ++a) n[a] /= 2;
    }
    *nl = l;
    long long last = (long long)lev_n[l - 1][0] * lev_n[l - 1][1] * lev_n[l - 1][2];
    if (last > DENSE_MAX) {
        set_error("grid cannot be coarsened to <= %d cells (coarsest %lld cells): use cell counts with more factors of 2",
                  DENSE_MAX, last);
        return CPIC_ERR_INVALID;
    }
    // every smoothed level needs even counts (colour ordering)
    for (int k = 0; k + 1 < l; ++k)
        for (int a = 0; a < c->dim; ++a)
            if (lev_n[k][a] & 1) {
                set_error("internal: odd smoothed level");
                return CPIC_ERR_INVALID;
            }
    return CPIC_OK;
}

void plan(cpic_run* r, Planner& P) {
    const cpic_config& c = r->cfg;
    int D = r->D;
    int S = D == 2 ? 9 : 27;  // 3D: the 19-point operator and the corners of Galerkin levels
    for (int l = 0; l < r->nlevels; ++l) {
        Level& L = r->lev[l];
        long long nv = (long long)(L.n[0] + 1) * (L.n[1] + 1) * (D == 3 ? L.n[2] + 1 : 1);
        L.S = S;
        L.A = P.take<double>((size_t)S * L.ncell);
        L.x = P.take<double>(L.ncell);
        L.b = P.take<double>(L.ncell);
        L.X = P.take<double>((size_t)nv * D);
        L.Jc = P.take<double>(L.ncell);
        L.omega = P.take<double>(L.ncell);
        L.dv = P.take<double>((size_t)D * nv * D);
        for (int a = 0; a < 3; ++a) {
            if (a >= D) {
                L.face[a] = nullptr;
                continue;
            }
            long long fn[3] = {L.n[0], L.n[1], D == 3 ? L.n[2] : 1};
            fn[a] += 1;
            L.face[a] = P.take<double>((size_t)D * fn[0] * fn[1] * fn[2]);
        }
    }
    r->k64 = P.take<double>((size_t)r->nvert * D * D);
    r->K32 = P.take<float>((size_t)r->nvert * (D == 2 ? 4 : 12));
    r->G32 = P.take<float>((size_t)r->nvert * (D == 2 ? 2 : 4));
    r->rhs_bc = P.take<double>(r->ncell);
    r->psi = P.take<double>(r->ncell);
    r->jcdf = P.take<double>(r->ncell);
    r->fcdf = r->D == 3 ? P.take<double>((size_t)2 * r->n[1] * r->n[2])
                        : (c.axisymmetric ? P.take<double>((size_t)2 * r->n[1]) : nullptr);
    r->R32 = c.axisymmetric ? P.take<float>((size_t)r->nvert) : nullptr;
    r->dcdf = D == 2 ? P.take<double>((size_t)CPIC_MAX_SPECIES * r->n[1]) : nullptr;
    r->charge = P.take<unsigned long long>((size_t)c.n_species * r->ncell);
    r->ncollect = D == 2 ? r->n[1] : r->n[1] * r->n[2];
    r->collect = P.take<unsigned long long>((size_t)c.n_species * 2 * r->ncollect);
    r->charge_h = P.take<unsigned long long>((size_t)c.n_species * r->ncell_h);
    long long total = 0;
    for (int s = 0; s < c.n_species; ++s) {
        r->pb.base[s] = total;
        r->pb.capacity[s] = c.capacity[s];
        total += (c.capacity[s] + 31) & ~31ll;
    }
    for (int s = c.n_species; s < CPIC_MAX_SPECIES; ++s) r->pb.base[s] = r->pb.capacity[s] = 0;
    if (total == 0) total = 32;
    r->pb.total = total;
    for (int b = 0; b < 2; ++b) {
        r->pb.cell[b] = P.take<int>(total);
        r->pb.t[b] = P.take<float>((size_t)D * total);
        r->pb.v[b] = P.take<float>((size_t)3 * total);
    }
    r->ctr = P.take<DevCounters>(1);
    r->red = P.take<double>(3 * KRY_BLOCKS + 16);
    r->kry = P.take<KrylovState>(1);
    r->kv = P.take<double>((size_t)2 * r->ncell + ((size_t)3 * r->ncell + 1) / 2);  // r, r^; FP32 p, v, s
    r->ph32 = P.take<float>(r->ncell);
    r->hist = P.take<int>((size_t)c.n_species * r->ncell);
    r->scan = P.take<long long>((size_t)c.n_species * r->ncell + 1);
    r->scan_blocks = P.take<long long>(1025);
    for (int l = 0; l < r->nlevels; ++l) {
        Level& L = r->lev[l];
        L.A32 = P.take<float>((size_t)S * L.ncell);
        L.x32 = P.take<float>(L.ncell);
        L.b32 = P.take<float>(L.ncell);
        L.dinv32 = P.take<float>(L.ncell);
        L.lw = P.take<float>((size_t)2 * L.ncell);     // line relaxation work
        L.pw = P.take<double>((size_t)D * L.ncell);    // operator-induced prolongation weights
        L.pw32 = P.take<float>((size_t)D * L.ncell);
    }
    const Level& Lc = r->lev[r->nlevels - 1];
    long long mm = Lc.ncell + 1;
    r->dense_inv = P.take<double>((size_t)mm * mm);
    r->dense_inv32 = P.take<float>((size_t)mm * mm);
    r->dense_tmp = P.take<double>((size_t)mm * mm);
    r->ticket = P.take<unsigned>(4);
}

void init_geometry_sizes(cpic_run* r, const cpic_config* cfg) {
    r->cfg = *cfg;
    r->D = cfg->dim;
    r->ncell = 1;
    r->nvert = 1;
    r->ncell_h = 1;
    for (int a = 0; a < 3; ++a) {
        r->n[a] = a < r->D ? cfg->n[a] : 1;
        r->nvert_axis[a] = a < r->D ? cfg->n[a] + 1 : 1;
        r->ncell *= r->n[a];
        r->nvert *= r->nvert_axis[a];
        if (a < r->D) r->ncell_h *= r->n[a] + 2;
    }
    // default cycle cap: the V-cycle iteration needs about 50 V-cycles on the 128^3 shell
    // (strong azimuthal coupling near the polar caps; BiCGStab about 22), 10-15 on the 2D maps
    if (r->cfg.mg_max_cycles <= 0) r->cfg.mg_max_cycles = 100;
    if (!(r->cfg.mg_rtol > 0.0)) r->cfg.mg_rtol = 1e-10;
    r->singular = true;
    for (int f = 0; f < 2 * r->D; ++f)
        if (cfg->field_bc[f] == CPIC_BC_DIRICHLET) r->singular = false;
}

int setup_levels(cpic_run* r) {
    int lev_n[MAX_LEVELS][3];
    int nl = 0;
    int st = plan_levels(&r->cfg, lev_n, &nl);
    if (st) return st;
    r->nlevels = nl;
    for (int l = 0; l < nl; ++l) {
        for (int a = 0; a < 3; ++a) r->lev[l].n[a] = lev_n[l][a];
        r->lev[l].ncell = (long long)lev_n[l][0] * lev_n[l][1] * lev_n[l][2];
        r->lev[l].cross = 0;
    }
    return CPIC_OK;
}

__global__ void set_count_kernel(DevCounters* ctr, int s, long long n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctr->count[s] = n;
        ctr->alive[s] = n;
    }
}

// Loaded particles with a cell index outside the grid, an offset outside [0, 1) or a
// non-finite velocity would make the mover read outside its vertex tables: they are
// turned into dead slots and counted as dropped.
__global__ void validate_load_kernel(int D, int n0, int n1, int n2, int* cell, const float* t, const float* v,
                                     long long T, long long n, DevCounters* ctr, int s) {
    long long bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int w = cell[i];
        if (w < 0) {
            ++bad;
            continue;
        }
        int c0, c1, c2 = 0;
        if (D == 2) {
            c0 = w & 0xFFFF;
            c1 = w >> 16;
        } else {
            c0 = w & 1023;
            c1 = (w >> 10) & 1023;
            c2 = w >> 20;
        }
        bool ok = c0 < n0 && c1 < n1 && (D == 2 || c2 < n2);
        for (int a = 0; a < D; ++a) {
            float x = t[a * T + i];
            ok = ok && (x >= 0.0f) && (x < 1.0f);
        }
        for (int a = 0; a < 3; ++a) ok = ok && isfinite(v[a * T + i]);
        if (!ok) {
            cell[i] = -1;
            ++bad;
        }
    }
    if (bad) {
        atomicAdd((unsigned long long*)&ctr->dropped[s], (unsigned long long)bad);
        atomicAdd((unsigned long long*)&ctr->alive[s], (unsigned long long)(-bad));
    }
}

#define CHECK_RUN(r)                         \
    do {                                     \
        if (!(r)) {                          \
            set_error("run handle is NULL"); \
            return CPIC_ERR_INVALID;         \
        }                                    \
    } while (0)
#define CHECK_MAP(r)                                            \
    do {                                                        \
        if (!(r)->map_set) {                                    \
            set_error("set the map (cpic_set_map_*) first");   \
            return CPIC_ERR_STATE;                              \
        }                                                       \
    } while (0)

// Stable compaction of one species' live slots (cell >= 0) into the other particle buffer
// (free between sorts), for cpic_get_particles: the slots are split into nb contiguous
// ranges; pass 1 counts the live slots of each range, pass 2 turns the counts into
// exclusive offsets, pass 3 writes each range's live particles in slot order.
constexpr int COMPACT_BLOCKS = 1024;

__global__ void compact_count_kernel(const int* cell, long long n, long long chunk, long long* counts) {
    const long long lo = (long long)blockIdx.x * chunk, hi = min(lo + chunk, n);
    int c = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) c += cell[i] >= 0;
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ int part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        counts[blockIdx.x] = t;
    }
}

__global__ void compact_offsets_kernel(long long* counts, int nb) {
    if (threadIdx.x == 0) {  // nb <= 1024 partial counts: one sequential pass
        long long acc = 0;
        for (int b = 0; b < nb; ++b) {
            const long long c = counts[b];
            counts[b] = acc;
            acc += c;
        }
        counts[nb] = acc;
    }
}

__global__ void compact_scatter_kernel(int D, const int* cell, const float* t, const float* v, long long stride,
                                       long long n, long long chunk, const long long* offsets, int* ocell, float* ot,
                                       float* ov, long long ostride) {
    const long long lo = (long long)blockIdx.x * chunk, hi = min(lo + chunk, n);
    __shared__ int warp_tot[32];
    long long dst0 = offsets[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long base = lo; base < hi; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool live = i < hi && cell[i] >= 0;
        const unsigned m = __ballot_sync(0xffffffffu, live);
        if (lane == 0) warp_tot[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            before += w < wid ? warp_tot[w] : 0;
            total += warp_tot[w];
        }
        if (live) {
            const long long d = dst0 + before + __popc(m & ((1u << lane) - 1u));
            ocell[d] = cell[i];
            for (int a = 0; a < D; ++a) ot[a * ostride + d] = t[a * stride + i];
            for (int a = 0; a < 3; ++a) ov[a * ostride + d] = v[a * stride + i];
        }
        dst0 += total;
        __syncthreads();
    }
}

// true for device, managed and page-locked host memory (a copy from it may stay in flight
// after the call returns); false for pageable host memory
bool stream_ordered_source(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged || at.type == cudaMemoryTypeHost;
}

// Drifting-Maxwellian injection (2D): per face segment j the inward unit normal from row 0
// of k averaged over the segment's two vertices (FP64), the inward drift u_j = drift . n_j,
// the one-sided flux density Gamma(u_j) = vth/sqrt(2 pi) exp(-u_j^2/2vth^2) + u_j/2 (1 +
// erf(u_j/(sqrt 2 vth))) times the segment's length (or surface of revolution); inclusive
// prefixes on the device (the segment draw), the total sets the rate.
int drift_setup(cpic_run* r, int s) {
    InjectSpec& q = r->inj[s];
    const int n1 = r->n[0], m = r->n[1], nv0 = n1 + 1;
    const int col = (q.face & 1) ? n1 : 0;
    std::vector<double> X((size_t)r->nvert * 2), k((size_t)r->nvert * 4);
    CPIC_CUDA(cudaMemcpyAsync(X.data(), r->lev[0].X, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaMemcpyAsync(k.data(), r->k64, sizeof(double) * k.size(), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    const double sgn = (q.face & 1) ? -1.0 : 1.0, vth = q.vth;
    std::vector<double> cdf(m);
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
        const size_t v0 = (size_t)col + (size_t)nv0 * j, v1 = v0 + nv0;
        const double g0 = 0.5 * (k[v0 * 4 + 0] + k[v1 * 4 + 0]), g1 = 0.5 * (k[v0 * 4 + 1] + k[v1 * 4 + 1]);
        const double gn = sqrt(g0 * g0 + g1 * g1);
        const double n0 = sgn * g0 / gn, nn1 = sgn * g1 / gn;
        const double u = q.drift[0] * n0 + q.drift[1] * nn1;
        const double gam = vth * (1.0 / sqrt(2.0 * M_PI)) * exp(-u * u / (2.0 * vth * vth)) +
                           0.5 * u * (1.0 + erf(u / (sqrt(2.0) * vth)));
        const double dx = X[v1 * 2] - X[v0 * 2], dy = X[v1 * 2 + 1] - X[v0 * 2 + 1];
        double a = sqrt(dx * dx + dy * dy);
        if (r->cfg.axisymmetric) a = 2.0 * M_PI * (0.5 * (X[v0 * 2] + X[v1 * 2])) * a;
        acc += gam * a;
        cdf[j] = acc;
    }
    CPIC_CUDA(cudaMemcpyAsync(r->dcdf + (size_t)s * m, cdf.data(), sizeof(double) * m, cudaMemcpyHostToDevice, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    q.dtot = acc;
    q.rate = q.density * acc * r->cfg.dt / r->cfg.w[s];
    return CPIC_OK;
}

int after_map(cpic_run* r) {
    int st = launch_geometry(r);
    if (st) return st;
    st = mg_setup(r);
    if (st) return st;
    st = mg_cluster_prepare(r);
    if (st) return st;
    // host-side constants: sum of J_c (singular projection) and face lengths (injection rate),
    // each summed sequentially in index order
    std::vector<double> jc(r->ncell), om(r->ncell);
    CPIC_CUDA(cudaMemcpyAsync(jc.data(), r->lev[0].Jc, sizeof(double) * r->ncell, cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaMemcpyAsync(om.data(), r->lev[0].omega, sizeof(double) * r->ncell, cudaMemcpyDeviceToHost, r->stream));
    std::vector<double> X((size_t)r->nvert * r->D);
    CPIC_CUDA(cudaMemcpyAsync(X.data(), r->lev[0].X, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    const bool axisym = r->cfg.axisymmetric != 0;
    double sj = 0.0, sl = 0.0;
    for (long long c = 0; c < r->ncell; ++c) {
        sj += jc[c];
        // inclusive prefix, for loading uniform in physical space: the cell's volume is J_c,
        // or the ring volume 2 pi Omega_c J_c of an axisymmetric run (2 pi drops out)
        sl += axisym ? om[c] * jc[c] : jc[c];
        jc[c] = sl;
    }
    r->sumJ = sj;
    r->load_total = sl;
    CPIC_CUDA(cudaMemcpyAsync(r->jcdf, jc.data(), sizeof(double) * r->ncell, cudaMemcpyHostToDevice, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));  // jc is a host temporary
    if (axisym) {  // FP32 vertex radius table of the axisymmetric mover (x^1, rounded once)
        std::vector<float> rad(r->nvert);
        for (long long v = 0; v < r->nvert; ++v) rad[v] = (float)X[(size_t)v * 2];
        CPIC_CUDA(cudaMemcpyAsync(r->R32, rad.data(), sizeof(float) * r->nvert, cudaMemcpyHostToDevice, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
    }
    for (int f = 0; f < 6; ++f) r->face_len[f] = 0.0;
    if (r->D == 2 && axisym) {
        // faces normal to axis 0 of an axisymmetric run are surfaces of revolution: segment
        // j has area 2 pi r_mid |dX| (r_mid the mean radius of its two vertices); inclusive
        // prefixes (injection positions) and totals (injection rates)
        const int nv0 = r->n[0] + 1;
        std::vector<double> cdf((size_t)2 * r->n[1]);
        for (int side = 0; side < 2; ++side) {
            const int col = side == 0 ? 0 : r->n[0];
            double acc = 0.0;
            for (int j = 0; j < r->n[1]; ++j) {
                const double* p0 = &X[((size_t)col + (size_t)nv0 * j) * 2];
                const double* p1 = &X[((size_t)col + (size_t)nv0 * (j + 1)) * 2];
                const double dx = p1[0] - p0[0], dy = p1[1] - p0[1];
                acc += 2.0 * M_PI * (0.5 * (p0[0] + p1[0])) * sqrt(dx * dx + dy * dy);
                cdf[(size_t)side * r->n[1] + j] = acc;
            }
            r->face_len[side] = acc;
        }
        CPIC_CUDA(cudaMemcpyAsync(r->fcdf, cdf.data(), sizeof(double) * cdf.size(), cudaMemcpyHostToDevice, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
    } else if (r->D == 2) {
        int nv0 = r->n[0] + 1;
        for (int side = 0; side < 2; ++side) {
            int col = side == 0 ? 0 : r->n[0];
            double acc = 0.0;
            for (int j = 0; j < r->n[1]; ++j) {
                const double* p0 = &X[((size_t)col + (size_t)nv0 * j) * 2];
                const double* p1 = &X[((size_t)col + (size_t)nv0 * (j + 1)) * 2];
                double dx = p1[0] - p0[0], dy = p1[1] - p0[1];
                acc += sqrt(dx * dx + dy * dy);
            }
            r->face_len[side] = acc;
        }
    } else {
        // 3D faces normal to axis 0: quadrilateral face-cell areas 1/2 |(X11 - X00) x (X01 - X10)|
        // in face-cell order j + N2 k, their inclusive prefix (injection positions) and total
        const int nv0 = r->n[0] + 1, nv1 = r->n[1] + 1;
        const long long nf = (long long)r->n[1] * r->n[2];
        std::vector<double> cdf(2 * nf);
        for (int side = 0; side < 2; ++side) {
            const int col = side == 0 ? 0 : r->n[0];
            auto V = [&](int j, int k) { return &X[(((size_t)k * nv1 + j) * nv0 + col) * 3]; };
            double acc = 0.0;
            for (int k = 0; k < r->n[2]; ++k)
                for (int j = 0; j < r->n[1]; ++j) {
                    const double *x00 = V(j, k), *x10 = V(j + 1, k), *x01 = V(j, k + 1), *x11 = V(j + 1, k + 1);
                    const double a0 = x11[0] - x00[0], a1 = x11[1] - x00[1], a2 = x11[2] - x00[2];
                    const double b0 = x01[0] - x10[0], b1 = x01[1] - x10[1], b2 = x01[2] - x10[2];
                    const double cx = a1 * b2 - a2 * b1, cy = a2 * b0 - a0 * b2, cz = a0 * b1 - a1 * b0;
                    acc += 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
                    cdf[side * nf + j + (long long)r->n[1] * k] = acc;
                }
            r->face_len[side] = acc;
        }
        CPIC_CUDA(cudaMemcpyAsync(r->fcdf, cdf.data(), sizeof(double) * cdf.size(), cudaMemcpyHostToDevice, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
    }
    CPIC_CUDA(cudaMemsetAsync(r->lev[0].x, 0, sizeof(double) * r->ncell, r->stream));
    CPIC_CUDA(cudaMemsetAsync(r->G32, 0, sizeof(float) * r->nvert * (r->D == 2 ? 2 : 4), r->stream));
    r->map_set = true;
    invalidate_graphs(r);
    for (int s = 0; s < CPIC_MAX_SPECIES; ++s)
        if (r->inj[s].enabled) {
            const InjectSpec& q = r->inj[s];
            if (q.drifting) {
                if (int e = drift_setup(r, s)) return e;
            } else {
                r->inj[s].rate =
                    (((q.density * q.vth) * (1.0 / sqrt(2.0 * M_PI))) * r->face_len[q.face & 1]) * r->cfg.dt / r->cfg.w[s];
            }
        }
    return CPIC_OK;
}

}  // namespace

void invalidate_graphs(cpic_run* r) {
    for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
            if (r->step_graph_ok[j][i]) cudaGraphExecDestroy(r->step_graph[j][i]);
            r->step_graph_ok[j][i] = false;
        }
}

namespace {

cudaEvent_t pool_event(cpic_run* r) {
    if (!r->prof_pool->empty()) {
        cudaEvent_t e = r->prof_pool->back();
        r->prof_pool->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// runs `fn` as phase `ph`, bracketed by events on the run's stream when profiling
template <class F>
int phase(cpic_run* r, int ph, F fn) {
    if (!r->profiling) return fn();
    cudaEvent_t a = pool_event(r), b = pool_event(r);
    CPIC_CUDA(cudaEventRecord(a, r->stream));
    int st = fn();
    CPIC_CUDA(cudaEventRecord(b, r->stream));
    r->prof_events->push_back({ph, {a, b}});
    return st;
}

// enqueue one step's work (stream order); `sort` selects the cell sort
}  // namespace

bool push2d_batchable(const cpic_run* r) {
    if (r->D != 2 || r->magnetized || r->cfg.axisymmetric) return false;
    for (int f = 0; f < 4; ++f)
        if (r->cfg.particle_bc[f] == CPIC_PBC_REFLECT) return false;
    return true;
}

int enqueue_step_pre(cpic_run* r, bool with_push) {
    int st = launch_vertex_field(r);
    if (!st) st = launch_push_prep(r);
    if (!st && with_push) st = launch_push_kernel(r);
    return st;
}

int enqueue_step_post(cpic_run* r, bool sort, bool fold, bool fused_sort) {
    int st = launch_finalize_step(r);
    if (!st) st = launch_inject(r);
    if (!st && fold) st = launch_fold(r);
    if (!st && sort) st = launch_sort(r, fused_sort);
    return st;
}

// a fused sort step: the push and the injection count the particles' new cells, so the
// sort skips its histogram pass
int begin_counted_step(cpic_run* r) {
    r->count_hist = true;
    CPIC_CUDA(cudaMemsetAsync(r->hist, 0, sizeof(int) * r->cfg.n_species * (size_t)r->ncell, r->stream));
    return CPIC_OK;
}

int enqueue_step(cpic_run* r, bool sort, bool fold, bool fused_sort = false) {
    int st = launch_vertex_field(r);
    if (st) return st;
    if (sort && fused_sort && (st = begin_counted_step(r))) return st;
    st = launch_push(r);
    if (st) return st;
    st = launch_inject(r);
    if (st) return st;
    if (fold) {  // the compact charge grid is read only by the solve and the charge readers
        st = launch_fold(r);
        if (st) return st;
    }
    if (sort) {
        st = launch_sort(r, fused_sort);
        if (st) return st;
    }
    return CPIC_OK;
}

namespace {


}  // namespace

// kernel nodes of a graph (top level; a conditional node's body runs a device-decided
// number of times and is not counted)
int count_kernel_nodes(cudaGraph_t g, int* out) {
    size_t n = 0;
    CPIC_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) CPIC_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        CPIC_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *out = k;
    return CPIC_OK;
}

namespace {

int build_step_graph(cpic_run* r, int with_solve, int with_sort) {
    if (!r->capture_stream) CPIC_CUDA(cudaStreamCreateWithFlags(&r->capture_stream, cudaStreamNonBlocking));
    cudaStream_t saved = r->stream;
    r->stream = r->capture_stream;
    int st = CPIC_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(r->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        r->stream = saved;
        return cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
    }
    // the graph is replayed in any order state: its push reads the device flag, and the host
    // flag is managed around each replay (step_once), not by what capture enqueues
    const bool pending = r->order_pending;
    r->order_pending = false;
    const bool fused = with_sort != 0 && push_fused_ok(r);
    st = enqueue_step(r, with_sort != 0, with_solve != 0, fused);
    r->order_pending = pending;
    r->count_hist = false;
    if (!st && with_solve) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        e = cudaStreamGetCaptureInfo(r->stream, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamGetCaptureInfo", __FILE__, __LINE__);
        else st = mg_capture_solve(r, cg, r->cfg.mg_rtol, r->cfg.mg_max_cycles);
    }
    e = cudaStreamEndCapture(r->stream, &g);
    r->stream = saved;
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    int nk = 0;
    st = count_kernel_nodes(g, &nk);
    if (st) {
        cudaGraphDestroy(g);
        return st;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    r->step_graph[with_solve][with_sort] = ex;
    r->step_graph_ok[with_solve][with_sort] = true;
    r->graph_kernels[with_solve][with_sort] = nk;
    r->graph_sort_fused[with_solve][with_sort] = fused;
    return CPIC_OK;
}

int step_once(cpic_run* r, bool solve) {
    bool sort = r->cfg.sort_interval > 0 && r->steps_since_sort + 1 >= r->cfg.sort_interval;
    if (r->order_pending && !push_fused_ok(r)) {
        if (int e = resolve_order(r)) return e;
    }
    if (!r->profiling) {
        const int wi = sort ? 1 : 0, ws = solve ? 1 : 0;
        if (!r->step_graph_ok[ws][wi]) {
            int st = build_step_graph(r, ws, wi);
            if (st) return st;
        }
        CPIC_CUDA(cudaGraphLaunch(r->step_graph[ws][wi], r->stream));
        g_launches.fetch_add(r->graph_kernels[ws][wi], std::memory_order_relaxed);
        // the replay's push took any pending order; a fused sort at its end leaves a new one
        r->order_pending = sort && r->graph_sort_fused[ws][wi];
        ++r->steps_since_sort;
        if (sort) {
            r->cur_host ^= 1;
            r->steps_since_sort = 0;
        }
        return CPIC_OK;
    }
    // profiled path: the same work launched stream-ordered, bracketed by events; the push
    // phase holds the fused push kernel alone
    const bool fused = sort && push_fused_ok(r);
    int st = phase(r, CPIC_PHASE_FIELD, [&] {
        int q = launch_vertex_field(r);
        if (!q && fused) q = begin_counted_step(r);
        return q ? q : launch_push_prep(r);
    });
    if (st) return st;
    st = phase(r, CPIC_PHASE_PUSH, [&] { return launch_push_kernel(r); });
    if (st) return st;
    st = phase(r, CPIC_PHASE_INJECT, [&] {
        int q = launch_finalize_step(r);
        if (!q) q = launch_inject(r);
        return q || !solve ? q : launch_fold(r);
    });
    if (st) return st;
    if (r->cfg.sort_interval > 0 && ++r->steps_since_sort >= r->cfg.sort_interval) {
        st = phase(r, CPIC_PHASE_SORT, [&] { return launch_sort(r, fused); });
        if (st) return st;
        r->cur_host ^= 1;
        r->steps_since_sort = 0;
    }
    if (!solve) return CPIC_OK;
    return phase(r, CPIC_PHASE_SOLVE,
                 [&] { return mg_solve(r, r->cfg.mg_rtol, r->cfg.mg_max_cycles, true, nullptr, nullptr); });
}

}  // namespace
}  // namespace cpic

using namespace cpic;

extern "C" {

const char* cpic_status_string(int s) {
    switch (s) {
        case CPIC_OK: return "ok";
        case CPIC_ERR_INVALID: return "invalid argument or configuration";
        case CPIC_ERR_OOM: return "out of device memory";
        case CPIC_ERR_CUDA: return "CUDA runtime error";
        case CPIC_ERR_NOT_CONVERGED: return "field solve did not converge";
        case CPIC_ERR_TIMEOUT: return "bounded device wait ran out";
        case CPIC_ERR_NONFINITE: return "non-finite particle positions";
        case CPIC_ERR_BUSY: return "not done yet";
        case CPIC_ERR_STATE: return "call out of order";
        case CPIC_ERR_CAPACITY: return "particle capacity exhausted";
        case CPIC_ERR_NOT_BUILT: return "not built in this version";
        case CPIC_ERR_CANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

const char* cpic_last_error(void) { return g_err; }

int64_t cpic_kernel_launches(void) { return g_launches.load(); }

int cpic_abi_version(void) { return CPIC_ABI_VERSION; }

int cpic_query_footprint(const cpic_config* cfg, size_t* bytes) {
    int st = validate(cfg);
    if (st) return st;
    if (!bytes) {
        set_error("bytes is NULL");
        return CPIC_ERR_INVALID;
    }
    cpic_run tmp;
    memset(&tmp, 0, sizeof(tmp));
    init_geometry_sizes(&tmp, cfg);
    st = setup_levels(&tmp);
    if (st) return st;
    Planner P;
    plan(&tmp, P);
    *bytes = P.used + 256;
    return CPIC_OK;
}

int cpic_get_config(const cpic_run* r, cpic_config* out) {
    if (!r || !out) {
        set_error("get_config: NULL run or out");
        return CPIC_ERR_INVALID;
    }
    *out = r->cfg;
    return CPIC_OK;
}

int cpic_set_sort_interval(cpic_run* r, int interval) {
    if (!r || interval < 0) {
        set_error("set_sort_interval: NULL run or negative interval");
        return CPIC_ERR_INVALID;
    }
    r->cfg.sort_interval = interval;
    return CPIC_OK;
}

int cpic_set_solver(cpic_run* r, int solver) {
    CHECK_RUN(r);
    if (solver != CPIC_SOLVER_MG && solver != CPIC_SOLVER_BICGSTAB) {
        set_error("set_solver: unknown solver %d", solver);
        return CPIC_ERR_INVALID;
    }
    if (r->solver != solver) {
        r->solver = solver;
        invalidate_graphs(r);  // captured steps hold the solve
    }
    return CPIC_OK;
}

int cpic_set_multigrid(cpic_run* r, int coarse, int interpolation, int smoother) {
    CHECK_RUN(r);
    if ((coarse != CPIC_MG_COARSE_REDISCRETIZED && coarse != CPIC_MG_COARSE_GALERKIN) ||
        (interpolation != CPIC_MG_INTERP_BILINEAR && interpolation != CPIC_MG_INTERP_OPERATOR) ||
        (smoother != CPIC_MG_SMOOTH_POINT && smoother != CPIC_MG_SMOOTH_LINE)) {
        set_error("set_multigrid: unknown coarse operator %d, interpolation %d or smoother %d", coarse, interpolation,
                  smoother);
        return CPIC_ERR_INVALID;
    }
    if (r->mg_coarse == coarse && r->mg_interp == interpolation && r->mg_smoother == smoother) return CPIC_OK;
    r->mg_coarse = coarse;
    r->mg_interp = interpolation;
    r->mg_smoother = smoother;
    invalidate_graphs(r);
    if (!r->map_set) return CPIC_OK;  // taken up when the map is set
    int st = mg_setup(r);
    if (!st) st = mg_cluster_prepare(r);
    return st;
}

int cpic_set_push_tuning(cpic_run* r, int chunk, int tile) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (chunk < 0 || chunk > (1 << 20) || (chunk % 256) != 0 || (tile != 0 && tile != 1)) {
        set_error("set_push_tuning: chunk must be 0 or a multiple of 256 up to 2^20, tile 0 or 1 (got %d, %d)", chunk,
                  tile);
        return CPIC_ERR_INVALID;
    }
    if (r->push_chunk != chunk || r->push_tile != tile) {
        r->push_chunk = chunk;
        r->push_tile = tile;
        invalidate_graphs(r);  // captured steps hold the push parameters
    }
    return CPIC_OK;
}

int cpic_create(const cpic_config* cfg, void* arena, size_t arena_bytes, void* stream, cpic_run** out) {
    if (!out) {
        set_error("out is NULL");
        return CPIC_ERR_INVALID;
    }
    *out = nullptr;
    int st = validate(cfg);
    if (st) return st;
    cpic_run* r = new cpic_run;
    memset(r, 0, sizeof(*r));
    r->solver = CPIC_SOLVER_BICGSTAB;
    r->floating_face = -1;
    r->kick_fraction = 1.0;
    r->push_tile = 1;
    init_geometry_sizes(r, cfg);
    st = setup_levels(r);
    if (st) {
        delete r;
        return st;
    }
    r->stream = (cudaStream_t)stream;
    Planner dry;
    plan(r, dry);
    size_t need = dry.used + 256;
    if (arena) {
        if (arena_bytes < need || (reinterpret_cast<uintptr_t>(arena) & 255)) {
            set_error("arena too small or misaligned: need %zu bytes, 256-byte aligned", need);
            delete r;
            return CPIC_ERR_OOM;
        }
        r->arena = (char*)arena;
        r->own_memory = false;
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
            delete r;
            return CPIC_ERR_OOM;
        }
        r->arena = (char*)p;
        r->own_memory = true;
    }
    r->arena_bytes = need;
    Planner P;
    P.base = r->arena;
    plan(r, P);
    cudaError_t e = cudaMemsetAsync(r->ctr, 0, sizeof(DevCounters), r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->charge, 0, sizeof(unsigned long long) * r->ncell * cfg->n_species, r->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(r->charge_h, 0, sizeof(unsigned long long) * r->ncell_h * cfg->n_species, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->pb.cell[0], 0xff, sizeof(int) * r->pb.total, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->pb.cell[1], 0xff, sizeof(int) * r->pb.total, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->ticket, 0, sizeof(unsigned) * 4, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->kry, 0, sizeof(KrylovState), r->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(r->collect, 0, sizeof(unsigned long long) * cfg->n_species * 2 * r->ncollect, r->stream);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "initial memset", __FILE__, __LINE__);
        if (r->own_memory) cudaFree(r->arena);
        delete r;
        return st;
    }
    r->prof_events = new std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>();
    r->prof_pool = new std::vector<cudaEvent_t>();
    *out = r;
    return CPIC_OK;
}

int cpic_destroy(cpic_run* r) {
    if (!r) return CPIC_OK;
    cudaError_t e = cudaStreamSynchronize(r->stream);
    if (r->own_memory) cudaFree(r->arena);
    for (auto& pe : *r->prof_events) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (cudaEvent_t ev : *r->prof_pool) cudaEventDestroy(ev);
    invalidate_graphs(r);
    if (r->capture_stream) cudaStreamDestroy(r->capture_stream);
    delete r->prof_events;
    delete r->prof_pool;
    delete r;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    return CPIC_OK;
}

int cpic_set_stream(cpic_run* r, void* stream) {
    CHECK_RUN(r);
    r->stream = (cudaStream_t)stream;
    return CPIC_OK;
}

int cpic_set_map_vertices(cpic_run* r, const double* xyz) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (!xyz) {
        set_error("xyz is NULL");
        return CPIC_ERR_INVALID;
    }
    CPIC_CUDA(cudaMemcpyAsync(r->lev[0].X, xyz, sizeof(double) * r->nvert * r->D, cudaMemcpyDefault, r->stream));
    return after_map(r);
}

int cpic_set_map_analytic(cpic_run* r, int map_id, const double* params, int nparams) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    int need = map_id == CPIC_MAP_SHELL ? 3 : (map_id == CPIC_MAP_SINE ? 1 : 2);
    bool dim_ok = map_id == CPIC_MAP_SHELL ? r->D == 3 : r->D == 2;
    if (map_id < CPIC_MAP_SINE || map_id > CPIC_MAP_SHELL || !dim_ok || !params || nparams < need) {
        set_error("bad analytic map %d for dim %d (needs %d parameters)", map_id, r->D, need);
        return CPIC_ERR_INVALID;
    }
    int st = launch_map_analytic(r, map_id, params, nparams);
    if (st) return st;
    return after_map(r);
}

int cpic_load_particles(cpic_run* r, int sp, int64_t n, const int32_t* cell, const float* t, const float* v) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (sp < 0 || sp >= r->cfg.n_species || n < 0 || n > r->pb.capacity[sp] || (n > 0 && (!cell || !t || !v))) {
        set_error("load_particles: bad species, count or pointers (n = %lld, capacity = %lld)", (long long)n,
                  sp >= 0 && sp < CPIC_MAX_SPECIES ? (long long)r->pb.capacity[sp] : -1ll);
        return CPIC_ERR_INVALID;
    }
    int b = r->cur_host;
    long long base = r->pb.base[sp], T = r->pb.total;
    if (n > 0) {
        CPIC_CUDA(cudaMemcpyAsync(r->pb.cell[b] + base, cell, sizeof(int) * n, cudaMemcpyDefault, r->stream));
        for (int a = 0; a < r->D; ++a)
            CPIC_CUDA(cudaMemcpyAsync(r->pb.t[b] + a * T + base, t + a * n, sizeof(float) * n, cudaMemcpyDefault, r->stream));
        for (int a = 0; a < 3; ++a)
            CPIC_CUDA(cudaMemcpyAsync(r->pb.v[b] + a * T + base, v + a * n, sizeof(float) * n, cudaMemcpyDefault, r->stream));
    }
    set_count_kernel<<<1, 32, 0, r->stream>>>(r->ctr, sp, n);
    CPIC_CHECK_LAUNCH();
    if (n > 0) {
        long long blocks = (n + 255) / 256;
        if (blocks > 4LL * device_sm_count()) blocks = 4LL * device_sm_count();
        validate_load_kernel<<<(int)blocks, 256, 0, r->stream>>>(r->D, r->n[0], r->n[1], r->n[2], r->pb.cell[b] + base,
                                                                 r->pb.t[b] + base, r->pb.v[b] + base, T, n, r->ctr, sp);
        CPIC_CHECK_LAUNCH();
    }
    // copies from pageable host memory must be complete before the caller may free or reuse
    // it; device and page-locked inputs stay stream-ordered (asynchronous)
    if (n > 0 && !(stream_ordered_source(cell) && stream_ordered_source(t) && stream_ordered_source(v)))
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_load_maxwellian(cpic_run* r, int sp, int64_t n, double vth, const double* drift, uint64_t seed) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    CHECK_MAP(r);
    if (sp < 0 || sp >= r->cfg.n_species || n < 0 || n > r->pb.capacity[sp] || !(vth >= 0.0)) {
        set_error("load_maxwellian: bad species, count (n = %lld) or vth", (long long)n);
        return CPIC_ERR_INVALID;
    }
    return launch_load_maxwellian(r, sp, n, vth, drift, seed);
}

int cpic_get_particles(cpic_run* r, int sp, int64_t room, int64_t* n, int32_t* cell, float* t, float* v) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (sp < 0 || sp >= r->cfg.n_species || !n) {
        set_error("get_particles: bad species or NULL count");
        return CPIC_ERR_INVALID;
    }
    DevCounters h;
    CPIC_CUDA(cudaMemcpyAsync(&h, r->ctr, sizeof(h), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    const long long cnt = h.count[sp], live = h.alive[sp];
    const int b = h.cur;
    const long long base = r->pb.base[sp], T = r->pb.total;
    *n = live;
    if (live > room) {
        set_error("get_particles: room %lld < %lld live particles", (long long)room, live);
        return CPIC_ERR_INVALID;
    }
    if (live == 0) return CPIC_OK;
    if (!cell || !t || !v) {
        set_error("get_particles: NULL output array");
        return CPIC_ERR_INVALID;
    }
    const int* src_c = r->pb.cell[b] + base;
    const float* src_t = r->pb.t[b] + base;
    const float* src_v = r->pb.v[b] + base;
    long long stride = T;
    if (live < cnt) {  // dead slots since the last sort: compact on the device first
        const int o = 1 - b;
        long long chunk = (cnt + COMPACT_BLOCKS - 1) / COMPACT_BLOCKS;
        if (chunk < 1024) chunk = 1024;
        const int nb = (int)((cnt + chunk - 1) / chunk);
        compact_count_kernel<<<nb, 256, 0, r->stream>>>(src_c, cnt, chunk, r->scan_blocks);
        CPIC_CHECK_LAUNCH();
        compact_offsets_kernel<<<1, 32, 0, r->stream>>>(r->scan_blocks, nb);
        CPIC_CHECK_LAUNCH();
        compact_scatter_kernel<<<nb, 256, 0, r->stream>>>(r->D, src_c, src_t, src_v, T, cnt, chunk, r->scan_blocks,
                                                         r->pb.cell[o] + base, r->pb.t[o] + base, r->pb.v[o] + base,
                                                         T);
        CPIC_CHECK_LAUNCH();
        src_c = r->pb.cell[o] + base;
        src_t = r->pb.t[o] + base;
        src_v = r->pb.v[o] + base;
        long long got = 0;  // the compaction's own count must be the live counter
        CPIC_CUDA(cudaMemcpyAsync(&got, r->scan_blocks + nb, sizeof(got), cudaMemcpyDeviceToHost, r->stream));
        CPIC_CUDA(cudaStreamSynchronize(r->stream));
        if (got != live) {
            set_error("get_particles: %lld live slots but the live counter is %lld", got, live);
            return CPIC_ERR_STATE;
        }
    }
    // one copy per array into the caller's buffers (host or device)
    CPIC_CUDA(cudaMemcpyAsync(cell, src_c, sizeof(int) * live, cudaMemcpyDefault, r->stream));
    for (int a = 0; a < r->D; ++a)
        CPIC_CUDA(cudaMemcpyAsync(t + a * live, src_t + a * stride, sizeof(float) * live, cudaMemcpyDefault, r->stream));
    for (int a = 0; a < 3; ++a)
        CPIC_CUDA(cudaMemcpyAsync(v + a * live, src_v + a * stride, sizeof(float) * live, cudaMemcpyDefault, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_set_magnetic_field(cpic_run* r, const double* B) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    double b[3] = {0.0, 0.0, 0.0};
    if (B)
        for (int a = 0; a < 3; ++a) b[a] = B[a];
    for (int a = 0; a < 3; ++a)
        if (!(b[a] == b[a]) || b[a] > 1e30 || b[a] < -1e30) {
            set_error("set_magnetic_field: non-finite component");
            return CPIC_ERR_INVALID;
        }
    if (r->cfg.axisymmetric && (b[0] != 0.0 || b[2] != 0.0)) {
        set_error("set_magnetic_field: an axisymmetric run takes a field along the axis (component 1) only");
        return CPIC_ERR_INVALID;
    }
    for (int a = 0; a < 3; ++a) r->B0[a] = b[a];
    r->magnetized = b[0] != 0.0 || b[1] != 0.0 || b[2] != 0.0;
    invalidate_graphs(r);
    return CPIC_OK;
}

int cpic_set_gyro_integrator(cpic_run* r, int kind) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (kind != CPIC_GYRO_BORIS && kind != CPIC_GYRO_CYCLOTRONIC) {
        set_error("set_gyro_integrator: CPIC_GYRO_BORIS or CPIC_GYRO_CYCLOTRONIC");
        return CPIC_ERR_INVALID;
    }
    r->gyro_kind = kind;
    invalidate_graphs(r);
    return CPIC_OK;
}

int cpic_get_collection(cpic_run* r, int sp, int face, int64_t* counts, int64_t n) {
    CHECK_RUN(r);
    if (sp < 0 || sp >= r->cfg.n_species || (face != 0 && face != 1) || !counts || n != r->ncollect) {
        set_error("get_collection: bad species, face, NULL array or size %lld (the face has %d cells)", (long long)n,
                  r->ncollect);
        return CPIC_ERR_INVALID;
    }
    CPIC_CUDA(cudaMemcpyAsync(counts, r->collect + ((size_t)sp * 2 + face) * r->ncollect,
                              sizeof(unsigned long long) * r->ncollect, cudaMemcpyDefault, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_set_floating(cpic_run* r, int face, double charge0) {
    CHECK_RUN(r);
    CHECK_MAP(r);
    if (r->initialized) {
        set_error("set_floating: call before cpic_initialize");
        return CPIC_ERR_STATE;
    }
    if ((face != 0 && face != 1) || r->cfg.field_bc[face] != CPIC_BC_DIRICHLET || !(charge0 == charge0)) {
        set_error("set_floating: a Dirichlet face normal to axis 0");
        return CPIC_ERR_INVALID;
    }
    r->floating_face = -1;  // no conductor correction while psi is solved
    double saved[6];
    memcpy(saved, r->cfg.field_bc_value, sizeof(saved));
    const double bg = r->cfg.background;
    // psi: charge-free space, this face at potential 1, every other Dirichlet face at 0
    for (int f = 0; f < 6; ++f)
        if (r->cfg.field_bc[f] == CPIC_BC_DIRICHLET) r->cfg.field_bc_value[f] = f == face ? 1.0 : 0.0;
    r->cfg.background = 0.0;
    int st = mg_setup(r);
    if (!st) {
        CPIC_CUDA(cudaMemsetAsync(r->charge, 0, sizeof(unsigned long long) * r->cfg.n_species * r->ncell, r->stream));
        CPIC_CUDA(cudaMemsetAsync(r->lev[0].x, 0, sizeof(double) * r->ncell, r->stream));
        st = mg_solve(r, 1e-13, 400, true, nullptr, nullptr);
    }
    if (!st) {
        CPIC_CUDA(cudaMemcpyAsync(r->psi, r->lev[0].x, sizeof(double) * r->ncell, cudaMemcpyDeviceToDevice, r->stream));
        r->floating_face = face;
        r->float_q0 = charge0;
        st = launch_floating_capacity(r);
    }
    // the run's own solves: the conductor's face at 0 (its potential is added after each solve)
    memcpy(r->cfg.field_bc_value, saved, sizeof(saved));
    r->cfg.field_bc_value[face] = 0.0;
    r->cfg.background = bg;
    if (!st) st = mg_setup(r);
    if (st) {
        r->floating_face = -1;
        return st;
    }
    CPIC_CUDA(cudaMemsetAsync(r->lev[0].x, 0, sizeof(double) * r->ncell, r->stream));
    invalidate_graphs(r);
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_set_injection(cpic_run* r, int sp, int face, double density, double vth, const double* drift, uint64_t seed) {
    CHECK_RUN(r);
    if (sp < 0 || sp >= r->cfg.n_species || (face != 0 && face != 1) ||
        r->cfg.particle_bc[face] != CPIC_PBC_ABSORB || !(density >= 0.0) || !(vth > 0.0)) {
        set_error("set_injection: faces normal to axis 0 with absorbing particle boundaries only");
        return CPIC_ERR_INVALID;
    }
    // the injection kernels wrap the last axis; an axisymmetric face ends on the z axis
    // instead (its draws stay on the face and the partial push drops what leaves it)
    if ((r->D == 2 && !r->cfg.axisymmetric && r->cfg.particle_bc[2] != CPIC_PBC_PERIODIC) ||
        (r->D == 3 && r->cfg.particle_bc[4] != CPIC_PBC_PERIODIC)) {
        set_error("set_injection: the last logical axis must be periodic (or the run axisymmetric)");
        return CPIC_ERR_INVALID;
    }
    const bool inplane = drift && (drift[0] != 0.0 || drift[1] != 0.0 || (r->D == 3 && drift[2] != 0.0));
    if (r->D == 3 && inplane) {
        set_error("set_injection: a drifting Maxwellian flux is built for 2D faces only");
        return CPIC_ERR_NOT_BUILT;
    }
    InjectSpec& q = r->inj[sp];
    q.enabled = density > 0.0;
    q.face = face;
    q.density = density;
    q.vth = vth;
    for (int a = 0; a < 3; ++a) q.drift[a] = drift ? drift[a] : 0.0;
    q.seed = seed;
    q.drifting = inplane ? 1 : 0;
    q.dtot = 0.0;
    q.rate = 0.0;
    if (r->map_set) {
        if (q.drifting) {
            if (int e = drift_setup(r, sp)) return e;
        } else {
            q.rate = (((density * vth) * (1.0 / sqrt(2.0 * M_PI))) * r->face_len[face & 1]) * r->cfg.dt / r->cfg.w[sp];
        }
    }
    invalidate_graphs(r);
    return CPIC_OK;
}

int cpic_initialize(cpic_run* r) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    CHECK_MAP(r);
    int st = launch_deposit(r);
    if (!st) st = launch_fold(r);
    if (st) return st;
    st = mg_solve(r, r->cfg.mg_rtol, r->cfg.mg_max_cycles, false, nullptr, nullptr);
    if (st) return st;
    st = launch_vertex_field(r);
    if (st) return st;
    st = launch_kick(r, -0.5);
    if (st) return st;
    r->initialized = true;
    return CPIC_OK;
}

int cpic_step(cpic_run* r, int nsteps) {
    CHECK_RUN(r);
    CHECK_MAP(r);
    for (int i = 0; i < nsteps; ++i) {
        int st = step_once(r, true);
        if (st) return st;
    }
    return CPIC_OK;
}

int cpic_step_particles(cpic_run* r, int nsteps) {
    CHECK_RUN(r);
    CHECK_MAP(r);
    for (int i = 0; i < nsteps; ++i) {
        int st = step_once(r, false);
        if (st) return st;
    }
    return CPIC_OK;
}

int cpic_vertex_field(cpic_run* r) {
    CHECK_RUN(r);
    CHECK_MAP(r);
    return launch_vertex_field(r);
}

int cpic_push(cpic_run* r) {
    CHECK_RUN(r);
    CHECK_MAP(r);
    int st = launch_push(r);
    return st ? st : launch_fold(r);
}

int cpic_deposit(cpic_run* r) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    CHECK_MAP(r);
    int st = launch_deposit(r);
    return st ? st : launch_fold(r);
}

int cpic_kick(cpic_run* r, double fraction) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    CHECK_MAP(r);
    return launch_kick(r, fraction);
}

int cpic_inject(cpic_run* r) {
    CHECK_RUN(r);
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    CHECK_MAP(r);
    int st = launch_inject(r);
    return st ? st : launch_fold(r);
}

int cpic_sort(cpic_run* r) {
    CHECK_RUN(r);
    int st = launch_sort(r);
    if (st) return st;
    r->cur_host ^= 1;
    r->steps_since_sort = 0;
    return CPIC_OK;
}

int cpic_solve_field(cpic_run* r, double rtol, int max_cycles, int* cycles, double* residual) {
    CHECK_RUN(r);
    CHECK_MAP(r);
    if (!(rtol > 0.0) || max_cycles < 0) {
        set_error("solve_field: rtol must be > 0 and max_cycles >= 0");
        return CPIC_ERR_INVALID;
    }
    int c = 0;
    double res = 0.0;
    int st = mg_solve(r, rtol, max_cycles, true, &c, &res);
    if (cycles) *cycles = c;
    if (residual) *residual = res;
    return st;
}

int cpic_get_diag(cpic_run* r, cpic_diag* out) {
    CHECK_RUN(r);
    if (!out) {
        set_error("out is NULL");
        return CPIC_ERR_INVALID;
    }
    DevCounters h;
    CPIC_CUDA(cudaMemcpyAsync(&h, r->ctr, sizeof(h), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    memset(out, 0, sizeof(*out));
    out->step = h.step;
    out->field_energy = h.field_energy;
    double ke = 0.0;
    for (int s = 0; s < r->cfg.n_species; ++s) {
        ke += 0.5 * r->cfg.m[s] * r->cfg.w[s] * ldexp((double)h.ke_fp[s], -KE_BITS);
        out->n_particles[s] = h.alive[s];
        for (int f = 0; f < 6; ++f) out->absorbed[s][f] = h.absorbed[s][f];
        out->injected[s] = h.injected[s];
        out->dropped[s] = h.dropped[s];
    }
    out->kinetic_energy = ke;
    out->nonfinite = h.nonfinite;
    out->mg_cycles = h.mg_cycles;
    out->mg_residual = h.mg_residual;
    out->pc_face_only = r->pc_face_only;
    out->object_potential = r->floating_face >= 0 ? h.object_potential : 0.0;
    out->object_charge = r->floating_face >= 0 ? h.object_charge : 0.0;
    return CPIC_OK;
}

int cpic_get_phi(cpic_run* r, double* phi) {
    CHECK_RUN(r);
    CPIC_CUDA(cudaMemcpyAsync(phi, r->lev[0].x, sizeof(double) * r->ncell, cudaMemcpyDefault, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_set_phi(cpic_run* r, const double* phi) {
    CHECK_RUN(r);
    CPIC_CUDA(cudaMemcpyAsync(r->lev[0].x, phi, sizeof(double) * r->ncell, cudaMemcpyDefault, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_get_charge(cpic_run* r, int sp, int64_t* counts) {
    CHECK_RUN(r);
    if (sp < 0 || sp >= r->cfg.n_species) {
        set_error("bad species");
        return CPIC_ERR_INVALID;
    }
    int st = launch_fold(r);  // fixed-field particle steps leave the charge in the padded grid
    if (st) return st;
    CPIC_CUDA(cudaMemcpyAsync(counts, r->charge + (long long)sp * r->ncell, sizeof(int64_t) * r->ncell, cudaMemcpyDefault,
                              r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_get_vertex_tables(cpic_run* r, float* k, float* g) {
    CHECK_RUN(r);
    const int D = r->D;
    const long long nv = r->nvert;
    // the device tables are padded records (2D: k one float4, G one float2 per vertex; 3D: k
    // and G in three float4 per vertex, G also as one float4); the output is unpadded
    std::vector<float> kraw, graw;
    if (k) {
        kraw.resize((size_t)nv * (D == 2 ? 4 : 12));
        CPIC_CUDA(cudaMemcpyAsync(kraw.data(), r->K32, sizeof(float) * kraw.size(), cudaMemcpyDeviceToHost, r->stream));
    }
    if (g) {
        graw.resize((size_t)nv * (D == 2 ? 2 : 4));
        CPIC_CUDA(cudaMemcpyAsync(graw.data(), r->G32, sizeof(float) * graw.size(), cudaMemcpyDeviceToHost, r->stream));
    }
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    if (k) {
        std::vector<float> out((size_t)nv * D * D);
        for (long long v = 0; v < nv; ++v)
            for (int q = 0; q < D * D; ++q)
                out[(size_t)v * D * D + q] = kraw[(size_t)v * (D == 2 ? 4 : 12) + q];
        CPIC_CUDA(cudaMemcpy(k, out.data(), sizeof(float) * out.size(), cudaMemcpyDefault));
    }
    if (g) {
        std::vector<float> out((size_t)nv * D);
        const int gw = D == 2 ? 2 : 4;
        for (long long v = 0; v < nv; ++v)
            for (int a = 0; a < D; ++a) out[(size_t)v * D + a] = graw[(size_t)v * gw + a];
        CPIC_CUDA(cudaMemcpy(g, out.data(), sizeof(float) * out.size(), cudaMemcpyDefault));
    }
    return CPIC_OK;
}

int cpic_get_geometry(cpic_run* r, double* k, double* jc) {
    CHECK_RUN(r);
    if (k) CPIC_CUDA(cudaMemcpyAsync(k, r->k64, sizeof(double) * r->nvert * r->D * r->D, cudaMemcpyDefault, r->stream));
    if (jc) CPIC_CUDA(cudaMemcpyAsync(jc, r->lev[0].Jc, sizeof(double) * r->ncell, cudaMemcpyDefault, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_synchronize(cpic_run* r) {
    CHECK_RUN(r);
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    return CPIC_OK;
}

int cpic_profile(cpic_run* r, int enable) {
    CHECK_RUN(r);
    r->profiling = enable != 0;
    return CPIC_OK;
}

int cpic_profile_read(cpic_run* r, double* ms, int64_t* count) {
    CHECK_RUN(r);
    if (!ms) {
        set_error("ms is NULL");
        return CPIC_ERR_INVALID;
    }
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    for (int p = 0; p < CPIC_NPHASES; ++p) {
        ms[p] = 0.0;
        if (count) count[p] = 0;
    }
    for (auto& pe : *r->prof_events) {
        float t = 0.0f;
        CPIC_CUDA(cudaEventElapsedTime(&t, pe.second.first, pe.second.second));
        ms[pe.first] += t;
        if (count) count[pe.first] += 1;
        r->prof_pool->push_back(pe.second.first);
        r->prof_pool->push_back(pe.second.second);
    }
    r->prof_events->clear();
    return CPIC_OK;
}

}  // extern "C"
