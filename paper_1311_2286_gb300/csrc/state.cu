// The run's dynamic state — particles of the current buffer, counters and diagnostics,
// the potential, and the host's sort phase — copied out and back in, for the sort-interval
// autotuner (a device snapshot around its trial steps) and for checkpoint files.
//
// Checkpoint file (host byte order, all integers little-endian on the supported hosts):
//   "CPICCKP1", u32 version, cpic_config, u64 nvert, f64 vertex map [nvert][D],
//   InjectSpec[CPIC_MAX_SPECIES], DevCounters, i32 steps_since_sort, i32 floating face,
//   f64 its initial charge, f64 B0[3], i32 gyro integrator, i32 multigrid coarse operator,
//   i32 interpolation, i32 smoother, u64 collection tally [species][2][face cells],
//   f64 phi [ncell],
//   per species: i64 count, i32 cell [count], f32 t [D][count], f32 v [3][count].
// A restored run is created from the stored configuration and vertex map (the same metric
// and multigrid hierarchy bit for bit), then takes the stored particles, counters, potential
// and injection sources, so stepping it continues the saved run exactly.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "internal.cuh"

namespace cpic {
namespace {

constexpr char kMagic[8] = {'C', 'P', 'I', 'C', 'C', 'K', 'P', '1'};
constexpr unsigned kVersion = 4;  // 2: floating conductor, 3: magnetic field, 4: gyro integrator,
                                  // multigrid components and the collection tally

size_t snapshot_bytes(const cpic_run* r) {
    size_t b = sizeof(DevCounters) + sizeof(double) * (size_t)r->ncell +
               sizeof(unsigned long long) * (size_t)r->cfg.n_species * 2 * r->ncollect;
    for (int s = 0; s < r->cfg.n_species; ++s) b += (size_t)r->pb.capacity[s] * (4 + 4 * r->D + 12);
    return b + 256;
}

// direction: true = run -> buf, false = buf -> run (device to device, on the run's stream)
int snapshot_copy(cpic_run* r, char* buf, bool save, int buffer) {
    const long long T = r->pb.total;
    size_t off = 0;
    auto cp = [&](void* dev, size_t bytes) -> int {
        void* dst = save ? (void*)(buf + off) : dev;
        const void* src = save ? (const void*)dev : (const void*)(buf + off);
        off += bytes;
        if (!bytes) return CPIC_OK;
        CPIC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, r->stream));
        return CPIC_OK;
    };
    int st = cp(r->ctr, sizeof(DevCounters));
    if (!st) st = cp(r->lev[0].x, sizeof(double) * (size_t)r->ncell);
    if (!st) st = cp(r->collect, sizeof(unsigned long long) * (size_t)r->cfg.n_species * 2 * r->ncollect);
    for (int s = 0; !st && s < r->cfg.n_species; ++s) {
        const long long b0 = r->pb.base[s], cap = r->pb.capacity[s];
        st = cp(r->pb.cell[buffer] + b0, sizeof(int) * cap);
        for (int a = 0; !st && a < r->D; ++a) st = cp(r->pb.t[buffer] + a * T + b0, sizeof(float) * cap);
        for (int a = 0; !st && a < 3; ++a) st = cp(r->pb.v[buffer] + a * T + b0, sizeof(float) * cap);
    }
    return st;
}

template <class T>
bool wr(FILE* f, const T* p, size_t n) {
    return n == 0 || fwrite(p, sizeof(T), n, f) == n;
}
template <class T>
bool rd(FILE* f, T* p, size_t n) {
    return n == 0 || fread(p, sizeof(T), n, f) == n;
}

}  // namespace
}  // namespace cpic

using namespace cpic;

extern "C" {

namespace {

// One autotuner trial with the run's current settings: a warm-up sort cycle (captures the
// graphs), then whole sort cycles of at least trial_steps fixed-field particle steps timed
// with CUDA events; afterwards the run's particles go back to the snapshot.
int tune_trial(cpic_run* r, char* buf, int saved_cur, int trial_steps, cudaEvent_t a, cudaEvent_t b, float* ms_per_step) {
    const int S = r->cfg.sort_interval > 0 ? r->cfg.sort_interval : 1;
    r->steps_since_sort = 0;
    int nsteps = trial_steps < S ? S : trial_steps;
    nsteps = (nsteps + S - 1) / S * S;
    int st = cpic_step_particles(r, S);
    if (!st && cudaEventRecord(a, r->stream) != cudaSuccess) st = CPIC_ERR_CUDA;
    if (!st) st = cpic_step_particles(r, nsteps);
    if (!st && cudaEventRecord(b, r->stream) != cudaSuccess) st = CPIC_ERR_CUDA;
    if (!st && cudaEventSynchronize(b) != cudaSuccess) st = CPIC_ERR_CUDA;
    float ms = 0.0f;
    if (!st) cudaEventElapsedTime(&ms, a, b);
    *ms_per_step = ms / nsteps;
    if (!st) st = snapshot_copy(r, buf, false, saved_cur);  // particles back to their buffer
    r->cur_host = saved_cur;
    r->order_pending = false;  // the snapshot was taken with the particles in slot order
    return st;
}

}  // namespace

int cpic_autotune(cpic_run* r, int trial_steps, cpic_tuning* out) {
    if (!r || !out || trial_steps < 1) {
        set_error("autotune: NULL run/out or trial_steps < 1");
        return CPIC_ERR_INVALID;
    }
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (!r->map_set) {
        set_error("autotune: the run has no map yet");
        return CPIC_ERR_STATE;
    }
    memset(out, 0, sizeof(*out));
    const int intervals[CPIC_TUNE_CANDIDATES] = {1, 2, 4, 8, 16};
    const int chunks[CPIC_TUNE_CANDIDATES] = {0, 1024, 2048, 4096, 8192};
    char* buf = nullptr;
    const size_t bytes = snapshot_bytes(r);
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) {
        set_error("autotune: cudaMalloc(%zu) for the snapshot failed", bytes);
        return CPIC_ERR_OOM;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int saved_interval = r->cfg.sort_interval, saved_since = r->steps_since_sort, saved_cur = r->cur_host;
    const int saved_chunk = r->push_chunk, saved_tile = r->push_tile;
    int st = snapshot_copy(r, buf, true, saved_cur);
    // 1. sort interval
    int best = saved_interval > 0 ? saved_interval : 4;
    float best_ms = 0.0f;
    for (int c = 0; !st && c < CPIC_TUNE_CANDIDATES; ++c) {
        r->cfg.sort_interval = intervals[c];
        out->interval[c] = intervals[c];
        st = tune_trial(r, buf, saved_cur, trial_steps, a, b, &out->ms_per_step[c]);
        if (!st && (best_ms == 0.0f || out->ms_per_step[c] < best_ms)) {
            best_ms = out->ms_per_step[c];
            best = intervals[c];
        }
    }
    r->cfg.sort_interval = st ? saved_interval : best;
    // 2. particles per block chunk, at that interval
    int best_chunk = saved_chunk;
    best_ms = 0.0f;
    for (int c = 0; !st && c < CPIC_TUNE_CANDIDATES; ++c) {
        st = cpic_set_push_tuning(r, chunks[c], saved_tile);
        out->chunks[c] = chunks[c];
        if (!st) st = tune_trial(r, buf, saved_cur, trial_steps, a, b, &out->ms_chunk[c]);
        if (!st && (best_ms == 0.0f || out->ms_chunk[c] < best_ms)) {
            best_ms = out->ms_chunk[c];
            best_chunk = chunks[c];
        }
    }
    // 3. deposit tiling, with that chunk
    int best_tile = saved_tile;
    best_ms = 0.0f;
    for (int t = 0; !st && t < 2; ++t) {
        st = cpic_set_push_tuning(r, best_chunk, t);
        if (!st) st = tune_trial(r, buf, saved_cur, trial_steps, a, b, &out->ms_tile[t]);
        if (!st && (best_ms == 0.0f || out->ms_tile[t] < best_ms)) {
            best_ms = out->ms_tile[t];
            best_tile = t;
        }
    }
    // 4. the sort interval once more, with the chunking and tiling chosen (the first pass
    //    ran with the tiling the run had; the best interval depends on the push's cost)
    if (!st) st = cpic_set_push_tuning(r, best_chunk, best_tile);
    if (!st && (best_chunk != saved_chunk || best_tile != saved_tile)) {
        best = r->cfg.sort_interval;
        best_ms = 0.0f;
        for (int c = 0; !st && c < CPIC_TUNE_CANDIDATES; ++c) {
            r->cfg.sort_interval = intervals[c];
            st = tune_trial(r, buf, saved_cur, trial_steps, a, b, &out->ms_per_step[c]);
            if (!st && (best_ms == 0.0f || out->ms_per_step[c] < best_ms)) {
                best_ms = out->ms_per_step[c];
                best = intervals[c];
            }
        }
        r->cfg.sort_interval = best;
    }
    r->steps_since_sort = saved_since;
    if (st) {
        r->cfg.sort_interval = saved_interval;
        cpic_set_push_tuning(r, saved_chunk, saved_tile);
    }
    out->sort_interval = r->cfg.sort_interval;
    out->chunk = r->push_chunk;
    out->tile = r->push_tile;
    cudaStreamSynchronize(r->stream);
    cudaFree(buf);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st == CPIC_ERR_CUDA) set_error("autotune: CUDA event or copy failed");
    return st;
}

int cpic_checkpoint(cpic_run* r, const char* path) {
    if (!r || !path) {
        set_error("checkpoint: NULL run or path");
        return CPIC_ERR_INVALID;
    }
    if (int e = resolve_order(r)) return e;  // the particles in slot order
    if (!r->map_set) {
        set_error("checkpoint: the run has no map yet");
        return CPIC_ERR_STATE;
    }
    const int D = r->D;
    std::vector<double> X((size_t)r->nvert * D), phi(r->ncell);
    std::vector<unsigned long long> coll((size_t)r->cfg.n_species * 2 * r->ncollect);
    CPIC_CUDA(cudaMemcpyAsync(coll.data(), r->collect, sizeof(unsigned long long) * coll.size(), cudaMemcpyDeviceToHost,
                              r->stream));
    DevCounters ctr;
    CPIC_CUDA(cudaMemcpyAsync(X.data(), r->lev[0].X, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaMemcpyAsync(phi.data(), r->lev[0].x, sizeof(double) * phi.size(), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaMemcpyAsync(&ctr, r->ctr, sizeof(ctr), cudaMemcpyDeviceToHost, r->stream));
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("checkpoint: cannot open %s for writing", path);
        return CPIC_ERR_INVALID;
    }
    const unsigned long long nvert = (unsigned long long)r->nvert;
    const int since = r->steps_since_sort;
    bool ok = wr(f, kMagic, 8) && wr(f, &kVersion, 1) && wr(f, &r->cfg, 1) && wr(f, &nvert, 1) &&
              wr(f, X.data(), X.size()) && wr(f, r->inj, CPIC_MAX_SPECIES) && wr(f, &ctr, 1) && wr(f, &since, 1) &&
              wr(f, &r->floating_face, 1) && wr(f, &r->float_q0, 1) && wr(f, r->B0, 3) && wr(f, &r->gyro_kind, 1) &&
              wr(f, &r->mg_coarse, 1) && wr(f, &r->mg_interp, 1) && wr(f, &r->mg_smoother, 1) &&
              wr(f, coll.data(), coll.size()) && wr(f, phi.data(), phi.size());
    const int b = ctr.cur;
    const long long T = r->pb.total;
    for (int s = 0; ok && s < r->cfg.n_species; ++s) {
        const long long n = ctr.count[s], b0 = r->pb.base[s];
        std::vector<int> cell(n);
        std::vector<float> t((size_t)D * n), v((size_t)3 * n);
        if (n) {
            CPIC_CUDA(cudaMemcpyAsync(cell.data(), r->pb.cell[b] + b0, sizeof(int) * n, cudaMemcpyDeviceToHost, r->stream));
            for (int a = 0; a < D; ++a)
                CPIC_CUDA(cudaMemcpyAsync(t.data() + a * n, r->pb.t[b] + a * T + b0, sizeof(float) * n,
                                          cudaMemcpyDeviceToHost, r->stream));
            for (int a = 0; a < 3; ++a)
                CPIC_CUDA(cudaMemcpyAsync(v.data() + a * n, r->pb.v[b] + a * T + b0, sizeof(float) * n,
                                          cudaMemcpyDeviceToHost, r->stream));
            CPIC_CUDA(cudaStreamSynchronize(r->stream));
        }
        ok = wr(f, &n, 1) && wr(f, cell.data(), cell.size()) && wr(f, t.data(), t.size()) && wr(f, v.data(), v.size());
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("checkpoint: write to %s failed", path);
        return CPIC_ERR_INVALID;
    }
    return CPIC_OK;
}

int cpic_restore(const char* path, void* arena, size_t arena_bytes, void* stream, cpic_run** out) {
    if (!path || !out) {
        set_error("restore: NULL path or out");
        return CPIC_ERR_INVALID;
    }
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("restore: cannot open %s", path);
        return CPIC_ERR_INVALID;
    }
    char magic[8];
    unsigned version = 0;
    cpic_config cfg;
    unsigned long long nvert = 0;
    bool ok = rd(f, magic, 8) && memcmp(magic, kMagic, 8) == 0 && rd(f, &version, 1) && version == kVersion &&
              rd(f, &cfg, 1) && rd(f, &nvert, 1);
    if (!ok || cfg.dim < 2 || cfg.dim > 3) {
        fclose(f);
        set_error("restore: %s is not a checkpoint of this library version", path);
        return CPIC_ERR_INVALID;
    }
    cpic_run* r = nullptr;
    int st = cpic_create(&cfg, arena, arena_bytes, stream, &r);
    if (st) {
        fclose(f);
        return st;
    }
    if ((unsigned long long)r->nvert != nvert) {
        fclose(f);
        cpic_destroy(r);
        set_error("restore: vertex count does not match the stored configuration");
        return CPIC_ERR_INVALID;
    }
    const int D = r->D;
    std::vector<double> X((size_t)nvert * D), phi(r->ncell);
    DevCounters ctr;
    int since = 0;
    ok = rd(f, X.data(), X.size());
    if (ok) st = cpic_set_map_vertices(r, X.data());
    int fface = -1;
    double fq0 = 0.0, B0[3] = {0.0, 0.0, 0.0};
    int gyro = CPIC_GYRO_BORIS, mgc = CPIC_MG_COARSE_REDISCRETIZED, mgi = CPIC_MG_INTERP_BILINEAR;
    int mgs = CPIC_MG_SMOOTH_POINT;
    ok = ok && !st && rd(f, r->inj, CPIC_MAX_SPECIES) && rd(f, &ctr, 1) && rd(f, &since, 1) && rd(f, &fface, 1) &&
         rd(f, &fq0, 1) && rd(f, B0, 3) && rd(f, &gyro, 1) && rd(f, &mgc, 1) && rd(f, &mgi, 1) && rd(f, &mgs, 1);
    // the multigrid components first: the conductor's psi is then solved as the saved run
    // solved it when its components were set before cpic_set_floating
    if (ok && !st) st = cpic_set_multigrid(r, mgc, mgi, mgs);
    if (ok && !st && fface >= 0) st = cpic_set_floating(r, fface, fq0);  // psi and its flux sum, recomputed
    if (ok && !st) st = cpic_set_magnetic_field(r, B0);
    if (ok && !st) st = cpic_set_gyro_integrator(r, gyro);
    std::vector<unsigned long long> coll((size_t)cfg.n_species * 2 * r->ncollect);
    ok = ok && !st && rd(f, coll.data(), coll.size()) && rd(f, phi.data(), phi.size());
    // particles into buffer 0, counters with cur = 0
    const long long T = r->pb.total;
    for (int s = 0; ok && s < cfg.n_species; ++s) {
        long long n = 0;
        ok = rd(f, &n, 1) && n >= 0 && n <= r->pb.capacity[s];
        if (!ok) break;
        std::vector<int> cell(n);
        std::vector<float> t((size_t)D * n), v((size_t)3 * n);
        ok = rd(f, cell.data(), cell.size()) && rd(f, t.data(), t.size()) && rd(f, v.data(), v.size());
        if (!ok || !n) continue;
        const long long b0 = r->pb.base[s];
        if (cudaMemcpy(r->pb.cell[0] + b0, cell.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
        for (int a = 0; ok && a < D; ++a)
            ok = cudaMemcpy(r->pb.t[0] + a * T + b0, t.data() + a * n, sizeof(float) * n, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
        for (int a = 0; ok && a < 3; ++a)
            ok = cudaMemcpy(r->pb.v[0] + a * T + b0, v.data() + a * n, sizeof(float) * n, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
    }
    fclose(f);
    if (ok) {
        ctr.cur = 0;
        for (int s = 0; s < CPIC_MAX_SPECIES; ++s) ctr.inject_ticket[s] = 0;
        ok = cudaMemcpy(r->ctr, &ctr, sizeof(ctr), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(r->lev[0].x, phi.data(), sizeof(double) * phi.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(r->collect, coll.data(), sizeof(unsigned long long) * coll.size(), cudaMemcpyHostToDevice) ==
                 cudaSuccess;
        r->cur_host = 0;
        r->steps_since_sort = since;
    }
    if (!ok || st) {
        cpic_destroy(r);
        if (!st) set_error("restore: %s is truncated or inconsistent", path);
        return st ? st : CPIC_ERR_INVALID;
    }
    *out = r;
    return CPIC_OK;
}

}  // extern "C"
