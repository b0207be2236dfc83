// Row a12: a request loop that serves parametric runs with continuous batching.
//
// A server owns one device memory pool (its HBM budget) and a scheduler thread. Requests
// (a cylinder- or sphere-in-plasma run: cells, particles, object bias, plasma density and
// temperature, steps) queue on submit. The scheduler
//   - admits queued requests while a slot is free and the pool holds the run's footprint
//     (cpic_query_footprint; first fit with backfill: a request that does not fit yet does
//     not block smaller ones behind it),
//   - sets each admitted run up on its own stream (map, device Maxwellian load of both
//     species, injection sources, start-up solve) with its state kept on the device,
//   - advances every active run by a slice of steps at a time (the run's own CUDA graphs,
//     launched asynchronously on its stream), so the runs' work overlaps on the device,
//   - and, when a run has taken all its steps, reads its diagnostics, releases its memory
//     and slot (making room for the queue) and files the result for cpic_server_poll.
// Each run's arithmetic is that of cpic_step on its own, so a result does not depend on the
// other requests in flight.
//
// Everything runs on the device that is current when cpic_server_start is called.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <stdio.h>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// first-fit allocator over one device allocation (offsets in 256-byte units)
struct Pool {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes;
                size_t roff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Job {
    uint64_t ticket = 0;
    cpic_request req{};
    cpic_config cfg{};
    size_t footprint = 0;
    size_t off = 0;
    cpic_run* run = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int steps_done = 0;
    int slice = 0;            // steps of the slice in flight
    long long slice_live = 0; // live particles when it was launched
    Clock::time_point t_submit, t_start;
    std::atomic<bool> cancel{false};  // set by cpic_server_cancel while the run is active
    cpic_result res{};
};

}  // namespace

struct cpic_server {
    cpic_server_opts opts{};
    int device = 0;
    Pool pool;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::vector<Job*> active;
    std::map<uint64_t, Job*> done;
    std::map<uint64_t, int> state;  // ticket -> 0 queued, 1 active, 2 done
    std::map<uint64_t, Job*> jobs;  // every ticket not yet polled
    uint64_t next_ticket = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
};

namespace cpic {
namespace {

constexpr double kThetaCap = M_PI / 32;  // sphere requests: polar caps cut out at theta_c

int make_config(const cpic_request& q, int sort_interval, cpic_config* c) {
    if (q.kind != CPIC_REQ_CYLINDER && q.kind != CPIC_REQ_SPHERE) {
        set_error("server: unknown request kind %d", q.kind);
        return CPIC_ERR_INVALID;
    }
    const bool sph = q.kind == CPIC_REQ_SPHERE;
    if (q.n[0] < 8 || q.n[1] < 8 || (sph && (q.n[2] < 8 || q.n[0] > 1023 || q.n[1] > 1023 || q.n[2] > 1023)) ||
        q.particles_per_species < 1 || q.steps < 0 || !(q.density > 0.0) || !(q.temperature > 0.0) ||
        !(q.mass_ratio > 0.0) || !(q.dt > 0.0) || !(q.r_outer > q.r_object) || !(q.r_object > 0.0)) {
        set_error("server: bad request (cells, particles, steps, density, temperature, mass ratio, dt or radii)");
        return CPIC_ERR_INVALID;
    }
    memset(c, 0, sizeof(*c));
    c->dim = sph ? 3 : 2;
    c->n[0] = q.n[0];
    c->n[1] = q.n[1];
    c->n[2] = sph ? q.n[2] : 1;
    c->field_bc[0] = c->field_bc[1] = CPIC_BC_DIRICHLET;
    c->field_bc_value[0] = q.phi_object;
    c->particle_bc[0] = c->particle_bc[1] = CPIC_PBC_ABSORB;
    if (sph) {  // shell: Neumann, specular polar caps; periodic azimuth
        c->field_bc[2] = c->field_bc[3] = CPIC_BC_NEUMANN;
        c->particle_bc[2] = c->particle_bc[3] = CPIC_PBC_REFLECT;
        c->field_bc[4] = c->field_bc[5] = CPIC_BC_PERIODIC;
        c->particle_bc[4] = c->particle_bc[5] = CPIC_PBC_PERIODIC;
    } else {
        c->field_bc[2] = c->field_bc[3] = CPIC_BC_PERIODIC;
        c->particle_bc[2] = c->particle_bc[3] = CPIC_PBC_PERIODIC;
    }
    c->dt = q.dt;
    c->n_species = 2;
    const double R = q.r_outer, r0 = q.r_object;
    const double volume = sph ? (4.0 / 3.0) * M_PI * (R * R * R - r0 * r0 * r0) * cos(kThetaCap) : M_PI * (R * R - r0 * r0);
    const double w = volume * q.density / (double)q.particles_per_species;
    c->q[0] = -1.0;
    c->m[0] = 1.0;
    c->q[1] = 1.0;
    c->m[1] = q.mass_ratio;
    c->w[0] = c->w[1] = w;
    c->capacity[0] = c->capacity[1] = q.particles_per_species + q.particles_per_species / 2 + 1024;
    c->sort_interval = sort_interval;
    return CPIC_OK;
}

// set up an admitted run on its stream (map, load, injection, start-up solve)
int start_job(cpic_server* sv, Job* j) {
    int st = cpic_create(&j->cfg, sv->pool.base + j->off, j->footprint, j->stream, &j->run);
    if (st) return st;
    const cpic_request& q = j->req;
    const double mp[3] = {q.r_object, q.r_outer, kThetaCap};
    st = q.kind == CPIC_REQ_SPHERE ? cpic_set_map_analytic(j->run, CPIC_MAP_SHELL, mp, 3)
                                   : cpic_set_map_analytic(j->run, CPIC_MAP_ANNULUS, mp, 2);
    const double vth[2] = {sqrt(q.temperature), sqrt(q.temperature / q.mass_ratio)};
    for (int s = 0; !st && s < 2; ++s)
        st = cpic_load_maxwellian(j->run, s, q.particles_per_species, vth[s], nullptr, q.seed * 16 + (uint64_t)s);
    for (int s = 0; !st && s < 2; ++s)
        st = cpic_set_injection(j->run, s, 1, q.density, vth[s], nullptr, q.seed * 1000 + 7 + (uint64_t)s);
    if (!st) st = cpic_sort(j->run);  // the load draws cells in random order
    if (!st) st = cpic_initialize(j->run);
    return st;
}

void finish_job(cpic_server* sv, Job* j, int status) {
    cpic_result& r = j->res;
    r.status = status;
    // the failure's message was written on this (the scheduler's) thread: keep it with the
    // result, where the client that polls for it can read it
    if (status == CPIC_ERR_CANCELLED)
        snprintf(r.message, sizeof(r.message), "cancelled after %d of %d steps", j->steps_done, j->req.steps);
    else if (status)
        snprintf(r.message, sizeof(r.message), "%s", cpic_last_error());
    r.ticket = j->ticket;
    r.steps = j->steps_done;
    if (j->run && !status) {
        cpic_diag d;
        int st = cpic_get_diag(j->run, &d);
        if (st) {
            r.status = st;
        } else {
            r.field_energy = d.field_energy;
            r.kinetic_energy = d.kinetic_energy;
            for (int s = 0; s < 2; ++s) {
                r.n_particles[s] = d.n_particles[s];
                r.absorbed_object[s] = d.absorbed[s][0];
                r.absorbed_outer[s] = d.absorbed[s][1];
                r.injected[s] = d.injected[s];
                const double t = j->steps_done * j->cfg.dt;
                r.current_object[s] = t > 0 ? j->cfg.q[s] * j->cfg.w[s] * (double)d.absorbed[s][0] / t : 0.0;
            }
            r.mg_cycles = d.mg_cycles;
        }
    }
    if (j->run) cpic_destroy(j->run);
    j->run = nullptr;
    if (j->ev) cudaEventDestroy(j->ev);
    if (j->stream) cudaStreamDestroy(j->stream);
    j->ev = nullptr;
    j->stream = nullptr;
    const auto now = Clock::now();
    r.queue_s = std::chrono::duration<double>(j->t_start - j->t_submit).count();
    r.latency_s = std::chrono::duration<double>(now - j->t_submit).count();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (j->footprint) sv->pool.release(j->off, j->footprint);
    sv->state[j->ticket] = 2;
    sv->done[j->ticket] = j;
}

void worker_loop(cpic_server* sv) {
    cudaSetDevice(sv->device);
    while (!sv->stop.load()) {
        bool progressed = false;
        // admission: first fit with backfill
        std::vector<Job*> admit;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto it = sv->queue.begin(); it != sv->queue.end();) {
                if ((int)(sv->active.size() + admit.size()) >= sv->opts.max_active) break;
                size_t off = 0;
                if (sv->pool.alloc((*it)->footprint, &off)) {
                    (*it)->off = off;
                    sv->state[(*it)->ticket] = 1;
                    admit.push_back(*it);
                    it = sv->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (Job* j : admit) {
            j->t_start = Clock::now();
            int st = CPIC_OK;
            if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                set_error("server: stream or event creation failed");
                st = CPIC_ERR_CUDA;
            }
            if (!st) st = start_job(sv, j);
            if (!st && cudaEventRecord(j->ev, j->stream) != cudaSuccess) st = CPIC_ERR_CUDA;
            if (st) {
                finish_job(sv, j, st);
                continue;
            }
            sv->active.push_back(j);
            progressed = true;
        }
        // advance the runs whose previous slice is done
        for (size_t i = 0; i < sv->active.size();) {
            Job* j = sv->active[i];
            cudaError_t q = cudaEventQuery(j->ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            int st = q == cudaSuccess ? CPIC_OK : CPIC_ERR_CUDA;
            // the stream is idle: account the finished slice and read the live count
            long long live = 0;
            if (!st) {
                cpic_diag d;
                st = cpic_get_diag(j->run, &d);
                if (!st) live = d.n_particles[0] + d.n_particles[1];
            }
            if (!st) j->res.particle_steps += (long long)j->slice * j->slice_live;
            j->slice = 0;
            if (!st && j->cancel.load()) st = CPIC_ERR_CANCELLED;
            if (!st && j->steps_done < j->req.steps) {
                const int k = std::min(sv->opts.steps_per_slice, j->req.steps - j->steps_done);
                st = cpic_step(j->run, k);
                if (!st) {
                    j->steps_done += k;
                    j->slice = k;
                    j->slice_live = live;
                    if (cudaEventRecord(j->ev, j->stream) != cudaSuccess) st = CPIC_ERR_CUDA;
                }
                if (!st) {
                    progressed = true;
                    ++i;
                    continue;
                }
            }
            // done (or failed): leave the active set
            sv->active.erase(sv->active.begin() + i);
            finish_job(sv, j, st);
            progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(100));
        }
    }
}

}  // namespace
}  // namespace cpic

using namespace cpic;

extern "C" {

int cpic_server_start(const cpic_server_opts* opts, cpic_server** out) {
    if (!out) {
        set_error("server_start: out is NULL");
        return CPIC_ERR_INVALID;
    }
    *out = nullptr;
    cpic_server* sv = new cpic_server;
    if (opts) sv->opts = *opts;
    if (sv->opts.max_active <= 0) sv->opts.max_active = 64;
    if (sv->opts.steps_per_slice <= 0) sv->opts.steps_per_slice = 10;
    if (sv->opts.sort_interval < 0) sv->opts.sort_interval = 0;
    if (sv->opts.sort_interval == 0) sv->opts.sort_interval = 4;
    cudaGetDevice(&sv->device);
    size_t budget = sv->opts.hbm_budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            delete sv;
            return cuda_fail(e, "cudaMemGetInfo", __FILE__, __LINE__);
        }
        budget = fr / 2;
    }
    budget &= ~size_t(255);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, budget);
    if (e != cudaSuccess) {
        delete sv;
        set_error("server_start: cudaMalloc(%zu) of the pool failed: %s", budget, cudaGetErrorString(e));
        return CPIC_ERR_OOM;
    }
    sv->pool.base = (char*)p;
    sv->pool.size = budget;
    sv->pool.free_[0] = budget;
    sv->opts.hbm_budget = budget;
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return CPIC_OK;
}

int cpic_server_submit(cpic_server* sv, const cpic_request* req, uint64_t* ticket) {
    if (!sv || !req || !ticket) {
        set_error("server_submit: NULL argument");
        return CPIC_ERR_INVALID;
    }
    Job* j = new Job;
    j->req = *req;
    int st = make_config(*req, sv->opts.sort_interval, &j->cfg);
    if (!st) st = cpic_query_footprint(&j->cfg, &j->footprint);
    if (st) {
        delete j;
        return st;
    }
    if (j->footprint > sv->pool.size) {
        set_error("server_submit: run needs %zu bytes, the pool holds %zu", j->footprint, sv->pool.size);
        delete j;
        return CPIC_ERR_CAPACITY;
    }
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        j->ticket = sv->next_ticket++;
        sv->state[j->ticket] = 0;
        sv->jobs[j->ticket] = j;
        sv->queue.push_back(j);
    }
    sv->cv.notify_one();
    *ticket = j->ticket;
    return CPIC_OK;
}

int cpic_server_poll(cpic_server* sv, uint64_t ticket, cpic_result* out) {
    if (!sv || !out) {
        set_error("server_poll: NULL argument");
        return CPIC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->state.find(ticket);
    if (it == sv->state.end()) {
        set_error("server_poll: unknown ticket %llu", (unsigned long long)ticket);
        return CPIC_ERR_INVALID;
    }
    if (it->second != 2) return CPIC_ERR_BUSY;
    Job* j = sv->done[ticket];
    *out = j->res;
    sv->done.erase(ticket);
    sv->jobs.erase(ticket);
    sv->state.erase(it);
    delete j;
    return CPIC_OK;
}

int cpic_server_cancel(cpic_server* sv, uint64_t ticket) {
    if (!sv) {
        set_error("server_cancel: NULL server");
        return CPIC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->state.find(ticket);
    if (it == sv->state.end()) {
        set_error("server_cancel: unknown ticket %llu", (unsigned long long)ticket);
        return CPIC_ERR_INVALID;
    }
    if (it->second == 2) {
        set_error("server_cancel: ticket %llu is already done", (unsigned long long)ticket);
        return CPIC_ERR_STATE;
    }
    if (it->second == 1) {  // active: the scheduler stops it when its slice in flight ends
        sv->jobs[ticket]->cancel.store(true);
        return CPIC_OK;
    }
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q) {
        if ((*q)->ticket != ticket) continue;
        Job* j = *q;
        sv->queue.erase(q);
        cpic_result& r = j->res;
        r.status = CPIC_ERR_CANCELLED;
        r.ticket = j->ticket;
        snprintf(r.message, sizeof(r.message), "cancelled before admission");
        r.latency_s = std::chrono::duration<double>(Clock::now() - j->t_submit).count();
        r.queue_s = r.latency_s;
        it->second = 2;
        sv->done[ticket] = j;
        return CPIC_OK;
    }
    return CPIC_OK;
}

int cpic_server_stats(cpic_server* sv, int* queued, int* active, size_t* pool_free) {
    if (!sv) {
        set_error("server_stats: NULL server");
        return CPIC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (queued) *queued = (int)sv->queue.size();
    if (active) {
        int a = 0;
        for (auto& kv : sv->state) a += kv.second == 1;
        *active = a;
    }
    if (pool_free) {
        size_t f = 0;
        for (auto& kv : sv->pool.free_) f += kv.second;
        *pool_free = f;
    }
    return CPIC_OK;
}

int cpic_server_stop(cpic_server* sv) {
    if (!sv) return CPIC_OK;
    sv->stop.store(true);
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    // runs still active: wait for their work, then release them
    for (Job* j : sv->active) {
        if (j->stream) cudaStreamSynchronize(j->stream);
        if (j->run) cpic_destroy(j->run);
        if (j->ev) cudaEventDestroy(j->ev);
        if (j->stream) cudaStreamDestroy(j->stream);
        delete j;
    }
    for (Job* j : sv->queue) delete j;
    for (auto& kv : sv->done) delete kv.second;
    cudaFree(sv->pool.base);
    delete sv;
    return CPIC_OK;
}

}  // extern "C"
