// Row a11: many independent runs stepped together.
//
// A batch step is one CUDA graph launch in three phases:
//   1. one branch per member run, forked off the batch stream: the run's vertex field and
//      the zeroing of its deposit grid (and the whole push for runs that cannot join the
//      batched launch: 3D, magnetised or reflecting runs);
//   2. the particle step (gather, push, boundaries, deposit: rows a2-a6) of every 2D member
//      in ONE persistent launch per combination of axis kinds: the resident blocks walk the
//      virtual blocks of all runs (a run's share in proportion to its particle capacity),
//      each taking its run's parameters from a device table;
//      (cpic_batch_set_mode; the default leaves the push in the run branches: on the
//      batched configuration, runs of 10^4..2 10^6 particles, the branches that do not wait
//      for each other measured faster, for full cycles and for particle steps alike);
//   3. one branch per run again: step counter, injection, halo fold, the cell sort when it
//      is due and, for full cycles, the field solve (the cluster kernel or the conditional
//      V-cycle loop).
// Branches have no dependencies on each other, so the device runs them concurrently: runs
// far smaller than the GPU (a few thousand cells, 10^4..10^6 particles, a 16-SM solve
// cluster) fill it together instead of one after another, and the host issues one launch
// per batch step instead of one per kernel.
//
// A graph is captured once per (field solve or not, pattern of which runs sort on this
// step) and replayed; adding or removing a run drops the cached graphs. A run must not
// change its map or injection while it is a member, and must not be stepped on its own
// meanwhile.
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "internal.cuh"

struct cpic_batch {
    int max_runs = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // created here when the caller passed none
    std::vector<cpic_run*> runs;
    std::vector<cudaStream_t> branch;  // one capture branch stream per member
    std::vector<cudaEvent_t> join;     // one join event per member
    cudaEvent_t fork = nullptr, fork2 = nullptr;
    std::vector<cudaEvent_t> join_pre;  // one per member: end of its pre-push branch
    cpic::PushParams* d_params = nullptr;  // device tables of the batched push (per capture)
    int* d_vbase = nullptr;
    size_t table_runs = 0;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int kernels = 0;
        std::vector<char> fused;  // per member: its sort in this graph leaves the order pending
    };
    std::map<std::string, Graph> graphs;
    int mode = CPIC_BATCH_AUTO;  // cpic_batch_set_mode
};

namespace cpic {
namespace {

void drop_graphs(cpic_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.exec);
    b->graphs.clear();
}

// The batched push's device tables: members that can join it, grouped by the kinds of their
// two axes (periodic or not); per group a run table and virtual-block offsets. Built once
// per membership (run parameters do not change between steps; counts are read on the
// device). Per group: its first table entry, runs, axis kinds, total virtual blocks; its
// n + 1 offsets follow the previous groups' in the offset table.
struct PushGroup {
    int first, n, per0, per1, vblocks;
};

int build_push_tables(cpic_batch* b, std::vector<PushGroup>* groups) {
    groups->clear();
    std::vector<PushParams> table;
    std::vector<int> vbase;
    for (int kind = 0; kind < 4; ++kind) {
        const int per0 = kind & 1, per1 = kind >> 1;
        PushGroup g{(int)table.size(), 0, per0, per1, 0};
        for (cpic_run* r : b->runs) {
            if (!push2d_batchable(r)) continue;
            if ((r->cfg.particle_bc[0] == CPIC_PBC_PERIODIC) != (per0 != 0) ||
                (r->cfg.particle_bc[2] == CPIC_PBC_PERIODIC) != (per1 != 0))
                continue;
            long long cap = 0;
            for (int s = 0; s < r->cfg.n_species; ++s) cap += r->pb.capacity[s];
            const int nb = (int)std::max<long long>(1, (cap + 2047) / 2048);  // ~2048 particles a block
            vbase.push_back(g.vblocks);
            g.vblocks += nb;
            table.push_back(make_push_params(r));
            ++g.n;
        }
        if (g.n) {  // the group's n + 1 virtual-block offsets follow the previous group's
            vbase.push_back(g.vblocks);
            groups->push_back(g);
        }
    }
    if (b->d_params) cudaFree(b->d_params);
    if (b->d_vbase) cudaFree(b->d_vbase);
    b->d_params = nullptr;
    b->d_vbase = nullptr;
    b->table_runs = table.size();
    if (table.empty()) return CPIC_OK;
    CPIC_CUDA(cudaMalloc(&b->d_params, sizeof(PushParams) * table.size()));
    CPIC_CUDA(cudaMalloc(&b->d_vbase, sizeof(int) * vbase.size()));
    CPIC_CUDA(cudaMemcpy(b->d_params, table.data(), sizeof(PushParams) * table.size(), cudaMemcpyHostToDevice));
    CPIC_CUDA(cudaMemcpy(b->d_vbase, vbase.data(), sizeof(int) * vbase.size(), cudaMemcpyHostToDevice));
    return CPIC_OK;
}

int capture(cpic_batch* b, bool solve, const std::string& key, cpic_batch::Graph* out) {
    std::vector<PushGroup> groups;
    const bool persistent = b->mode == CPIC_BATCH_PERSISTENT;  // AUTO: branches (measured faster)
    (void)solve;
    int st = persistent ? build_push_tables(b, &groups) : CPIC_OK;  // before the capture: it allocates
    if (st) return st;
    // members that sort in this step and push with a kernel that reads through a pending
    // order (not through the persistent batched push) sort with the fused order: their push
    // counts the histogram and their next push does the gather. The graph runs in any order
    // state (the kernels read the device flag); the host flags are managed around launches.
    const size_t nr = b->runs.size();
    out->fused.assign(nr, 0);
    std::vector<char> pending(nr, 0);
    for (size_t i = 0; i < nr; ++i) {
        cpic_run* r = b->runs[i];
        out->fused[i] = key[i] == '1' && push_fused_ok(r) && !(persistent && push2d_batchable(r));
        pending[i] = r->order_pending;
        r->order_pending = false;
    }
    CPIC_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaEventRecord(fork)", __FILE__, __LINE__);
    // 1. pre-push branches
    for (size_t i = 0; !st && i < b->runs.size(); ++i) {
        cpic_run* r = b->runs[i];
        e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaStreamWaitEvent(fork)", __FILE__, __LINE__);
            break;
        }
        cudaStream_t saved = r->stream;
        r->stream = b->branch[i];
        if (out->fused[i]) st = begin_counted_step(r);
        if (!st) st = enqueue_step_pre(r, !persistent || !push2d_batchable(r));
        r->stream = saved;
        if (st) break;
        e = cudaEventRecord(b->join_pre[i], b->branch[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join_pre[i], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "join (pre-push)", __FILE__, __LINE__);
    }
    // 2. the batched particle step, one persistent launch per group
    int vfirst = 0;
    for (const PushGroup& g : groups) {
        if (st) break;
        const int blocks = std::min(g.vblocks, push2d_batch_blocks());
        st = launch_push2d_batch(b->d_params + g.first, b->d_vbase + vfirst, g.n, g.per0, g.per1, blocks, b->stream);
        vfirst += g.n + 1;
    }
    if (!st) {
        e = cudaEventRecord(b->fork2, b->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaEventRecord(fork2)", __FILE__, __LINE__);
    }
    // 3. post-push branches (injection, fold, sort, field solve)
    for (size_t i = 0; !st && i < b->runs.size(); ++i) {
        cpic_run* r = b->runs[i];
        e = cudaStreamWaitEvent(b->branch[i], b->fork2, 0);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaStreamWaitEvent(fork2)", __FILE__, __LINE__);
            break;
        }
        cudaStream_t saved = r->stream;
        r->stream = b->branch[i];
        st = enqueue_step_post(r, key[i] == '1', solve, out->fused[i] != 0);
        if (!st && solve) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg = nullptr;
            e = cudaStreamGetCaptureInfo(r->stream, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamGetCaptureInfo", __FILE__, __LINE__);
            else st = mg_capture_solve(r, cg, r->cfg.mg_rtol, r->cfg.mg_max_cycles);
        }
        r->stream = saved;
        if (st) break;
        e = cudaEventRecord(b->join[i], b->branch[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "join", __FILE__, __LINE__);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    for (size_t i = 0; i < nr; ++i) {
        b->runs[i]->order_pending = pending[i] != 0;
        b->runs[i]->count_hist = false;
    }
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(batch)", __FILE__, __LINE__);
    st = count_kernel_nodes(g, &out->kernels);
    if (!st) {
        e = cudaGraphInstantiate(&out->exec, g, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate(batch)", __FILE__, __LINE__);
    }
    cudaGraphDestroy(g);
    return st;
}

}  // namespace
}  // namespace cpic

using namespace cpic;

extern "C" {

int cpic_batch_create(int max_runs, void* stream, cpic_batch** out) {
    if (!out || max_runs < 1 || max_runs > 4096) {
        set_error("batch_create: need out != NULL and 1 <= max_runs <= 4096");
        return CPIC_ERR_INVALID;
    }
    cpic_batch* b = new cpic_batch;
    b->max_runs = max_runs;
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->stream) {  // graphs cannot be captured on the legacy default stream
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "cudaEventCreate(fork)", __FILE__, __LINE__);
    }
    *out = b;
    return CPIC_OK;
}

int cpic_batch_destroy(cpic_batch* b) {
    if (!b) return CPIC_OK;
    drop_graphs(b);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto ev : b->join) cudaEventDestroy(ev);
    for (auto ev : b->join_pre) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->fork2) cudaEventDestroy(b->fork2);
    if (b->d_params) cudaFree(b->d_params);
    if (b->d_vbase) cudaFree(b->d_vbase);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return CPIC_OK;
}

int cpic_batch_add(cpic_batch* b, cpic_run* r) {
    if (!b || !r) {
        set_error("batch_add: NULL batch or run");
        return CPIC_ERR_INVALID;
    }
    if (!r->map_set) {
        set_error("batch_add: the run has no map yet");
        return CPIC_ERR_STATE;
    }
    if ((int)b->runs.size() >= b->max_runs) {
        set_error("batch_add: batch is full (%d runs)", b->max_runs);
        return CPIC_ERR_CAPACITY;
    }
    for (auto x : b->runs)
        if (x == r) {
            set_error("batch_add: run is already a member");
            return CPIC_ERR_INVALID;
        }
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr, ev_pre = nullptr;
    CPIC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_pre, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        cudaStreamDestroy(s);
        return cuda_fail(e, "cudaEventCreate(join)", __FILE__, __LINE__);
    }
    // the run's earlier work (load, initialise, a pending sort order, which the batch's
    // kernels do not read through) is on its own stream: order the batch after it
    if (int st = resolve_order(r)) return st;
    CPIC_CUDA(cudaStreamSynchronize(r->stream));
    b->runs.push_back(r);
    b->branch.push_back(s);
    b->join.push_back(ev);
    b->join_pre.push_back(ev_pre);
    drop_graphs(b);
    return CPIC_OK;
}

int cpic_batch_remove(cpic_batch* b, cpic_run* r) {
    if (!b || !r) {
        set_error("batch_remove: NULL batch or run");
        return CPIC_ERR_INVALID;
    }
    for (size_t i = 0; i < b->runs.size(); ++i)
        if (b->runs[i] == r) {
            CPIC_CUDA(cudaStreamSynchronize(b->stream));
            cudaStreamDestroy(b->branch[i]);
            cudaEventDestroy(b->join[i]);
            cudaEventDestroy(b->join_pre[i]);
            b->runs.erase(b->runs.begin() + i);
            b->branch.erase(b->branch.begin() + i);
            b->join.erase(b->join.begin() + i);
            b->join_pre.erase(b->join_pre.begin() + i);
            drop_graphs(b);
            return CPIC_OK;
        }
    set_error("batch_remove: run is not a member");
    return CPIC_ERR_INVALID;
}

int cpic_batch_size(const cpic_batch* b, int* n) {
    if (!b || !n) {
        set_error("batch_size: NULL argument");
        return CPIC_ERR_INVALID;
    }
    *n = (int)b->runs.size();
    return CPIC_OK;
}

int cpic_batch_set_mode(cpic_batch* b, int mode) {
    if (!b || mode < CPIC_BATCH_AUTO || mode > CPIC_BATCH_PERSISTENT) {
        set_error("batch_set_mode: NULL batch or unknown mode %d", mode);
        return CPIC_ERR_INVALID;
    }
    if (mode != b->mode) {
        CPIC_CUDA(cudaStreamSynchronize(b->stream));
        drop_graphs(b);
    }
    b->mode = mode;
    return CPIC_OK;
}

int cpic_batch_step(cpic_batch* b, int nsteps, int with_solve) {
    if (!b || nsteps < 0) {
        set_error("batch_step: NULL batch or negative step count");
        return CPIC_ERR_INVALID;
    }
    if (b->runs.empty()) return CPIC_OK;
    const bool persistent = b->mode == CPIC_BATCH_PERSISTENT;
    for (cpic_run* r : b->runs)  // a pending order the member's batched push does not take
        if (r->order_pending && !(push_fused_ok(r) && !(persistent && push2d_batchable(r)))) {
            if (int st = resolve_order(r)) return st;
            CPIC_CUDA(cudaStreamSynchronize(r->stream));
        }
    for (int k = 0; k < nsteps; ++k) {
        std::string key(b->runs.size(), '0');
        for (size_t i = 0; i < b->runs.size(); ++i) {
            const cpic_run* r = b->runs[i];
            if (r->cfg.sort_interval > 0 && r->steps_since_sort + 1 >= r->cfg.sort_interval) key[i] = '1';
        }
        const std::string full = (with_solve ? "S" : "P") + key;
        auto it = b->graphs.find(full);
        if (it == b->graphs.end()) {
            // bounded cache; runs whose sort intervals are powers of two up to 16 repeat
            // their joint pattern every 16 steps (32 graphs with and without the solve)
            if (b->graphs.size() >= 64) drop_graphs(b);
            cpic_batch::Graph g;
            int st = capture(b, with_solve != 0, key, &g);
            if (st) return st;
            it = b->graphs.emplace(full, g).first;
        }
        CPIC_CUDA(cudaGraphLaunch(it->second.exec, b->stream));
        add_launches(it->second.kernels);
        for (size_t i = 0; i < b->runs.size(); ++i) {
            cpic_run* r = b->runs[i];
            // the push took any pending order; a fused sort at the end leaves a new one
            r->order_pending = key[i] == '1' && it->second.fused[i];
            if (key[i] == '1') {
                r->cur_host ^= 1;
                r->steps_since_sort = 0;
            } else {
                ++r->steps_since_sort;
            }
        }
    }
    return CPIC_OK;
}

int cpic_batch_synchronize(cpic_batch* b) {
    if (!b) {
        set_error("batch_synchronize: NULL batch");
        return CPIC_ERR_INVALID;
    }
    CPIC_CUDA(cudaStreamSynchronize(b->stream));
    return CPIC_OK;
}

}  // extern "C"
