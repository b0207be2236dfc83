// Internal declarations of the CUDA library behind include/cpic.h (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cpic.h"

namespace cpic {

// ---------------------------------------------------------------- constants
constexpr int QK = 16;  // spec Q: offsets quantised to 2^-QK of a cell
constexpr int QB = 16;  // spec Q: per-axis weights to 2^-QB
constexpr int QF = 24;  // spec Q: one particle deposits exactly 2^QF charge units
constexpr int KE_BITS = 24;  // spec D: kinetic energy products in units of 2^-24
constexpr int MAX_LEVELS = 16;
constexpr int COARSE_CELLS = 2048;  // levels at or below this size run in one CTA (shared memory)
constexpr int DENSE_MAX = 512;      // coarsest level solved densely (inverse) up to this size

// ---------------------------------------------------------------- error handling
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
#define CPIC_CUDA(call)                                                      \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)
// streaming multiprocessors of the current device (queried once per device, cached)
int device_sm_count();
// every kernel launch of the library is followed by this check, which also counts it
void count_launch();
void add_launches(long long n);  // kernels launched by a graph replay
#define CPIC_CHECK_LAUNCH()           \
    do {                              \
        ::cpic::count_launch();       \
        CPIC_CUDA(cudaGetLastError()); \
    } while (0)

// ---------------------------------------------------------------- device-side run state
// Counters written by kernels (one struct in device memory per run).
struct DevCounters {
    long long count[CPIC_MAX_SPECIES];     // occupied slots (live + dead until the next sort)
    long long alive[CPIC_MAX_SPECIES];     // live particles
    long long absorbed[CPIC_MAX_SPECIES][6];
    long long injected[CPIC_MAX_SPECIES];
    long long dropped[CPIC_MAX_SPECIES];
    long long nonfinite;
    long long ke_fp[CPIC_MAX_SPECIES];     // sum of round(v_old . v_new * 2^24) of the last push
    long long step;                        // completed pushes
    int cur;                               // current particle buffer (0/1)
    unsigned inject_ticket[CPIC_MAX_SPECIES];  // blocks of the running injection that are done
    double field_energy;
    double mg_residual;
    double mg_bnorm;
    int mg_cycles;
    int mg_converged;
    // floating conductor (cpic_set_floating): its potential and charge after the last solve,
    // and the flux sum of the unit-potential solution (set once)
    double object_potential;
    double object_charge;
    double float_cpsi;
    // 1: a sort's new order is pending: slot i of the other buffer's cell array holds the
    // index (in the current buffer) of the particle that belongs in slot i, and the counts
    // are already the sorted ones; the next fused 3D push reads through it and the step's
    // finalisation flips the buffers (see launch_sort)
    int perm;
};

// Scalars and reduction partials of the Krylov solve (device).
// blocks of the operator passes over the finest level (the FP64 residual, the Krylov
// products): up to one per eight rows of cells, so that these passes fill the GPU; each
// block leaves its partial sums in a reduction array of this many entries
constexpr int KRY_BLOCKS = 2048;
struct KrylovState {
    double rho, alpha, omega, beta;
    int restart;       // the next direction step starts over: r_hat = r, p = r
    unsigned ticket;   // last-block counter of the Krylov reductions
    double part[3 * KRY_BLOCKS];
};

// Particle storage: two buffers (sort ping-pong), each a structure of arrays over all
// species; species s owns slots [base[s], base[s] + capacity[s]).
struct ParticleBuffers {
    int* cell[2];
    float* t[2];  // [D][total] per buffer
    float* v[2];  // [3][total] per buffer
    long long total;
    long long base[CPIC_MAX_SPECIES];
    long long capacity[CPIC_MAX_SPECIES];
};

// Everything a particle kernel needs, passed by value.
struct PushParams {
    int D;
    int n[3];
    int pbc[6];
    int nsp;
    float dtqm[CPIC_MAX_SPECIES];  // (float)(dt q/m)
    float hdt;                     // (float)(dt/2)
    float dt;                      // (float)dt
    const float* K;                // vertex k table: 2D float4 [K00 K01 K10 K11]; 3D 3 x float4 (9 used)
    const float* G;                // vertex G table: 2D float2; 3D float4 (3 used)
    ParticleBuffers pb;
    unsigned long long* charge;    // padded deposit grid [nsp][ncell_h]
    long long ncell_h;             // cells of the padded grid: prod (n_a + 2)
    int hs1, hs2;                  // padded strides of axes 1 and 2
    int origin;                    // padded index of cell (0, 0, 0)
    const float* R;                // axisymmetric runs: vertex table of the cylindrical radius
                                   // (FP32); nullptr otherwise
    int magnetized;                // uniform B0 (cpic_set_magnetic_field): Boris kick
    float bh[CPIC_MAX_SPECIES];    // Boris constants per species: half kick (float)(dt q/m / 2),
    float bt[CPIC_MAX_SPECIES][3]; // t = (float)(dt q/m B0 / 2),
    float bs[CPIC_MAX_SPECIES][3]; // s = (float)(2 t / (1 + |t|^2)) (t, s from FP64 values)
    unsigned long long* collect;   // absorbed particles per [species][face 0/1][face cell]
    int ncollect;                  // face cells of a face normal to axis 0
    int gyro;                      // cyclotronic integrator (exact gyration) instead of Boris
    float gb[3];                   // its unit field direction b (velocity components' basis)
    float gy[CPIC_MAX_SPECIES][4]; // per species cos th, sin th, sin th / th, (1 - cos th) / th
    int chunk;                     // particles per block chunk (0: one wave of blocks)
    int* hist;                     // when set: count each kept particle's new cell here
                                   // ([species][cell], the next sort's histogram)
    int tile;                      // 1: shared-memory deposit tile when the chunk fits
    DevCounters* ctr;
};

// Multigrid level (cell-centred finite volume, rediscretised from the level's vertex map).
struct Level {
    int n[3];
    long long ncell;
    int S;            // stencil entries stored: 9 (2D) / 27 (3D: 19-point operator + Galerkin corners)
    int cross;        // 1 if any cross coefficient is non-zero (9/19-point), else 5/7-point
    double* A;        // [S][ncell]
    double* x;        // solution (finest: phi) / correction
    double* b;        // right-hand side
    double* X;        // vertex map of this level [vertex][D]
    double* Jc;       // cell Jacobians
    double* omega;    // cell Omega
    double* face[3];  // face coefficients per axis: [D][nface_a] (a^{a0}, a^{a1}, a^{a2})
    double* dv;       // vertex derivatives [D][nvertex][D] (scratch for setup)
    float* A32;       // FP32 copy of the stencil for the correction cycles
    float* x32;       // FP32 correction
    float* b32;       // FP32 residual / right-hand side of the correction
    float* dinv32;    // FP32 inverse diagonal (Gauss-Seidel)
    float* lw;        // line-relaxation work [2][ncell] (eliminated upper diagonal, 2nd solve)
    double* pw;       // operator-induced prolongation weights [D][ncell] of this (fine) level
    float* pw32;      // their FP32 copy (the V-cycle's prolongation)
};

struct InjectSpec {
    int enabled;
    int face;
    double density, vth, drift[3];
    unsigned long long seed;
    double rate;   // particles per step
    int drifting;  // 2D, in-plane drift: the drifting-Maxwellian flux and normal speeds
    double dtot;   // drifting: sum over the face segments of Gamma(u_j) A_j
};

}  // namespace cpic

// The run (opaque handle of the ABI).
struct cpic_run {
    cpic_config cfg;
    int D;
    int n[3];
    long long ncell, nvert;
    int nvert_axis[3];
    cudaStream_t stream;
    bool own_memory;
    char* arena;
    size_t arena_bytes, arena_used;
    bool map_set;
    bool initialized;
    // geometry (finest level lives in levels[0])
    double* k64;      // [nvert][D][D]
    float* K32;       // vertex k table (padded records)
    float* G32;       // vertex G table (padded records)
    float* R32;       // axisymmetric runs: vertex cylindrical radius x^1 (FP32), else nullptr
    double* rhs_bc;   // Dirichlet part of the right-hand side (finest)
    double* jcdf;     // inclusive prefix sums of the cell Jacobians (device loading)
    double* dcdf;     // 2D drifting injection: per species, inclusive prefixes of Gamma(u_j) A_j
    double* fcdf;     // inclusive prefix sums of the face-cell areas of faces 0 and 1 (3D), or
                      // of the face segments' surfaces of revolution (axisymmetric 2D)
    unsigned long long* charge;  // [nsp][ncell] folded charge counts (what the field solve reads)
    unsigned long long* charge_h;  // [nsp][ncell_h] deposit grid with one halo layer per side
    long long ncell_h;
    cpic::ParticleBuffers pb;
    cpic::DevCounters* ctr;      // device
    int cur_host;                // host mirror of ctr->cur (every sort flips both)
    // multigrid
    int nlevels;
    cpic::Level lev[cpic::MAX_LEVELS];
    double* dense_inv;           // coarsest inverse [(m+1)^2] (FP64, setup)
    float* dense_inv32;          // FP32 copy used by the correction cycles
    double* dense_tmp;           // setup scratch [(m+1)^2]
    unsigned* ticket;            // last-block counter of the residual reduction
    // CUDA graphs of one PIC step (index 1: with the cell sort), captured on capture_stream
    cudaGraphExec_t step_graph[2][2];  // [with field solve][with sort]
    bool step_graph_ok[2][2];
    int graph_kernels[2][2];           // kernel nodes launched by one replay
    bool graph_sort_fused[2][2];       // the graph's sort leaves its order to the next push
    cudaStream_t capture_stream;
    int cluster_cs;              // cluster size of the cluster solver (0: not applicable)
    bool order_pending;          // a fused sort's order may be pending on the device (DevCounters::perm)
    bool count_hist;             // this step's direct 3D push and injection build the sort's histogram
    int dense_m;                 // coarsest unknowns (+1 row when singular)
    bool singular;
    double sumJ;                 // sum of finest J_c (singular projection)
    double load_total;           // last entry of jcdf: sum J_c, or sum Omega_c J_c (axisymmetric)
    double* red;                 // reduction scratch [3 * KRY_BLOCKS + 16]
    int solver;                  // CPIC_SOLVER_* of the stream solve
    int pc_face_only;            // the FP32 V-cycle uses the stencil's face entries only
    double B0[3];                // uniform magnetic field (cpic_set_magnetic_field)
    double kick_fraction;        // fraction of dt of the kick being launched (1 otherwise)
    int magnetized;              // B0 != 0
    int gyro_kind;               // CPIC_GYRO_*: Boris step or cyclotronic integrator
    int mg_coarse;               // CPIC_MG_COARSE_*: rediscretised or Galerkin coarse operators
    int mg_smoother;             // CPIC_MG_SMOOTH_*: point or alternating zebra line Gauss-Seidel
    int mg_interp;               // CPIC_MG_INTERP_*: bilinear or operator-induced prolongation
    unsigned long long* collect; // collection tally [species][face 0/1][face cell] (Fig. 7)
    int ncollect;                // face cells of a face normal to axis 0: n1 (2D), n1 n2 (3D)
    int floating_face;           // face whose conductor floats (cpic_set_floating), -1: none
    double float_q0;             // its charge before any particle was collected
    double* psi;                 // potential of the unit-potential conductor in charge-free space
    int push_chunk;              // push kernel: particles per block chunk (0: one wave)
    int push_tile;               // push kernel: shared-memory deposit tile (1) or direct (0)
    cpic::KrylovState* kry;      // device scalars of the Krylov solve
    double* kv;                  // Krylov vectors, FP64 [5][ncell]: r, r_hat, p, v, s
    float* ph32;                 // preconditioned direction p_hat (FP32)
    // sort scratch
    int* hist;                   // [nsp][ncell] counts -> cursors
    long long* scan;             // [nsp*ncell + 1] exclusive prefix
    long long* scan_blocks;      // block partials
    // injection
    cpic::InjectSpec inj[CPIC_MAX_SPECIES];
    double face_len[6];
    int steps_since_sort;
    // tracing: event pairs recorded around each phase of cpic_step
    bool profiling;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* prof_events;
    std::vector<cudaEvent_t>* prof_pool;
};

namespace cpic {
// ---------------------------------------------------------------- launchers (per .cu)
// geometry.cu
int launch_map_analytic(cpic_run* r, int map_id, const double* params, int nparams);
int launch_geometry(cpic_run* r);
// fields.cu
int launch_vertex_field(cpic_run* r);
int launch_rhs(cpic_run* r, double* b);
int launch_field_energy(cpic_run* r);
// floating conductor: Gauss's-law potential of the face's conductor, then phi += V psi
int launch_floating(cpic_run* r);
// flux sum of the face's unit-potential solution (set-up of the floating conductor)
int launch_floating_capacity(cpic_run* r);
// push.cu
int launch_push(cpic_run* r);
int launch_deposit(cpic_run* r);
int launch_kick(cpic_run* r, double fraction);
int launch_finalize_step(cpic_run* r);
int launch_fold(cpic_run* r);
int launch_push_prep(cpic_run* r);    // zero the deposit grid and kinetic-energy tallies
int launch_push_kernel(cpic_run* r);  // the fused push + deposit kernel alone
PushParams make_push_params(cpic_run* r);
void set_boris_constants(const cpic_run* r, PushParams* p, double fraction);
int launch_push2d(cpic_run* r, const PushParams& p);
// batched 2D particle step (row a11): one launch over a device table of runs' parameters
int push2d_batch_blocks();  // resident blocks of the batched kernel (one wave)
int launch_push2d_batch(const PushParams* runs, const int* vbase, int nruns, int per0, int per1, int blocks,
                        cudaStream_t stream);
// true when the run's particle step can join the batched 2D launch
bool push2d_batchable(const cpic_run* r);
// one step's work split around the particle push (for the batched launch): vertex field and
// the zeroing of the deposit grid (and the push itself for runs that cannot join it); then
// the step counter, injection, halo fold and sort
int enqueue_step_pre(cpic_run* r, bool with_push);
int enqueue_step_post(cpic_run* r, bool sort, bool fold, bool fused_sort = false);
// a fused sort step: the push and the injection count the sort's histogram (zeroed here)
int begin_counted_step(cpic_run* r);
int launch_push3d(cpic_run* r, const PushParams& p);  // CPIC_ERR_NOT_BUILT: no specialisation
// one PIC step without the field solve, enqueued on r->stream (also inside stream capture)
int enqueue_step(cpic_run* r, bool sort, bool fold);
int count_kernel_nodes(cudaGraph_t g, int* out);
int launch_load_maxwellian(cpic_run* r, int sp, long long n, double vth, const double* drift, unsigned long long seed);
// inject.cu
int launch_inject(cpic_run* r);
// sort.cu
// the cell sort; fused: leave the reordering to the next push (the direct 3D kernel and the
// 2D kernel read through the pending order; only when push_fused_ok), else gather now
int launch_sort(cpic_run* r, bool fused = false);
// carry out a pending sort order (gather; a no-op when none is pending): before anything
// other than a fused 3D push touches the particles
int resolve_order(cpic_run* r);
bool push_fused_ok(const cpic_run* r);
bool push3d_direct_taken(const cpic_run* r);
// mg.cu
int mg_setup(cpic_run* r);
int mg_solve(cpic_run* r, double rtol, int max_cycles, bool host_loop, int* cycles, double* res);
// enqueue the whole solve on the stream being captured into graph `g` after `deps`;
// returns the node the rest of the step must depend on
int mg_capture_solve(cpic_run* r, cudaGraph_t g, double rtol, int max_cycles);
void invalidate_graphs(cpic_run* r);
// mg_cluster.cu
int mg_cluster_prepare(cpic_run* r);
int mg_cluster_solve(cpic_run* r, double rtol, int max_cycles);
}  // namespace cpic
