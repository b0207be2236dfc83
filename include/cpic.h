/*
 * cpic.h - C ABI of the GB300-native curvilinear particle-in-cell hot path.
 *
 * Method: electrostatic PIC in curvilinear geometry (Delzanno et al., CPIC, arXiv 1311.2286).
 * Particles keep a logical position xi in the unit cube (split into an int32 cell index per
 * axis and an FP32 offset in [0, 1), "cell units") and a physical velocity (hybrid mover,
 * Sec. II.B.4, eq. (hybridx)). One PIC step (Sec. II, four-step cycle): vertex field ->
 * fused gather / push / boundary / deposit -> injection -> (sort) -> field solve.
 *
 * Conventions for every call:
 *  - Return value: CPIC_OK (0) or a negative CPIC_ERR_* code; cpic_last_error() returns a
 *    message for the calling thread's last failure (static storage, overwritten by the next
 *    failure on that thread).
 *  - Layout: logical axis a = 0, 1, 2 (xi, eta, zeta); cell arrays are indexed
 *    i + N1 (j + N2 k) (i fastest); vertex arrays have N_a + 1 entries per axis (a periodic
 *    axis repeats vertex 0 as vertex N_a) and are indexed i + (N1+1)(j + (N2+1) k).
 *    Face f = 2 * axis + side (side 0 = low end, 1 = high end of the logical axis).
 *  - Particle format (structure of arrays, one species per call): cell = int32 packed
 *    per-axis cell indices (2D: i | j << 16, 3D: i | j << 10 | k << 20; dead = -1),
 *    t = FP32 offsets [D][n], v = FP32 physical velocity [3][n] (three components also in
 *    2D, Sec. III).
 *  - Pointers marked "host or device" may point to either (unified addressing); every
 *    other pointer is host memory. Host arrays are copied before the call returns.
 *  - Work is enqueued on the run's stream (cpic_create / cpic_set_stream) and is
 *    asynchronous unless the call says it synchronises; cpic_get_* calls synchronise.
 *  - Ownership: a run owns the device memory it allocates; with a caller arena
 *    (cpic_create) it allocates nothing and the caller keeps the arena alive until
 *    cpic_destroy returns. A run is not thread safe: one thread at a time per run.
 */
#ifndef CPIC_H
#define CPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPIC_ABI_VERSION 1
#define CPIC_MAX_SPECIES 4

/* status codes */
#define CPIC_OK 0
#define CPIC_ERR_INVALID (-1)        /* bad argument or configuration */
#define CPIC_ERR_OOM (-2)            /* device allocation failed or arena too small */
#define CPIC_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define CPIC_ERR_NOT_CONVERGED (-4)  /* field solve hit its cycle limit */
#define CPIC_ERR_TIMEOUT (-5)        /* a bounded device wait ran out */
#define CPIC_ERR_NONFINITE (-6)      /* particles with non-finite positions were removed */
#define CPIC_ERR_BUSY (-7)           /* not done yet (serving) */
#define CPIC_ERR_STATE (-8)          /* call out of order (e.g. step before a map is set) */
#define CPIC_ERR_CAPACITY (-9)       /* particles dropped: species capacity exhausted */
#define CPIC_ERR_NOT_BUILT (-10)     /* the library was built without the requested part */
#define CPIC_ERR_CANCELLED (-11)     /* a served request was cancelled (cpic_server_cancel) */

/* field boundary conditions (Sec. II.B.3: imposed through ghost cells) */
#define CPIC_BC_PERIODIC 0
#define CPIC_BC_DIRICHLET 1
#define CPIC_BC_NEUMANN 2
/* particle boundary conditions (Sec. II.B.4, Sec. III.A-B) */
#define CPIC_PBC_PERIODIC 0
#define CPIC_PBC_ABSORB 1
#define CPIC_PBC_REFLECT 2

/* analytic maps evaluated on the device (Sec. II.A eq. (map); Sec. II.B.4 eq. (map2);
 * Sec. II.B.3 eqs. (r), (z)) */
#define CPIC_MAP_SINE 1          /* params: eps            x = xi + eps sin(2 pi xi) sin(2 pi eta), y likewise */
#define CPIC_MAP_ANNULUS 2       /* params: r0, R          r = r0 (R/r0)^xi, theta = 2 pi eta */
#define CPIC_MAP_SPHERE_AXISYM 3 /* params: r1, r2         (r, z) = [r1 + (r2-r1) xi](sin, cos)(pi (1 - eta)) */
#define CPIC_MAP_SHELL 4         /* params: r0, R, theta_c 3D: r = r0 (R/r0)^xi, theta = theta_c + (pi - 2 theta_c) eta, phi = 2 pi zeta */

typedef struct cpic_run cpic_run;

/* Run configuration (Sec. II: grid, boundary conditions, species in normalised units,
 * Sec. II.B). Fixed for the life of a run. */
typedef struct cpic_config {
    int32_t dim;                  /* 2 or 3 */
    int32_t n[3];                 /* cells per logical axis; 2D: n[2] ignored.
                                     Limits: 2D n[0] < 65536, n[1] < 32768; 3D each < 1024 */
    int32_t field_bc[6];          /* CPIC_BC_* per face; a periodic axis has both faces periodic */
    double field_bc_value[6];     /* Dirichlet potential per face */
    int32_t particle_bc[6];       /* CPIC_PBC_* per face; periodic iff the field axis is */
    double dt;                    /* time step (normalised to 1/omega_pe) */
    double background;            /* uniform immobile charge density (e.g. +1: neutralising ions) */
    int32_t axisymmetric;         /* 1 (2D only): azimuthal symmetry about the axis x^1 = 0
                                     (Sec. II.B): geometric factor Omega = x^1 in the solver
                                     (eq. (poiscurv)); a macro-particle is a ring of charge
                                     q w (its deposit is divided by 2 pi Omega_c); the mover
                                     moves it on a straight line in 3D and turns (v_r, v_theta)
                                     with the frame, v = (v_r, v_z, v_theta); loading is
                                     uniform in the 3D volume and injection faces are surfaces
                                     of revolution */
    int32_t n_species;            /* 1 .. CPIC_MAX_SPECIES */
    double q[CPIC_MAX_SPECIES];   /* charge of a physical particle */
    double m[CPIC_MAX_SPECIES];   /* mass of a physical particle */
    double w[CPIC_MAX_SPECIES];   /* physical particles per macro-particle */
    int64_t capacity[CPIC_MAX_SPECIES]; /* particle slots per species (load + injection) */
    int32_t sort_interval;        /* cpic_step sorts every this many steps (0 = never) */
    int32_t mg_max_cycles;        /* V-cycle limit of the solve inside cpic_step (0: 100) */
    double mg_rtol;               /* relative residual target of that solve (0: 1e-10, the
                                     paper's tolerance, Sec. II.B.3) */
} cpic_config;

/* Diagnostics (Sec. III: potential, currents from absorbed particles, particle counts;
 * Table IV: solver iterations). Energies: W_E = 1/2 sum_c phi_c Q_c at the current time
 * level, W_K = sum_s 1/2 m_s w_s sum_p v^{n-1/2} . v^{n+1/2} of the last push. */
typedef struct cpic_diag {
    int64_t step;                          /* completed pushes */
    double field_energy;
    double kinetic_energy;
    int64_t n_particles[CPIC_MAX_SPECIES]; /* live particles */
    int64_t absorbed[CPIC_MAX_SPECIES][6]; /* cumulative, per face */
    int64_t injected[CPIC_MAX_SPECIES];    /* cumulative */
    int64_t dropped[CPIC_MAX_SPECIES];     /* cumulative, for lack of capacity */
    int64_t nonfinite;                     /* cumulative */
    int32_t mg_cycles;                     /* V-cycles of the last solve */
    double mg_residual;                    /* relative residual of the last solve */
    int32_t pc_face_only;                  /* 1: the FP32 V-cycle uses the stencil's face
                                              entries only (cross entries below 2% of the
                                              diagonal; the FP64 residual keeps the full
                                              operator); 0: the full stencil. The environment
                                              variable CPIC_PC_FULL_STENCIL, set when the map
                                              is set, forces 0. */
    double object_potential;               /* floating conductor (cpic_set_floating): its
                                              potential after the last solve (0 without one) */
    double object_charge;                  /* and its charge (initial + collected) */
} cpic_diag;

/* ---------------------------------------------------------------- general */

/* Message for a status code (static string). */
const char* cpic_status_string(int status);
/* Message of the calling thread's last failure (static thread-local storage). */
const char* cpic_last_error(void);
/* ABI version of the loaded library (CPIC_ABI_VERSION when it matches this header). */
int cpic_abi_version(void);
/* Number of CUDA kernels this library has launched since it was loaded (all runs). */
int64_t cpic_kernel_launches(void);

/* ---------------------------------------------------------------- setup */

/* Device bytes a run with this configuration needs (the size of a caller arena).
 * Pure host computation; no GPU work. */
int cpic_query_footprint(const cpic_config* cfg, size_t* device_bytes);

/* Create a run on the current device. arena: NULL (the run cudaMallocs its memory) or a
 * device buffer of at least cpic_query_footprint bytes, 256-byte aligned, owned by the
 * caller. stream: cudaStream_t to enqueue on (NULL = legacy default stream). */
int cpic_create(const cpic_config* cfg, void* arena, size_t arena_bytes, void* stream,
                cpic_run** out);
/* The run's configuration as in use (the sort interval as last chosen by cpic_autotune). */
int cpic_get_config(const cpic_run* run, cpic_config* out);
/* Changes the cell-sort interval of cpic_step / cpic_step_particles (0 = never); the
 * steps already taken since the last sort count towards the new interval. */
int cpic_set_sort_interval(cpic_run* run, int interval);
/* Synchronise the run's stream and release it (frees what it allocated). NULL is a no-op. */
int cpic_destroy(cpic_run* run);
/* Enqueue subsequent work on another stream. */
int cpic_set_stream(cpic_run* run, void* stream);

/* Map from logical to physical space known at cell vertices (Sec. II.A, eq. (map) and its
 * last paragraph: metric coefficients by finite differences of the vertex map).
 * xyz: host or device, FP64 [vertex][D] in the vertex layout above. Computes on the device
 * (FP64): k = j^-1 at vertices (eqs. (jcov), (jcon)), the cell Jacobians (eq. (jac)), the
 * face coefficients Omega J g^{ab} (eqs. (gcon), (poiscurv)) for every multigrid level,
 * and the FP32 vertex table of k used by the mover. */
int cpic_set_map_vertices(cpic_run* run, const double* xyz);
/* Same, with the map evaluated on the device from a CPIC_MAP_* formula. */
int cpic_set_map_analytic(cpic_run* run, int map_id, const double* params, int nparams);

/* ---------------------------------------------------------------- particles */

/* Replace species sp's particles (Sec. III.B: initial load). cell, t, v: host or device,
 * particle format above, n <= capacity. Asynchronous on the run's stream when all three
 * arrays are device, managed or page-locked host memory (the caller keeps them unchanged
 * until the stream has passed the call); synchronises for pageable host memory. Slots
 * outside the grid are dropped (counted in dropped[sp]). */
int cpic_load_particles(cpic_run* run, int sp, int64_t n, const int32_t* cell, const float* t,
                        const float* v);
/* Copy species sp's live particles out (synchronises). cell, t, v: host or device with room
 * for `room` particles; *n receives the count (CPIC_ERR_INVALID if room is too small). The
 * order is the storage order (cell-sorted after cpic_sort, unspecified within a cell).
 * Dead slots left by absorption since the last sort are compacted on the device (into the
 * run's second particle buffer, which is free between sorts); then one copy per array goes
 * straight into the caller's buffers. */
int cpic_get_particles(cpic_run* run, int sp, int64_t room, int64_t* n, int32_t* cell, float* t,
                       float* v);
/* Maxwellian flux injection through face `face` for species sp (Sec. III.A-B): density,
 * thermal speed vth, drift (host, 3 doubles, may be NULL), Philox4x32-10 key `seed`.
 * Faces normal to axis 0 (face 0 or 1) with absorbing particle boundaries, and the last
 * logical axis periodic or (2D) the run axisymmetric, whose face is then a surface of
 * revolution: segments drawn by ring area 2 pi r_mid |dX|, rate from the total. Otherwise
 * CPIC_ERR_INVALID. A drift with an in-plane part (drift[0] or drift[1] nonzero) is a
 * drifting Maxwellian source (Sec. III.A, the ions of the wall test), 2D only: per face
 * segment j the inward drift u_j = drift . n_j (n_j the inward unit normal averaged over the
 * segment's vertices) weighs the segment by its one-sided flux density
 * Gamma(u_j) = vth/sqrt(2 pi) exp(-u_j^2/2 vth^2) + u_j/2 (1 + erf(u_j/(sqrt 2 vth))) times
 * its length (or ring area); the rate is density sum_j Gamma(u_j) A_j dt / w; the normal
 * speed follows the flux-weighted density v exp(-(v - u)^2/2 vth^2) on v > 0 (inverted by 64
 * FP64 bisections), the tangential speed is Gaussian about the drift's tangential part, and
 * drift[2] shifts the out-of-plane component. A 2D drift along z only keeps the resting
 * flux and adds the drift to the drawn velocity; in 3D a nonzero drift returns
 * CPIC_ERR_NOT_BUILT. */
int cpic_set_injection(cpic_run* run, int sp, int face, double density, double vth,
                       const double* drift, uint64_t seed);

/* Uniform magnetic field B0 (host, 3 doubles in physical space; NULL or zero: none), for
 * the magnetised mover of Sec. II.B.4: the kick of eq. (step1) with the v x B term, taken
 * by the Boris split (half kick, rotation, half kick) with t = (dt/2)(q/m) B0 and
 * s = 2 t / (1 + |t|^2); the positions advance as before (the hybrid predictor-corrector
 * with v^{n+1/2}; in 2D the velocity keeps three components). The start-up kick of
 * cpic_initialize then takes the Boris step over -dt/2. Magnetised runs push with the
 * generic particle kernel. Invalidates the run's captured step graphs. An axisymmetric run
 * (v = (v_r, v_z, v_theta)) takes only a field along the symmetry axis, B = (0, B_z, 0)
 * (CPIC_ERR_INVALID otherwise): the only uniform field that keeps the symmetry. */
int cpic_set_magnetic_field(cpic_run* run, const double* B);

/* Integrator of the gyration in the uniform field B0 (Sec. II.B: for a uniform field the
 * mover can resolve the gyromotion exactly, relaxing the time step constraint when the
 * cyclotron frequency is large). CPIC_GYRO_BORIS (the default): the Boris step above.
 * CPIC_GYRO_CYCLOTRONIC: the cyclotronic integrator, read as the splitting of the step
 * into the electric kick v+ = v + dt (q/m) E(xi^n) and the exact motion in B0 alone over
 * dt: with b = B0/|B0|, th = (q/m)|B0| dt, u = v+ x b, par = (v+ . b) b, perp = v+ - par,
 * the new velocity is par + cos th perp + sin th u and the physical displacement
 * d = dt (par + (sin th / th) perp + ((1 - cos th) / th) u) moves xi through the same
 * predictor-corrector (xi' = xi^n + k(xi^n) d / 2, xi^{n+1} = xi^n + k(xi') d). Exact for
 * E = 0 at any th, and exact E x B drift for a uniform E. The start-up kick is then the
 * plain half kick -dt/2 (q/m) E. Axisymmetric runs start the displacement at the
 * particle's point in 3D and turn the velocity with the frame. Takes effect only with a
 * nonzero B0. CPIC_ERR_INVALID for another kind. Invalidates captured step graphs. */
#define CPIC_GYRO_BORIS 0
#define CPIC_GYRO_CYCLOTRONIC 1
int cpic_set_gyro_integrator(cpic_run* run, int kind);

/* Collection tally (Sec. III.C, Fig. 7: where on the object the particles are collected):
 * counts[i] = particles of species sp removed at face `face` (0 or 1, the ends of axis 0)
 * since the run started, by face cell i (2D: the cell index j along axis 1, n = n[1]; 3D:
 * j + n[1] k, n = n[1] n[2]), taken at the particle's corrector point with the transverse
 * indices clamped into the face. counts: host or device, n int64 values; CPIC_ERR_INVALID
 * for a bad species, face or size. Synchronous. */
int cpic_get_collection(cpic_run* run, int sp, int face, int64_t* counts, int64_t n);

/* Floating conductor (Sec. III.A-B: the object collects the particles that reach it and
 * charges up to a floating potential; Figs. of the wall and sphere potential against time).
 * From now on the Dirichlet face `face` (0 or 1: the ends of axis 0, e.g. the object at
 * xi = 0) is a conductor whose potential V is set at every field solve by Gauss's law from
 * its charge Q = charge0 + sum_s q_s w_s (particles of species s absorbed at that face,
 * counted since the run started): Q equals minus the flux of grad phi out through the face,
 * 2 a^{00} (phi_c - V) summed over the face's cells in the finite-volume scheme. The solve
 * computes phi_0 with the conductor at 0 and adds V psi, psi the charge-free potential of
 * the conductor at 1 (solved here, once, with the other Dirichlet faces at 0). The face's
 * configured Dirichlet value is no longer used; cpic_get_diag reports V and Q. In an
 * axisymmetric run the flux sum is that of the Omega-weighted scheme, so Q / (2 pi) takes
 * the place of Q. Requires the map and a run that is not yet initialised (CPIC_ERR_STATE
 * otherwise) and a Dirichlet face (CPIC_ERR_INVALID otherwise). Synchronous. */
int cpic_set_floating(cpic_run* run, int face, double charge0);

/* Loads n particles of species sp on the device, replacing its particles: a Maxwellian
 * plasma of uniform physical density (the paper's runs start from one, Sec. III.A-B).
 * Cells are drawn with probability J_c / sum J_c (J_c the cell Jacobian; Omega_c J_c, the
 * ring volume / 2 pi, in an axisymmetric run), offsets uniform
 * in each cell, velocities vth * N(0, 1) per component plus drift (host, 3 doubles, may be
 * NULL). Draws: Philox4x32-10, counter (i, 0x10AD, sp, word), key seed. Requires the map
 * (CPIC_ERR_STATE otherwise); n <= capacity[sp] (CPIC_ERR_INVALID otherwise). Asynchronous
 * on the run's stream. */
int cpic_load_maxwellian(cpic_run* run, int sp, int64_t n, double vth, const double* drift, uint64_t seed);

/* ---------------------------------------------------------------- the PIC cycle */

/* Start-up: deposit rho^0 and solve phi^0, then v^{-1/2} = v^0 - dt/2 (q/m) E(xi^0)
 * (standard leapfrog start-up for eq. (step1)). */
int cpic_initialize(cpic_run* run);
/* nsteps full PIC steps (Sec. II cycle): vertex field, push (+ deposit), injection, sort
 * every sort_interval steps, charge -> RHS, multigrid solve to mg_rtol, diagnostics.
 * When the push is the direct 3D kernel or the 2D kernel, a sort takes its histogram from
 * the step's push and injection and leaves its reordering to the next push, which reads
 * each sorted slot's particle through the sort's index; every other call that touches the
 * particles (reads, loads, injection, checkpoints, another push kernel) carries out such a
 * pending order first, so the particles are always seen in sorted slot order. */
int cpic_step(cpic_run* run, int nsteps);
/* nsteps particle steps with the field held fixed: vertex field, push (+ deposit),
 * injection, sort every sort_interval steps; no charge -> RHS and no field solve. This is
 * the mover with its grid coupling on its own, as timed with fixed fields in Sec. III
 * (Tables II and III); the deposited charge of the last step is kept (cpic_get_charge
 * returns it). */
int cpic_step_particles(cpic_run* run, int nsteps);

/* Rows of one step, for callers that drive the cycle themselves: */
/* a1: G = d phi / d u at vertices from the cell potential (Sec. II.B staggering). */
int cpic_vertex_field(cpic_run* run);
/* a2-a6: for every live particle: b1 gather of G and k at xi^n (eqs. (vvp), (Wvp), (b1)),
 * E = -k^T G, kick (eq. (step1)), predictor (eq. (step2)), k re-gather (eq. (step3)),
 * corrector (eq. (step4)), boundaries (periodic / absorb), then the b2 deposit
 * (eqs. (pg), (Wpc), (b2)) in 64-bit fixed point into freshly zeroed charge grids.
 * Advances the step counter. */
int cpic_push(cpic_run* run);
/* a6 alone: zero the charge grids and deposit every live particle. */
int cpic_deposit(cpic_run* run);
/* Gather and kick only: v += fraction * dt (q/m) E(xi) (fraction = -0.5: start-up). */
int cpic_kick(cpic_run* run, double fraction);
/* a8: inject this step's particles (step index = completed pushes - 1) and deposit them. */
int cpic_inject(cpic_run* run);
/* a7: counting sort of every species by cell (row-major cell index), dropping dead slots. */
int cpic_sort(cpic_run* run);
/* a9: RHS from the charge grids (Omega_c Q_c plus Dirichlet terms), then multigrid
 * V-cycles (Sec. II.B.3) until ||r||/||b|| <= rtol or max_cycles; synchronises once per
 * cycle. cycles, residual: host, may be NULL. CPIC_ERR_NOT_CONVERGED if rtol was not met. */
int cpic_solve_field(cpic_run* run, double rtol, int max_cycles, int* cycles, double* residual);

/* Outer iteration of the field solve on the kernel-chain path (3D runs, and 2D runs that the
 * one-cluster solver does not take; the cluster solver always iterates V-cycles):
 *   CPIC_SOLVER_MG        x += V-cycle(b - M x) until ||r||/||b|| <= rtol (Sec. II.B.3's
 *                         multigrid iteration);
 *   CPIC_SOLVER_BICGSTAB  BiCGStab (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) on
 *                         M x = b, right-preconditioned by the same FP32 V-cycle: two V-cycles,
 *                         two FP64 products with M and one FP64 residual per iteration, the
 *                         residual recomputed from x every iteration (the default: about half
 *                         the V-cycles on the 3D shell, and it converges where point smoothing
 *                         alone stalls on strongly anisotropic cells). The stopping test and
 *                         the result's accuracy are the same; mg_cycles counts V-cycles.
 * Invalidates the run's captured step graphs. CPIC_ERR_INVALID for another value. */
#define CPIC_SOLVER_MG 0
#define CPIC_SOLVER_BICGSTAB 1
int cpic_set_solver(cpic_run* run, int solver);

/* Multigrid components (Sec. II.B.3: BoxMG's variational coarse operators and
 * operator-induced interpolation, and line relaxation for anisotropic problems).
 * coarse: CPIC_MG_COARSE_REDISCRETIZED (default: each coarse level assembled from the map
 * sampled at every other vertex) or CPIC_MG_COARSE_GALERKIN (A_coarse = R A_fine P with the
 * V-cycle's own restriction, the sum over the 2^D children, and prolongation; 9-point
 * coarse stencils in 2D, 27-point in 3D). interpolation: CPIC_MG_INTERP_BILINEAR (default: weights 3/4, 1/4 per
 * axis, homogeneous ghost rules) or CPIC_MG_INTERP_OPERATOR (per axis, the weights of the
 * flux-continuous 1D solution between the fine cell's parent and the parent's neighbour,
 * from the fine operator's couplings across faces collapsed over the transverse direction;
 * uniform couplings give the bilinear weights). smoother: CPIC_MG_SMOOTH_POINT (default:
 * colour-ordered point Gauss-Seidel) or CPIC_MG_SMOOTH_LINE (alternating zebra line
 * Gauss-Seidel: every line of cells along axis 0, then along axis 1 (then axis 2), solved
 * exactly, cyclic on a periodic axis). Any non-default choice runs the solve on the kernel
 * chain (not the one-cluster solver). CPIC_ERR_INVALID for an unknown value. Synchronous when the map is already set (the hierarchy is rebuilt);
 * invalidates captured step graphs. */
#define CPIC_MG_COARSE_REDISCRETIZED 0
#define CPIC_MG_COARSE_GALERKIN 1
#define CPIC_MG_INTERP_BILINEAR 0
#define CPIC_MG_INTERP_OPERATOR 1
#define CPIC_MG_SMOOTH_POINT 0
#define CPIC_MG_SMOOTH_LINE 1
int cpic_set_multigrid(cpic_run* run, int coarse, int interpolation, int smoother);

/* ---------------------------------------------------------------- data out / in */

int cpic_get_diag(cpic_run* run, cpic_diag* out);              /* synchronises */
int cpic_get_phi(cpic_run* run, double* phi);                  /* host or device, cells */
int cpic_set_phi(cpic_run* run, const double* phi);            /* host or device, cells */
int cpic_get_charge(cpic_run* run, int sp, int64_t* counts);   /* host or device, cells;
                                                                  units of 2^-24 particles */
/* FP32 vertex tables used by the mover: k [vertex][D][D] (cell units, k[a][alpha]) and
 * G [vertex][D]; host or device; either may be NULL. */
int cpic_get_vertex_tables(cpic_run* run, float* k, float* g);
/* FP64 metric of the finest grid: k [vertex][D][D], cell Jacobians J_c [cell]; host or
 * device; either may be NULL. */
int cpic_get_geometry(cpic_run* run, double* k, double* jc);
/* Wait for the run's stream. */
int cpic_synchronize(cpic_run* run);

/* ---------------------------------------------------------------- no-allocation sort */

/* Largest grid (cells) cpic_sort_cells_noalloc accepts: its scratch is fixed in size. */
#define CPIC_NOALLOC_MAX_CELLS (1 << 20)

/* Cell sort for callers that cannot allocate device memory (code running during CUDA graph
 * capture, hosts whose memory manager owns all device memory, loops that must not pay for
 * an allocation). The paper has no counterpart: this is a data-layout utility. It does what
 * cpic_sort does for a run, on arrays the caller provides: counting sort of `count`
 * particles by row-major cell index (i + N1 (j + N2 k)), dropping slots whose cell is -1
 * or outside the grid. The order inside a cell is unspecified.
 *   dim, n:   2 or 3, cells per axis (host array of dim ints), n[0]*n[1](*n[2]) <=
 *             CPIC_NOALLOC_MAX_CELLS, else CPIC_ERR_INVALID;
 *   cell_in, t_in [dim][count], v_in [3][count]: device arrays in the particle format;
 *   cell_out, t_out [dim][count], v_out [3][count]: device arrays with the same strides
 *             (count); the first *live_out entries receive the sorted particles;
 *   live_out: device int64 receiving the number of live particles;
 *   stream:   cudaStream_t the work is enqueued on (asynchronous).
 * It allocates nothing: its histogram and prefix sums live in a fixed 8 MiB device array of
 * the library, held on every GPU that loads the library until the process exits. The first
 * call on a device looks up that array's device address (make it before any stream
 * capture). All calls share the array: calls whose work overlaps on the GPU race and give
 * wrong results; order them on one stream. */
int cpic_sort_cells_noalloc(int dim, const int32_t* n, int64_t count, const int32_t* cell_in,
                            const float* t_in, const float* v_in, int32_t* cell_out, float* t_out,
                            float* v_out, int64_t* live_out, void* stream);

/* ---------------------------------------------------------------- tuning and checkpoints */

#define CPIC_TUNE_CANDIDATES 5

typedef struct cpic_tuning {
    int32_t sort_interval;                     /* chosen (and set in the run) */
    int32_t interval[CPIC_TUNE_CANDIDATES];    /* candidates tried: 1, 2, 4, 8, 16 */
    float ms_per_step[CPIC_TUNE_CANDIDATES];   /* measured fixed-field particle step time */
    int32_t chunk;                             /* chosen particles per block chunk (0: one wave) */
    int32_t chunks[CPIC_TUNE_CANDIDATES];      /* candidates tried: 0, 1024, 2048, 4096, 8192 */
    float ms_chunk[CPIC_TUNE_CANDIDATES];      /* step time per chunk candidate */
    int32_t tile;                              /* chosen deposit tiling (1 shared tile, 0 direct) */
    float ms_tile[2];                          /* step time with [0] direct, [1] tiled deposit */
} cpic_tuning;

/* Chooses, in this order, the run's cell-sort interval, the particles per block chunk of
 * the push kernel and its deposit tiling, then (when chunk or tiling changed) the sort
 * interval again with them (ms_per_step then holds the second pass): for each candidate,
 * times whole sort cycles of at
 * least trial_steps fixed-field particle steps on the run's own particles (CUDA events on
 * the run's stream), restoring the run's particles, counters and potential from a device
 * snapshot after each trial, so the simulation is unchanged; the fastest setting of each
 * knob is kept for the next. The result is set in the run. The snapshot is a temporary
 * device allocation (CPIC_ERR_OOM if it fails). Synchronous. Not in the paper (the sort and
 * the chunking are GPU locality devices). */
int cpic_autotune(cpic_run* run, int trial_steps, cpic_tuning* out);

/* Push kernel knobs (the autotuner's second and third): chunk = particles per block chunk
 * (0: the particles split evenly over one wave of resident blocks; otherwise a multiple of
 * 256 in [256, 2^20]); tile = 1 to deposit through the block's shared-memory tile when the
 * chunk's cells fit it, 0 to deposit straight into the global grid. The result is the same
 * either way (integer deposit). CPIC_ERR_INVALID for other values. Invalidates the run's
 * captured step graphs. */
int cpic_set_push_tuning(cpic_run* run, int chunk, int tile);

/* Writes the run's configuration, vertex map, injection sources, counters, potential,
 * conductor, magnetic field, gyro integrator, multigrid components and live-slot particles
 * to a file (synchronous). A restored run continues bit for bit; a floating conductor's
 * charge-free potential is solved again on restore with the saved multigrid components, so
 * a run that changed its components after cpic_set_floating continues to the solve
 * tolerance instead. */
int cpic_checkpoint(cpic_run* run, const char* path);
/* Creates a run from a checkpoint (arena/stream as in cpic_create); stepping it continues
 * the saved run exactly (particles, charge, potential and diagnostics bit for bit).
 * CPIC_ERR_INVALID for a missing, foreign or truncated file. */
int cpic_restore(const char* path, void* arena, size_t arena_bytes, void* stream, cpic_run** out);

/* ---------------------------------------------------------------- batched runs (row a11) */

/* A batch steps many independent runs together: one CUDA graph launch per batch step, whose
 * branches (one per member run, no dependencies between them) hold each run's step, so the
 * device runs them concurrently; the 2D members' particle push can be one persistent launch
 * over all of them (cpic_batch_set_mode). Runs keep their own arenas and streams; a member
 * must not be stepped alone, nor change its map or injection. Not in the paper (its runs
 * are single simulations); the physics of each run is unchanged, so each run's result is
 * the same in a batch as alone. */
typedef struct cpic_batch cpic_batch;

/* max_runs: 1 .. 4096. stream: cudaStream_t the batch's graphs are launched on (NULL: the
 * batch creates and owns a non-blocking stream; graphs cannot be captured on the legacy
 * default stream). */
int cpic_batch_create(int max_runs, void* stream, cpic_batch** out);
int cpic_batch_destroy(cpic_batch* batch);
/* The run must have its map (CPIC_ERR_STATE) and be initialised; CPIC_ERR_CAPACITY when the
 * batch is full. Synchronises the run's stream. */
int cpic_batch_add(cpic_batch* batch, cpic_run* run);
int cpic_batch_remove(cpic_batch* batch, cpic_run* run);
int cpic_batch_size(const cpic_batch* batch, int* n);
/* How a batch step runs the particle push of its 2D members (the others always push in
 * their own branch of the step's graph):
 *   CPIC_BATCH_BRANCHES    each run's push in its branch, next to its other work;
 *   CPIC_BATCH_PERSISTENT  one persistent launch for all of them between a pre-push and a
 *                          post-push phase of per-run branches (the resident blocks walk the
 *                          runs' chunks from a device table of run parameters);
 *   CPIC_BATCH_AUTO        (default) the form measured faster on the batched configuration
 *                          (uneven runs of 10^4..2 10^6 particles): branches.
 * The results are the same in every mode. CPIC_ERR_INVALID for another value. */
#define CPIC_BATCH_AUTO 0
#define CPIC_BATCH_BRANCHES 1
#define CPIC_BATCH_PERSISTENT 2
int cpic_batch_set_mode(cpic_batch* batch, int mode);
/* nsteps batch steps; with_solve != 0: full PIC cycles (cpic_step), 0: fixed-field particle
 * steps (cpic_step_particles). Each run sorts on its own schedule. Asynchronous. */
int cpic_batch_step(cpic_batch* batch, int nsteps, int with_solve);
int cpic_batch_synchronize(cpic_batch* batch);

/* ---------------------------------------------------------------- served runs (row a12) */

/* A server runs parametric requests with continuous batching: requests queue on submit, a
 * scheduler thread admits them while a slot is free and the server's device pool holds the
 * run's footprint (first fit, smaller requests may pass one that does not fit yet), keeps
 * each admitted run's particles and fields on the device, advances all active runs a slice
 * of steps at a time on their own streams (their work overlaps on the GPU), and files each
 * result when its run has taken all its steps. A run's arithmetic is cpic_step's, so its
 * result does not depend on the other requests. Not in the paper (its runs are single
 * simulations). */
typedef struct cpic_server cpic_server;

#define CPIC_REQ_CYLINDER 0 /* 2D cylinder in plasma (annulus map, object at xi = 0, injection at xi = 1) */
#define CPIC_REQ_SPHERE 1   /* 3D sphere in plasma (shell map r0 (R/r0)^xi, polar caps cut at pi/32 and
                               specular, azimuth periodic, injection at the outer shell) */

typedef struct cpic_server_opts {
    size_t hbm_budget;     /* bytes of the device pool (0: half of the free device memory) */
    int32_t max_active;    /* runs on the device at once (0: 64) */
    int32_t steps_per_slice; /* steps a run advances per scheduling turn (0: 10) */
    int32_t sort_interval; /* cell sort interval of the runs (0: 4) */
} cpic_server_opts;

typedef struct cpic_request {
    int32_t kind;                  /* CPIC_REQ_* */
    int32_t n[3];                  /* cells per logical axis (radial, azimuthal[, polar]) */
    int64_t particles_per_species; /* initial macro-particles of electrons and of ions */
    double phi_object;             /* object potential (Dirichlet), in kT_e/e */
    double density;                /* plasma density (1 = the normalisation density) */
    double temperature;            /* electron temperature (1 = normalisation; vth_e = sqrt(T)) */
    double mass_ratio;             /* m_i / m_e (T_i = T_e) */
    double r_object, r_outer;      /* object and outer radius (Debye lengths) */
    double dt;                     /* time step (1/omega_pe) */
    int32_t steps;                 /* PIC cycles to run */
    uint64_t seed;                 /* load and injection streams */
} cpic_request;

typedef struct cpic_result {
    int32_t status;                /* CPIC_OK or the run's failure */
    uint64_t ticket;
    int32_t steps;                 /* cycles taken */
    double queue_s;                /* submit -> admission */
    double latency_s;              /* submit -> result (time-to-result) */
    int64_t particle_steps;        /* sum over the cycles of the live particles */
    double field_energy, kinetic_energy;
    int64_t n_particles[2], absorbed_object[2], absorbed_outer[2], injected[2];
    double current_object[2];      /* collected current per species, q w absorbed / (steps dt) */
    int32_t mg_cycles;             /* V-cycles of the last solve */
    char message[160];             /* when status != CPIC_OK: why the request failed (the
                                      scheduler thread's cpic_last_error text) */
} cpic_result;

int cpic_server_start(const cpic_server_opts* opts, cpic_server** out);
/* Queues a request (host memory, copied); ticket receives its id. CPIC_ERR_CAPACITY when
 * the run cannot fit the pool at all; CPIC_ERR_INVALID for a bad request. */
int cpic_server_submit(cpic_server* server, const cpic_request* req, uint64_t* ticket);
/* CPIC_OK and the result once the run is done (the ticket is then retired), CPIC_ERR_BUSY
 * while it is queued or running, CPIC_ERR_INVALID for an unknown ticket. */
int cpic_server_poll(cpic_server* server, uint64_t ticket, cpic_result* out);
/* Cancels a request: a queued one leaves the queue at once, an active one stops when the
 * slice of steps it has in flight ends (its device memory then returns to the pool). Its
 * result (cpic_server_poll) then has status CPIC_ERR_CANCELLED and the steps it took.
 * CPIC_ERR_STATE when the request is already done, CPIC_ERR_INVALID for an unknown ticket. */
int cpic_server_cancel(cpic_server* server, uint64_t ticket);
/* Requests queued, runs active, free bytes of the pool (any pointer may be NULL). */
int cpic_server_stats(cpic_server* server, int* queued, int* active, size_t* pool_free);
/* Stops the scheduler; active runs are finished on the device and discarded. */
int cpic_server_stop(cpic_server* server);

/* ---------------------------------------------------------------- tracing */

/* Phases of cpic_step timed with CUDA events recorded on the run's stream. */
#define CPIC_PHASE_FIELD 0   /* a1 vertex field, zeroing of the deposit grid */
#define CPIC_PHASE_PUSH 1    /* a2-a6 the fused push + deposit kernel alone */
#define CPIC_PHASE_INJECT 2  /* a8 injection, step counter, halo fold of the deposit grid */
#define CPIC_PHASE_SORT 3    /* a7 */
#define CPIC_PHASE_SOLVE 4   /* a9 right-hand side + multigrid + field energy */
#define CPIC_NPHASES 5
/* Enable (1) or disable (0) per-phase event timing of cpic_step (off by default). */
int cpic_profile(cpic_run* run, int enable);
/* Milliseconds per phase (ms[CPIC_NPHASES], host) and timed occurrences (count, host, may
 * be NULL) accumulated since the last read; synchronises and resets the accumulators. */
int cpic_profile_read(cpic_run* run, double* ms, int64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* CPIC_H */
