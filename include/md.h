/*
 * md.h -- C ABI of the GB300 molecular-dynamics hot path.
 *
 * One call of md_step advances every replica of an md_sim by leapfrog timesteps of a
 * Lennard-Jones 12-6 pair potential with the shifted-potential cutoff, evaluated over a Verlet
 * neighbour list that is rebuilt from a spatially sorted cell list whenever any particle of the
 * replica has moved more than half the skin since the last build.  This is the method of
 * Bailey et al., "RUMD: A general purpose molecular dynamics package optimized to utilize GPU
 * hardware down to a few thousand particles":
 *   - force, per-particle energy and virial over the neighbour list ........ Sec. 5, Fig. 2
 *   - neighbour list of all pairs within rc + s, column-major, with skin s .. Sec. 4, Sec. 5
 *   - rebuild when any particle moved more than s/2 (device-side flag) ..... Sec. 6 (O(N^2) text)
 *   - cell-index binning, sort of all particle data by cell, list build .... Sec. 7, Fig. 4
 *   - O(N^2) list build (with an occasional re-sort) and the no-list mode .. Sec. 6, Appendix
 *   - leapfrog NVE and Nose-Hoover NVT integrators .......................... Sec. 2
 *   - shifted-potential and shifted-force cutoffs ........................... Sec. 2
 *   - Coulomb interactions with a shifted-force cutoff ...................... Sec. 9
 *   - parameter search over list method, skin, threads per particle, block
 *     size and cell size, with a cache of tuned parameters .................. Appendix
 *
 * Conventions.
 *   - Every function returns an md_status (0 = MD_OK).  Errors are sticky per md_sim: after a
 *     failure of md_step / md_sync (MD_EUNSTABLE, MD_ECUDA, MD_ETIMEOUT) every later call that
 *     needs the device returns the same code until md_destroy.  Argument errors (MD_EINVAL)
 *     are not sticky.
 *   - All array arguments are HOST pointers owned by the caller; getters copy out, setters copy
 *     in.  The library owns every device buffer it allocates (cudaMalloc on the current
 *     device at md_create time) and frees them in md_destroy.
 *   - Particles of a replica are addressed in the caller's ("user") order 0..n_r-1 in every
 *     getter and setter, whatever order the library keeps them in on the device.
 *   - Positions are (n,3) row-major doubles; velocities (n,3) doubles holding v(t - dt/2) (the
 *     leapfrog half step); images (n,3) int32 periodic image counters.
 *   - Work is issued on the stream given by md_set_stream (default: a stream the library
 *     creates).  md_step returns after the requested steps have completed on the device.
 *   - Not thread-safe: one host thread per md_sim at a time.
 */
#ifndef GB300_MD_H
#define GB300_MD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_sim md_sim;

typedef enum {
    MD_OK = 0,
    MD_EINVAL = 1,     /* bad argument or violated precondition (no state change) */
    MD_ENOMEM = 2,     /* device or host allocation failed */
    MD_ECUDA = 3,      /* a CUDA runtime call failed (sticky) */
    MD_EUNSTABLE = 4,  /* non-finite position or a displacement > L/4 in one step (sticky) */
    MD_ETIMEOUT = 5,   /* a bounded device wait ran out (sticky) */
    MD_ESTATE = 6      /* call out of order, e.g. md_step before md_set_state of every replica */
} md_status;

/* cutoff methods (Sec. 2 "Pair potentials"): shift of the potential (continuous u), or shift of
 * the force (continuous u and F: a linear term (r - rc) |F|(rc) is added to the potential) */
enum { MD_SHIFTED_POTENTIAL = 0, MD_SHIFTED_FORCE = 1 };
enum { MD_MIXED = 0, MD_FP64 = 1 };             /* precision modes, see md_create */
enum { MD_NVE_LEAPFROG = 0, MD_NVT_NOSE_HOOVER = 1 };

/* LJ parameters of one (ordered) type pair; the matrix must be symmetric.  rc is absolute. */
typedef struct {
    double eps, sigma, rc;
} md_pair;

/* Thermodynamic record of the last completed step of one replica.  A completed step n evaluates
 * the forces at r_n, so after s completed steps the record describes time index n = s - 1. */
typedef struct {
    long long step;      /* n = completed steps - 1; -1 before the first step */
    int n;               /* particles in the replica */
    double V;            /* box volume L^3 */
    double U;            /* potential energy at r_n: sum_i u_i, u_i = 1/2 sum_j u_SP(r_ij) */
    double W;            /* virial at r_n: 1/3 sum_{i<j} r_ij . F_ij */
    double K;            /* kinetic energy at n: (K_{n-1/2} + K_{n+1/2}) / 2 */
    double K_minus;      /* K_{n-1/2} */
    double K_plus;       /* K_{n+1/2} */
    double T_kin;        /* 2 K / (3n - 3) */
    double P;            /* (n T_kin + W) / V */
    double xi;           /* Nose-Hoover friction xi_n (0 for NVE) */
    double xi_int;       /* sum_k xi_k dt */
    double H;            /* U + K (+ g T0 (tau^2 xi^2 / 2 + xi_int) for NVT): conserved */
    double sum_p[3];     /* total momentum of v_{n+1/2} */
} md_energies;

/* Counters kept by the runtime (host side; read after md_sync). */
typedef struct {
    long long steps;            /* completed steps */
    long long rebuild_passes;   /* device rebuild passes (any replica rebuilt) */
    long long replica_rebuilds; /* sum over replicas of list rebuilds */
    long long overflows;        /* neighbour-list overflows recovered by doubling n_max */
    int n_max;                  /* current neighbour-list capacity per particle */
    int max_neighbors;          /* largest neighbour count at the most recent build */
    int tp, block, reach;       /* threads per particle, threads per block, cell stencil reach */
    int build_lanes;            /* lanes per particle in the list build */
    int path;                   /* 1 grid, 2 replica-resident, 3 grid with staged positions */
    int list_method;            /* 0 sorted cells, 1 O(N^2) scan, 2 no list */
    int rebuild_batch;          /* K of md_set_rebuild_batch */
    int resort;                 /* interval of md_set_resort_interval */
    int rebuild_kernels;        /* kernels launched per rebuild pass on the grid path */
    int step_kernels;           /* step kernels per graph step (2: split around the rebuild) */
    int graph_block;            /* steps per captured CUDA graph (0 = plain launches) */
    long long n_total;          /* particles over all replicas */
    long long neighbor_entries; /* sum of neighbour counts at the most recent build */
    long long graph_builds;     /* CUDA graphs captured and instantiated so far (a timed region
                                   that must not include host-side graph construction can
                                   compare this before and after) */
} md_stats;

/* Average device durations measured with CUDA events by md_profile (milliseconds). */
typedef struct {
    double step_kernel_ms;       /* fused force + integrate + check + reduction kernel */
    double rebuild_ms;           /* one full rebuild pass (bin, scan, scatter, sort, gather, build) */
    double rebuild_fraction;     /* rebuild passes per step during the profiled steps */
    long long neighbor_entries;  /* sum of neighbour counts (for algorithmic bytes) */
    int steps;                   /* profiled steps */
} md_timing;

/* Create a simulation of n_replicas independent systems in cubic periodic boxes.
 *   n_particles[r] >= 2, box[r] = edge L_r > 2 (rc_max + skin) (minimum image, Sec. 4);
 *   params: n_types x n_types row-major LJ parameters (Sec. 2), symmetric, rc > 0, sigma > 0;
 *   mass: n_types masses (NULL = all 1);  skin > 0 (Sec. 4: list holds pairs with r < rc + s);
 *   cutoff_method: MD_SHIFTED_POTENTIAL or MD_SHIFTED_FORCE (the replica-resident and staged
 *   kernel paths support the shifted potential only);  precision: MD_MIXED (FP32 pair math and FP32
 *   per-particle accumulation; FP64 master positions, image update and energy/virial/momentum
 *   reductions) or MD_FP64 (every quantity in FP64).
 * n_types <= 8, n_replicas >= 1.  On success *out owns device memory for all replicas. */
int md_create(md_sim **out, int n_replicas, const int *n_particles, const double *box,
              int n_types, const md_pair *params, const double *mass, double skin,
              int cutoff_method, int precision);

/* Integrator (Sec. 2): MD_NVE_LEAPFROG, or MD_NVT_NOSE_HOOVER with target T and relaxation time
 * tau (friction update xi_n = xi_{n-1} + dt (K_{n-1/2}/K0 - 1)/tau^2, K0 = (3N-3) T / 2). */
int md_set_integrator(md_sim *sim, int kind, double dt, double T, double tau);

/* Load replica r (Sec. 2, Fig. 1: the simulation object starts from an initial configuration of
 * positions, types and velocities; here the caller passes it as arrays instead of a file):
 * pos (n,3) in any periodic image (wrapped into [0,L) here, the wrap added to the image
 * counters), type (n) in [0,n_types), vel (n,3) = v(t - dt/2) (the leapfrog half step of the
 * Sec. 2 integrators), image (n,3) or NULL.  Host arrays, read before the call returns; the
 * caller keeps them.  The state is packed on the host into a pinned staging area and loaded on
 * the md_sim's stream behind the steps already queued there, so the call does not wait for
 * the device (a later call on this md_sim, or md_sync, sees it complete).
 * Resets the replica's thermostat (xi = 0) and step record, and forces a list rebuild.
 * MD_EINVAL for a bad replica index, a NULL array, a type outside [0,n_types) or a non-finite
 * value (nothing is changed); MD_ECUDA (sticky) if a copy or launch fails. */
int md_set_state(md_sim *sim, int replica, const double *pos, const int *type, const double *vel,
                 const int *image);

/* Issue all device work on this cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream).
 * The paper runs one simulation per GPU (Sec. 2) and says nothing about streams; this call lets
 * the caller order the library's kernels with its own work.  The stream stays the caller's (it is
 * not destroyed); pending work on the previous stream is waited for first.  MD_ECUDA (sticky)
 * if that wait fails. */
int md_set_stream(md_sim *sim, void *cuda_stream);

/* Advance all replicas by n_steps >= 0 timesteps (Fig. 2 force kernel fused with the
 * integrator; rebuild of Fig. 4 on the device when the skin criterion fires).  Neighbour-list
 * overflow is recovered inside the call (capacity doubled, list rebuilt, the step redone),
 * as in Sec. 4.  Returns after the steps completed, or the first sticky error. */
int md_step(md_sim *sim, long long n_steps);

/* Wait for outstanding work on the md_sim's stream (the end of a Sec. 2 / Fig. 1 "Run" of
 * steps); surfaces sticky device errors (MD_ECUDA, MD_EUNSTABLE). */
int md_sync(md_sim *sim);

/* Copy replica r out in user order (the configuration that Sec. 2 saves to disk, positions with
 * their periodic images): pos (n,3) wrapped into [0,L), image (n,3), vel (n,3) = v(t - dt/2).
 * Host arrays owned by the caller; any pointer may be NULL.  Waits for the steps queued on the
 * md_sim's stream.  MD_ESTATE before md_set_state of this replica, MD_EINVAL for a bad replica
 * index. */
int md_get_state(md_sim *sim, int replica, double *pos, int *image, double *vel);

/* Thermodynamic record of replica r (see md_energies): the energy, virial, pressure and
 * temperature that Sec. 2 lists among RUMD's basic statistics, computed on the device with FP64
 * reductions at every step.  *out is caller-owned.  MD_EINVAL for a bad index or NULL out. */
int md_get_energies(md_sim *sim, int replica, md_energies *out);

/* Test hook: forces f (n,3), u_i (n), w_i (n) at the CURRENT positions of replica r (rebuilding
 * the list first if needed), user order; u_i = 1/2 sum_j u_SP, w_i = 1/6 sum_j r_ij . F_ij
 * (Fig. 2: per-particle energy halved for the double counting).  Any output may be NULL. */
int md_get_forces(md_sim *sim, int replica, double *f, double *u, double *w);

/* Test hook: neighbour list of replica r at its most recent build, as user indices.  counts[n];
 * nbrs (n, max_per_particle) row-major, each row in list order, unused slots -1.  Requires a
 * prior md_step or md_get_forces (the list exists only after a build).  MD_ESTATE when the list
 * method is MD_LIST_NONE (no list is kept). */
int md_get_neighbors(md_sim *sim, int replica, int max_per_particle, int *counts, int *nbrs);

/* Kernel shape: tp in {1,2,4,8,16,32} threads per particle in the force kernel (Sec. 3 t_p),
 * block threads per CTA (multiple of 32, tp <= block <= 1024), reach in {1,2,3}: cell edge
 * >= (rc_max + skin)/reach with a (2 reach + 1)^3 stencil (Sec. 7 uses reach 2), build_lanes in
 * {1,2,4,8,16,32} lanes per particle in the list build (Sec. 7 uses one thread per particle), or
 * MD_BUILD_CELL: one warp per cell builds the lists of all the cell's particles, loading each
 * stencil candidate once for the whole cell (grid kernel paths only).  The list order, hence
 * every result bit, does not depend on build_lanes.  0 keeps the current value. */
enum { MD_BUILD_CELL = 64 };
int md_set_tuning(md_sim *sim, int tp, int block, int reach, int build_lanes);
int md_get_tuning(md_sim *sim, int *tp, int *block, int *reach, int *build_lanes);

/* Neighbour-list capacity per particle (Sec. 4: a fixed N x n_max array, doubled automatically
 * when a build overflows).  The initial capacity is 1.35 x the ideal-gas count within
 * rc_max + skin plus 24.  Reallocates the list and forces a rebuild of every replica. */
int md_set_list_capacity(md_sim *sim, int n_max);

/* Kernel path: 1 = grid kernels (one CTA per tile of any replica; the rebuild is a chain of
 * kernels behind a CUDA-graph IF node), 2 = replica-resident kernel (persistent CTAs that each
 * run a whole step of one replica at a time in shared memory, rebuild included), 3 = grid kernels
 * with each tile's replica positions staged in shared memory for the neighbour gathers.  2 and 3
 * are mixed precision only and need replicas that fit in shared memory.  4 = the grid kernels
 * with the step kernel limited to 48 registers a thread (more resident warps to hide the
 * neighbour gathers' latency, at the price of a few register spills; faster for large single
 * systems, slower for small mixed ones).  0 = automatic (1; the autotuner times the others).
 * All paths give the same results bit for bit.  MD_EINVAL if the requested path does not apply. */
enum { MD_PATH_AUTO = 0, MD_PATH_GRID = 1, MD_PATH_REPLICA = 2, MD_PATH_STAGED = 3,
       MD_PATH_LEAN = 4 };
int md_set_path(md_sim *sim, int path);

/* Steps captured per CUDA graph replay (>= 1; graphs are kept per starting step parity, so an odd
 * block uses two), or 0 for plain kernel launches with device-side early exit of the rebuild
 * kernels (the baseline launch mode).  MD_EINVAL for a negative value. */
int md_set_graph_block(md_sim *sim, int steps);

/* Neighbour-list method (Appendix phase I): 0 = sorted cells (Sec. 7, Fig. 4: bin, sort all
 * particle data by cell, build over the cell stencil); 1 = O(N^2) scan of every particle of the
 * replica (Sec. 6, Fig. 3; no sort, for small replicas); 2 = no list, every pair of the replica is
 * evaluated each step (the paper's choice for very small systems).  All three follow the same
 * pair rule; forces agree to FP32 summation order.  0 is the default. */
enum { MD_LIST_CELLS = 0, MD_LIST_N2 = 1, MD_LIST_NONE = 2 };
int md_set_list_method(md_sim *sim, int method);

/* With the O(N^2) list method: every `passes`-th rebuild pass first sorts the particles by cell
 * and builds that pass's list from the cells, which keeps neighbours close in memory (Appendix,
 * step 5: near the crossover to the cell method a sort every few hundred rebuilds can pay).
 * 0 (default) never sorts; the other list methods ignore it.  MD_EINVAL for passes < 0. */
int md_set_resort_interval(md_sim *sim, int passes);

/* Shifted-force Coulomb term between charged particles (Sec. 9, the molten-salt benchmark: Coulomb
 * forces with a large shifted-force cutoff instead of a mesh method).  charge[n_types] in units of
 * sqrt(4 pi eps0 eps sigma) (the paper's reduced units), rc_coulomb the Coulomb cutoff rc_C:
 *   u_C(r) = q_a q_b (1/r - 1/rc_C + (r - rc_C)/rc_C^2),  F_ij = q_a q_b (1/r^2 - 1/rc_C^2) r_ij/r
 * for r < rc_C, added to the LJ term (which keeps its own rc_ab and cutoff method).  The list
 * range of every pair becomes max(rc_ab, rc_C) + s.  charge NULL switches the term off.  Needs
 * L > 2 (max(rc_max, rc_C) + s); MD_EINVAL otherwise, or for rc_coulomb <= 0 with charges, or a
 * non-finite charge (no state change).  Forces a rebuild of every replica; the Coulomb term runs
 * on the grid kernel path (paths 2 and 3 are not used while it is on). */
int md_set_coulomb(md_sim *sim, const double *charge, double rc_coulomb);

/* Rebuild slots for batches of replicas (the paper runs one system and has no counterpart; its
 * rule, a rebuild once some particle has moved more than s/2, Sec. 6, is kept).  K = 1 (default):
 * a replica rebuilds exactly when that rule fires.  K > 1: in addition, at every K-th step a
 * replica whose largest displacement since its build, grown by 1.5 x its largest one-step
 * displacement per step, would pass s/2 within K - 1 more steps rebuilds now, so that rebuilds
 * gather on the slot steps and one rebuild pass serves many replicas; the other steps usually
 * rebuild nothing and skip the pass.  The list is valid either way (the s/2 rule still fires
 * on any step); only the rebuild times, hence the list order and FP32 summation order, change.
 * 1 <= K <= 64, MD_EINVAL otherwise. */
int md_set_rebuild_batch(md_sim *sim, int k);

/* List skin s (Sec. 4): pairs within rc + s are listed and the list is rebuilt when a particle
 * has moved more than s/2.  Changes only the work done, never the physics.  Needs
 * L > 2 (rc_max + s) for every replica; forces a rebuild of every replica. */
int md_set_skin(md_sim *sim, double skin);
int md_get_skin(md_sim *sim, double *skin);

/* Parameter search of the Appendix, over the kernel path, the list method, the rebuild slots K
 * (batches of 8 or more replicas), tp, block, reach and build_lanes (and
 * the skin when flags has MD_TUNE_SKIN: 20% then 10% steps until the time stops falling): short
 * timed runs from the
 * current state (restored after every trial), single-minimum line searches with the break rules
 * of the Appendix.  cache_path (may be NULL) is a text file of tuned parameters keyed by the
 * user parameters and the GPU name; a hit skips the search.  The state is unchanged. */
enum { MD_TUNE_SKIN = 1 };
int md_autotune(md_sim *sim, const char *cache_path, int steps_per_trial, int flags);

/* Runtime counters. */
int md_get_stats(md_sim *sim, md_stats *out);

/* Run n_steps with plain launches and a CUDA event pair around every kernel; report average
 * durations.  Advances the simulation by n_steps (it is a real run). */
int md_profile(md_sim *sim, int n_steps, md_timing *out);

/* Per-step thermodynamic log on the device: capacity rows per replica (0 disables).  Each
 * completed step n writes (n, U, W, K_minus, K_plus, xi, xi_int, H, p_x, p_y, p_z). */
int md_set_log(md_sim *sim, int capacity);
/* Copy up to max_rows most recent rows of replica r, oldest first, 11 doubles per row; the
 * number of rows written is returned in *rows. */
int md_get_log(md_sim *sim, int replica, int max_rows, double *out, int *rows);

/* Bit-exact checkpoint: the full device state (positions, images, velocities, build positions,
 * thermostat carry, step counters, pending rebuild flags) in user order.  Loading it into an
 * md_sim created with the same arguments and tuning reproduces the uninterrupted trajectory
 * bit for bit. */
int md_checkpoint_size(md_sim *sim, size_t *bytes);
int md_save_checkpoint(md_sim *sim, void *buf, size_t bytes);
int md_load_checkpoint(md_sim *sim, const void *buf, size_t bytes);

/* Free every device and host buffer of the md_sim (the end of the Fig. 1 script's simulation
 * object, Sec. 2), after waiting for its stream.  NULL is ignored.  A stream given to
 * md_set_stream is not destroyed. */
void md_destroy(md_sim *sim);
/* Static text for an md_status code (the conventions above; unknown codes give a generic text).
 * The paper has no error interface; this is the C counterpart of the Python exceptions the
 * Fig. 1 script would see. */
const char *md_strerror(int status);

/* Measurement utility (the paper has no counterpart): the FP32 fused multiply-add throughput of
 * the current GPU in TFLOP/s (2 flops per FMA), the denominator of the step kernel's FP32
 * roofline.  Every SM is filled with independent FMA chains; the best of `repeats` >= 1 timed
 * launches on cuda_stream (NULL = legacy default stream) is returned in *tflops, the SM count in
 * *sms and that launch's duration in *ms (either may be NULL).  Allocates and frees a small
 * device buffer.  MD_EINVAL for repeats < 1 or a NULL tflops, MD_ENOMEM, MD_ECUDA. */
int md_measure_fp32_peak(void *cuda_stream, int repeats, double *tflops, int *sms, double *ms);

/* Forces of one system for callers that cannot allocate device memory at call time.
 *
 * The paper has no counterpart: this entry point exists for callers that may not call
 * cudaMalloc when they need forces -- a host framework that owns all device memory through its
 * own pool and forbids libraries from allocating their own, or a latency-critical loop that must
 * never enter the CUDA allocator (cudaMalloc / cudaFree can synchronise the device).  It needs no
 * md_sim and allocates nothing: inputs and outputs are the caller's device buffers, and the
 * scratch it needs (the particles sorted by cell) lives in one fixed array that every GPU loading
 * this library reserves (about 160 KB) and keeps until the process exits.
 *
 *   pos   (n,3) FP64 device array, any periodic image (folded into [0,L) on the device exactly
 *         as md_set_state folds it);  type (n) int32 device array, every entry in [0,n_types)
 *         (a particle with another type, and every particle within the stencil of one, gets NaN
 *         outputs; nothing is read out of bounds);
 *   L     cubic box edge, > 2 rc_max;  params n_types x n_types HOST array (symmetric);
 *   f     (n,3) FP64 device output;  u, w (n) FP64 device outputs or NULL (u_i = 1/2 sum u_SP,
 *         w_i = 1/6 sum r.F);  uw: 2 FP64 device outputs (U, W) or NULL;
 *   cuda_stream: stream to run on (NULL = the legacy default stream).
 * Limits: n <= MD_STATIC_MAX_PARTICLES and (floor(L / rc_max))^3 <= MD_STATIC_MAX_CELLS; larger
 * inputs return MD_EINVAL with a message on stderr.  Arithmetic is the mixed-precision pair math
 * of md_sim (forces agree with md_get_forces to FP32 summation order).
 * The first call on a device looks up the scratch array's device address (once per device);
 * make that first call before any stream capture.  All calls share the one scratch array, which
 * keeps the last call's contents: calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.  Returns MD_OK once the work is
 * queued on the stream. */
enum { MD_STATIC_MAX_PARTICLES = 8192, MD_STATIC_MAX_CELLS = 4096 };
int md_forces_static(const double *pos, const int *type, int n, double L, int n_types,
                     const md_pair *params, double *f, double *u, double *w, double *uw,
                     void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_MD_H */
