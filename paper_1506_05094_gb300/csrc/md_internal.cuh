// md_internal.cuh -- device-side data layout and kernel argument blocks shared by the kernels
// and the host runtime of the GB300 MD path.  Not part of the public ABI.
//
// Layout (all per-particle arrays are indexed by the device's cell-sorted slot; replica r owns
// slots [off_r, off_r + n_r), and the order inside a replica is (cell, user id)):
//   pos[2]      : position mirror, ping-pong by step parity.  Mixed precision: int4 of 32-bit
//                 fixed-point coordinates (unit L / 2^32, so 2^32 units are one period and the
//                 minimum image of a difference is its wrap to int32) and the type in .w.
//                 FP64: double4 with the type's bits in .w
//   xm,ym,zm    : master positions in [0, L), 8 bytes each.  Mixed precision: 64-bit fixed point
//                 (unit L / 2^64: the update is an exact integer add and the periodic wrap is the
//                 add's own wrap-around, no FP64 instruction).  FP64: doubles
//   img         : int4 periodic image counters (touched only when a particle wraps)
//   vel         : Real4 velocities v(t - dt/2), .w unused (float4 / double4)
//   id          : user index inside the replica
//   pos_build   : Real4 positions at the last list build (rebuild check, Sec. 6)
//   nbl         : int32 neighbour slots, column-major within 32-particle slices: neighbour k of
//                 slot i at ((i/32) * nmax + k) * 32 + i%32 (Sec. 5: first neighbours of the
//                 particles contiguous, then second, ...; one slice per warp)
//   nnb         : int32 neighbour counts
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MD_MAX_TYPES 8
#define MD_MAX_PAIRS (MD_MAX_TYPES * MD_MAX_TYPES)
#define MD_LOG_COLS 11
#define MD_NRED 6   // reduced quantities per tile: U, W, K, px, py, pz

// position mirror (V4T), velocities and forces (F4T), master positions (MT) per precision
template <typename R> struct V4T;
template <> struct V4T<float> { typedef int4 t; };
template <> struct V4T<double> { typedef double4_32a t; };
template <typename R> struct F4T;
template <> struct F4T<float> { typedef float4 t; };
template <> struct F4T<double> { typedef double4_32a t; };
template <typename R> struct MT;
template <> struct MT<float> { typedef unsigned long long t; };
template <> struct MT<double> { typedef double t; };

// Per replica description (device array, read-only inside a step).
struct SysDesc {
    int off, n;            // first slot, particle count
    int cell_off, nc;      // first cell, cells per box edge
    int tile_off, ntiles;  // first tile of the step kernel, tile count
    int reach;             // stencil half width in cells
    int span;              // cells visited per dimension (min(2 reach + 1, nc))
    double L, invL;
    float Lf, invLf, cell_scale;   // cell_scale = nc / L rounded to float (FP64 mode binning)
    float s64;             // (float)(2^64 / L): master-position units per unit length (mixed)
    float ps, ps2;         // (float)(L / 2^32) and (float)((L / 2^32)^2): the mirror unit (mixed)
    float ps_lo, ps2_lo;   // their rounding remainders: ps + ps_lo and ps2 + ps2_lo are exact to
                           // ~2^-48, so a length scaled from mirror units carries no systematic
                           // error of the unit's own rounding
    float pad2[2];
    double K0;             // (3n - 3) T0 / 2
};

// Work list of one rebuild pass (written by k_plan): the replicas rebuilt and prefix sums of
// their particle and cell counts (arrays plan_rep, plan_pp, plan_pc).
struct Plan {
    int nflag, tot_p, tot_c;
    int sort_now;   // O(N^2) method: this pass sorts by cell and builds from the cells
};

// Per type-pair LJ table (shifted potential, Sec. 2).
//   u(r)   = c12 r^-12 - c6 r^-6 - ushift    (c12 = 4 eps sigma^12, c6 = 4 eps sigma^6)
//   F_ij   = r^-2 (a12 r^-12 - a6 r^-6) r_ij (a12 = 12 c12, a6 = 6 c6)
//   rc2    = rc^2,  thr2 = (rc + s)^2 (neighbour threshold)
//   shifted force adds (r - rc) fc to u and removes fc / r from the scalar force, fc = |F|(rc)
struct PairTab {
    float rc2, c12, c6, ushift, a12, a6, thr2, pad;
    float fc, rc, padf[2];
    double rc2d, c12d, c6d, ushiftd, a12d, a6d, thr2d, padd;
    double fcd, rcd;
    // shifted-force Coulomb (Sec. 9): rc_C^2, q_a q_b, q_a q_b / rc_C^2, 2 q_a q_b / rc_C
    float qrc2, qq, qf, qu;
    double qrc2d, qqd, qfd, qud;
};

// Per replica thermostat carry and last-step record (FP64).
struct Thermo {
    double xi_prev;   // xi_{n-1}
    double K_prev;    // K_{n-1/2}
    double xi_next;   // xi_n of the next step (from the two above), and its leapfrog factors
    double A_next;    // 1 - xi_n dt / 2
    double B_next;    // 1 / (1 + xi_n dt / 2)
    double xi_int;    // sum_k xi_k dt
    double U, W, K_minus, K_plus, xi, px, py, pz;
    long long step;   // completed steps of this replica
    long long rebuilds;
};

// Global control block.
struct Ctrl {
    int halt;           // nonzero: every kernel returns at once
    int overflow;       // neighbour list overflowed at the last build
    int unstable;       // non-finite or runaway displacement seen
    int need_any;       // some replica needs a rebuild before the next step
    int max_count;      // largest neighbour count seen by the most recent builds
    unsigned int global_ticket;
    long long step;     // completed steps (all replicas step together)
    long long rebuild_passes;
    int q1, q2;         // replica queue cursors of the replica-resident kernel
    int rep_overflow;   // a replica-resident build overflowed (results stay exact; grow n_max)
    int pad;
};

template <typename R> struct StepArgs {
    typedef typename V4T<R>::t V4;
    typedef typename F4T<R>::t F4;
    typedef typename MT<R>::t M;
    const V4 *pos_in;
    V4 *pos_out;
    M *xm, *ym, *zm;
    F4 *vel;
    int4 *img;
    const V4 *pos_build;
    const int *nbl;
    const int *nnb;
    int nmax;                 // list capacity per particle (slice stride)
    const int *tile_rep;      // tile -> replica
    const SysDesc *sys;
    const PairTab *tab;
    int ntypes;
    int nrep;
    double inv_mass[MD_MAX_TYPES];
    double mass[MD_MAX_TYPES];
    Thermo *th;
    Ctrl *ctrl;
    int *moved;               // per replica: some particle moved > s/2 this step
    const int *need_in;       // per replica: rebuild before this step (read)
    int *need_out;            // per replica: rebuild before the next step (written)
    int *id_g;                // user ids (the replica-resident kernel permutes them)
    const int *rep_order;     // replicas by descending size (replica-resident queue)
    int rep_nmax, rep_cmax;   // largest replica and cell count (shared-memory sizing)
    int tile_threads;         // threads per tile (the grid kernel's block size)
    unsigned int *rep_ticket; // per replica tile tickets
    double *partial;          // per tile MD_NRED partial sums
    double *log;              // MD_LOG_COLS doubles per (row, replica) or null
    int log_cap;
    int integrator;           // 0 NVE, 1 Nose-Hoover
    double dt;
    double T0;
    double inv_tau2;
    R half_skin2;             // (s/2)^2
    float half_skin;          // s/2
    int rebuild_batch;        // K: rebuild slots every K steps (1: rebuild exactly when needed)
    unsigned *disp;           // per replica: max |r - r_build|^2 and max one-step |dr|^2 (float bits)
    int force_only;           // 1: write f_out / w_out, no integration and no bookkeeping
    F4 *f_out;                // fx, fy, fz, u_i
    R *w_out;
    cudaGraphConditionalHandle next_handle;
    int has_next;
    int need_filter;          // -1 all replicas; 0 / 1: only replicas whose need_in is 0 / nonzero
    int cutoff;               // 0 shifted potential, 1 shifted force
    int coulomb;              // 1: shifted-force Coulomb term between charged types
    int nolist;               // 1: no neighbour list, every pair of the replica is evaluated
    int launch_prio;          // host side: CUDA launch priority of this launch (0 = default)
    int lean;                 // host side: launch the register-capped step kernel (path 4)
};

template <typename R> struct RebuildArgs {
    typedef typename V4T<R>::t V4;
    typedef typename F4T<R>::t F4;
    typedef typename MT<R>::t M;
    V4 *pos;                 // current mirror (in/out, permuted)
    const V4 *key;           // positions the cells and the list are built from (== pos normally)
    int key_is_pos;
    M *xm, *ym, *zm;
    F4 *vel;
    int4 *img;
    int *id;
    V4 *pos_build;
    // scratch
    V4 *tpos, *tkey;
    M *txm, *tym, *tzm;
    F4 *tvel;
    int4 *timg;
    int *tid;
    int *cell_of, *rank, *perm;
    int *cell_start;         // Ctot + 1 entries
    int *count;              // Ctot entries, zero between passes
    const int *prep;         // slot -> replica
    const int *crep;         // cell -> replica
    int *nbl;
    int *nnb;
    int nmax;
    Plan *plan;
    int *plan_rep, *plan_pp, *plan_pc;
    int nsm;                 // SMs, for the persistent grids
    int tpb;                 // lanes per particle in the list build
    int pad;                 // lists are padded with the particle's own slot to a multiple of this
                             // (4 x the step kernel's threads per particle; n_max is a multiple)
    int sort_small;          // 1: one-CTA-per-replica fused sort (k_sort_small)
    int sort_nmax, sort_cmax;
    size_t sort_smem;
    int launch_prio;         // host side: CUDA launch priority of these launches (0 = default)
    int list_method;         // 0 sorted cells (Sec. 7), 1 O(N^2) scan (Sec. 6)
    int resort;              // O(N^2) method: every resort-th pass sorts by cell (0 never)
    const SysDesc *sys;
    const PairTab *tab;
    int ntypes;
    int nrep;
    int ntot;
    int ctot;
    const int *need_in;
    Ctrl *ctrl;
    Thermo *th;
};

// Launchers (defined in md_kernels_*.cu, one translation unit per precision).
template <typename R> cudaError_t launch_step(const StepArgs<R> &a, int tp, int block, int ntiles,
                                              cudaStream_t s);
template <typename R> cudaError_t launch_rebuild(const RebuildArgs<R> &a, cudaStream_t s);
template <typename R> cudaError_t launch_rebuild_timed(const RebuildArgs<R> &a, cudaStream_t s,
                                                       cudaEvent_t e0, cudaEvent_t e1);
cudaError_t launch_arm(const Ctrl *ctrl, cudaGraphConditionalHandle h, cudaStream_t s);
template <typename R> cudaError_t prepare_sort_small(size_t smem);

inline size_t sort_small_smem_bytes(int nmax, int cmax) {
    return (size_t)(2 * cmax + 1 + 3 * nmax) * 4;
}
// Replica-resident step kernel (FP32 / mixed precision only).
cudaError_t launch_rep(const StepArgs<float> &a, const RebuildArgs<float> &b, int tp, int block,
                       int grid, size_t smem, cudaStream_t s);
cudaError_t prepare_rep(int tp, int tpb, bool single, size_t smem);
// Grid step kernel with the replica's positions staged in shared memory (FP32 only).
cudaError_t launch_step_staged(const StepArgs<float> &a, int tp, int block, int ntiles,
                               size_t smem, cudaStream_t s);
cudaError_t prepare_step_staged(int tp, bool single, size_t smem);
// Dynamic shared memory of the replica-resident kernel for replicas of up to nmax particles and
// cmax cells with `block` threads and tp threads per particle.
inline size_t rep_smem_bytes(int nmax, int cmax, int block, int tp, int cta_threads) {
    const int P = block / tp;
    // tile partials, rounded up to whole rounds of cta_threads / block tiles
    const size_t per_round = (size_t)(cta_threads / block);
    const size_t tiles = (((size_t)(nmax + P - 1) / P + per_round - 1) / per_round) * per_round;
    return (size_t)nmax * 16 + (size_t)(2 * cmax + 1) * 4 + (size_t)2 * nmax * 4 + 16 +
           tiles * MD_NRED * 8;
}
