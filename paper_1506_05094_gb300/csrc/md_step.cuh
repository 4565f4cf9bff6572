// md_step.cuh -- the grid step kernel (k_step) and the per-particle pieces it shares with the
// replica-resident kernel: force sum over the list, integrator, tile and replica reductions.
#pragma once
#include "md_common.cuh"

namespace md {

// ------------------------------------------------------------------------------------------------
// Per-particle pieces shared by the grid kernel (k_step) and the replica-resident kernel (k_rep).
// ------------------------------------------------------------------------------------------------

// Neighbour positions read from global memory through the read-only path (grid kernel) ...
template <typename R> struct GlobalPos {
    const typename V4T<R>::t *p;
    __device__ __forceinline__ typename V4T<R>::t operator()(int j) const { return ld_nc(p + j); }
};
// ... or from the replica's positions staged in shared memory (slot j - off).
template <typename R> struct SharedPos {
    const typename V4T<R>::t *p;
    int off;
    __device__ __forceinline__ typename V4T<R>::t operator()(int j) const { return p[j - off]; }
};

// Force, u and w sums of slot i over its neighbour list (Fig. 2): TP lanes per particle, lane lt
// takes neighbours lt, lt + TP, ...; the next four indices are prefetched while four pairs are
// evaluated.
template <bool NC> __device__ __forceinline__ int ld_idx(const int *p) {
    if (NC) return __ldg(p);
    return *p;
}

// NC: the list may be read through the non-coherent read-only path (it was written by an
// earlier kernel); false when the same kernel has just built it.
template <typename R, int TP, bool SINGLE, typename Src, bool NC = true, int SF = 0>
__device__ __forceinline__ void force_sum(const StepArgs<R> &a, const Src &P4, int i,
                                          const typename V4T<R>::t &ri, int ti, const Frame<R> &F,
                                          int lt, const typename Coef4<R>::t *s_c0,
                                          const typename Coef4<R>::t *s_c1, R &fx, R &fy, R &fz,
                                          R &u, R &w,
                                          const typename Coef4<R>::t *s_cq = nullptr) {
    typedef typename V4T<R>::t V4;
    const typename Coef4<R>::t c1 = s_c0[0];
    const typename Coef4<R>::t c1b = s_c1[0];
    const int nn = a.nnb[i];
    // entries of this lane, rounded up to whole groups of four: the list is padded with the
    // particle's own slot (pad_list), so every index read is a valid entry and no lane tests bounds
    const int m = ((nn > lt ? (nn - lt + TP - 1) / TP : 0) + 3) & ~3;
    const int stride = TP * 32;
    const int *q = a.nbl + nbl_offset(i, lt, a.nmax);
    // groups of four entries, the indices of the next group loaded while this one is evaluated
    int j0 = 0, j1 = 0, j2 = 0, j3 = 0;
    if (m > 0) {
        j0 = ld_idx<NC>(q); j1 = ld_idx<NC>(q + stride); j2 = ld_idx<NC>(q + 2 * stride);
        j3 = ld_idx<NC>(q + 3 * stride);
    }
    for (int e = 0; e < m; e += 4) {
        const V4 r0 = P4(j0), r1 = P4(j1), r2 = P4(j2), r3 = P4(j3);
        q += 4 * stride;
        if (e + 4 < m) {   // prefetch the next four indices (Sec. 5 prefetching)
            j0 = ld_idx<NC>(q); j1 = ld_idx<NC>(q + stride); j2 = ld_idx<NC>(q + 2 * stride);
            j3 = ld_idx<NC>(q + 3 * stride);
        }
        interact<R, SINGLE, SF>(ri, ti, r0, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w, s_cq);
        interact<R, SINGLE, SF>(ri, ti, r1, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w, s_cq);
        interact<R, SINGLE, SF>(ri, ti, r2, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w, s_cq);
        interact<R, SINGLE, SF>(ri, ti, r3, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w, s_cq);
    }
}

// No list: every other particle of the replica, TP lanes per particle (the mode the paper uses
// for very small systems, Appendix).
template <typename R, int TP, bool SINGLE, int SF, typename Src>
__device__ __forceinline__ void force_all(const StepArgs<R> &a, const Src &P4, const SysDesc &S,
                                          int i, const typename V4T<R>::t &ri, int ti,
                                          const Frame<R> &F, int lt,
                                          const typename Coef4<R>::t *s_c0,
                                          const typename Coef4<R>::t *s_c1, R &fx, R &fy, R &fz,
                                          R &u, R &w,
                                          const typename Coef4<R>::t *s_cq = nullptr) {
    const typename Coef4<R>::t c1 = s_c0[0];
    const typename Coef4<R>::t c1b = s_c1[0];
    for (int j = S.off + lt; j < S.off + S.n; j += TP)
        if (j != i)
            interact<R, SINGLE, SF>(ri, ti, P4(j), F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz,
                                    u, w, s_cq);
}

// Merge the TP partial sums of each particle (replaces the serial shared-memory sum of Fig. 2).
template <typename R, int TP>
__device__ __forceinline__ void merge_lanes(R &fx, R &fy, R &fz, R &u, R &w) {
#pragma unroll
    for (int o = TP / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(FULL_MASK, fx, o);
        fy += __shfl_xor_sync(FULL_MASK, fy, o);
        fz += __shfl_xor_sync(FULL_MASK, fz, o);
        u += __shfl_xor_sync(FULL_MASK, u, o);
        w += __shfl_xor_sync(FULL_MASK, w, o);
    }
}

// Leapfrog NVE / Nose-Hoover NVT update of slot i (Sec. 2): velocity, master position with image
// counters, new mirror, skin check (Sec. 6).  Returns whether the particle moved more than s/2
// since the build, its kinetic energy and momentum, and the displacement measures of the rebuild
// slots.  A, B: Nose-Hoover factors (1 - xi dt/2) and 1/(1 + xi dt/2).
template <typename R>
__device__ __forceinline__ void kick(const StepArgs<R> &a, int i, R fx, R fy, R fz, R im, R m,
                                     R A, R B, typename F4T<R>::t &v, R &ke, R &px, R &py, R &pz) {
    const R dt = (R)a.dt;
    v = a.vel[i];
    if (a.integrator == 1) {
        v.x = (A * v.x + dt * fx * im) * B;
        v.y = (A * v.y + dt * fy * im) * B;
        v.z = (A * v.z + dt * fz * im) * B;
    } else {
        v.x += dt * fx * im;
        v.y += dt * fy * im;
        v.z += dt * fz * im;
    }
    a.vel[i] = v;
    ke = R(0.5) * m * (v.x * v.x + v.y * v.y + v.z * v.z);
    px = m * v.x;
    py = m * v.y;
    pz = m * v.z;
}

// runaway / non-finite displacement (more than L/4 in one step): halt
__device__ __forceinline__ void check_runaway(const Ctrl *c, bool ok) {
    if (!ok) {
        atomicExch((int *)&c->unstable, 1);
        atomicExch((int *)&c->halt, 1);
    }
}

// Mixed precision: the master position is 64-bit fixed point (2^64 units per period).  The
// FP32 displacement dt v is converted to those units (one rounding, 2^-24 relative, the FP32
// precision of v itself) and added as an integer: the add is exact, and a carry out of 64 bits is
// exactly a crossing of the box face, which moves the image counter.  The mirror is the master
// rounded to 32 bits.  No FP64 instruction.
__device__ __forceinline__ bool integrate_one(const StepArgs<float> &a, const SysDesc &S, int i,
                                              const int4 &ri, float fx, float fy, float fz,
                                              float im, float m, float A, float B, float &ke,
                                              float &px, float &py, float &pz, float &d2,
                                              float &st2) {
    float4 v;
    kick(a, i, fx, fy, fz, im, m, A, B, v, ke, px, py, pz);
    const float dt = (float)a.dt;
    const float ex = dt * v.x, ey = dt * v.y, ez = dt * v.z;
    const float lim = 0.25f * S.Lf;
    check_runaway(a.ctrl, fabsf(ex) < lim && fabsf(ey) < lim && fabsf(ez) < lim);
    const long long qx = __float2ll_rn(ex * S.s64), qy = __float2ll_rn(ey * S.s64),
                    qz = __float2ll_rn(ez * S.s64);
    const unsigned long long ox = a.xm[i], oy = a.ym[i], oz = a.zm[i];
    const unsigned long long nx = ox + (unsigned long long)qx, ny = oy + (unsigned long long)qy,
                             nz = oz + (unsigned long long)qz;
    a.xm[i] = nx;
    a.ym[i] = ny;
    a.zm[i] = nz;
    // a wrap of the unsigned add is a crossing of the face at 0 == L
    const int wx = qx > 0 ? (nx < ox) : -(int)(nx > ox);
    const int wy = qy > 0 ? (ny < oy) : -(int)(ny > oy);
    const int wz = qz > 0 ? (nz < oz) : -(int)(nz > oz);
    if (wx | wy | wz) {
        int4 g = a.img[i];
        g.x += wx; g.y += wy; g.z += wz;
        a.img[i] = g;
    }
    const int4 rn = make_int4((int)((nx + 0x80000000ull) >> 32), (int)((ny + 0x80000000ull) >> 32),
                              (int)((nz + 0x80000000ull) >> 32), ri.w);
    a.pos_out[i] = rn;
    const int4 pb = a.pos_build[i];
    const float bx = fixed_diff(rn.x, pb.x), by = fixed_diff(rn.y, pb.y), bz = fixed_diff(rn.z, pb.z);
    const float b2 = bx * bx + by * by + bz * bz;
    const float db2 = __fmaf_rn(b2, S.ps2, b2 * S.ps2_lo);
    d2 = db2;
    st2 = ex * ex + ey * ey + ez * ez;
    return db2 > a.half_skin2;
}

// FP64: the master position is a double; the wrap is decided exactly in FP64.
__device__ __forceinline__ bool integrate_one(const StepArgs<double> &a, const SysDesc &S, int i,
                                              const double4_32a &ri, double fx, double fy,
                                              double fz, double im, double m, double A, double B,
                                              double &ke, double &px, double &py, double &pz,
                                              float &d2, float &st2) {
    double4_32a v;
    kick(a, i, fx, fy, fz, im, m, A, B, v, ke, px, py, pz);
    const double dt = a.dt;
    double x = a.xm[i] + dt * v.x, y = a.ym[i] + dt * v.y, z = a.zm[i] + dt * v.z;
    int wx = 0, wy = 0, wz = 0;
    if (x >= S.L) { x -= S.L; wx = 1; } else if (x < 0.0) { x += S.L; wx = -1; }
    if (y >= S.L) { y -= S.L; wy = 1; } else if (y < 0.0) { y += S.L; wy = -1; }
    if (z >= S.L) { z -= S.L; wz = 1; } else if (z < 0.0) { z += S.L; wz = -1; }
    a.xm[i] = x;
    a.ym[i] = y;
    a.zm[i] = z;
    if (wx | wy | wz) {
        int4 g = a.img[i];
        g.x += wx; g.y += wy; g.z += wz;
        a.img[i] = g;
    }
    const double lim = 0.25 * S.L;
    check_runaway(a.ctrl, fabs(dt * v.x) < lim && fabs(dt * v.y) < lim && fabs(dt * v.z) < lim);
    const double4_32a rn = make_double4_32a(x, y, z, ri.w);
    a.pos_out[i] = rn;
    const double4_32a pb = a.pos_build[i];
    const double bx = min_image_fast(rn.x - pb.x, S.L, S.invL);
    const double by = min_image_fast(rn.y - pb.y, S.L, S.invL);
    const double bz = min_image_fast(rn.z - pb.z, S.L, S.invL);
    const double db2 = bx * bx + by * by + bz * bz;
    d2 = (float)db2;
    st2 = (float)(dt * dt * (v.x * v.x + v.y * v.y + v.z * v.z));
    return db2 > a.half_skin2;
}

// Warp maxima of the displacement measures into the replica's slots (non-negative floats order
// like their bit patterns, so the maximum is independent of the order of the atomics).
__device__ __forceinline__ void disp_max_warp(unsigned *slot, float d2, float st2) {
    const unsigned m1 = __reduce_max_sync(FULL_MASK, __float_as_uint(d2));
    const unsigned m2 = __reduce_max_sync(FULL_MASK, __float_as_uint(st2));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(slot, m1);
        atomicMax(slot + 1, m2);
    }
}

// Rebuild decision for the next step.  moved: some particle is more than s/2 from its build
// position, so the list is not valid for the next step (Sec. 6) -- always a rebuild.  With
// rebuild slots (K > 1) a replica that reaches a slot step also rebuilds when its largest
// displacement since the build, grown by 1.5 x its largest one-step displacement per step,
// would pass s/2 before the next slot: rebuilds then fall on the slot steps and a rebuild pass
// serves many replicas at once.  The list stays valid either way.
template <typename R>
__device__ __forceinline__ int rebuild_needed(const StepArgs<R> &a, long long next_step, int moved,
                                              float d2max, float st2max) {
    if (moved) return 1;
    const int K = a.rebuild_batch;
    if (K <= 1 || (next_step % K) != 0) return 0;
    const float grow = 1.5f * (float)(K - 1) * sqrtf(st2max);
    return (sqrtf(d2max) + grow > a.half_skin) ? 1 : 0;
}

// Exact sum of two floats as an unevaluated pair s + e (Knuth's TwoSum; every operation rounded
// on its own, none contracted).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// One level of the warp's pair tree: slot k of this lane and its partner at distance `off` are
// added exactly (hi by TwoSum, the rounding error and both lo parts into lo).
__device__ __forceinline__ void pair_add(float &h, float &l, float rh, float rl) {
    float s, e;
    two_sum(h, rh, s, e);
    h = s;
    l = __fadd_rn(__fadd_rn(l, rl), e);
}

// Warp sums of the MD_NRED per-particle quantities, each accurate to FP64 precision, written to
// out[q] (shared memory, the warp's row) by one lane each.  Mixed precision: the FP32 values are summed as exact float pairs (hi + lo) in a
// transposed tree -- at distance 16 each half of the warp keeps half of 8 slots (6 quantities, 2
// zeros), at 8 a quarter, at 4 an eighth, then every lane adds one slot -- so each lane does 9
// exact pair additions instead of 30 plain ones, and no FP64 instruction runs in the tree (the
// FP64 pipe of this GPU is a small fraction of the FP32 one).  The pair's relative error is about
// 2^-48, below FP64 rounding of the sum; hi + lo is then formed in FP64.  FP64 mode: plain FP64
// shuffle tree.  The tree is fixed, so the result is deterministic.  Call with the whole warp.
__device__ __forceinline__ void warp_sums(const float v[MD_NRED], double out[MD_NRED]) {
    const int lane = threadIdx.x & 31;
    float h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        h[k] = k < MD_NRED ? v[k] : 0.f;
        l[k] = 0.f;
    }
#pragma unroll
    for (int half = 4; half >= 1; half >>= 1) {   // distances 16, 8, 4: keep `half` slots
        const int off = half * 4;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float mh = up ? h[k + half] : h[k], ml = up ? l[k + half] : l[k];
            const float sh = up ? h[k] : h[k + half], sl = up ? l[k] : l[k + half];
            const float rh = __shfl_xor_sync(FULL_MASK, sh, off);
            const float rl = __shfl_xor_sync(FULL_MASK, sl, off);
            h[k] = mh;
            l[k] = ml;
            pair_add(h[k], l[k], rh, rl);
        }
    }
#pragma unroll
    for (int off = 2; off >= 1; off >>= 1) {
        const float rh = __shfl_xor_sync(FULL_MASK, h[0], off);
        const float rl = __shfl_xor_sync(FULL_MASK, l[0], off);
        pair_add(h[0], l[0], rh, rl);
    }
    // slot 0 of lane 4 q (lane bits 4, 3, 2 = the bits of q) holds quantity q: those lanes form
    // hi + lo in FP64 side by side and store it
    if ((lane & 3) == 0 && (lane >> 2) < MD_NRED) out[lane >> 2] = (double)h[0] + (double)l[0];
}
__device__ __forceinline__ void warp_sums(const double v[MD_NRED], double out[MD_NRED]) {
#pragma unroll
    for (int q = 0; q < MD_NRED; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL_MASK, x, o);
        if ((threadIdx.x & 31) == 0) out[q] = x;
    }
}

// Sum of one tile's per-particle values (u_i, w_i, kinetic energy, momentum): FP64-accurate warp
// sums (warp_sums), then across the tile's warps in FP64 in warp order; a tile is `tw`
// consecutive warps of the block (tw = blockDim/32 in the grid kernel).  Thread (k, q), k < tiles
// in the block, writes quantity q of tile k to out[k * MD_NRED + q].  Call with the whole block.
template <typename R>
__device__ __forceinline__ void tile_partial(const R vals[MD_NRED], double (*s_tmp)[MD_NRED],
                                             double *out, int tw) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_sums(vals, s_tmp[warp]);
    __syncthreads();
    const int ntile = nw / tw;
    if (threadIdx.x < ntile * MD_NRED) {
        const int k = threadIdx.x / MD_NRED, q = threadIdx.x % MD_NRED;
        double acc = 0.0;
        for (int ww = k * tw; ww < (k + 1) * tw; ++ww) acc += s_tmp[ww][q];
        out[k * MD_NRED + q] = acc;
    }
}

// Nose-Hoover friction of the next step from the carry (Sec. 2), and its leapfrog factors:
// xi_n = xi_{n-1} + dt (K_{n-1/2} / K0 - 1) / tau^2 (0 for NVE), A = 1 - xi_n dt / 2,
// B = 1 / (1 + xi_n dt / 2).  Computed once per replica when a step closes (and by the host when
// a state is loaded), so a tile only reads them; every operation is rounded on its own, so the
// host's copy of the formula gives the same bits.
__device__ __forceinline__ void next_factors(Thermo *T, int integrator, double dt, double K0,
                                             double inv_tau2) {
    double xi = 0.0;
    if (integrator == 1)
        xi = __dadd_rn(T->xi_prev,
                       __dmul_rn(__dmul_rn(dt, __dsub_rn(__ddiv_rn(T->K_prev, K0), 1.0)), inv_tau2));
    const double h = __dmul_rn(__dmul_rn(0.5, xi), dt);
    T->xi_next = xi;
    T->A_next = __dsub_rn(1.0, h);
    T->B_next = __ddiv_rn(1.0, __dadd_rn(1.0, h));
}

// Replica sums over its tile partials (fixed order for a fixed blockDim), thermostat carry,
// per-step log row and the rebuild flag of the next step.  Call with the whole block.
// Threads below nthr take tiles tt = thread, thread + nthr, ...; the others add exact zeros, so a
// larger block reproduces the grid kernel's tree (nthr = its blockDim) bit for bit.
template <typename R>
__device__ __forceinline__ void replica_finish(const StepArgs<R> &a, int r, const SysDesc &S,
                                               const double *partial, double xi, int moved,
                                               double (*s_tmp)[MD_NRED], double *s_red,
                                               bool from_global, int nthr, float d2max,
                                               float st2max) {
    double acc[MD_NRED];
#pragma unroll
    for (int q2 = 0; q2 < MD_NRED; ++q2) acc[q2] = 0.0;
    for (int tt = threadIdx.x; threadIdx.x < nthr && tt < S.ntiles; tt += nthr) {
        const double *pp = partial + (long long)tt * MD_NRED;
#pragma unroll
        for (int q2 = 0; q2 < MD_NRED; ++q2) acc[q2] += from_global ? __ldcg(pp + q2) : pp[q2];
    }
    block_reduce_nred(acc, s_tmp, s_red);
    if (threadIdx.x == 0) {
        Thermo *T = a.th + r;
        const double U = s_red[0], W = s_red[1], K = s_red[2];
        T->U = U;
        T->W = W;
        T->K_minus = T->K_prev;
        T->K_plus = K;
        T->xi = xi;
        T->px = s_red[3];
        T->py = s_red[4];
        T->pz = s_red[5];
        T->xi_int += xi * a.dt;
        T->xi_prev = xi;
        T->K_prev = K;
        next_factors(T, a.integrator, a.dt, S.K0, a.inv_tau2);
        const long long n = T->step;
        T->step = n + 1;
        if (a.log != nullptr && a.log_cap > 0) {
            double *row = a.log + ((long long)(n % a.log_cap) * a.nrep + r) * MD_LOG_COLS;
            const double Kn = 0.5 * (T->K_minus + K);
            double H = U + Kn;
            if (a.integrator == 1) {
                const double g = 2.0 * S.K0 / a.T0;
                H += g * a.T0 * (0.5 * xi * xi / a.inv_tau2 + T->xi_int);
            }
            row[0] = (double)n; row[1] = U; row[2] = W; row[3] = T->K_minus; row[4] = K;
            row[5] = xi; row[6] = T->xi_int; row[7] = H; row[8] = s_red[3]; row[9] = s_red[4];
            row[10] = s_red[5];
        }
        a.need_out[r] = rebuild_needed(a, n + 1, moved, d2max, st2max);
    }
}


template <typename R>
__device__ __forceinline__ void load_tables(const StepArgs<R> &a, typename Coef4<R>::t *s_c0,
                                            typename Coef4<R>::t *s_c1, R *s_im, R *s_m) {
    const int npair = a.ntypes * a.ntypes;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        s_c0[p] = coef0_of<R>(a.tab[p]);
        s_c1[p] = coef1_of<R>(a.tab[p]);
    }
    if (threadIdx.x < MD_MAX_TYPES) {
        s_im[threadIdx.x] = (R)a.inv_mass[threadIdx.x];
        s_m[threadIdx.x] = (R)a.mass[threadIdx.x];
    }
}

// The last block of a launch closes the step: OR of the next step's rebuild flags, step counter,
// IF-node condition of the next graph step.  Call with the whole block after s_glast is known.
template <typename R> __device__ __forceinline__ void close_step(const StepArgs<R> &a) {
    __threadfence();
    int any = 0;
    for (int rr = threadIdx.x; rr < a.nrep; rr += blockDim.x) any |= __ldcg(a.need_out + rr);
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        a.ctrl->need_any = any;
        a.ctrl->global_ticket = 0u;
        a.ctrl->q1 = 0;
        a.ctrl->q2 = 0;
        a.ctrl->step += 1;
        if (a.has_next) cudaGraphSetConditional(a.next_handle, (any && !a.ctrl->halt) ? 1u : 0u);
    }
}

// ------------------------------------------------------------------------------------------------
// Grid step kernel (any replica size).  One CTA = one tile of (blockDim / TP) particles of one
// replica; the last tile of a replica reduces its tile partials, the last replica closes the step.
// ------------------------------------------------------------------------------------------------
// STAGE: the CTA first copies its replica's positions into shared memory and gathers the
// neighbour positions from there (replicas that fit; the copy is repeated by every tile of the
// replica and is served from L2).
// SF: potential kind of interact() (bit 0 LJ shifted force, bit 1 Coulomb).
template <typename R, int TP, bool SINGLE, bool STAGE, int SF>
__device__ __forceinline__ void step_body(const StepArgs<R> &a) {
    typedef typename V4T<R>::t V4;
    typedef typename Coef4<R>::t C4;
    typedef typename Coef4<R>::t C2;
    extern __shared__ __align__(16) unsigned char k_step_smem[];

    __shared__ C4 s_c0[MD_MAX_PAIRS];
    __shared__ C2 s_c1[MD_MAX_PAIRS];
    __shared__ C4 s_cq[(SF & 2) ? MD_MAX_PAIRS : 1];
    __shared__ R s_im[MD_MAX_TYPES], s_m[MD_MAX_TYPES];
    __shared__ double s_tmp[32][MD_NRED];
    __shared__ double s_red[MD_NRED];
    __shared__ double s_xi;
    __shared__ R s_A, s_B;
    __shared__ int s_skip, s_last, s_glast;

    const int tile = blockIdx.x;
    const int r = a.tile_rep[tile];
    // split steps: replicas that rebuild this step and those that do not run in two launches
    // (the second overlaps the rebuild); a tile of the other class exits at once
    if (a.need_filter >= 0 && ((a.need_in[r] != 0) != (a.need_filter != 0))) return;
    const SysDesc S = a.sys[r];
    load_tables(a, s_c0, s_c1, s_im, s_m);
    if (SF & 2)
        for (int p = threadIdx.x; p < a.ntypes * a.ntypes; p += blockDim.x)
            s_cq[p] = coef2_of<R>(a.tab[p]);
    if (threadIdx.x == 0) {
        // one uniform decision per block: a halt or an unrecovered list overflow stops the step
        s_skip = *(volatile int *)&a.ctrl->halt | *(volatile int *)&a.ctrl->overflow;
        const Thermo *T = a.th + r;   // this step's friction and factors, set when the last closed
        s_xi = a.force_only ? 0.0 : T->xi_next;
        s_A = a.force_only ? R(1) : (R)T->A_next;
        s_B = a.force_only ? R(1) : (R)T->B_next;
    }
    __syncthreads();
    if (s_skip) return;
    V4 *s_pos = reinterpret_cast<V4 *>(k_step_smem);
    if (STAGE) {
        for (int k = threadIdx.x; k < S.n; k += blockDim.x) s_pos[k] = ld_nc(a.pos_in + S.off + k);
        __syncthreads();
    }

    const int P = blockDim.x / TP;
    const int lp = threadIdx.x / TP, lt = threadIdx.x % TP;
    const int li = (tile - S.tile_off) * P + lp;
    const bool active = li < S.n;
    const int i = S.off + li;

    R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    V4 ri{};
    int ti = 0;
    if (active) {
        ri = STAGE ? s_pos[li] : a.pos_in[i];
        ti = type_of(ri);
        const Frame<R> F = make_frame(ri, S);
        if (STAGE) {
            SharedPos<R> src{s_pos, S.off};
            force_sum<R, TP, SINGLE, SharedPos<R>, true, SF>(a, src, i, ri, ti, F, lt, s_c0, s_c1,
                                                             fx, fy, fz, u, w, s_cq);
        } else if (a.nolist) {
            GlobalPos<R> src{a.pos_in};
            force_all<R, TP, SINGLE, SF>(a, src, S, i, ri, ti, F, lt, s_c0, s_c1, fx, fy, fz, u, w,
                                         s_cq);
        } else {
            GlobalPos<R> src{a.pos_in};
            force_sum<R, TP, SINGLE, GlobalPos<R>, true, SF>(a, src, i, ri, ti, F, lt, s_c0, s_c1,
                                                             fx, fy, fz, u, w, s_cq);
        }
    }
    merge_lanes<R, TP>(fx, fy, fz, u, w);
    scale_force(S, fx, fy, fz);
    const bool leader = active && lt == 0;
    u *= R(0.5);          // Fig. 2: compensate the double counting of the full list
    w *= R(1.0 / 6.0);    // 1/2 (double counting) * 1/3 (virial)

    if (a.force_only) {
        if (leader) {
            a.f_out[i] = make_v4(fx, fy, fz, u);
            a.w_out[i] = w;
        }
        return;
    }

    const double xi = s_xi;
    R ke = 0, px = 0, py = 0, pz = 0;
    bool moved = false;
    float d2 = 0.f, st2 = 0.f;
    if (leader)
        moved = integrate_one(a, S, i, ri, fx, fy, fz, s_im[ti], s_m[ti], s_A, s_B, ke, px, py,
                              pz, d2, st2);
    if (__ballot_sync(FULL_MASK, moved) != 0u && (threadIdx.x & 31) == 0) atomicOr(a.moved + r, 1);
    if (a.rebuild_batch > 1) disp_max_warp(a.disp + 2 * r, d2, st2);

    const R vals[MD_NRED] = {leader ? u : R(0), leader ? w : R(0), ke, px, py, pz};
    tile_partial(vals, s_tmp, a.partial + (long long)tile * MD_NRED, blockDim.x >> 5);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(a.rep_ticket + r, 1u);
        s_last = (prev == (unsigned)(S.ntiles - 1));
    }
    __syncthreads();
    if (!s_last) return;

    // ---- last tile of replica r: FP64 replica sums in a fixed order, thermostat carry ----
    __threadfence();
    const int mv = __ldcg(a.moved + r);
    const float d2max = __uint_as_float(__ldcg(a.disp + 2 * r));
    const float st2max = __uint_as_float(__ldcg(a.disp + 2 * r + 1));
    replica_finish(a, r, S, a.partial + (long long)S.tile_off * MD_NRED, xi, mv, s_tmp, s_red,
                   true, (int)blockDim.x, d2max, st2max);
    if (threadIdx.x == 0) {
        a.moved[r] = 0;
        a.disp[2 * r] = 0u;
        a.disp[2 * r + 1] = 0u;
        a.rep_ticket[r] = 0u;
        __threadfence();
        const unsigned g = atomicAdd(&a.ctrl->global_ticket, 1u);
        s_glast = (g == (unsigned)(a.nrep - 1));
    }
    __syncthreads();
    if (!s_glast) return;
    close_step(a);
}

// The step kernel, and its register-capped form (kernel path 4): at most 48 registers a thread,
// so more warps are resident to hide the neighbour gathers' latency, at the price of a few spills.
// Which is faster depends on the system (measured: 10 % faster for 10^6 LJ particles, slower for
// the two-type ensemble); the autotuner times both.
template <typename R, int TP, bool SINGLE, bool STAGE = false, int SF = 0>
__global__ void __launch_bounds__(1024) k_step(const StepArgs<R> a) {
    step_body<R, TP, SINGLE, STAGE, SF>(a);
}
template <typename R, int TP, bool SINGLE, int SF = 0>
__global__ void __maxnreg__(48) k_step_lean(const StepArgs<R> a) {
    step_body<R, TP, SINGLE, false, SF>(a);
}

}  // namespace md
