// md_kernels.cuh -- sm_103a kernels of one MD timestep (included by one translation unit per
// precision, which instantiates the templates for its Real type).
//
//   k_step      force + energy + virial over the neighbour list (Sec. 5, Fig. 2) fused with the
//               leapfrog / Nose-Hoover update (Sec. 2), the skin check (Sec. 6) and the FP64
//               energy / virial / momentum reductions; tp threads per particle merged by warp
//               shuffles (Sec. 3 t_p).
//   k_bin .. k_build   the cell-sorted O(N) list rebuild of Sec. 7 / Fig. 4: cell index and
//               per-cell counts, per-replica exclusive scan (cellStart), slot assignment,
//               deterministic in-cell order by user id, permutation of all particle data, list
//               build over the (2 reach + 1)^3 cell stencil.
#pragma once
#include "md_internal.cuh"

namespace md {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ int type_of(float4 p) { return __float_as_int(p.w); }
__device__ __forceinline__ int type_of(double4_32a p) { return (int)__double_as_longlong(p.w); }

__device__ __forceinline__ float4 ld_nc(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ double4_32a ld_nc(const double4_32a *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float4 make_v4(float x, float y, float z, float w) {
    return make_float4(x, y, z, w);
}
__device__ __forceinline__ double4_32a make_v4(double x, double y, double z, double w) {
    return make_double4_32a(x, y, z, w);
}
__device__ __forceinline__ float type_word(float, int t) { return __int_as_float(t); }
__device__ __forceinline__ double type_word(double, int t) { return __longlong_as_double((long long)t); }

// Sliced column-major neighbour list (32-particle slices): neighbour k of slot i.  Within a
// slice the first neighbours of all 32 particles are contiguous, then the second, ... (Sec. 5),
// so a warp reads 128 B per k and walks its slice sequentially.
__host__ __device__ __forceinline__ long long nbl_offset(int i, int k, int nmax) {
    return (((long long)(i >> 5) * nmax + k) << 5) + (i & 31);
}

// Minimum image in the force kernel: d - L * rne(d / L) with round-to-nearest-even done by the
// 1.5 * 2^23 (resp. 2^52) shift, valid for |d / L| < 2^22; positions are wrapped so |d| < L.
__device__ __forceinline__ float min_image_fast(float d, float L, float invL) {
    float q = __fadd_rn(__fmaf_rn(d, invL, 12582912.0f), -12582912.0f);
    return __fmaf_rn(-L, q, d);
}
__device__ __forceinline__ double min_image_fast(double d, double L, double invL) {
    double q = __dadd_rn(__fma_rn(d, invL, 6755399441055744.0), -6755399441055744.0);
    return __fma_rn(-L, q, d);
}

// Minimum image of the list build, bit-defined: every product and sum rounded on its own.
__device__ __forceinline__ float min_image_exact(float d, float L, float invL) {
    float t = rintf(__fmul_rn(d, invL));
    return __fsub_rn(d, __fmul_rn(L, t));
}
__device__ __forceinline__ double min_image_exact(double d, double L, double invL) {
    double t = rint(__dmul_rn(d, invL));
    return __dsub_rn(d, __dmul_rn(L, t));
}
__device__ __forceinline__ float dist2_exact(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}
__device__ __forceinline__ double dist2_exact(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

template <typename R> __device__ __forceinline__ R box_L(const SysDesc &S);
template <> __device__ __forceinline__ float box_L<float>(const SysDesc &S) { return S.Lf; }
template <> __device__ __forceinline__ double box_L<double>(const SysDesc &S) { return S.L; }
template <typename R> __device__ __forceinline__ R box_invL(const SysDesc &S);
template <> __device__ __forceinline__ float box_invL<float>(const SysDesc &S) { return S.invLf; }
template <> __device__ __forceinline__ double box_invL<double>(const SysDesc &S) { return S.invL; }

// Per type-pair coefficients in shared memory: {rc2, c12, c6, ushift} and {a12, a6}.
template <typename R> struct Coef4;
template <> struct Coef4<float> { typedef float4 t; };
template <> struct Coef4<double> { typedef double4_32a t; };
template <typename R> struct Coef2;
template <> struct Coef2<float> { typedef float2 t; };
template <> struct Coef2<double> { typedef double2 t; };

template <typename R> __device__ __forceinline__ typename Coef4<R>::t coef0_of(const PairTab &p);
template <> __device__ __forceinline__ float4 coef0_of<float>(const PairTab &p) {
    return make_float4(p.rc2, p.c12, p.c6, p.ushift);
}
template <> __device__ __forceinline__ double4_32a coef0_of<double>(const PairTab &p) {
    return make_double4_32a(p.rc2d, p.c12d, p.c6d, p.ushiftd);
}
template <typename R> __device__ __forceinline__ typename Coef2<R>::t coef1_of(const PairTab &p);
template <> __device__ __forceinline__ float2 coef1_of<float>(const PairTab &p) {
    return make_float2(p.a12, p.a6);
}
template <> __device__ __forceinline__ double2 coef1_of<double>(const PairTab &p) {
    return make_double2(p.a12d, p.a6d);
}

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// One pair's contribution (the fij / ComputeInteraction of Sec. 5) for LJ with shifted potential:
// F_ij = r^-2 (a12 r^-12 - a6 r^-6) r_ij, u += c12 r^-12 - c6 r^-6 - ushift, w += r_ij . F_ij.
template <typename R, typename C4, typename C2>
__device__ __forceinline__ void lj_pair(R dx, R dy, R dz, R r2, const C4 &c, const C2 &b, R &fx,
                                        R &fy, R &fz, R &u, R &w) {
    const R r2i = fast_rcp(r2);
    const R r6i = r2i * r2i * r2i;
    const R fs = r2i * r6i * (b.x * r6i - b.y);
    fx += fs * dx;
    fy += fs * dy;
    fz += fs * dz;
    u += r6i * (c.y * r6i - c.z) - c.w;
    w += fs * r2;
}

// Per-particle minimum-image frame.
//
// FP32: the plain d - L*rint(d/L) loses up to ulp(L)/2 on pairs that cross the periodic boundary
// (the difference of a coordinate near L and one near 0 is rounded before L is removed), and
// (float)L != L adds a systematic offset.  Instead the coordinate near L is shifted by L first,
// which is exact (Sterbenz), and L - (float)L is folded into the particle's own shifted
// coordinate once per particle:
//   t = x_i - x_j;  if |t| > L/2:  d = xa_i - (x_j - n_i L)   else  d = t
// with, for x_i >= L/2 (partners can only cross upward): xa_i = x_i - L, n_i = 0, and for
// x_i < L/2: xa_i = x_i + (L - (float)L), n_i = 1 (the partner near L is shifted instead).
// Five FP32 instructions per dimension, all on the FMA pipe.
// FP64: the plain rint form is accurate to the FP64 rounding of the coordinates.
template <typename R> struct Frame;
template <> struct Frame<float> { float xa, ya, za, nx, ny, nz, half, L; };
template <> struct Frame<double> { double L, invL; };

__device__ __forceinline__ Frame<float> make_frame(const float4 &ri, const SysDesc &S) {
    // x_i - L is exact for x_i >= L/2 (Sterbenz); the L - (float)L remainder (Llo) is then
    // removed from a small number, and added to x_i < L/2 whose crossing partners sit near L.
    Frame<float> F;
    const float L = S.Lf, h = S.halfLf, lo = S.Llo;
    const bool ux = ri.x >= h, uy = ri.y >= h, uz = ri.z >= h;
    F.xa = ux ? __fsub_rn(__fsub_rn(ri.x, L), lo) : __fadd_rn(ri.x, lo);
    F.ya = uy ? __fsub_rn(__fsub_rn(ri.y, L), lo) : __fadd_rn(ri.y, lo);
    F.za = uz ? __fsub_rn(__fsub_rn(ri.z, L), lo) : __fadd_rn(ri.z, lo);
    F.nx = ux ? 0.0f : 1.0f;
    F.ny = uy ? 0.0f : 1.0f;
    F.nz = uz ? 0.0f : 1.0f;
    F.half = h;
    F.L = L;
    return F;
}
__device__ __forceinline__ Frame<double> make_frame(const double4_32a &, const SysDesc &S) {
    Frame<double> F;
    F.L = S.L;
    F.invL = S.invL;
    return F;
}

__device__ __forceinline__ float mi_axis(float xi, float xj, float xa, float n, float half,
                                         float L) {
    const float t = __fsub_rn(xi, xj);
    const float e = __fsub_rn(xa, __fmaf_rn(-n, L, xj));
    return fabsf(t) > half ? e : t;
}

__device__ __forceinline__ void pair_delta(const Frame<float> &F, const float4 &ri,
                                           const float4 &rj, float &dx, float &dy, float &dz) {
    dx = mi_axis(ri.x, rj.x, F.xa, F.nx, F.half, F.L);
    dy = mi_axis(ri.y, rj.y, F.ya, F.ny, F.half, F.L);
    dz = mi_axis(ri.z, rj.z, F.za, F.nz, F.half, F.L);
}
__device__ __forceinline__ void pair_delta(const Frame<double> &F, const double4_32a &ri,
                                           const double4_32a &rj, double &dx, double &dy,
                                           double &dz) {
    dx = min_image_fast(ri.x - rj.x, F.L, F.invL);
    dy = min_image_fast(ri.y - rj.y, F.L, F.invL);
    dz = min_image_fast(ri.z - rj.z, F.L, F.invL);
}

template <typename R, bool SINGLE>
__device__ __forceinline__ void interact(const typename V4T<R>::t &ri, int ti,
                                         const typename V4T<R>::t &rj, const Frame<R> &F, int nt,
                                         const typename Coef4<R>::t *s_c0,
                                         const typename Coef2<R>::t *s_c1,
                                         const typename Coef4<R>::t &c1,
                                         const typename Coef2<R>::t &c1b, R &fx, R &fy, R &fz,
                                         R &u, R &w) {
    R dx, dy, dz;
    pair_delta(F, ri, rj, dx, dy, dz);
    const R r2 = dx * dx + dy * dy + dz * dz;
    if (SINGLE) {
        if (r2 < c1.x) lj_pair(dx, dy, dz, r2, c1, c1b, fx, fy, fz, u, w);
    } else {
        const int p = ti * nt + type_of(rj);
        const typename Coef4<R>::t c = s_c0[p];
        if (r2 < c.x) lj_pair(dx, dy, dz, r2, c, s_c1[p], fx, fy, fz, u, w);
    }
}

// Deterministic block reduction of MD_NRED doubles (fixed tree for a fixed blockDim).
__device__ __forceinline__ void block_reduce_nred(double v[MD_NRED], double (*s_tmp)[MD_NRED],
                                                  double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < MD_NRED; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(FULL_MASK, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < MD_NRED; ++q) s_tmp[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < MD_NRED) {
        double acc = 0.0;
        for (int ww = 0; ww < nw; ++ww) acc += s_tmp[ww][threadIdx.x];
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

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
template <typename R, int TP, bool SINGLE, typename Src, bool NC = true>
__device__ __forceinline__ void force_sum(const StepArgs<R> &a, const Src &P4, int i,
                                          const typename V4T<R>::t &ri, int ti, const Frame<R> &F,
                                          int lt, const typename Coef4<R>::t *s_c0,
                                          const typename Coef2<R>::t *s_c1, R &fx, R &fy, R &fz,
                                          R &u, R &w) {
    typedef typename V4T<R>::t V4;
    const typename Coef4<R>::t c1 = s_c0[0];
    const typename Coef2<R>::t c1b = s_c1[0];
    const int nn = a.nnb[i];
    // sliced column-major list: neighbour k of slot i at ((i/32)*nmax + k)*32 + i%32
    const int stride = TP * 32;
    const int *q = a.nbl + nbl_offset(i, lt, a.nmax);
    int k = lt;
    int j0 = 0, j1 = 0, j2 = 0, j3 = 0;
    if (k + 3 * TP < nn) {
        j0 = ld_idx<NC>(q); j1 = ld_idx<NC>(q + stride); j2 = ld_idx<NC>(q + 2 * stride); j3 = ld_idx<NC>(q + 3 * stride);
    }
    for (; k + 3 * TP < nn; k += 4 * TP) {
        const V4 r0 = P4(j0), r1 = P4(j1), r2 = P4(j2), r3 = P4(j3);
        q += 4 * stride;
        if (k + 7 * TP < nn) {   // prefetch the next four indices (Sec. 5 prefetching)
            j0 = ld_idx<NC>(q); j1 = ld_idx<NC>(q + stride); j2 = ld_idx<NC>(q + 2 * stride);
            j3 = ld_idx<NC>(q + 3 * stride);
        }
        interact<R, SINGLE>(ri, ti, r0, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
        interact<R, SINGLE>(ri, ti, r1, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
        interact<R, SINGLE>(ri, ti, r2, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
        interact<R, SINGLE>(ri, ti, r3, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
    }
    for (; k < nn; k += TP) {
        const int j = ld_idx<NC>(q);
        q += stride;
        interact<R, SINGLE>(ri, ti, P4(j), F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
    }
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

// Leapfrog NVE / Nose-Hoover NVT update of slot i (Sec. 2), FP64 master position with image
// counters, new FP32 mirror, skin check (Sec. 6).  Returns the particle's kinetic energy and
// momentum.  A, B: Nose-Hoover factors (1 - xi dt/2) and 1/(1 + xi dt/2).
template <typename R>
__device__ __forceinline__ bool integrate_one(const StepArgs<R> &a, const SysDesc &S, int i,
                                              const typename V4T<R>::t &ri, R fx, R fy, R fz,
                                              R im, R m, R A, R B, R &ke, R &px, R &py, R &pz) {
    typedef typename V4T<R>::t V4;
    const R dt = (R)a.dt;
    V4 v = a.vel[i];
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
    // FP64 master position, wrap and image (the mixed-precision contract).  The wrap is detected
    // on the rounded mirror (it can only round up to L, never below 0) and decided exactly in FP64
    // only when the mirror says the particle may have left [0, L).
    double x = a.xd[i] + (double)(dt * v.x), y = a.yd[i] + (double)(dt * v.y),
           z = a.zd[i] + (double)(dt * v.z);
    const R Lr = box_L<R>(S);
    int wx = 0, wy = 0, wz = 0;
    if (!((R)x < Lr && (R)x >= R(0))) {
        if (x >= S.L) { x -= S.L; wx = 1; } else if (x < 0.0) { x += S.L; wx = -1; }
    }
    if (!((R)y < Lr && (R)y >= R(0))) {
        if (y >= S.L) { y -= S.L; wy = 1; } else if (y < 0.0) { y += S.L; wy = -1; }
    }
    if (!((R)z < Lr && (R)z >= R(0))) {
        if (z >= S.L) { z -= S.L; wz = 1; } else if (z < 0.0) { z += S.L; wz = -1; }
    }
    a.xd[i] = x;
    a.yd[i] = y;
    a.zd[i] = z;
    if (wx | wy | wz) {
        int4 g = a.img[i];
        g.x += wx; g.y += wy; g.z += wz;
        a.img[i] = g;
    }
    const R lim = (R)(0.25 * S.L);   // runaway / non-finite displacement
    if (!(fabs(dt * v.x) < lim && fabs(dt * v.y) < lim && fabs(dt * v.z) < lim)) {
        atomicExch(&a.ctrl->unstable, 1);
        atomicExch(&a.ctrl->halt, 1);
    }
    const V4 rn = make_v4((R)x, (R)y, (R)z, ri.w);
    a.pos_out[i] = rn;
    const V4 pb = a.pos_build[i];
    const R L = box_L<R>(S), invL = box_invL<R>(S);
    const R bx = min_image_fast(rn.x - pb.x, L, invL);
    const R by = min_image_fast(rn.y - pb.y, L, invL);
    const R bz = min_image_fast(rn.z - pb.z, L, invL);
    return (bx * bx + by * by + bz * bz) > a.half_skin2;
}

// Sum of one tile's per-particle values: within a warp in R, across the tile's warps in FP64 in
// warp order; a tile is `tw` consecutive warps of the block (tw = blockDim/32 in the grid kernel).
// Thread (k, q), k < tiles in the block, writes quantity q of tile k to out[k * MD_NRED + q].
// Call with the whole block.
template <typename R>
__device__ __forceinline__ void tile_partial(R vals[MD_NRED], double (*s_tmp)[MD_NRED],
                                             double *out, int tw) {
#pragma unroll
    for (int q2 = 0; q2 < MD_NRED; ++q2)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vals[q2] += __shfl_down_sync(FULL_MASK, vals[q2], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q2 = 0; q2 < MD_NRED; ++q2) s_tmp[warp][q2] = (double)vals[q2];
    __syncthreads();
    const int ntile = nw / tw;
    if (threadIdx.x < ntile * MD_NRED) {
        const int k = threadIdx.x / MD_NRED, q = threadIdx.x % MD_NRED;
        double acc = 0.0;
        for (int ww = k * tw; ww < (k + 1) * tw; ++ww) acc += s_tmp[ww][q];
        out[k * MD_NRED + q] = acc;
    }
}

// Replica sums over its tile partials (fixed order for a fixed blockDim), thermostat carry,
// per-step log row and the rebuild flag of the next step.  Call with the whole block.
// Threads below nthr take tiles tt = thread, thread + nthr, ...; the others add exact zeros, so a
// larger block reproduces the grid kernel's tree (nthr = its blockDim) bit for bit.
template <typename R>
__device__ __forceinline__ void replica_finish(const StepArgs<R> &a, int r, const SysDesc &S,
                                               const double *partial, double xi, int moved,
                                               double (*s_tmp)[MD_NRED], double *s_red,
                                               bool from_global, int nthr) {
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
        a.need_out[r] = moved;
    }
}

// Nose-Hoover friction of this step from the previous step's carry (one thread).
template <typename R>
__device__ __forceinline__ double step_xi(const StepArgs<R> &a, const SysDesc &S, int r) {
    if (a.integrator != 1 || a.force_only) return 0.0;
    const Thermo *T = a.th + r;
    return T->xi_prev + a.dt * (T->K_prev / S.K0 - 1.0) * a.inv_tau2;
}

template <typename R>
__device__ __forceinline__ void load_tables(const StepArgs<R> &a, typename Coef4<R>::t *s_c0,
                                            typename Coef2<R>::t *s_c1, R *s_im, R *s_m) {
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
template <typename R, int TP, bool SINGLE>
__global__ void __launch_bounds__(1024) k_step(const StepArgs<R> a) {
    typedef typename V4T<R>::t V4;
    typedef typename Coef4<R>::t C4;
    typedef typename Coef2<R>::t C2;

    __shared__ C4 s_c0[MD_MAX_PAIRS];
    __shared__ C2 s_c1[MD_MAX_PAIRS];
    __shared__ R s_im[MD_MAX_TYPES], s_m[MD_MAX_TYPES];
    __shared__ double s_tmp[32][MD_NRED];
    __shared__ double s_red[MD_NRED];
    __shared__ double s_xi;
    __shared__ R s_A, s_B;
    __shared__ int s_skip, s_last, s_glast;

    const int tile = blockIdx.x;
    const int r = a.tile_rep[tile];
    const SysDesc S = a.sys[r];
    load_tables(a, s_c0, s_c1, s_im, s_m);
    if (threadIdx.x == 0) {
        // one uniform decision per block: a halt or an unrecovered list overflow stops the step
        s_skip = *(volatile int *)&a.ctrl->halt | *(volatile int *)&a.ctrl->overflow;
        const double xi = step_xi(a, S, r);
        s_xi = xi;
        s_A = (R)(1.0 - 0.5 * xi * a.dt);
        s_B = (R)(1.0 / (1.0 + 0.5 * xi * a.dt));
    }
    __syncthreads();
    if (s_skip) return;

    const int P = blockDim.x / TP;
    const int lp = threadIdx.x / TP, lt = threadIdx.x % TP;
    const int li = (tile - S.tile_off) * P + lp;
    const bool active = li < S.n;
    const int i = S.off + li;

    R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    V4 ri = make_v4(R(0), R(0), R(0), R(0));
    int ti = 0;
    if (active) {
        ri = a.pos_in[i];
        ti = type_of(ri);
        const Frame<R> F = make_frame(ri, S);
        GlobalPos<R> src{a.pos_in};
        force_sum<R, TP, SINGLE>(a, src, i, ri, ti, F, lt, s_c0, s_c1, fx, fy, fz, u, w);
    }
    merge_lanes<R, TP>(fx, fy, fz, u, w);
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
    if (leader)
        moved = integrate_one(a, S, i, ri, fx, fy, fz, s_im[ti], s_m[ti], s_A, s_B, ke, px, py,
                              pz);
    if (__ballot_sync(FULL_MASK, moved) != 0u && (threadIdx.x & 31) == 0) atomicOr(a.moved + r, 1);

    R vals[MD_NRED] = {u * R(leader), w * R(leader), ke, px, py, pz};
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
    replica_finish(a, r, S, a.partial + (long long)S.tile_off * MD_NRED, xi, mv, s_tmp, s_red,
                   true, (int)blockDim.x);
    if (threadIdx.x == 0) {
        a.moved[r] = 0;
        a.rep_ticket[r] = 0u;
        __threadfence();
        const unsigned g = atomicAdd(&a.ctrl->global_ticket, 1u);
        s_glast = (g == (unsigned)(a.nrep - 1));
    }
    __syncthreads();
    if (!s_glast) return;
    close_step(a);
}

// ------------------------------------------------------------------------------------------------
// Rebuild (Sec. 7).  k_plan compacts the replicas whose need flag is set into a work list; the
// other kernels grid-stride over that list only (no blocks are spent on replicas that keep their
// list).  halt and need_any only change between passes, so every thread sees the same values.
// An overflow does not stop a pass: the copy back of the permuted data must always complete.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool rebuild_off(const Ctrl *c) {
    return *(volatile const int *)&c->halt || !*(volatile const int *)&c->need_any;
}

// largest k in [0, n) with pfx[k] <= t  (pfx ascending, pfx[0] = 0)
__device__ __forceinline__ int find_seg(const int *pfx, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pfx[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename V4> __device__ __forceinline__ int cell_index(const V4 &p, const SysDesc &S) {
    const float cs = S.cell_scale;
    int cx = __float2int_rd(__fmul_rn((float)p.x, cs));
    int cy = __float2int_rd(__fmul_rn((float)p.y, cs));
    int cz = __float2int_rd(__fmul_rn((float)p.z, cs));
    cx = min(max(cx, 0), S.nc - 1);
    cy = min(max(cy, 0), S.nc - 1);
    cz = min(max(cz, 0), S.nc - 1);
    return (cz * S.nc + cy) * S.nc + cx;
}

// One CTA: exclusive scans over replicas of (flagged, particles, cells) -> the pass's work list.
template <typename R> __global__ void k_plan(const RebuildArgs<R> a) {
    __shared__ int s_w[3][32];
    const int R_ = a.nrep, nt = blockDim.x;
    if (rebuild_off(a.ctrl)) {
        if (threadIdx.x == 0) { a.plan->nflag = 0; a.plan->tot_p = 0; a.plan->tot_c = 0; }
        return;
    }
    const int chunk = (R_ + nt - 1) / nt;
    const int r0 = min(R_, (int)threadIdx.x * chunk), r1 = min(R_, r0 + chunk);
    int f = 0, np = 0, nc = 0;
    for (int r = r0; r < r1; ++r)
        if (a.need_in[r]) {
            const SysDesc &S = a.sys[r];
            ++f; np += S.n; nc += S.nc * S.nc * S.nc;
        }
    int v[3] = {f, np, nc}, x[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        x[q] = v[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, x[q], o);
            if (lane >= o) x[q] += y;
        }
        if (lane == 31) s_w[q][warp] = x[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            int t = (lane < (nt >> 5)) ? s_w[q][lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL_MASK, t, o);
                if (lane >= o) t += y;
            }
            s_w[q][lane] = t;
        }
    }
    __syncthreads();
    int of = x[0] - v[0] + (warp ? s_w[0][warp - 1] : 0);
    int op = x[1] - v[1] + (warp ? s_w[1][warp - 1] : 0);
    int oc = x[2] - v[2] + (warp ? s_w[2][warp - 1] : 0);
    for (int r = r0; r < r1; ++r)
        if (a.need_in[r]) {
            const SysDesc &S = a.sys[r];
            a.plan_rep[of] = r;
            a.plan_pp[of] = op;
            a.plan_pc[of] = oc;
            ++of; op += S.n; oc += S.nc * S.nc * S.nc;
        }
    if (threadIdx.x == nt - 1) {
        a.plan->nflag = of;
        a.plan->tot_p = op;
        a.plan->tot_c = oc;
        a.plan_pp[of] = op;
        a.plan_pc[of] = oc;
        if (of > 0) a.ctrl->rebuild_passes += 1;
    }
}

// particle t of the pass's work list -> (replica, slot)
__device__ __forceinline__ void pass_particle(const int *pp, const int *rep, int nflag, int t,
                                              const SysDesc *sys, int &r, int &i) {
    const int k = find_seg(pp, nflag, t);
    r = rep[k];
    i = sys[r].off + (t - pp[k]);
}

template <typename R> __global__ void k_bin(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int r, i;
        pass_particle(a.plan_pp, a.plan_rep, nf, t, a.sys, r, i);
        const SysDesc &S = a.sys[r];
        const int c = S.cell_off + cell_index(a.key[i], S);
        a.cell_of[i] = c;
        a.rank[i] = atomicAdd(a.count + c, 1);
    }
}

// Per replica: exclusive scan of the cell counts -> cellStart (Sec. 7); counts re-zeroed.
template <typename R> __global__ void k_scan(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    __shared__ int s_warp[32];
    const int nf = a.plan->nflag;
    for (int b = blockIdx.x; b < nf; b += gridDim.x) {
        const int r = a.plan_rep[b];
        const SysDesc &S = a.sys[r];
        const int C = S.nc * S.nc * S.nc;
        const int nt = blockDim.x;
        const int chunk = (C + nt - 1) / nt;
        const int c0 = min(C, (int)threadIdx.x * chunk), c1 = min(C, c0 + chunk);
        int sum = 0;
        for (int c = c0; c < c1; ++c) sum += a.count[S.cell_off + c];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int v = (lane < (nt >> 5)) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL_MASK, v, o);
                if (lane >= o) v += y;
            }
            s_warp[lane] = v;
        }
        __syncthreads();
        int run = S.off + (x - sum) + (warp > 0 ? s_warp[warp - 1] : 0);
        for (int c = c0; c < c1; ++c) {
            const int n = a.count[S.cell_off + c];
            a.cell_start[S.cell_off + c] = run;
            a.count[S.cell_off + c] = 0;
            run += n;
        }
        if (threadIdx.x == 0) a.th[r].rebuilds += 1;
        __syncthreads();
    }
}

template <typename R> __global__ void k_scatter(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int r, i;
        pass_particle(a.plan_pp, a.plan_rep, nf, t, a.sys, r, i);
        a.perm[a.cell_start[a.cell_of[i]] + a.rank[i]] = i;
    }
}

// Atomic slot order inside a cell is arbitrary (as with atomicInc in Sec. 6); restore a
// deterministic order: by user id.
template <typename R> __global__ void k_cellsort(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int tot = a.plan->tot_c, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        const int k = find_seg(a.plan_pc, nf, t);
        const int c = a.sys[a.plan_rep[k]].cell_off + (t - a.plan_pc[k]);
        const int s = a.cell_start[c], e = a.cell_start[c + 1];
        for (int q = s + 1; q < e; ++q) {
            const int v = a.perm[q];
            const int key = a.id[v];
            int m = q - 1;
            while (m >= s && a.id[a.perm[m]] > key) {
                a.perm[m + 1] = a.perm[m];
                --m;
            }
            a.perm[m + 1] = v;
        }
    }
}

template <typename R> __global__ void k_gather(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int r, s;
        pass_particle(a.plan_pp, a.plan_rep, nf, t, a.sys, r, s);
        const int o = a.perm[s];
        a.tpos[s] = a.pos[o];
        if (!a.key_is_pos) a.tkey[s] = a.key[o];
        a.txd[s] = a.xd[o];
        a.tyd[s] = a.yd[o];
        a.tzd[s] = a.zd[o];
        a.tvel[s] = a.vel[o];
        a.timg[s] = a.img[o];
        a.tid[s] = a.id[o];
    }
}

// List build from sorted cells (Fig. 4) for one particle.  TPB lanes per particle walk the
// stencil as rows of cells along x: the cells (cx-reach .. cx+reach) of one (cy, cz) row hold one
// contiguous range of sorted slots (two when the row wraps), so a row costs two cellStart reads
// and its candidates are tested TPB at a time.  Accepted slots are compacted by ballot within the
// lane group, in candidate order, so the list order -- and hence every force bit -- is the same
// for every TPB.  Candidate indices are local (0..n-1 of the replica, or global slots when
// base = 0 and the cell starts are global); the list stores slot = base + j.
// Returns the full count (which may exceed nmax).
template <typename R, int TPB, bool STAGE, typename KeySrc, typename StartSrc>
__device__ __forceinline__ int build_one(const SysDesc &S, const KeySrc &K, const StartSrc &CS,
                                         int self, int slot_i, int base, int *nbl, int nmax,
                                         const R *s_thr, int ntypes, int2 *s_rng) {
    typedef typename V4T<R>::t V4;
    const int lt = threadIdx.x % TPB;
    const int lane = threadIdx.x & 31;
    const unsigned gmask = (TPB == 32) ? FULL_MASK : (((1u << TPB) - 1u) << (lane & ~(TPB - 1)));
    const unsigned below = (1u << lane) - 1u;
    const V4 ki = K(self);
    const int ti = type_of(ki);
    const R L = box_L<R>(S), invL = box_invL<R>(S);
    const int nc = S.nc, span = S.span, reach = S.reach;
    const int c = cell_index(ki, S);
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const bool full = (span == nc);
    int xa0, xa1, xb0 = 0, xb1 = -1;   // x range of every row as one or two cell ranges
    if (full) { xa0 = 0; xa1 = nc - 1; }
    else {
        const int x0 = cx - reach, x1 = cx + reach;
        if (x0 < 0) { xa0 = x0 + nc; xa1 = nc - 1; xb0 = 0; xb1 = x1; }
        else if (x1 >= nc) { xa0 = x0; xa1 = nc - 1; xb0 = 0; xb1 = x1 - nc; }
        else { xa0 = x0; xa1 = x1; }
    }
    // range q of the stencil: row q/2 in (z, y) order, part q%2 of its x extent
    auto range = [&](int q) -> int2 {
        const int rowi = q >> 1, part = q & 1;
        const int oz = rowi / span, oy = rowi % span;
        const int zz = full ? oz : (cz - reach + oz + nc) % nc;
        const int yy = full ? oy : (cy - reach + oy + nc) % nc;
        const int row = (zz * nc + yy) * nc;
        const int lo = part ? xb0 : xa0, hi = part ? xb1 : xa1;
        return (hi < lo) ? make_int2(0, 0) : make_int2(CS(row + lo), CS(row + hi + 1));
    };
    const int nr = span * span * 2;
    if (STAGE) {
        // stage every range with independent loads spread over the lanes, so the cellStart
        // latency is paid once instead of once per row
        for (int q = lt; q < nr; q += TPB) s_rng[q] = range(q);
        __syncwarp(gmask);
    }
    int cnt = 0;
    for (int q = 0; q < nr; ++q) {
        const int2 rg = STAGE ? s_rng[q] : range(q);
        for (int b0 = rg.x; b0 < rg.y; b0 += TPB) {
            const int j = b0 + lt;
            bool ok = false;
            if (j < rg.y && j != self) {
                const V4 kj = K(j);
                const R dx = min_image_exact(kj.x - ki.x, L, invL);
                const R dy = min_image_exact(kj.y - ki.y, L, invL);
                const R dz = min_image_exact(kj.z - ki.z, L, invL);
                ok = dist2_exact(dx, dy, dz) < s_thr[ti * ntypes + type_of(kj)];
            }
            const unsigned m = __ballot_sync(gmask, ok);
            if (ok) {
                const int sl = cnt + __popc(m & below);
                if (sl < nmax) nbl[nbl_offset(slot_i, sl, nmax)] = base + j;
            }
            cnt += __popc(m);
        }
    }
    if (STAGE) __syncwarp(gmask);   // the staged ranges are reused by the group's next particle
    return cnt;
}

template <typename R> struct GlobalKey {
    const typename V4T<R>::t *p;
    __device__ __forceinline__ typename V4T<R>::t operator()(int j) const { return p[j]; }
};
struct GlobalStart {   // cell starts of replica S in the global cellStart array
    const int *cs;
    int cell_off;
    __device__ __forceinline__ int operator()(int c) const { return cs[cell_off + c]; }
};

// largest stencil: reach 3 -> 7 x 7 rows, two ranges each
#define MD_MAX_RANGES 98
#define MD_BUILD_BLOCK 128

template <typename R, int TPB> __global__ void __launch_bounds__(MD_BUILD_BLOCK) k_build(const RebuildArgs<R> a) {
    typedef typename V4T<R>::t V4;
    if (rebuild_off(a.ctrl)) return;
    __shared__ R s_thr[MD_MAX_PAIRS];
    __shared__ int2 s_rng_all[MD_BUILD_BLOCK / TPB][MD_MAX_RANGES];
    const int npair = a.ntypes * a.ntypes;
    for (int p = threadIdx.x; p < npair; p += blockDim.x)
        s_thr[p] = sizeof(R) == 4 ? (R)a.tab[p].thr2 : (R)a.tab[p].thr2d;
    __syncthreads();
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    const int groups = gridDim.x * (blockDim.x / TPB);
    const V4 *Kp = a.key_is_pos ? a.tpos : a.tkey;
    for (int g = blockIdx.x * (blockDim.x / TPB) + threadIdx.x / TPB; g < tot; g += groups) {
        int r, i;
        pass_particle(a.plan_pp, a.plan_rep, nf, g, a.sys, r, i);
        const SysDesc &S = a.sys[r];
        GlobalKey<R> K{Kp};
        GlobalStart CS{a.cell_start, S.cell_off};
        int cnt = build_one<R, TPB, true>(S, K, CS, i, i, 0, a.nbl, a.nmax, s_thr, a.ntypes,
                                          s_rng_all[threadIdx.x / TPB]);
        if (threadIdx.x % TPB == 0) {
            if (cnt > a.nmax) {   // Sec. 4: out of space -> flag for the host, which doubles n_max
                atomicMax(&a.ctrl->max_count, cnt);
                atomicExch(&a.ctrl->overflow, 1);
                cnt = a.nmax;
            }
            a.nnb[i] = cnt;
            a.pos[i] = a.tpos[i];
            a.pos_build[i] = Kp[i];
            a.xd[i] = a.txd[i];
            a.yd[i] = a.tyd[i];
            a.zd[i] = a.tzd[i];
            a.vel[i] = a.tvel[i];
            a.img[i] = a.timg[i];
            a.id[i] = a.tid[i];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Replica-resident step kernel (the batched form): persistent CTAs claim whole replicas from a
// queue (replicas that must rebuild first, then the rest, each in descending size), stage the
// replica's positions in shared memory and run the whole step in the CTA: the cell-sorted
// rebuild of Sec. 7 when the skin criterion fired, forces with neighbour positions gathered from
// shared memory, the integrator and the replica's reductions.  Slot order, list order and the
// reduction tree are the same as in the grid path, so both paths give the same bits.
// If a list overflows, that replica's forces in this step are evaluated directly over the cell
// stencil (no list), so no replica falls behind; the host then grows n_max.
// ------------------------------------------------------------------------------------------------
struct SharedStart {
    const int *cs;
    __device__ __forceinline__ int operator()(int c) const { return cs[c]; }
};
template <typename R> struct SharedKey {
    const typename V4T<R>::t *p;
    __device__ __forceinline__ typename V4T<R>::t operator()(int j) const { return p[j]; }
};

// List-free forces of local particle `self` over the stencil candidates (overflow fallback).
template <typename R, int TP, bool SINGLE>
__device__ __forceinline__ void force_direct(const StepArgs<R> &a, const SysDesc &S,
                                             const typename V4T<R>::t *s_pos, const int *s_cs,
                                             int self, const typename V4T<R>::t &ri, int ti,
                                             const Frame<R> &F, int lt,
                                             const typename Coef4<R>::t *s_c0,
                                             const typename Coef2<R>::t *s_c1, R &fx, R &fy,
                                             R &fz, R &u, R &w) {
    const typename Coef4<R>::t c1 = s_c0[0];
    const typename Coef2<R>::t c1b = s_c1[0];
    const int nc = S.nc, span = S.span, reach = S.reach;
    const int c = cell_index(ri, S);
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const bool full = (span == nc);
    for (int oz = 0; oz < span; ++oz) {
        const int zz = full ? oz : (cz - reach + oz + nc) % nc;
        for (int oy = 0; oy < span; ++oy) {
            const int yy = full ? oy : (cy - reach + oy + nc) % nc;
            const int row = (zz * nc + yy) * nc;
            for (int ox = 0; ox < span; ++ox) {
                const int xx = full ? ox : (cx - reach + ox + nc) % nc;
                for (int j = s_cs[row + xx] + lt; j < s_cs[row + xx + 1]; j += TP)
                    if (j != self)
                        interact<R, SINGLE>(ri, ti, s_pos[j], F, a.ntypes, s_c0, s_c1, c1, c1b,
                                            fx, fy, fz, u, w);
            }
        }
    }
}

// Block-wide exclusive scan of cnt[0..C) into start[0..C] (start[C] = total); chunked per thread.
__device__ __forceinline__ void block_scan_cells(const int *cnt, int *start, int C, int *s_warp) {
    const int nt = blockDim.x;
    const int chunk = (C + nt - 1) / nt;
    const int c0 = min(C, (int)threadIdx.x * chunk), c1 = min(C, c0 + chunk);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += cnt[c];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = (lane < (nt >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, v, o);
            if (lane >= o) v += y;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    int run = (x - sum) + (warp > 0 ? s_warp[warp - 1] : 0);
    for (int c = c0; c < c1; ++c) {
        start[c] = run;
        run += cnt[c];
    }
    if (threadIdx.x == nt - 1) start[C] = run;
    __syncthreads();
}

template <typename R, int TP, bool SINGLE, int TPB>
__global__ void __launch_bounds__(1024) k_rep(const StepArgs<R> a, const RebuildArgs<R> b) {
    typedef typename V4T<R>::t V4;
    typedef typename Coef4<R>::t C4;
    typedef typename Coef2<R>::t C2;
    extern __shared__ __align__(16) unsigned char smem[];
    // dynamic shared memory: positions, cell starts/counters, per-particle cell and slot scratch,
    // tile partials
    V4 *s_pos = reinterpret_cast<V4 *>(smem);
    int *s_cs = reinterpret_cast<int *>(s_pos + a.rep_nmax);    // cmax + 1
    int *s_cnt = s_cs + a.rep_cmax + 1;                          // cmax
    int *s_cell = s_cnt + a.rep_cmax;                            // rep_nmax
    int *s_perm = s_cell + a.rep_nmax;                           // rep_nmax
    double *s_part = reinterpret_cast<double *>(                 // tile partials, 16 B aligned
        ((size_t)(s_perm + a.rep_nmax) + 15) & ~(size_t)15);

    __shared__ C4 s_c0[MD_MAX_PAIRS];
    __shared__ C2 s_c1[MD_MAX_PAIRS];
    __shared__ R s_im[MD_MAX_TYPES], s_m[MD_MAX_TYPES], s_thr[MD_MAX_PAIRS];
    __shared__ double s_tmp[32][MD_NRED];
    __shared__ double s_red[MD_NRED];
    __shared__ int s_warp[32];
    __shared__ double s_xi;
    __shared__ R s_A, s_B;
    __shared__ int s_job, s_skip, s_ovf;
    __shared__ SysDesc S;   // the replica being processed (shared: keeps registers free)

    load_tables(a, s_c0, s_c1, s_im, s_m);
    for (int p = threadIdx.x; p < a.ntypes * a.ntypes; p += blockDim.x)
        s_thr[p] = sizeof(R) == 4 ? (R)a.tab[p].thr2 : (R)a.tab[p].thr2d;
    if (threadIdx.x == 0) s_skip = *(volatile int *)&a.ctrl->halt;
    __syncthreads();
    if (s_skip) return;   // uniform for the whole launch: halt is only set by a finished step

    // the block runs blockDim / tile_threads tiles of the grid kernel's shape side by side
    const int TT = a.tile_threads;
    const int P = TT / TP;
    const int tpb_tiles = blockDim.x / TT;
    const int tsub = threadIdx.x / TT;
    const int lp = (threadIdx.x % TT) / TP, lt = threadIdx.x % TP;
    for (;;) {
        if (threadIdx.x == 0) {
            // two passes over the size-ordered queue: replicas that rebuild, then the others
            int r = -1;
            while (r < 0) {
                const int k1 = atomicAdd(&a.ctrl->q1, 1);
                if (k1 < a.nrep) {
                    const int c = a.rep_order[k1];
                    if (a.need_in[c]) r = c;
                    continue;
                }
                const int k2 = atomicAdd(&a.ctrl->q2, 1);
                if (k2 < a.nrep) {
                    const int c = a.rep_order[k2];
                    if (!a.need_in[c]) r = c;
                    continue;
                }
                break;
            }
            s_job = r;
        }
        __syncthreads();
        const int r = s_job;
        if (r < 0) break;
        if (threadIdx.x == 0) S = a.sys[r];
        __syncthreads();
        const int n = S.n, off = S.off;
        const bool rebuild = a.need_in[r] != 0;
        if (threadIdx.x == 0) {
            const double xi = step_xi(a, S, r);
            s_xi = xi;
            s_A = (R)(1.0 - 0.5 * xi * a.dt);
            s_B = (R)(1.0 / (1.0 + 0.5 * xi * a.dt));
            s_ovf = 0;
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_pos[k] = a.pos_in[off + k];
        __syncthreads();

        if (rebuild) {
            // ---- Sec. 7 rebuild inside the CTA: bin, scan, scatter, order by id, permute, build
            const int C = S.nc * S.nc * S.nc;
            for (int c = threadIdx.x; c < C; c += blockDim.x) s_cnt[c] = 0;
            __syncthreads();
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                const int c = cell_index(s_pos[k], S);
                s_cell[k] = c;
                atomicAdd(s_cnt + c, 1);
            }
            __syncthreads();
            block_scan_cells(s_cnt, s_cs, C, s_warp);
            for (int c = threadIdx.x; c < C; c += blockDim.x) s_cnt[c] = s_cs[c];
            __syncthreads();
            for (int k = threadIdx.x; k < n; k += blockDim.x)
                s_perm[atomicAdd(s_cnt + s_cell[k], 1)] = k;
            __syncthreads();
            const int *idg = a.id_g + off;   // user ids (pre-permutation)
            for (int c = threadIdx.x; c < C; c += blockDim.x) {   // deterministic: by user id
                const int s0 = s_cs[c], e0 = s_cs[c + 1];
                for (int q = s0 + 1; q < e0; ++q) {
                    const int v = s_perm[q], key = idg[v];
                    int m = q - 1;
                    while (m >= s0 && idg[s_perm[m]] > key) { s_perm[m + 1] = s_perm[m]; --m; }
                    s_perm[m + 1] = v;
                }
            }
            __syncthreads();
            // permute the particle data through the scratch arrays (global, same block)
            for (int s = threadIdx.x; s < n; s += blockDim.x) {
                const int o = off + s_perm[s], d = off + s;
                b.tpos[d] = s_pos[s_perm[s]];
                b.txd[d] = a.xd[o]; b.tyd[d] = a.yd[o]; b.tzd[d] = a.zd[o];
                b.tvel[d] = a.vel[o];
                b.timg[d] = a.img[o];
                b.tid[d] = a.id_g[o];
            }
            __syncthreads();
            for (int s = threadIdx.x; s < n; s += blockDim.x) {
                const int d = off + s;
                s_pos[s] = b.tpos[d];
                a.xd[d] = b.txd[d]; a.yd[d] = b.tyd[d]; a.zd[d] = b.tzd[d];
                a.vel[d] = b.tvel[d];
                a.img[d] = b.timg[d];
                a.id_g[d] = b.tid[d];
            }
            __syncthreads();
            // list build from the shared positions and cell starts
            SharedKey<R> K{s_pos};
            SharedStart CS{s_cs};
            for (int g = threadIdx.x / TPB; g < n; g += blockDim.x / TPB) {
                int cnt = build_one<R, TPB, false>(S, K, CS, g, off + g, off, b.nbl, b.nmax,
                                                   s_thr, a.ntypes, nullptr);
                if (threadIdx.x % TPB == 0) {
                    if (cnt > b.nmax) {
                        atomicMax(&a.ctrl->max_count, cnt);
                        atomicExch(&a.ctrl->rep_overflow, 1);
                        s_ovf = 1;
                        cnt = b.nmax;
                    }
                    b.nnb[off + g] = cnt;
                    b.pos_build[off + g] = s_pos[g];
                }
            }
            if (threadIdx.x == 0) a.th[r].rebuilds += 1;
            __syncthreads();
        }

        // ---- forces over the list (shared-memory gathers), integration, tile partials ----
        const bool direct = s_ovf != 0;
        int moved_any = 0;
        for (int t0 = 0; t0 < S.ntiles; t0 += tpb_tiles) {
            const int t = t0 + tsub;
            const int li = t * P + lp;
            const bool active = t < S.ntiles && li < n;
            const int i = off + li;
            R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
            V4 ri = make_v4(R(0), R(0), R(0), R(0));
            int ti = 0;
            if (active) {
                ri = s_pos[li];
                ti = type_of(ri);
                const Frame<R> F = make_frame(ri, S);
                if (!direct) {
                    SharedPos<R> src{s_pos, off};
                    force_sum<R, TP, SINGLE, SharedPos<R>, false>(a, src, i, ri, ti, F, lt, s_c0,
                                                                 s_c1, fx, fy, fz, u, w);
                } else {
                    force_direct<R, TP, SINGLE>(a, S, s_pos, s_cs, li, ri, ti, F, lt, s_c0, s_c1,
                                                fx, fy, fz, u, w);
                }
            }
            merge_lanes<R, TP>(fx, fy, fz, u, w);
            const bool leader = active && lt == 0;
            u *= R(0.5);
            w *= R(1.0 / 6.0);
            R ke = 0, px = 0, py = 0, pz = 0;
            bool moved = false;
            if (leader)
                moved = integrate_one(a, S, i, ri, fx, fy, fz, s_im[ti], s_m[ti], s_A, s_B, ke,
                                      px, py, pz);
            moved_any |= (int)moved;
            R vals[MD_NRED] = {u * R(leader), w * R(leader), ke, px, py, pz};
            // partials of tiles past the replica's last one are written to spare rows and ignored
            tile_partial(vals, s_tmp, s_part + (long long)t0 * MD_NRED, TT >> 5);
            __syncthreads();
        }
        moved_any = __syncthreads_or(moved_any);
        // an overflowed list stays flagged: every step rebuilds and evaluates list-free until the
        // host has grown the capacity
        replica_finish(a, r, S, s_part, s_xi, (moved_any || direct) ? 1 : 0, s_tmp, s_red, false,
                       TT);
        __syncthreads();
    }
    // last CTA closes the step
    __shared__ int s_glast;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = atomicAdd(&a.ctrl->global_ticket, 1u);
        s_glast = (g == gridDim.x - 1);
    }
    __syncthreads();
    if (s_glast) close_step(a);
}


// ------------------------------------------------------------------------------------------------
// Fused sort for replicas that fit in shared memory (grid path): one CTA per rebuilt replica
// performs bin, exclusive scan (cellStart), slot scatter, in-cell order by user id and the gather
// into the scratch arrays -- the work of k_bin .. k_gather in one launch.  k_build follows.
// ------------------------------------------------------------------------------------------------
template <typename R> __global__ void __launch_bounds__(512) k_sort_small(const RebuildArgs<R> a) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int s_warp[32];
    if (rebuild_off(a.ctrl)) return;
    int *s_cnt = sm;                          // sort_cmax
    int *s_cs = s_cnt + a.sort_cmax;          // sort_cmax + 1
    int *s_cell = s_cs + a.sort_cmax + 1;     // sort_nmax
    int *s_perm = s_cell + a.sort_nmax;       // sort_nmax
    int *s_id = s_perm + a.sort_nmax;         // sort_nmax
    const int nf = a.plan->nflag;
    for (int b = blockIdx.x; b < nf; b += gridDim.x) {
        const int r = a.plan_rep[b];
        const SysDesc S = a.sys[r];
        const int n = S.n, off = S.off, C = S.nc * S.nc * S.nc;
        for (int c = threadIdx.x; c < C; c += blockDim.x) s_cnt[c] = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int c = cell_index(a.key[off + k], S);
            s_cell[k] = c;
            s_id[k] = a.id[off + k];
            atomicAdd(s_cnt + c, 1);
        }
        __syncthreads();
        block_scan_cells(s_cnt, s_cs, C, s_warp);
        for (int c = threadIdx.x; c < C; c += blockDim.x) s_cnt[c] = s_cs[c];
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x)
            s_perm[atomicAdd(s_cnt + s_cell[k], 1)] = k;
        __syncthreads();
        for (int c = threadIdx.x; c < C; c += blockDim.x) {   // deterministic: by user id
            const int s0 = s_cs[c], e0 = s_cs[c + 1];
            for (int q = s0 + 1; q < e0; ++q) {
                const int v = s_perm[q], key = s_id[v];
                int m = q - 1;
                while (m >= s0 && s_id[s_perm[m]] > key) { s_perm[m + 1] = s_perm[m]; --m; }
                s_perm[m + 1] = v;
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int o = off + s_perm[q], d = off + q;
            a.tpos[d] = a.pos[o];
            if (!a.key_is_pos) a.tkey[d] = a.key[o];
            a.txd[d] = a.xd[o];
            a.tyd[d] = a.yd[o];
            a.tzd[d] = a.zd[o];
            a.tvel[d] = a.vel[o];
            a.timg[d] = a.img[o];
            a.tid[d] = s_id[s_perm[q]];
        }
        for (int c = threadIdx.x; c < C; c += blockDim.x) a.cell_start[S.cell_off + c] = off + s_cs[c];
        if (threadIdx.x == 0) a.th[r].rebuilds += 1;
        __syncthreads();
    }
}

}  // namespace md
