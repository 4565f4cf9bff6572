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
    Frame<float> F;
    const double L = S.L, lo = S.L - (double)S.Lf;
    const bool ux = (double)ri.x >= 0.5 * L, uy = (double)ri.y >= 0.5 * L,
               uz = (double)ri.z >= 0.5 * L;
    F.xa = (float)(ux ? (double)ri.x - L : (double)ri.x + lo);
    F.ya = (float)(uy ? (double)ri.y - L : (double)ri.y + lo);
    F.za = (float)(uz ? (double)ri.z - L : (double)ri.z + lo);
    F.nx = ux ? 0.0f : 1.0f;
    F.ny = uy ? 0.0f : 1.0f;
    F.nz = uz ? 0.0f : 1.0f;
    F.half = (float)(0.5 * L);
    F.L = S.Lf;
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
// Fused step kernel.  One CTA = one tile of (blockDim / TP) particles of a single replica.
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
    Thermo *T = a.th + r;
    const int npair = a.ntypes * a.ntypes;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        s_c0[p] = coef0_of<R>(a.tab[p]);
        s_c1[p] = coef1_of<R>(a.tab[p]);
    }
    if (threadIdx.x < MD_MAX_TYPES) {
        s_im[threadIdx.x] = (R)a.inv_mass[threadIdx.x];
        s_m[threadIdx.x] = (R)a.mass[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        // one uniform decision per block: a halt or an unrecovered list overflow stops the step
        s_skip = *(volatile int *)&a.ctrl->halt | *(volatile int *)&a.ctrl->overflow;
        double xi = 0.0;  // Nose-Hoover friction of this step, from the previous step's carry
        if (a.integrator == 1 && !a.force_only)
            xi = T->xi_prev + a.dt * (T->K_prev / S.K0 - 1.0) * a.inv_tau2;
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
    const R L = box_L<R>(S), invL = box_invL<R>(S);
    const C4 c1 = s_c0[0];
    const C2 c1b = s_c1[0];

    R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    V4 ri = make_v4(R(0), R(0), R(0), R(0));
    int ti = 0;
    if (active) {
        ri = a.pos_in[i];
        ti = type_of(ri);
        const Frame<R> F = make_frame(ri, S);
        const int nn = a.nnb[i];
        const V4 *__restrict__ P4 = a.pos_in;
        const long long stride = (long long)TP * a.ncap;
        const int *q = a.nbl + (long long)lt * a.ncap + i;
        int k = lt;
        for (; k + 3 * TP < nn; k += 4 * TP) {
            const int j0 = __ldg(q), j1 = __ldg(q + stride), j2 = __ldg(q + 2 * stride),
                      j3 = __ldg(q + 3 * stride);
            q += 4 * stride;
            const V4 r0 = ld_nc(P4 + j0), r1 = ld_nc(P4 + j1), r2 = ld_nc(P4 + j2),
                     r3 = ld_nc(P4 + j3);
            interact<R, SINGLE>(ri, ti, r0, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
            interact<R, SINGLE>(ri, ti, r1, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
            interact<R, SINGLE>(ri, ti, r2, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
            interact<R, SINGLE>(ri, ti, r3, F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy, fz, u, w);
        }
        for (; k < nn; k += TP) {
            const int j = __ldg(q);
            q += stride;
            interact<R, SINGLE>(ri, ti, ld_nc(P4 + j), F, a.ntypes, s_c0, s_c1, c1, c1b, fx, fy,
                                fz, u, w);
        }
    }
    // merge the TP partial sums of each particle (replaces the serial shared-memory sum of Fig. 2)
#pragma unroll
    for (int o = TP / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(FULL_MASK, fx, o);
        fy += __shfl_xor_sync(FULL_MASK, fy, o);
        fz += __shfl_xor_sync(FULL_MASK, fz, o);
        u += __shfl_xor_sync(FULL_MASK, u, o);
        w += __shfl_xor_sync(FULL_MASK, w, o);
    }
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

    // ---- integrate (Sec. 2: leapfrog NVE / Nose-Hoover NVT) ----
    const double xi = s_xi;
    R ke = 0, px = 0, py = 0, pz = 0;
    bool moved = false;
    if (leader) {
        const R im = s_im[ti], m = s_m[ti], dt = (R)a.dt;
        V4 v = a.vel[i];
        if (a.integrator == 1) {
            const R A = s_A, B = s_B;
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
        // FP64 master position, wrap and image (the mixed-precision contract)
        const double ddx = a.dt * (double)v.x, ddy = a.dt * (double)v.y, ddz = a.dt * (double)v.z;
        double x = a.xd[i] + ddx, y = a.yd[i] + ddy, z = a.zd[i] + ddz;
        int wx = 0, wy = 0, wz = 0;
        if (x >= S.L) { x -= S.L; wx = 1; } else if (x < 0.0) { x += S.L; wx = -1; }
        if (y >= S.L) { y -= S.L; wy = 1; } else if (y < 0.0) { y += S.L; wy = -1; }
        if (z >= S.L) { z -= S.L; wz = 1; } else if (z < 0.0) { z += S.L; wz = -1; }
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
        // skin check (Sec. 6): moved more than s/2 since the last build
        const V4 pb = a.pos_build[i];
        const R bx = min_image_fast(rn.x - pb.x, L, invL);
        const R by = min_image_fast(rn.y - pb.y, L, invL);
        const R bz = min_image_fast(rn.z - pb.z, L, invL);
        moved = (bx * bx + by * by + bz * bz) > a.half_skin2;
    }
    if (__ballot_sync(FULL_MASK, moved) != 0u && (threadIdx.x & 31) == 0) atomicOr(a.moved + r, 1);

    // ---- per-tile partial sums: values within a warp in R, everything above in FP64 ----
    R vals[MD_NRED] = {u * R(leader), w * R(leader), ke, px, py, pz};
#pragma unroll
    for (int q2 = 0; q2 < MD_NRED; ++q2)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vals[q2] += __shfl_down_sync(FULL_MASK, vals[q2], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q2 = 0; q2 < MD_NRED; ++q2) s_tmp[warp][q2] = (double)vals[q2];
    __syncthreads();
    if (threadIdx.x < MD_NRED) {
        double acc = 0.0;
        for (int ww = 0; ww < nw; ++ww) acc += s_tmp[ww][threadIdx.x];
        a.partial[(long long)tile * MD_NRED + threadIdx.x] = acc;
    }
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
    double acc[MD_NRED];
#pragma unroll
    for (int q2 = 0; q2 < MD_NRED; ++q2) acc[q2] = 0.0;
    for (int tt = threadIdx.x; tt < S.ntiles; tt += blockDim.x) {
        const double *pp = a.partial + (long long)(S.tile_off + tt) * MD_NRED;
#pragma unroll
        for (int q2 = 0; q2 < MD_NRED; ++q2) acc[q2] += __ldcg(pp + q2);
    }
    block_reduce_nred(acc, s_tmp, s_red);
    if (threadIdx.x == 0) {
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
        a.need[r] = __ldcg(a.moved + r);
        a.moved[r] = 0;
        a.rep_ticket[r] = 0u;
        __threadfence();
        const unsigned g = atomicAdd(&a.ctrl->global_ticket, 1u);
        s_glast = (g == (unsigned)(a.nrep - 1));
    }
    __syncthreads();
    if (!s_glast) return;
    __threadfence();
    int any = 0;
    for (int rr = threadIdx.x; rr < a.nrep; rr += blockDim.x) any |= __ldcg(a.need + rr);
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        a.ctrl->need_any = any;
        a.ctrl->global_ticket = 0u;
        a.ctrl->step += 1;
        if (a.has_next) cudaGraphSetConditional(a.next_handle, (any && !a.ctrl->halt) ? 1u : 0u);
    }
}

// ------------------------------------------------------------------------------------------------
// Rebuild (Sec. 7): only replicas with need[r] != 0 take part; the rest exit at once.
// ------------------------------------------------------------------------------------------------
// halt and need_any only change between passes (halt is set by step kernels, need_any by the
// last block of a step), so every thread of a pass sees the same values.  An overflow does not
// stop a pass: the copy back of the permuted data must always complete.
__device__ __forceinline__ bool rebuild_off(const Ctrl *c) {
    return *(volatile const int *)&c->halt || !*(volatile const int *)&c->need_any;
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

template <typename R> __global__ void k_bin(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) a.ctrl->rebuild_passes += 1;   // one thread per pass
    if (i >= a.ntot) return;
    const int r = a.prep[i];
    if (!a.need[r]) return;
    const SysDesc S = a.sys[r];
    const int c = S.cell_off + cell_index(a.key[i], S);
    a.cell_of[i] = c;
    a.rank[i] = atomicAdd(a.count + c, 1);
}

// One CTA per replica: exclusive scan of the cell counts -> cellStart (Sec. 7), counts re-zeroed.
template <typename R> __global__ void k_scan(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int r = blockIdx.x;
    if (!a.need[r]) return;
    __shared__ int s_warp[32];
    const SysDesc S = a.sys[r];
    const int C = S.nc * S.nc * S.nc;
    const int nt = blockDim.x;
    const int chunk = (C + nt - 1) / nt;
    const int c0 = min(C, (int)threadIdx.x * chunk), c1 = min(C, c0 + chunk);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += a.count[S.cell_off + c];
    // block exclusive scan of per-thread sums
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
}

template <typename R> __global__ void k_scatter(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ntot) return;
    if (!a.need[a.prep[i]]) return;
    a.perm[a.cell_start[a.cell_of[i]] + a.rank[i]] = i;
}

// Atomic slot order inside a cell is arbitrary (as with atomicInc in Sec. 6); restore a
// deterministic order: by user id.
template <typename R> __global__ void k_cellsort(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.ctot) return;
    if (!a.need[a.crep[c]]) return;
    const int s = a.cell_start[c], e = a.cell_start[c + 1];
    for (int k = s + 1; k < e; ++k) {
        const int v = a.perm[k];
        const int key = a.id[v];
        int m = k - 1;
        while (m >= s && a.id[a.perm[m]] > key) {
            a.perm[m + 1] = a.perm[m];
            --m;
        }
        a.perm[m + 1] = v;
    }
}

template <typename R> __global__ void k_gather(const RebuildArgs<R> a) {
    if (rebuild_off(a.ctrl)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.ntot) return;
    if (!a.need[a.prep[s]]) return;
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

// List build from sorted cells (Fig. 4), one thread per particle, plus the copy back of the
// permuted particle data and the build positions (kept for the skin check).
template <typename R> __global__ void k_build(const RebuildArgs<R> a) {
    typedef typename V4T<R>::t V4;
    if (rebuild_off(a.ctrl)) return;
    __shared__ R s_thr[MD_MAX_PAIRS];
    const int npair = a.ntypes * a.ntypes;
    for (int p = threadIdx.x; p < npair; p += blockDim.x)
        s_thr[p] = sizeof(R) == 4 ? (R)a.tab[p].thr2 : (R)a.tab[p].thr2d;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ntot) return;
    const int r = a.prep[i];
    if (!a.need[r]) return;
    const SysDesc S = a.sys[r];
    const V4 *K = a.key_is_pos ? a.tpos : a.tkey;
    const V4 ki = K[i];
    const int ti = type_of(ki);
    const R L = box_L<R>(S), invL = box_invL<R>(S);
    const int nc = S.nc, span = S.span;
    const int c = cell_index(ki, S);
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    // visit each stencil cell once: offsets -reach..reach, or every cell when 2 reach + 1 >= nc
    const int b0 = (span == nc) ? 0 : -S.reach;
    int cnt = 0;
    int *col = a.nbl + i;
    for (int oz = 0; oz < span; ++oz) {
        const int zz = (span == nc) ? oz : (cz + b0 + oz + nc) % nc;
        for (int oy = 0; oy < span; ++oy) {
            const int yy = (span == nc) ? oy : (cy + b0 + oy + nc) % nc;
            for (int ox = 0; ox < span; ++ox) {
                const int xx = (span == nc) ? ox : (cx + b0 + ox + nc) % nc;
                const int cell = S.cell_off + (zz * nc + yy) * nc + xx;
                const int js = a.cell_start[cell], je = a.cell_start[cell + 1];
                for (int j = js; j < je; ++j) {
                    if (j == i) continue;
                    const V4 kj = K[j];
                    const R dx = min_image_exact(kj.x - ki.x, L, invL);
                    const R dy = min_image_exact(kj.y - ki.y, L, invL);
                    const R dz = min_image_exact(kj.z - ki.z, L, invL);
                    const R d2 = dist2_exact(dx, dy, dz);
                    if (d2 < s_thr[ti * a.ntypes + type_of(kj)]) {
                        if (cnt < a.nmax) col[(long long)cnt * a.ncap] = j;
                        ++cnt;
                    }
                }
            }
        }
    }
    if (cnt > a.nmax) {   // Sec. 4: out of space -> flag for the host, which doubles n_max
        atomicMax(&a.ctrl->max_count, cnt);
        atomicExch(&a.ctrl->overflow, 1);
        cnt = a.nmax;
    }
    a.nnb[i] = cnt;
    a.pos[i] = a.tpos[i];
    a.pos_build[i] = ki;
    a.xd[i] = a.txd[i];
    a.yd[i] = a.tyd[i];
    a.zd[i] = a.tzd[i];
    a.vel[i] = a.tvel[i];
    a.img[i] = a.timg[i];
    a.id[i] = a.tid[i];
}

}  // namespace md
