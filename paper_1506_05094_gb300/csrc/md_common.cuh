// md_common.cuh -- device helpers shared by the step, rebuild and replica-resident kernels:
// vector types, list layout, minimum image, LJ pair term, deterministic block reduction.
//
// Kernels: md_step.cuh (k_step), md_rebuild.cuh (k_plan .. k_build), md_rep.cuh (k_rep,
// k_sort_small); md_kernels.cuh includes them all.
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

// Per type-pair coefficients in shared memory: {rc2, c12, c6, ushift} and {a12, a6, fc, rc}.
template <typename R> struct Coef4;
template <> struct Coef4<float> { typedef float4 t; };
template <> struct Coef4<double> { typedef double4_32a t; };

template <typename R> __device__ __forceinline__ typename Coef4<R>::t coef0_of(const PairTab &p);
template <> __device__ __forceinline__ float4 coef0_of<float>(const PairTab &p) {
    return make_float4(p.rc2, p.c12, p.c6, p.ushift);
}
template <> __device__ __forceinline__ double4_32a coef0_of<double>(const PairTab &p) {
    return make_double4_32a(p.rc2d, p.c12d, p.c6d, p.ushiftd);
}
template <typename R> __device__ __forceinline__ typename Coef4<R>::t coef1_of(const PairTab &p);
template <> __device__ __forceinline__ float4 coef1_of<float>(const PairTab &p) {
    return make_float4(p.a12, p.a6, p.fc, p.rc);
}
template <> __device__ __forceinline__ double4_32a coef1_of<double>(const PairTab &p) {
    return make_double4_32a(p.a12d, p.a6d, p.fcd, p.rcd);
}

template <typename R> __device__ __forceinline__ typename Coef4<R>::t coef2_of(const PairTab &p);
template <> __device__ __forceinline__ float4 coef2_of<float>(const PairTab &p) {
    return make_float4(p.qrc2, p.qq, p.qf, p.qu);
}
template <> __device__ __forceinline__ double4_32a coef2_of<double>(const PairTab &p) {
    return make_double4_32a(p.qrc2d, p.qqd, p.qfd, p.qud);
}

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }

// One pair's contribution (the fij / ComputeInteraction of Sec. 5) for LJ, shifted potential:
// F_ij = r^-2 (a12 r^-12 - a6 r^-6) r_ij, u += c12 r^-12 - c6 r^-6 - ushift, w += r_ij . F_ij;
// shifted force (SF) also subtracts fc / r from the scalar force and adds (r - rc) fc to u.
// c = {rc2, c12, c6, ushift}, b = {a12, a6, fc, rc}.
template <bool SF, typename R, typename C4, typename C2>
__device__ __forceinline__ void lj_pair(R dx, R dy, R dz, R r2, const C4 &c, const C2 &b, R &fx,
                                        R &fy, R &fz, R &u, R &w) {
    const R r2i = fast_rcp(r2);
    const R r6i = r2i * r2i * r2i;
    R fs = r2i * r6i * (b.x * r6i - b.y);
    u += r6i * (c.y * r6i - c.z) - c.w;
    if (SF) {
        const R ri = fast_rsqrt(r2);
        fs -= b.z * ri;
        u += (r2 * ri - b.w) * b.z;
    }
    fx += fs * dx;
    fy += fs * dy;
    fz += fs * dz;
    w += fs * r2;
}

// Shifted-force Coulomb term (Sec. 9, molten salt) for r < rc_C:
// u = qq (1/r - 2/rc_C + r/rc_C^2), F_ij = (qq/r) (1/r^2 - 1/rc_C^2) r_ij.
// q = {rc_C^2, qq, qq / rc_C^2, 2 qq / rc_C}.
template <typename R, typename C4>
__device__ __forceinline__ void coulomb_pair(R dx, R dy, R dz, R r2, const C4 &q, R &fx, R &fy,
                                             R &fz, R &u, R &w) {
    const R ri = fast_rsqrt(r2);
    const R fs = ri * (q.y * ri * ri - q.z);
    u += q.y * ri - q.w + q.z * (r2 * ri);
    fx += fs * dx;
    fy += fs * dy;
    fz += fs * dz;
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

// Potential kind (template POT, a bit set): bit 0 = LJ with the shifted-force cutoff (else
// shifted potential), bit 1 = shifted-force Coulomb term (s_cq holds its coefficients; only
// with per-pair tables, SINGLE = false).
template <typename R, bool SINGLE, int POT = 0>
__device__ __forceinline__ void interact(const typename V4T<R>::t &ri, int ti,
                                         const typename V4T<R>::t &rj, const Frame<R> &F, int nt,
                                         const typename Coef4<R>::t *s_c0,
                                         const typename Coef4<R>::t *s_c1,
                                         const typename Coef4<R>::t &c1,
                                         const typename Coef4<R>::t &c1b, R &fx, R &fy, R &fz,
                                         R &u, R &w,
                                         const typename Coef4<R>::t *s_cq = nullptr) {
    static_assert(!(SINGLE && (POT & 2)), "the Coulomb term needs the per-pair tables");
    constexpr bool SF = (POT & 1) != 0;
    R dx, dy, dz;
    pair_delta(F, ri, rj, dx, dy, dz);
    const R r2 = dx * dx + dy * dy + dz * dz;
    if (sizeof(R) == 4) {
        // FP32: branch-free.  Nearly every warp has some lane inside rc, so a branch saves no
        // work; without it the compiler interleaves the unrolled candidates' arithmetic.  A pair
        // outside rc contributes exact zeros (the scalar force and energy term are selected to 0).
        // The shifted-potential terms need only c = {rc2, c12, c6, ushift}: with a12 = 12 c12 and
        // a6 = 6 c6, F = 6 r^-2 r^-6 (2 c12 r^-6 - c6) r_ij, so one shared-memory load per pair.
        typename Coef4<R>::t c;
        int p = 0;
        if (SINGLE) {
            c = c1;
        } else {
            p = ti * nt + type_of(rj);
            c = s_c0[p];
        }
        const bool in = r2 < c.x;
        const R r2i = fast_rcp(r2);
        const R r6i = r2i * r2i * r2i;
        const R t = c.y * r6i - c.z;                    // c12 r^-6 - c6
        R uu = r6i * t - c.w;
        R fs = (R(6) * r2i) * r6i * (c.y * r6i + t);    // 6 r^-8 (2 c12 r^-6 - c6)
        if (SF) {
            const typename Coef4<R>::t b = SINGLE ? c1b : s_c1[p];
            const R rinv = fast_rsqrt(r2);
            fs -= b.z * rinv;
            uu += (r2 * rinv - b.w) * b.z;
        }
        fs = in ? fs : R(0);
        u += in ? uu : R(0);
        if (POT & 2) {
            const typename Coef4<R>::t q = s_cq[p];
            const bool inq = r2 < q.x;
            const R rinv = fast_rsqrt(r2);
            const R fq = rinv * (q.y * rinv * rinv - q.z);
            const R uq = q.y * rinv - q.w + q.z * (r2 * rinv);
            fs += inq ? fq : R(0);
            u += inq ? uq : R(0);
        }
        fx += fs * dx;
        fy += fs * dy;
        fz += fs * dz;
        w += fs * r2;
        return;
    }
    if (SINGLE) {
        if (r2 < c1.x) lj_pair<SF>(dx, dy, dz, r2, c1, c1b, fx, fy, fz, u, w);
    } else {
        const int p = ti * nt + type_of(rj);
        const typename Coef4<R>::t c = s_c0[p];
        if (r2 < c.x) lj_pair<SF>(dx, dy, dz, r2, c, s_c1[p], fx, fy, fz, u, w);
        if (POT & 2) {
            const typename Coef4<R>::t q = s_cq[p];
            if (r2 < q.x) coulomb_pair(dx, dy, dz, r2, q, fx, fy, fz, u, w);
        }
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

}  // namespace md
