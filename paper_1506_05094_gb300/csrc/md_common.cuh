// md_common.cuh -- device helpers shared by the step, rebuild and replica-resident kernels:
// vector types, list layout, minimum image, LJ pair term, deterministic block reduction.
//
// Kernels: md_step.cuh (k_step), md_rebuild.cuh (k_plan .. k_build), md_rep.cuh (k_rep,
// k_sort_small); md_kernels.cuh includes them all.
#pragma once
#include "md_internal.cuh"

namespace md {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ int type_of(int4 p) { return p.w; }
__device__ __forceinline__ int type_of(double4_32a p) { return (int)__double_as_longlong(p.w); }

__device__ __forceinline__ int4 ld_nc(const int4 *p) { return __ldg(p); }
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

// Difference of two fixed-point mirror coordinates as a float in mirror units: the 32-bit
// difference wraps to the nearest periodic image by itself (2^32 units are one period), and the
// int -> float conversion rounds to nearest.
__device__ __forceinline__ float fixed_diff(int a, int b) {
    return __int2float_rn((int)((unsigned)a - (unsigned)b));
}

// Squared distance of the list rule, bit-defined (every product and sum rounded on its own, none
// contracted).  Mixed precision: d = float(x_j - x_i) per axis in mirror units,
// dist^2 = ((dx dx + dy dy) + dz dz) ps2.  FP64: d = x_j - x_i; d -= L rint(d / L).
__device__ __forceinline__ float key_dist2(const int4 &ki, const int4 &kj, const SysDesc &S) {
    const float dx = fixed_diff(kj.x, ki.x), dy = fixed_diff(kj.y, ki.y),
                dz = fixed_diff(kj.z, ki.z);
    return __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)),
                     S.ps2);
}
__device__ __forceinline__ double min_image_exact(double d, double L, double invL) {
    double t = rint(__dmul_rn(d, invL));
    return __dsub_rn(d, __dmul_rn(L, t));
}
__device__ __forceinline__ double key_dist2(const double4_32a &ki, const double4_32a &kj,
                                            const SysDesc &S) {
    const double dx = min_image_exact(kj.x - ki.x, S.L, S.invL);
    const double dy = min_image_exact(kj.y - ki.y, S.L, S.invL);
    const double dz = min_image_exact(kj.z - ki.z, S.L, S.invL);
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

// Per-particle minimum-image frame of the force loop.
//
// Mixed precision: the mirror is 32-bit fixed point with 2^32 units per box edge, so the minimum
// image of x_i - x_j is the 32-bit difference itself (two's-complement wrap), converted to float:
// two instructions per axis, exact up to the conversion's rounding (2^-24 relative), and no
// per-particle state.  The pair loop works with d in mirror units: r^2 = |d|^2 ps2 (real units),
// the force sum accumulates the scalar force times d, and the particle's force is multiplied by
// the unit ps once at the end (scale_force, after the lanes are merged).
// FP64: the plain rint form on the FP64 mirror.
template <typename R> struct Frame;
template <> struct Frame<float> { float ps2, ps2_lo; };
template <> struct Frame<double> { double L, invL; };

__device__ __forceinline__ Frame<float> make_frame(const int4 &, const SysDesc &S) {
    Frame<float> F;
    F.ps2 = S.ps2;
    F.ps2_lo = S.ps2_lo;
    return F;
}
__device__ __forceinline__ Frame<double> make_frame(const double4_32a &, const SysDesc &S) {
    Frame<double> F;
    F.L = S.L;
    F.invL = S.invL;
    return F;
}

__device__ __forceinline__ void pair_delta(const Frame<float> &, const int4 &ri, const int4 &rj,
                                           float &dx, float &dy, float &dz) {
    dx = fixed_diff(ri.x, rj.x);
    dy = fixed_diff(ri.y, rj.y);
    dz = fixed_diff(ri.z, rj.z);
}
__device__ __forceinline__ void pair_delta(const Frame<double> &F, const double4_32a &ri,
                                           const double4_32a &rj, double &dx, double &dy,
                                           double &dz) {
    dx = min_image_fast(ri.x - rj.x, F.L, F.invL);
    dy = min_image_fast(ri.y - rj.y, F.L, F.invL);
    dz = min_image_fast(ri.z - rj.z, F.L, F.invL);
}
// r^2 in real units from the pair_delta components (mixed: |d|^2 (ps2 + ps2_lo), so the rounding
// of the squared unit adds no common scale error to every distance)
__device__ __forceinline__ float pair_r2(const Frame<float> &F, float dx, float dy, float dz) {
    const float d2 = dx * dx + dy * dy + dz * dz;
    return __fmaf_rn(d2, F.ps2, d2 * F.ps2_lo);
}
__device__ __forceinline__ double pair_r2(const Frame<double> &, double dx, double dy, double dz) {
    return dx * dx + dy * dy + dz * dz;
}
// A particle's force sum in real units (mixed: the sum was taken over d in mirror units)
__device__ __forceinline__ void scale_force(const SysDesc &S, float &fx, float &fy, float &fz) {
    fx = __fmaf_rn(fx, S.ps, fx * S.ps_lo);
    fy = __fmaf_rn(fy, S.ps, fy * S.ps_lo);
    fz = __fmaf_rn(fz, S.ps, fz * S.ps_lo);
}
__device__ __forceinline__ void scale_force(const SysDesc &, double &, double &, double &) {}

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
    const R r2 = pair_r2(F, dx, dy, dz);
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
        const bool in = r2 < c.x && r2 > R(0);   // r2 = 0: a pad entry (the particle itself)
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
            const bool inq = r2 < q.x && r2 > R(0);
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
    if (!(r2 > R(0))) return;   // a pad entry (the particle itself)
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
