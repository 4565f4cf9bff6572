// md_static.cu -- md_forces_static: forces of one system without allocating any device memory.
//
// Who needs this: code that may not call cudaMalloc at the moment it wants forces -- a host
// framework that owns all device memory through its own pool and forbids libraries from
// allocating behind its back (its memory budget is fixed up front), or a latency-critical loop
// that must never enter the CUDA allocator (cudaMalloc and cudaFree can synchronise the device
// and take far longer than the force evaluation itself).  Such a caller hands in device buffers
// for the inputs and outputs; the scratch space this computation needs (positions sorted by cell
// and their original indices) lives in one fixed array below, reserved when the library is
// loaded on a device and held until the process exits.
//
// The computation is a one-CTA variant of the force evaluation: bin the particles into cells of
// edge >= rc_max (27-cell stencil), sort them by cell into the scratch array, then sum the shifted-
// potential LJ pair forces over the stencil directly (no neighbour list), with the same FP32 pair
// arithmetic as the main path.  It is meant for small systems; larger ones go through md_sim.
#include "md.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

constexpr int kMaxParticles = 8192;   // MD_STATIC_MAX_PARTICLES
constexpr int kMaxCells = 4096;       // MD_STATIC_MAX_CELLS
constexpr int kMaxTypes = 8;
constexpr int kThreads = 1024;

// The scratch area: kMaxParticles sorted positions (float4: x, y, z, type bits) followed by
// kMaxParticles original indices.  Every call reuses (and overwrites) it.
constexpr size_t kScratchBytes = (size_t)kMaxParticles * sizeof(float4) + (size_t)kMaxParticles * sizeof(int);
static __device__ __align__(256) unsigned char g_md_static_scratch[kScratchBytes];

struct StaticParams {
    int n, nt, nc;
    float L, invL, halfL, Llo, cell_scale;
    double Ld;
    float rc2[kMaxTypes * kMaxTypes], c12[kMaxTypes * kMaxTypes], c6[kMaxTypes * kMaxTypes];
    float ush[kMaxTypes * kMaxTypes], a12[kMaxTypes * kMaxTypes], a6[kMaxTypes * kMaxTypes];
};

// Fold one coordinate into [0, L) with the steps of the host-side wrap in md_set_state: subtract
// floor(v / L) periods, fold a result that rounded to L or below 0, and map L itself to 0.  Every
// product and sum is rounded on its own (no contraction), so the counting pass and the scatter
// pass, which both call this, bin every particle into the same cell.
__device__ __forceinline__ double wrap_coord(double v, double L) {
    v = __dsub_rn(v, __dmul_rn(L, floor(__ddiv_rn(v, L))));
    if (v >= L) v = __dsub_rn(v, L);
    if (v < 0.0) v = __dadd_rn(v, L);
    if (v >= L) v = 0.0;   // -tiny + L rounded up to L
    return v;
}

// Wrapped FP32 mirror of particle k (x, y, z, type bits) and its cell.
__device__ __forceinline__ float4 wrapped_pos(const double *pos, const int *type, int k,
                                              double Ld) {
    const double x = wrap_coord(pos[3 * k], Ld), y = wrap_coord(pos[3 * k + 1], Ld),
                 z = wrap_coord(pos[3 * k + 2], Ld);
    return make_float4((float)x, (float)y, (float)z, __int_as_float(type[k]));
}
__device__ __forceinline__ int cell_of(const float4 &q, float cell_scale, int nc) {
    const int cx = min(max(__float2int_rd(q.x * cell_scale), 0), nc - 1);
    const int cy = min(max(__float2int_rd(q.y * cell_scale), 0), nc - 1);
    const int cz = min(max(__float2int_rd(q.z * cell_scale), 0), nc - 1);
    return (cz * nc + cy) * nc + cx;
}

__device__ __forceinline__ float mi(float xi, float xj, float xa, float nfl, float half, float L) {
    // minimum image with the coordinate near L shifted first (exact), as in the main path
    const float t = __fsub_rn(xi, xj);
    const float e = __fsub_rn(xa, __fmaf_rn(-nfl, L, xj));
    return fabsf(t) > half ? e : t;
}

__global__ void __launch_bounds__(kThreads) k_forces_static(StaticParams p, void *scratch,
                                                              const double *pos, const int *type,
                                                              double *f, double *u, double *w,
                                                              double *uw) {
    __shared__ int s_cnt[kMaxCells];
    __shared__ int s_start[kMaxCells + 1];
    __shared__ int s_warp[32];
    __shared__ double s_red[32][2];
    float4 *spos = reinterpret_cast<float4 *>(scratch);
    int *sidx = reinterpret_cast<int *>(spos + kMaxParticles);
    const int n = p.n, nc = p.nc, C = nc * nc * nc;

    // 1. cell counts start at zero on every call (the previous call left its own)
    for (int c = threadIdx.x; c < C; c += blockDim.x) s_cnt[c] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        atomicAdd(s_cnt + cell_of(wrapped_pos(pos, type, k, p.Ld), p.cell_scale, nc), 1);
    __syncthreads();
    // 2. exclusive scan of the counts (one chunk of cells per thread)
    {
        const int nt = blockDim.x, chunk = (C + nt - 1) / nt;
        const int c0 = min(C, (int)threadIdx.x * chunk), c1 = min(C, c0 + chunk);
        int sum = 0;
        for (int c = c0; c < c1; ++c) sum += s_cnt[c];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int yv = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += yv;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int v = lane < (nt >> 5) ? s_warp[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int yv = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += yv;
            }
            s_warp[lane] = v;
        }
        __syncthreads();
        int run = (x - sum) + (warp ? s_warp[warp - 1] : 0);
        for (int c = c0; c < c1; ++c) {
            s_start[c] = run;
            const int m = s_cnt[c];
            s_cnt[c] = run;          // becomes the fill cursor of the scatter
            run += m;
        }
        if (threadIdx.x == nt - 1) s_start[C] = run;
    }
    __syncthreads();
    // 3. scatter positions (FP32 mirror of the wrapped FP64 input) and indices into the scratch
    //    (the same wrap and cell as the counting pass, so every cell's slots are filled exactly)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float4 q = wrapped_pos(pos, type, k, p.Ld);
        const int slot = atomicAdd(s_cnt + cell_of(q, p.cell_scale, nc), 1);
        spos[slot] = q;
        sidx[slot] = k;
    }
    __syncthreads();
    // 4. forces over the 27-cell stencil (every cell once when nc < 3), summed per particle
    double Uacc = 0.0, Wacc = 0.0;
    const int span = nc < 3 ? nc : 3;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const float4 ri = spos[s];
        const int ti = __float_as_int(ri.w);
        // a type outside [0, n_types) would index past the coefficient tables: such a particle,
        // and every particle that meets one in its stencil, gets NaN outputs instead
        bool bad = (unsigned)ti >= (unsigned)p.nt;
        const bool ux = ri.x >= p.halfL, uy = ri.y >= p.halfL, uz = ri.z >= p.halfL;
        const float xa = ux ? __fsub_rn(__fsub_rn(ri.x, p.L), p.Llo) : __fadd_rn(ri.x, p.Llo);
        const float ya = uy ? __fsub_rn(__fsub_rn(ri.y, p.L), p.Llo) : __fadd_rn(ri.y, p.Llo);
        const float za = uz ? __fsub_rn(__fsub_rn(ri.z, p.L), p.Llo) : __fadd_rn(ri.z, p.Llo);
        const float nx = ux ? 0.f : 1.f, ny = uy ? 0.f : 1.f, nz = uz ? 0.f : 1.f;
        const int ci = cell_of(ri, p.cell_scale, nc);
        const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
        float fx = 0.f, fy = 0.f, fz = 0.f, uu = 0.f, ww = 0.f;
        for (int oz = 0; oz < span; ++oz) {
            const int zz = span == nc ? oz : (cz - 1 + oz + nc) % nc;
            for (int oy = 0; oy < span; ++oy) {
                const int yy = span == nc ? oy : (cy - 1 + oy + nc) % nc;
                for (int ox = 0; ox < span; ++ox) {
                    const int xx = span == nc ? ox : (cx - 1 + ox + nc) % nc;
                    const int c = (zz * nc + yy) * nc + xx;
                    for (int j = s_start[c]; j < s_start[c + 1] && !bad; ++j) {
                        if (j == s) continue;
                        const float4 rj = spos[j];
                        if ((unsigned)__float_as_int(rj.w) >= (unsigned)p.nt) {
                            bad = true;
                            break;
                        }
                        const float dx = mi(ri.x, rj.x, xa, nx, p.halfL, p.L);
                        const float dy = mi(ri.y, rj.y, ya, ny, p.halfL, p.L);
                        const float dz = mi(ri.z, rj.z, za, nz, p.halfL, p.L);
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const int q = ti * p.nt + __float_as_int(rj.w);
                        if (r2 < p.rc2[q]) {
                            const float r2i = __fdividef(1.0f, r2), r6i = r2i * r2i * r2i;
                            const float fs = r2i * r6i * (p.a12[q] * r6i - p.a6[q]);
                            fx += fs * dx; fy += fs * dy; fz += fs * dz;
                            uu += r6i * (p.c12[q] * r6i - p.c6[q]) - p.ush[q];
                            ww += fs * r2;
                        }
                    }
                }
            }
        }
        const int k = sidx[s];
        if (bad) fx = fy = fz = uu = ww = __int_as_float(0x7fc00000);   // NaN
        f[3 * k] = fx; f[3 * k + 1] = fy; f[3 * k + 2] = fz;
        const float ui = 0.5f * uu, wi = ww * (1.0f / 6.0f);
        if (u) u[k] = ui;
        if (w) w[k] = wi;
        Uacc += (double)ui;
        Wacc += (double)wi;
    }
    // 5. totals: FP64 sums, warp then block
    for (int o = 16; o > 0; o >>= 1) {
        Uacc += __shfl_down_sync(0xffffffffu, Uacc, o);
        Wacc += __shfl_down_sync(0xffffffffu, Wacc, o);
    }
    if ((threadIdx.x & 31) == 0) { s_red[threadIdx.x >> 5][0] = Uacc; s_red[threadIdx.x >> 5][1] = Wacc; }
    __syncthreads();
    if (threadIdx.x < 2 && uw) {
        double acc = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) acc += s_red[k][threadIdx.x];
        uw[threadIdx.x] = acc;
    }
}

// Device address of the scratch array, looked up once per device (host code cannot use the
// symbol itself: in host code it names a host-side stand-in, not device memory).
std::mutex g_mu;
void *g_scratch_ptr[64] = {};

int scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_md_static_scratch);
        if (e != cudaSuccess || !ptr) {
            std::fprintf(stderr, "md_forces_static: cudaGetSymbolAddress failed: %s\n",
                         cudaGetErrorString(e));
            cudaGetLastError();
            return MD_ECUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return MD_OK;
}

}  // namespace

extern "C" int md_forces_static(const double *pos, const int *type, int n, double L, int n_types,
                                const md_pair *params, double *f, double *u, double *w,
                                double *uw, void *cuda_stream) {
    if (!pos || !type || !f || !params || n < 1 || n_types < 1 || n_types > kMaxTypes ||
        !(L > 0.0) || !std::isfinite(L))
        return MD_EINVAL;
    double rc_max = 0.0;
    for (int q = 0; q < n_types * n_types; ++q) {
        const md_pair &pp = params[q];
        if (!(pp.sigma > 0.0) || !(pp.rc > 0.0) || !(pp.eps >= 0.0)) return MD_EINVAL;
        rc_max = std::fmax(rc_max, pp.rc);
    }
    if (!(L > 2.0 * rc_max)) return MD_EINVAL;   // minimum image
    if (n > kMaxParticles) {
        std::fprintf(stderr,
                     "md_forces_static: %d particles exceed the fixed scratch limit of %d "
                     "(MD_STATIC_MAX_PARTICLES); use md_create/md_get_forces instead\n",
                     n, kMaxParticles);
        return MD_EINVAL;
    }
    int nc = (int)std::floor(L / (rc_max * (1.0 + 1e-4)));
    if (nc < 1) nc = 1;
    if ((long long)nc * nc * nc > kMaxCells) {
        std::fprintf(stderr,
                     "md_forces_static: %d^3 cells exceed the fixed limit of %d cells "
                     "(MD_STATIC_MAX_CELLS)\n", nc, kMaxCells);
        return MD_EINVAL;
    }
    StaticParams p;
    p.n = n;
    p.nt = n_types;
    p.nc = nc;
    p.Ld = L;
    p.L = (float)L;
    p.invL = (float)(1.0 / L);
    p.halfL = (float)(0.5 * L);
    p.Llo = (float)(L - (double)p.L);
    p.cell_scale = (float)(nc / L);
    for (int q = 0; q < n_types * n_types; ++q) {
        const md_pair &pp = params[q];
        const double s6 = std::pow(pp.sigma, 6.0), c12 = 4.0 * pp.eps * s6 * s6, c6 = 4.0 * pp.eps * s6;
        const double rc6 = std::pow(pp.rc, 6.0);
        p.rc2[q] = (float)(pp.rc * pp.rc);
        p.c12[q] = (float)c12;
        p.c6[q] = (float)c6;
        p.ush[q] = (float)(c12 / (rc6 * rc6) - c6 / rc6);
        p.a12[q] = (float)(12.0 * c12);
        p.a6[q] = (float)(6.0 * c6);
    }
    void *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    k_forces_static<<<1, kThreads, 0, (cudaStream_t)cuda_stream>>>(p, scratch, pos, type, f, u, w,
                                                                     uw);
    if (cudaGetLastError() != cudaSuccess) return MD_ECUDA;
    return MD_OK;
}
