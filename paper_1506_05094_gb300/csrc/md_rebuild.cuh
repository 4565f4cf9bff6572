// md_rebuild.cuh -- the cell-sorted rebuild of the neighbour list (Sec. 7, Fig. 4) on the grid
// path: work plan, bin / scan / scatter / in-cell order / gather (or the fused one-CTA sort), build.
#pragma once
#include "md_step.cuh"

namespace md {

// ------------------------------------------------------------------------------------------------
// Rebuild (Sec. 7).  k_plan compacts the replicas whose need flag is set into a work list; the
// other kernels grid-stride over that list only (no blocks are spent on replicas that keep their
// list).  halt and need_any only change between passes, so every thread sees the same values.
// An overflow does not stop a pass: the copy back of the permuted data must always complete.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool rebuild_off(const Ctrl *c) {
    return *(volatile const int *)&c->halt || !*(volatile const int *)&c->need_any;
}

// The cell sort and the cell-list build run in this pass: always with the cell method, and with
// the O(N^2) method only on its periodic re-sort passes (Appendix, step 5).
template <typename A> __device__ __forceinline__ bool cells_off(const A &a) {
    return rebuild_off(a.ctrl) || (a.list_method == 1 && !a.plan->sort_now);
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

// Cell of a mirror position (Sec. 7).  Mixed precision: exact integer binning of the fixed-point
// coordinate, floor(x nc / 2^32), always in [0, nc).  FP64: floor of the FP32 product x nc / L,
// clamped to [0, nc).
__device__ __forceinline__ int cell_index(const int4 &p, const SysDesc &S) {
    const unsigned nc = (unsigned)S.nc;
    const int cx = (int)__umulhi((unsigned)p.x, nc), cy = (int)__umulhi((unsigned)p.y, nc),
              cz = (int)__umulhi((unsigned)p.z, nc);
    return (cz * S.nc + cy) * S.nc + cx;
}
__device__ __forceinline__ int cell_index(const double4_32a &p, const SysDesc &S) {
    const float cs = S.cell_scale;
    int cx = __float2int_rd(__fmul_rn((float)p.x, cs));
    int cy = __float2int_rd(__fmul_rn((float)p.y, cs));
    int cz = __float2int_rd(__fmul_rn((float)p.z, cs));
    cx = min(max(cx, 0), S.nc - 1);
    cy = min(max(cy, 0), S.nc - 1);
    cz = min(max(cz, 0), S.nc - 1);
    return (cz * S.nc + cy) * S.nc + cx;
}
// Position of a particle along one axis relative to its cell c, in cell edges (the clipping of
// the list build's stencil needs only an estimate: it carries a slack far above these roundings).
// Mixed precision: the exact fraction in [0, 1).  FP64: x nc / L - c (it may reach 1 where the
// binning clamped a coordinate that rounded up to L).
__device__ __forceinline__ float cell_frac(int x, int, const SysDesc &S) {
    const unsigned lo = (unsigned)((unsigned long long)(unsigned)x * (unsigned)S.nc);
    return (float)lo * 2.3283064365386963e-10f;   // 2^-32
}
__device__ __forceinline__ float cell_frac(double x, int c, const SysDesc &S) {
    return __fmul_rn((float)x, S.cell_scale) - (float)c;
}

// One CTA: exclusive scans over replicas of (flagged, particles, cells) -> the pass's work list.
template <typename R> __global__ void k_plan(const RebuildArgs<R> a) {
    __shared__ int s_w[3][32];
    const int R_ = a.nrep, nt = blockDim.x;
    if (rebuild_off(a.ctrl)) {
        if (threadIdx.x == 0) {
            a.plan->nflag = 0; a.plan->tot_p = 0; a.plan->tot_c = 0; a.plan->sort_now = 0;
        }
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
        int sort_now = 0;
        if (of > 0) {
            const int passes = a.ctrl->rebuild_passes + 1;
            a.ctrl->rebuild_passes = passes;
            sort_now = (a.list_method == 1 && a.resort > 0 && passes % a.resort == 0) ? 1 : 0;
        }
        a.plan->sort_now = sort_now;
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
    if (cells_off(a)) return;
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
    if (cells_off(a)) return;
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
    if (cells_off(a)) return;
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int r, i;
        pass_particle(a.plan_pp, a.plan_rep, nf, t, a.sys, r, i);
        a.perm[a.cell_start[a.cell_of[i]] + a.rank[i]] = i;
    }
}

// Atomic slot order inside a cell is arbitrary (as with atomicInc in Sec. 6); restore a
// deterministic order: by user id.  Each particle counts the members of its cell (listed in
// atomic order by k_scatter) that have a smaller id: that count is its place in the cell's
// id-sorted order.  The counts reuse the atomic-rank array, which k_scatter has consumed.
template <typename R> __global__ void k_cellsort(const RebuildArgs<R> a) {
    if (cells_off(a)) return;
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int r, i;
        pass_particle(a.plan_pp, a.plan_rep, nf, t, a.sys, r, i);
        const int c = a.cell_of[i];
        const int s = a.cell_start[c], e = a.cell_start[c + 1];
        const int key = a.id[i];
        int below = 0;
        for (int q = s; q < e; ++q) below += a.id[a.perm[q]] < key ? 1 : 0;
        a.rank[i] = below;
    }
}

// Every rebuilt particle's data to its sorted slot (cell start + place in the cell) in scratch.
template <typename R> __global__ void k_gather(const RebuildArgs<R> a) {
    if (cells_off(a)) return;
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int r, o;
        pass_particle(a.plan_pp, a.plan_rep, nf, t, a.sys, r, o);
        const int s = a.cell_start[a.cell_of[o]] + a.rank[o];
        a.tpos[s] = a.pos[o];
        if (!a.key_is_pos) a.tkey[s] = a.key[o];
        a.txm[s] = a.xm[o];
        a.tym[s] = a.ym[o];
        a.tzm[s] = a.zm[o];
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
    const int nc = S.nc, span = S.span, reach = S.reach;
    const int c = cell_index(ki, S);
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const bool full = (span == nc);
    // Per-particle clipping of the stencil (the search volume of Sec. 7 is a cube of cells around
    // the particle's cell; only cells that reach within rc + s of the particle itself can hold a
    // neighbour).  In cell units the particle sits at fraction f of its cell along each axis; a
    // cell d cells away is at least max(0, d - f) (d > 0) or f + |d| - 1 (d < 0) away along that
    // axis.  Rows whose (y, z) gap already exceeds the particle's largest threshold are skipped
    // and every row's x extent is cut to the cells within reach.  The bound carries a slack
    // (1e-3 cell, 0.1 % of the threshold) far above FP32 rounding, so no accepted pair is ever
    // dropped; the cells that remain are visited in the same order, so the list is unchanged.
    float fxc = 0.f, fyc = 0.f, fzc = 0.f, lim2 = 0.f;
    if (!full) {
        const float cs = S.cell_scale;
        fxc = cell_frac(ki.x, cx, S);
        fyc = cell_frac(ki.y, cy, S);
        fzc = cell_frac(ki.z, cz, S);
        float thr = 0.f;
        for (int t = 0; t < ntypes; ++t) thr = fmaxf(thr, (float)s_thr[ti * ntypes + t]);
        lim2 = thr * cs * cs * 1.001f + 1e-3f;
    }
    auto gap = [](int d, float f) -> float {
        const float g = d > 0 ? (float)d - f : (d < 0 ? f - (float)d - 1.f : 0.f);
        return fmaxf(g - 1e-3f, 0.f);
    };
    // range q of the stencil: row q/2 in (z, y) order, part q%2 of its x extent (two parts when
    // the row wraps around the box)
    auto range = [&](int q) -> int2 {
        const int rowi = q >> 1, part = q & 1;
        const int oz = rowi / span, oy = rowi % span;
        int lo, hi;
        if (full) {
            if (part) return make_int2(0, 0);
            lo = 0;
            hi = nc - 1;
        } else {
            const float gy = gap(oy - reach, fyc), gz = gap(oz - reach, fzc);
            const float rem = lim2 - gy * gy - gz * gz;
            if (rem <= 0.f) return make_int2(0, 0);
            const float w = sqrtf(rem);
            const int x0 = cx - min(reach, (int)(w - fxc + 1.001f));
            const int x1 = cx + min(reach, (int)(w + fxc + 0.001f));
            int a0, a1, b0 = 0, b1 = -1;
            if (x0 < 0) { a0 = x0 + nc; a1 = nc - 1; b0 = 0; b1 = x1; }
            else if (x1 >= nc) { a0 = x0; a1 = nc - 1; b0 = 0; b1 = x1 - nc; }
            else { a0 = x0; a1 = x1; }
            lo = part ? b0 : a0;
            hi = part ? b1 : a1;
        }
        const int zz = full ? oz : (cz - reach + oz + nc) % nc;
        const int yy = full ? oy : (cy - reach + oy + nc) % nc;
        const int row = (zz * nc + yy) * nc;
        return (hi < lo) ? make_int2(0, 0) : make_int2(CS(row + lo), CS(row + hi + 1));
    };
    const int nr = span * span * 2;
    if (STAGE) {
        // stage every range with independent loads spread over the lanes, so the cellStart
        // latency is paid once instead of once per row
        for (int q = lt; q < nr; q += TPB) s_rng[q] = range(q);
        __syncwarp(gmask);
    }
    // each lane tests U candidates per pass, then U ballots in candidate order keep the
    // compaction order of a one-candidate-per-lane walk (U = 1: rows hold ~20 candidates, wider
    // passes leave lanes idle and measured slower)
    constexpr int U = 1;
    int cnt = 0;
    for (int q = 0; q < nr; ++q) {
        const int2 rg = STAGE ? s_rng[q] : range(q);
        for (int b0 = rg.x; b0 < rg.y; b0 += TPB * U) {
            bool ok[U];
#pragma unroll
            for (int uu = 0; uu < U; ++uu) {
                const int j = b0 + uu * TPB + lt;
                ok[uu] = false;
                if (j < rg.y && j != self) {
                    const V4 kj = K(j);
                    ok[uu] = key_dist2(ki, kj, S) < s_thr[ti * ntypes + type_of(kj)];
                }
            }
#pragma unroll
            for (int uu = 0; uu < U; ++uu) {
                const unsigned m = __ballot_sync(gmask, ok[uu]);
                if (ok[uu]) {
                    const int sl = cnt + __popc(m & below);
                    if (sl < nmax) nbl[nbl_offset(slot_i, sl, nmax)] = base + b0 + uu * TPB + lt;
                }
                cnt += __popc(m);
            }
        }
    }
    if (STAGE) __syncwarp(gmask);   // the staged ranges are reused by the group's next particle
    return cnt;
}

// Pad a list of cnt entries with the particle's own slot up to the next multiple of `pad`
// (4 x the step kernel's threads per particle, and n_max is a multiple of it), so every lane of
// the force loop runs whole groups of four entries with no bounds test; a padded entry is the
// particle itself, at distance 0, which the pair arithmetic excludes.  TPB lanes share the work.
__device__ __forceinline__ void pad_list(int *nbl, int slot_i, int cnt, int nmax, int pad, int lt,
                                         int TPB) {
    const int end = min(nmax, (cnt + pad - 1) / pad * pad);
    for (int k = cnt + lt; k < end; k += TPB) nbl[nbl_offset(slot_i, k, nmax)] = slot_i;
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

template <typename R, int TPB> __global__ void __launch_bounds__(MD_BUILD_BLOCK, 12) k_build(const RebuildArgs<R> a) {
    typedef typename V4T<R>::t V4;
    if (cells_off(a)) return;
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
        const SysDesc S = a.sys[r];   // a copy: the list stores cannot alias it
        GlobalKey<R> K{Kp};
        GlobalStart CS{a.cell_start, S.cell_off};
        int cnt = build_one<R, TPB, true>(S, K, CS, i, i, 0, a.nbl, a.nmax, s_thr, a.ntypes,
                                          s_rng_all[threadIdx.x / TPB]);
        pad_list(a.nbl, i, cnt, a.nmax, a.pad, threadIdx.x % TPB, TPB);
        if (threadIdx.x % TPB == 0) {
            if (cnt > a.nmax) {   // Sec. 4: out of space -> flag for the host, which doubles n_max
                atomicMax(&a.ctrl->max_count, cnt);
                atomicExch(&a.ctrl->overflow, 1);
                cnt = a.nmax;
            }
            a.nnb[i] = cnt;
            a.pos[i] = a.tpos[i];
            a.pos_build[i] = Kp[i];
            a.xm[i] = a.txm[i];
            a.ym[i] = a.tym[i];
            a.zm[i] = a.tzm[i];
            a.vel[i] = a.tvel[i];
            a.img[i] = a.timg[i];
            a.id[i] = a.tid[i];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// List build with one warp per cell (build_lanes = MD_BUILD_CELL).  Every particle of a cell
// searches the same stencil of cells (Fig. 4), so the warp walks the cell's stencil ranges once,
// 32 candidates at a time (one per lane, consecutive sorted slots), and tests each batch against
// up to MD_CELL_CHUNK particles of the cell read from shared memory.  Accepted candidates are
// compacted per particle by ballot in candidate order.  The ranges are build_one's in the same
// order without its per-particle clipping; the clipping drops only cells that hold no neighbour
// of the particle and keeps the order of the rest, so every list is the same as build_one's, bit
// for bit.
// ------------------------------------------------------------------------------------------------
#define MD_CELL_CHUNK 8

template <typename R>
__global__ void __launch_bounds__(MD_BUILD_BLOCK, 8) k_build_cell(const RebuildArgs<R> a) {
    typedef typename V4T<R>::t V4;
    constexpr int NW = MD_BUILD_BLOCK / 32;
    if (cells_off(a)) return;
    __shared__ R s_thr[MD_MAX_PAIRS];
    __shared__ int s_lo[NW][MD_MAX_RANGES];        // first slot of each nonempty range
    __shared__ int s_pre[NW][MD_MAX_RANGES + 1];   // its first candidate in the cell's order
    __shared__ V4 s_ki[NW][MD_CELL_CHUNK];
    const int npair = a.ntypes * a.ntypes;
    for (int p = threadIdx.x; p < npair; p += blockDim.x)
        s_thr[p] = sizeof(R) == 4 ? (R)a.tab[p].thr2 : (R)a.tab[p].thr2d;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int tot = a.plan->tot_c, nf = a.plan->nflag;
    const V4 *Kp = a.key_is_pos ? a.tpos : a.tkey;
    int *lo_w = s_lo[warp], *pre_w = s_pre[warp];
    V4 *ki_w = s_ki[warp];
    for (int t = blockIdx.x * NW + warp; t < tot; t += gridDim.x * NW) {
        const int k = find_seg(a.plan_pc, nf, t);
        const SysDesc S = a.sys[a.plan_rep[k]];   // a copy: the list stores cannot alias it
        const int cl = t - a.plan_pc[k];
        const int p0 = a.cell_start[S.cell_off + cl], p1 = a.cell_start[S.cell_off + cl + 1];
        if (p0 == p1) continue;
        const int nc = S.nc, span = S.span, reach = S.reach;
        const int cx = cl % nc, cy = (cl / nc) % nc, cz = cl / (nc * nc);
        const bool full = (span == nc);
        // the stencil's ranges: row q/2 in (z, y) order, part q%2 of its x extent
        const int nr = span * span * 2;
        int total = 0, nq = 0;
        for (int q0 = 0; q0 < nr; q0 += 32) {
            const int q = q0 + lane;
            int lo = 0, len = 0;
            if (q < nr) {
                const int rowi = q >> 1, part = q & 1;
                const int oz = rowi / span, oy = rowi % span;
                int x0 = 0, x1 = nc - 1;
                bool has = (part == 0);
                if (!full) {
                    const int a0 = cx - reach, a1 = cx + reach;
                    if (a0 < 0) { has = true; x0 = part ? 0 : a0 + nc; x1 = part ? a1 : nc - 1; }
                    else if (a1 >= nc) { has = true; x0 = part ? 0 : a0; x1 = part ? a1 - nc : nc - 1; }
                    else { x0 = a0; x1 = a1; }
                }
                if (has) {
                    const int zz = full ? oz : (cz - reach + oz + nc) % nc;
                    const int yy = full ? oy : (cy - reach + oy + nc) % nc;
                    const int row = S.cell_off + (zz * nc + yy) * nc;
                    lo = a.cell_start[row + x0];
                    len = a.cell_start[row + x1 + 1] - lo;
                }
            }
            // keep the nonempty ranges in order, with the running candidate count
            const unsigned ne = __ballot_sync(FULL_MASK, len > 0);
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL_MASK, incl, o);
                if (lane >= o) incl += v;
            }
            if (len > 0) {
                const int pos = nq + __popc(ne & below);
                lo_w[pos] = lo;
                pre_w[pos] = total + incl - len;
            }
            total += __shfl_sync(FULL_MASK, incl, 31);
            nq += __popc(ne);
        }
        if (lane == 0) pre_w[nq] = total;
        __syncwarp();
        for (int pb = p0; pb < p1; pb += MD_CELL_CHUNK) {
            const int np = min(MD_CELL_CHUNK, p1 - pb);
            if (lane < np) ki_w[lane] = Kp[pb + lane];
            __syncwarp();
            int cnt[MD_CELL_CHUNK];
#pragma unroll
            for (int p = 0; p < MD_CELL_CHUNK; ++p) cnt[p] = 0;
            int q = 0;   // this lane's current range
            for (int f0 = 0; f0 < total; f0 += 32) {
                const int f = f0 + lane;
                const bool valid = f < total;
                int j = -1, tj = 0;
                V4 kj = ki_w[0];
                if (valid) {
                    while (pre_w[q + 1] <= f) ++q;
                    j = lo_w[q] + (f - pre_w[q]);
                    kj = Kp[j];
                    tj = type_of(kj);
                }
#pragma unroll
                for (int p = 0; p < MD_CELL_CHUNK; ++p) {
                    if (p < np) {
                        const V4 ki = ki_w[p];
                        const bool ok = valid && j != pb + p &&
                                        key_dist2(ki, kj, S) < s_thr[type_of(ki) * a.ntypes + tj];
                        const unsigned m = __ballot_sync(FULL_MASK, ok);
                        if (ok) {
                            const int sl = cnt[p] + __popc(m & below);
                            if (sl < a.nmax) a.nbl[nbl_offset(pb + p, sl, a.nmax)] = j;
                        }
                        cnt[p] += __popc(m);
                    }
                }
            }
            int mine = 0;
#pragma unroll
            for (int p = 0; p < MD_CELL_CHUNK; ++p) {
                if (p < np) pad_list(a.nbl, pb + p, cnt[p], a.nmax, a.pad, lane, 32);
                if (lane == p) mine = cnt[p];
            }
            if (lane < np) {
                const int i = pb + lane;
                if (mine > a.nmax) {   // Sec. 4: out of space -> flag for the host
                    atomicMax(&a.ctrl->max_count, mine);
                    atomicExch(&a.ctrl->overflow, 1);
                    mine = a.nmax;
                }
                a.nnb[i] = mine;
                a.pos[i] = a.tpos[i];
                a.pos_build[i] = Kp[i];
                a.xm[i] = a.txm[i];
                a.ym[i] = a.tym[i];
                a.zm[i] = a.tzm[i];
                a.vel[i] = a.tvel[i];
                a.img[i] = a.timg[i];
                a.id[i] = a.tid[i];
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------------------------------------
// O(N^2) list build (Sec. 6, Fig. 3): TPB lanes per rebuilt particle scan every particle of its
// replica in slot order (no cell sort), test the same bit-defined FP32 rule as the cell build and
// compact the accepted slots by ballot in slot order.  The build positions are the current ones.
// ------------------------------------------------------------------------------------------------
template <typename R, int TPB>
__global__ void __launch_bounds__(MD_BUILD_BLOCK) k_build_n2(const RebuildArgs<R> a) {
    typedef typename V4T<R>::t V4;
    if (rebuild_off(a.ctrl) || a.plan->sort_now) return;   // re-sort passes build from cells
    __shared__ R s_thr[MD_MAX_PAIRS];
    const int npair = a.ntypes * a.ntypes;
    for (int p = threadIdx.x; p < npair; p += blockDim.x)
        s_thr[p] = sizeof(R) == 4 ? (R)a.tab[p].thr2 : (R)a.tab[p].thr2d;
    __syncthreads();
    const int tot = a.plan->tot_p, nf = a.plan->nflag;
    const int groups = gridDim.x * (blockDim.x / TPB);
    const int lt = threadIdx.x % TPB, lane = threadIdx.x & 31;
    const unsigned gmask = (TPB == 32) ? FULL_MASK : (((1u << TPB) - 1u) << (lane & ~(TPB - 1)));
    const unsigned below = (1u << lane) - 1u;
    for (int g = blockIdx.x * (blockDim.x / TPB) + threadIdx.x / TPB; g < tot; g += groups) {
        int r, i;
        pass_particle(a.plan_pp, a.plan_rep, nf, g, a.sys, r, i);
        const SysDesc S = a.sys[r];   // a copy: the list stores cannot alias it
        const V4 ki = a.key[i];
        const int ti = type_of(ki);
        int cnt = 0;
        for (int b0 = S.off; b0 < S.off + S.n; b0 += TPB) {
            const int j = b0 + lt;
            bool ok = false;
            if (j < S.off + S.n && j != i) {
                const V4 kj = a.key[j];
                ok = key_dist2(ki, kj, S) < s_thr[ti * a.ntypes + type_of(kj)];
            }
            const unsigned m = __ballot_sync(gmask, ok);
            if (ok) {
                const int sl = cnt + __popc(m & below);
                if (sl < a.nmax) a.nbl[nbl_offset(i, sl, a.nmax)] = j;
            }
            cnt += __popc(m);
        }
        pad_list(a.nbl, i, cnt, a.nmax, a.pad, lt, TPB);
        if (lt == 0) {
            if (cnt > a.nmax) {
                atomicMax(&a.ctrl->max_count, cnt);
                atomicExch(&a.ctrl->overflow, 1);
                cnt = a.nmax;
            }
            a.nnb[i] = cnt;
            // build positions = the keys; not rewritten when the keys are the build positions
            // themselves (other groups are still reading them)
            if (a.key != a.pos_build) a.pos_build[i] = ki;
            if (S.off == i) a.th[r].rebuilds += 1;
        }
    }
}

}  // namespace md
