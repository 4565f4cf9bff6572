// md_rep.cuh -- the replica-resident step kernel (k_rep) and the fused one-CTA-per-replica sort.
#pragma once
#include "md_rebuild.cuh"

namespace md {

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
                                             const typename Coef4<R>::t *s_c1, R &fx, R &fy,
                                             R &fz, R &u, R &w) {
    const typename Coef4<R>::t c1 = s_c0[0];
    const typename Coef4<R>::t c1b = s_c1[0];
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
                        interact<R, SINGLE, false>(ri, ti, s_pos[j], F, a.ntypes, s_c0, s_c1, c1, c1b,
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

// In-CTA rebuild of one replica (Sec. 7): bin its particles into cells, exclusive scan of the
// counts (cellStart), scatter, in-cell order by user id, permutation of all particle data, and the
// list build of Fig. 4 from the shared-memory positions and cell starts (TPB lanes per particle).
// On entry s_pos holds the replica's positions in its current slot order; on exit the sorted
// ones, s_cs the cell starts (local slots).  An overfull list stores n_max entries, raises
// *ovf_flag and the largest count, and the call returns 1 (block-uniform); else 0.
// The slot order, list order and list contents are those of the grid path's sort and build.
// Call with the whole block; uses s_cnt (cmax), s_cell and s_perm (n entries each), s_warp (32).
template <typename R, int TPB>
__device__ __forceinline__ int cta_rebuild(const RebuildArgs<R> &b, const SysDesc &S, int r,
                                           typename V4T<R>::t *s_pos, int *s_cs, int *s_cnt,
                                           int *s_cell, int *s_perm, int *s_warp, const R *s_thr,
                                           int *ovf_flag) {
    const int n = S.n, off = S.off;
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
    for (int k = threadIdx.x; k < n; k += blockDim.x) s_perm[atomicAdd(s_cnt + s_cell[k], 1)] = k;
    __syncthreads();
    const int *idg = b.id + off;   // user ids (pre-permutation)
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
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int o = off + s_perm[q], d = off + q;
        b.tpos[d] = s_pos[s_perm[q]];
        b.txm[d] = b.xm[o]; b.tym[d] = b.ym[o]; b.tzm[d] = b.zm[o];
        b.tvel[d] = b.vel[o];
        b.timg[d] = b.img[o];
        b.tid[d] = b.id[o];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int d = off + q;
        s_pos[q] = b.tpos[d];
        b.xm[d] = b.txm[d]; b.ym[d] = b.tym[d]; b.zm[d] = b.tzm[d];
        b.vel[d] = b.tvel[d];
        b.img[d] = b.timg[d];
        b.id[d] = b.tid[d];
    }
    __syncthreads();
    // list build from the shared positions and cell starts
    SharedKey<R> K{s_pos};
    SharedStart CS{s_cs};
    int ovf = 0;
    for (int g = threadIdx.x / TPB; g < n; g += blockDim.x / TPB) {
        int cnt = build_one<R, TPB, false>(S, K, CS, g, off + g, off, b.nbl, b.nmax, s_thr,
                                           b.ntypes, nullptr);
        pad_list(b.nbl, off + g, cnt, b.nmax, b.pad, threadIdx.x % TPB, TPB);
        if (threadIdx.x % TPB == 0) {
            if (cnt > b.nmax) {
                atomicMax(&b.ctrl->max_count, cnt);
                atomicExch(ovf_flag, 1);
                ovf = 1;
                cnt = b.nmax;
            }
            b.nnb[off + g] = cnt;
            b.pos_build[off + g] = s_pos[g];
        }
    }
    if (threadIdx.x == 0) b.th[r].rebuilds += 1;
    return __syncthreads_or(ovf);
}

template <typename R, int TP, bool SINGLE, int TPB>
__global__ void __launch_bounds__(1024) k_rep(const StepArgs<R> a, const RebuildArgs<R> b) {
    typedef typename V4T<R>::t V4;
    typedef typename Coef4<R>::t C4;
    typedef typename Coef4<R>::t C2;
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
    __shared__ unsigned s_disp[2];   // replica maxima of the displacement measures
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
            const Thermo *T = a.th + r;
            s_xi = T->xi_next;
            s_A = (R)T->A_next;
            s_B = (R)T->B_next;
            s_ovf = 0;
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_pos[k] = a.pos_in[off + k];
        __syncthreads();

        if (rebuild) {
            // ---- Sec. 7 rebuild inside the CTA: bin, scan, scatter, order by id, permute, build
            if (cta_rebuild<R, TPB>(b, S, r, s_pos, s_cs, s_cnt, s_cell, s_perm, s_warp, s_thr,
                                    &a.ctrl->rep_overflow) &&
                threadIdx.x == 0)
                s_ovf = 1;
            __syncthreads();
        }

        // ---- forces over the list (shared-memory gathers), integration, tile partials ----
        const bool direct = s_ovf != 0;
        int moved_any = 0;
        if (threadIdx.x < 2) s_disp[threadIdx.x] = 0u;
        __syncthreads();
        for (int t0 = 0; t0 < S.ntiles; t0 += tpb_tiles) {
            const int t = t0 + tsub;
            const int li = t * P + lp;
            const bool active = t < S.ntiles && li < n;
            const int i = off + li;
            R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
            V4 ri{};
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
            scale_force(S, fx, fy, fz);
            const bool leader = active && lt == 0;
            u *= R(0.5);
            w *= R(1.0 / 6.0);
            R ke = 0, px = 0, py = 0, pz = 0;
            bool moved = false;
            float d2 = 0.f, st2 = 0.f;
            if (leader)
                moved = integrate_one(a, S, i, ri, fx, fy, fz, s_im[ti], s_m[ti], s_A, s_B, ke,
                                      px, py, pz, d2, st2);
            moved_any |= (int)moved;
            if (a.rebuild_batch > 1) disp_max_warp(s_disp, d2, st2);
            const R vals[MD_NRED] = {leader ? u : R(0), leader ? w : R(0), ke, px, py, pz};
            // partials of tiles past the replica's last one are written to spare rows and ignored
            tile_partial(vals, s_tmp, s_part + (long long)t0 * MD_NRED, TT >> 5);
            __syncthreads();
        }
        moved_any = __syncthreads_or(moved_any);
        // an overflowed list stays flagged: every step rebuilds and evaluates list-free until the
        // host has grown the capacity
        replica_finish(a, r, S, s_part, s_xi, (moved_any || direct) ? 1 : 0, s_tmp, s_red, false,
                       TT, __uint_as_float(s_disp[0]), __uint_as_float(s_disp[1]));
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
template <typename R> __global__ void __launch_bounds__(1024) k_sort_small(const RebuildArgs<R> a) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int s_warp[32];
    if (cells_off(a)) return;
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
            a.txm[d] = a.xm[o];
            a.tym[d] = a.ym[o];
            a.tzm[d] = a.zm[o];
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
