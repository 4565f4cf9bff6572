// md_runtime.cu -- host runtime behind the C ABI of include/md.h: device memory, replica layout,
// state upload / download in user order, the step scheduler (CUDA graphs with IF nodes around
// the rebuild, or plain launches), overflow recovery, checkpoints, logging and profiling.
#include "md.h"
#include "md_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

const int kMaxTypes = MD_MAX_TYPES;

struct Buffers {
    void *pos[2] = {nullptr, nullptr};
    double *xd = nullptr, *yd = nullptr, *zd = nullptr;
    void *vel = nullptr;
    int4 *img = nullptr;
    int *id = nullptr;
    void *pos_build = nullptr;
    void *tpos = nullptr, *tkey = nullptr;
    double *txd = nullptr, *tyd = nullptr, *tzd = nullptr;
    void *tvel = nullptr;
    int4 *timg = nullptr;
    int *tid = nullptr;
    int *cell_of = nullptr, *rank = nullptr, *perm = nullptr;
    int *cell_start = nullptr, *count = nullptr, *crep = nullptr, *prep = nullptr;
    int *nbl = nullptr, *nnb = nullptr;
    Plan *plan = nullptr;
    int *plan_arr = nullptr;
    SysDesc *sys = nullptr;
    PairTab *tab = nullptr;
    Thermo *th = nullptr;
    Ctrl *ctrl = nullptr;
    int *moved = nullptr, *need = nullptr;
    unsigned *disp = nullptr;   // 2 per replica: displacement maxima of the current step
    unsigned *ticket = nullptr;
    double *partial = nullptr;
    int *tile_rep = nullptr;
    double *log = nullptr;
    void *f_out = nullptr, *w_out = nullptr;
};

}  // namespace

struct md_sim {
    int R = 0, nt = 0, precision = MD_MIXED, cutoff = MD_SHIFTED_POTENTIAL;
    int ntot = 0, ctot = 0, ntiles = 0;
    std::vector<int> n, off;
    std::vector<double> L;
    std::vector<md_pair> params;
    std::vector<PairTab> tab;
    std::vector<SysDesc> sys;
    double mass[kMaxTypes], inv_mass[kMaxTypes];
    double skin = 0.3, rc_max = 0.0;
    bool coul = false;                 // shifted-force Coulomb term on (Sec. 9)
    double charge[kMaxTypes] = {};
    double rcc = 0.0;                  // Coulomb cutoff rc_C
    int integrator = MD_NVE_LEAPFROG;
    double dt = 0.005, T0 = 1.0, tau = 0.2;
    int tp = 1, block = 128, reach = 2, tpb = 8;
    int path = 0;            // 0 auto, 1 grid, 2 replica-resident
    int list_method = 0;     // 0 sorted cells, 1 O(N^2) scan, 2 no list
    int rebuild_batch = 1;   // K: rebuild slots every K steps (1: rebuild exactly when needed)
    int resort = 0;          // O(N^2) method: sort by cell every resort-th rebuild pass (0 never)
    bool rep_ok = false;     // replica-resident kernel usable with the current shape
    size_t rep_smem = 0;
    int rep_threads = 512, rep_ctas = 1;
    bool sort_small = false;
    size_t sort_smem = 0;
    bool staged_ok = false;   // path 3: grid step kernel with replica positions in shared memory
    size_t staged_smem = 0;
    int rep_nmax = 0, rep_cmax = 0;
    int *rep_order = nullptr;
    int nsm = 148;
    int graph_block = 100;
    int nmax = 0;
    int log_cap = 0;
    std::vector<char> loaded;
    size_t r4 = 16;   // bytes of one Real4
    Buffers b;
    cudaStream_t stream = nullptr, cap_stream = nullptr, body_stream = nullptr;
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int prio_hi = 0, prio_lo = 0;   // launch priorities of the split step's two branches
    bool own_stream = false;
    Ctrl *h_ctrl = nullptr;  // pinned
    long long h_step = 0;    // completed steps (host view)
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int graph_len[2] = {0, 0};
    long long graph_builds = 0;   // graphs captured and instantiated (md_stats)
    int sticky = MD_OK;
    long long overflows = 0;
    int device = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    // state transfers (md_set_state / md_get_state) go through one packed staging area: two
    // pinned host halves (one is packed while the other's copy runs) and one device buffer,
    // each for stage_cap particles
    unsigned char *stage_h[2] = {nullptr, nullptr};
    void *stage_d = nullptr;
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int stage_k = 0, stage_cap = 0;
};

namespace {

#define CK(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            std::fprintf(stderr, "md: CUDA error %s at %s:%d: %s\n", cudaGetErrorName(e_),      \
                         __FILE__, __LINE__, cudaGetErrorString(e_));                           \
            return fail(s, MD_ECUDA);                                                           \
        }                                                                                       \
    } while (0)

int fail(md_sim *s, int code) {
    if (s && (code == MD_ECUDA || code == MD_EUNSTABLE || code == MD_ETIMEOUT) &&
        s->sticky == MD_OK)
        s->sticky = code;
    return code;
}

template <typename T> int dalloc(md_sim *s, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return MD_ENOMEM;
    }
    return MD_OK;
}
int dallocb(md_sim *s, void **p, size_t bytes) {
    (void)s;
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return MD_ENOMEM;
    }
    return MD_OK;
}
template <typename T> void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void destroy_graphs(md_sim *s) {
    for (int k = 0; k < 2; ++k) {
        if (s->exec[k]) cudaGraphExecDestroy(s->exec[k]);
        if (s->graph[k]) cudaGraphDestroy(s->graph[k]);
        s->exec[k] = nullptr;
        s->graph[k] = nullptr;
        s->graph_len[k] = 0;
    }
}

bool is_pow2_tp(int tp) {
    return tp == 1 || tp == 2 || tp == 4 || tp == 8 || tp == 16 || tp == 32;
}
bool valid_lanes(int lanes) { return is_pow2_tp(lanes) || lanes == MD_BUILD_CELL; }

// Cells per box edge for a stencil reach: edge >= (rc_max + skin) / reach with a 1e-4 margin
// so that FP32 rounding of the cell coordinate never breaks the stencil guarantee.
int cells_per_edge(double L, double rc_max, double skin, int reach) {
    const double min_edge = (rc_max + skin) / reach * (1.0 + 1e-4);
    int nc = (int)std::floor(L / min_edge);
    return nc < 1 ? 1 : nc;
}

// (Re)compute cells and tiles for the current tuning; (re)allocate what depends on them.
int configure_layout(md_sim *s, bool realloc_cells) {
    int ctot = 0, ntiles = 0;
    const int P = s->block / s->tp;
    for (int r = 0; r < s->R; ++r) {
        SysDesc &d = s->sys[r];
        d.nc = cells_per_edge(s->L[r], s->rc_max, s->skin, s->reach);
        d.reach = s->reach;
        d.span = std::min(2 * s->reach + 1, d.nc);
        d.cell_scale = (float)(d.nc / s->L[r]);
        d.cell_off = ctot;
        ctot += d.nc * d.nc * d.nc;
        d.tile_off = ntiles;
        d.ntiles = (d.n + P - 1) / P;
        ntiles += d.ntiles;
    }
    if (realloc_cells || ctot != s->ctot) {
        dfree(s->b.cell_start);
        dfree(s->b.count);
        dfree(s->b.crep);
        s->ctot = ctot;
        if (dalloc(s, &s->b.cell_start, (size_t)ctot + 1) || dalloc(s, &s->b.count, ctot) ||
            dalloc(s, &s->b.crep, ctot))
            return MD_ENOMEM;
        std::vector<int> cs((size_t)ctot + 1), cr(ctot);
        for (int r = 0; r < s->R; ++r) {
            const SysDesc &d = s->sys[r];
            const int C = d.nc * d.nc * d.nc;
            for (int c = 0; c < C; ++c) {
                cs[d.cell_off + c] = d.off;   // all cells empty until the first build
                cr[d.cell_off + c] = r;
            }
        }
        cs[ctot] = s->ntot;
        if (cudaMemcpy(s->b.cell_start, cs.data(), cs.size() * sizeof(int),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->b.crep, cr.data(), cr.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemset(s->b.count, 0, sizeof(int) * (size_t)std::max(ctot, 1)) != cudaSuccess)
            return fail(s, MD_ECUDA);
    }
    if (ntiles != s->ntiles || s->b.tile_rep == nullptr) {
        dfree(s->b.tile_rep);
        dfree(s->b.partial);
        s->ntiles = ntiles;
        if (dalloc(s, &s->b.tile_rep, ntiles) ||
            dalloc(s, &s->b.partial, (size_t)ntiles * MD_NRED))
            return MD_ENOMEM;
    }
    // replica-resident kernel: shared memory for the largest replica
    s->rep_nmax = 0;
    s->rep_cmax = 0;
    for (int r = 0; r < s->R; ++r) {
        s->rep_nmax = std::max(s->rep_nmax, s->sys[r].n);
        s->rep_cmax = std::max(s->rep_cmax, s->sys[r].nc * s->sys[r].nc * s->sys[r].nc);
    }
    // fused one-CTA-per-replica sort when the largest replica fits in shared memory
    {
        int optin2 = 0;
        cudaDeviceGetAttribute(&optin2, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
        s->sort_smem = sort_small_smem_bytes(s->rep_nmax, s->rep_cmax);
        s->sort_small = s->rep_nmax <= 16384 && s->sort_smem + 1024 <= (size_t)optin2 &&
                        (s->precision == MD_FP64 ? prepare_sort_small<double>(s->sort_smem)
                                                 : prepare_sort_small<float>(s->sort_smem)) ==
                            cudaSuccess;
        cudaGetLastError();
    }
    {
        int optin3 = 0;
        cudaDeviceGetAttribute(&optin3, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
        s->staged_smem = (size_t)s->rep_nmax * 16;
        s->staged_ok = s->precision == MD_MIXED && s->cutoff == MD_SHIFTED_POTENTIAL && !s->coul &&
                       s->staged_smem + 8192 <= (size_t)optin3 &&
                       s->staged_smem <= 100 * 1024 &&
                       prepare_step_staged(s->tp, s->nt == 1, s->staged_smem) == cudaSuccess;
        cudaGetLastError();
    }
    s->rep_threads = std::max(s->block, 512);
    s->rep_smem = rep_smem_bytes(s->rep_nmax, s->rep_cmax, s->block, s->tp, s->rep_threads);
    int optin = 0, per_sm = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device);
    // resident CTAs per SM: shared memory (plus ~8 KB static) and 64 registers x threads
    s->rep_ctas = std::max(1, std::min(per_sm / (int)(s->rep_smem + 8192),
                                       65536 / (64 * s->rep_threads)));
    s->rep_ok = s->precision == MD_MIXED && s->cutoff == MD_SHIFTED_POTENTIAL && !s->coul &&
                s->rep_smem + 8192 <= (size_t)optin &&
                (s->tpb == 8 || s->tpb == 32) &&
                prepare_rep(s->tp, s->tpb, s->nt == 1, s->rep_smem) == cudaSuccess;
    cudaGetLastError();
    std::vector<int> tr(ntiles);
    for (int r = 0; r < s->R; ++r)
        for (int t = 0; t < s->sys[r].ntiles; ++t) tr[s->sys[r].tile_off + t] = r;
    if (cudaMemcpy(s->b.tile_rep, tr.data(), tr.size() * sizeof(int), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(s->b.sys, s->sys.data(), s->sys.size() * sizeof(SysDesc),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(s, MD_ECUDA);
    return MD_OK;
}

// Lists are padded to a multiple of 4 x tp entries (the force loop's groups of four per lane), and
// the capacity n_max is kept a multiple of that.
int list_pad(const md_sim *s) { return 4 * s->tp; }
int round_nmax(const md_sim *s, int n) {
    const int p = list_pad(s);
    return (n + p - 1) / p * p;
}

// sliced layout: ceil(ntot / 32) slices of nmax x 32 entries
size_t nbl_entries(const md_sim *s) { return (((size_t)s->ntot + 31) / 32) * 32 * (size_t)s->nmax; }

// Initial list capacity (Sec. 4): 1.35 x the ideal-gas count within rc_max + skin, plus 24.
int estimate_nmax(const md_sim *s) {
    double est = 0.0;
    int n_big = 0;
    for (int r = 0; r < s->R; ++r) {
        const double rho = s->n[r] / (s->L[r] * s->L[r] * s->L[r]);
        const double rl = s->rc_max + s->skin;
        est = std::max(est, rho * 4.18879020478639 * rl * rl * rl);
        n_big = std::max(n_big, s->n[r]);
    }
    const int nmax = std::min((int)std::ceil(est * 1.35) + 24, n_big - 1);
    return std::max(nmax, 1);
}

int alloc_nbl(md_sim *s) {
    dfree(s->b.nbl);
    return dalloc(s, &s->b.nbl, nbl_entries(s));
}

// Force a full rebuild of every replica before the next step (device flags, stream-ordered).
int *need_now(md_sim *s) { return s->b.need + (size_t)(s->h_step & 1) * s->R; }

int request_rebuild_all(md_sim *s) {
    std::vector<int> ones(s->R, 1);
    if (cudaMemcpyAsync(need_now(s), ones.data(), sizeof(int) * s->R, cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess)
        return fail(s, MD_ECUDA);
    const int one = 1;
    if (cudaMemcpyAsync(&s->b.ctrl->need_any, &one, sizeof(int), cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return fail(s, MD_ECUDA);
    return MD_OK;
}

template <typename R> StepArgs<R> step_args(md_sim *s, int parity, int force_only) {
    typedef typename V4T<R>::t V4;
    StepArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.pos_in = (const V4 *)s->b.pos[parity];
    a.pos_out = (V4 *)s->b.pos[parity ^ 1];
    typedef typename MT<R>::t M;
    a.xm = (M *)s->b.xd; a.ym = (M *)s->b.yd; a.zm = (M *)s->b.zd;
    a.vel = (typename F4T<R>::t *)s->b.vel;
    a.img = s->b.img;
    a.pos_build = (const V4 *)s->b.pos_build;
    a.nbl = s->b.nbl;
    a.nnb = s->b.nnb;
    a.nmax = s->nmax;
    a.tile_rep = s->b.tile_rep;
    a.sys = s->b.sys;
    a.tab = s->b.tab;
    a.ntypes = s->nt;
    a.nrep = s->R;
    for (int t = 0; t < kMaxTypes; ++t) {
        a.inv_mass[t] = s->inv_mass[t];
        a.mass[t] = s->mass[t];
    }
    a.th = s->b.th;
    a.ctrl = s->b.ctrl;
    a.moved = s->b.moved;
    a.need_in = s->b.need + (size_t)parity * s->R;
    a.need_out = s->b.need + (size_t)(parity ^ 1) * s->R;
    a.id_g = s->b.id;
    a.rep_order = s->rep_order;
    a.rep_nmax = s->rep_nmax;
    a.rep_cmax = s->rep_cmax;
    a.tile_threads = s->block;
    a.rep_ticket = s->b.ticket;
    a.partial = s->b.partial;
    a.log = s->b.log;
    a.log_cap = s->log_cap;
    a.integrator = s->integrator;
    a.dt = s->dt;
    a.T0 = s->T0;
    a.inv_tau2 = (s->integrator == MD_NVT_NOSE_HOOVER) ? 1.0 / (s->tau * s->tau) : 0.0;
    a.half_skin2 = (R)(0.25 * s->skin * s->skin);
    a.half_skin = (float)(0.5 * s->skin);
    a.rebuild_batch = s->rebuild_batch;
    a.disp = s->b.disp;
    a.force_only = force_only;
    a.f_out = (typename F4T<R>::t *)s->b.f_out;
    a.w_out = (R *)s->b.w_out;
    a.has_next = 0;
    a.need_filter = -1;
    a.cutoff = s->cutoff;
    a.coulomb = s->coul ? 1 : 0;
    a.nolist = s->list_method == 2 ? 1 : 0;
    return a;
}

template <typename R> RebuildArgs<R> rebuild_args(md_sim *s, int parity, const void *key) {
    typedef typename V4T<R>::t V4;
    RebuildArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.pos = (V4 *)s->b.pos[parity];
    a.key = key ? (const V4 *)key : (const V4 *)s->b.pos[parity];
    a.key_is_pos = key ? 0 : 1;
    typedef typename MT<R>::t M;
    a.xm = (M *)s->b.xd; a.ym = (M *)s->b.yd; a.zm = (M *)s->b.zd;
    a.vel = (typename F4T<R>::t *)s->b.vel;
    a.img = s->b.img;
    a.id = s->b.id;
    a.pos_build = (V4 *)s->b.pos_build;
    a.tpos = (V4 *)s->b.tpos;
    a.tkey = (V4 *)s->b.tkey;
    a.txm = (M *)s->b.txd; a.tym = (M *)s->b.tyd; a.tzm = (M *)s->b.tzd;
    a.tvel = (typename F4T<R>::t *)s->b.tvel;
    a.timg = s->b.timg;
    a.tid = s->b.tid;
    a.cell_of = s->b.cell_of;
    a.rank = s->b.rank;
    a.perm = s->b.perm;
    a.cell_start = s->b.cell_start;
    a.count = s->b.count;
    a.prep = s->b.prep;
    a.crep = s->b.crep;
    a.nbl = s->b.nbl;
    a.nnb = s->b.nnb;
    a.nmax = s->nmax;
    a.plan = s->b.plan;
    a.plan_rep = s->b.plan_arr;
    a.plan_pp = s->b.plan_arr + s->R;
    a.plan_pc = s->b.plan_arr + 2 * s->R + 1;
    a.nsm = s->nsm;
    a.tpb = s->tpb;
    a.pad = list_pad(s);
    a.sort_small = s->sort_small ? 1 : 0;
    a.list_method = s->list_method == 1 ? 1 : 0;
    a.resort = s->list_method == 1 ? s->resort : 0;
    a.sort_nmax = s->rep_nmax;
    a.sort_cmax = s->rep_cmax;
    a.sort_smem = s->sort_smem;
    a.sys = s->b.sys;
    a.tab = s->b.tab;
    a.ntypes = s->nt;
    a.nrep = s->R;
    a.ntot = s->ntot;
    a.ctot = s->ctot;
    a.need_in = s->b.need + (size_t)parity * s->R;
    a.ctrl = s->b.ctrl;
    a.th = s->b.th;
    return a;
}

cudaError_t do_rebuild(md_sim *s, int parity, cudaStream_t st, const void *key = nullptr,
                       int prio = 0) {
    if (s->list_method == 2) return cudaSuccess;   // no list: nothing to rebuild
    if (s->precision == MD_FP64) {
        RebuildArgs<double> a = rebuild_args<double>(s, parity, key);
        a.launch_prio = prio;
        return launch_rebuild<double>(a, st);
    }
    RebuildArgs<float> a = rebuild_args<float>(s, parity, key);
    a.launch_prio = prio;
    return launch_rebuild<float>(a, st);
}

bool use_rep(const md_sim *s) {
    if (!s->rep_ok || s->list_method != 0) return false;
    if (s->path == 2) return true;
    return false;   // auto: the grid path (the replica-resident kernel is chosen by tuning)
}

// Graph steps are split (unflagged replicas step while flagged ones rebuild) for batches.
// With rebuild slots (K > 1) most steps rebuild nothing and the IF-node graph skips the rebuild.
bool split_steps(const md_sim *s) {
    return s->R >= 8 && !use_rep(s) && s->list_method != 2 && s->rebuild_batch <= 1;
}

cudaError_t do_step(md_sim *s, int parity, cudaStream_t st, int force_only,
                    cudaGraphConditionalHandle next = 0, int has_next = 0, int filter = -1) {
    if (!force_only && use_rep(s)) {
        StepArgs<float> a = step_args<float>(s, parity, 0);
        a.has_next = 0;
        RebuildArgs<float> b = rebuild_args<float>(s, parity, nullptr);
        const int grid = std::min(s->R, s->rep_ctas * s->nsm);
        return launch_rep(a, b, s->tp, s->rep_threads, grid, s->rep_smem, st);
    }
    if (s->precision == MD_FP64) {
        StepArgs<double> a = step_args<double>(s, parity, force_only);
        a.next_handle = next;
        a.has_next = has_next;
        a.need_filter = filter;
        a.launch_prio = filter == 0 ? s->prio_lo : (filter == 1 ? s->prio_hi : 0);
        a.lean = s->path == 4 ? 1 : 0;
        return launch_step<double>(a, s->tp, s->block, s->ntiles, st);
    }
    StepArgs<float> a = step_args<float>(s, parity, force_only);
    a.next_handle = next;
    a.has_next = has_next;
    a.need_filter = filter;
    a.launch_prio = filter == 0 ? s->prio_lo : (filter == 1 ? s->prio_hi : 0);
    a.lean = s->path == 4 ? 1 : 0;
    if (s->path == 3 && s->staged_ok && s->list_method != 2)
        return launch_step_staged(a, s->tp, s->block, s->ntiles, s->staged_smem, st);
    return launch_step<float>(a, s->tp, s->block, s->ntiles, st);
}

// Capture graph_block steps starting at step parity p: [IF need_any {rebuild}] -> step, repeated.
int build_graph(md_sim *s, int p) {
    const int B = s->graph_block;
    cudaGraph_t g = nullptr;
    if (use_rep(s) || s->list_method == 2) {   // one launch per step: rebuild inside / none
        if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(s, MD_ECUDA);
        bool okr = true;
        for (int k = 0; okr && k < B; ++k) okr = do_step(s, (p + k) & 1, s->cap_stream, 0) == cudaSuccess;
        cudaGraph_t outg = nullptr;
        cudaError_t ee = cudaStreamEndCapture(s->cap_stream, &outg);
        if (!okr || ee != cudaSuccess || !outg) {
            if (outg) cudaGraphDestroy(outg);
            cudaGetLastError();
            return fail(s, MD_ECUDA);
        }
        cudaGraphExec_t exr = nullptr;
        if (cudaGraphInstantiate(&exr, outg, 0) != cudaSuccess) {
            cudaGraphDestroy(outg);
            return fail(s, MD_ECUDA);
        }
        s->graph[p] = outg;
        s->exec[p] = exr;
        s->graph_len[p] = B;
        s->graph_builds++;
        return MD_OK;
    }
    if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(s, MD_ECUDA);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    std::vector<cudaGraphConditionalHandle> h(B, 0);
    const bool split = split_steps(s);   // split steps use no IF nodes (see below)
    bool ok = cudaStreamGetCaptureInfo(s->cap_stream, &st, nullptr, &g, &deps, nullptr, &ndeps) ==
              cudaSuccess;
    for (int k = 0; ok && !split && k < B; ++k)
        ok = cudaGraphConditionalHandleCreate(&h[k], g, 0, cudaGraphCondAssignDefault) ==
             cudaSuccess;
    ok = ok && (split || launch_arm(s->b.ctrl, h[0], s->cap_stream) == cudaSuccess);
    for (int k = 0; ok && k < B; ++k) {
        const int q = (p + k) & 1;
        if (split) {   // branch: the replicas that keep their list step now
            ok = cudaEventRecord(s->ev_fork, s->cap_stream) == cudaSuccess &&
                 cudaStreamWaitEvent(s->side_stream, s->ev_fork, 0) == cudaSuccess &&
                 do_step(s, q, s->side_stream, 0, 0, 0, 0) == cudaSuccess &&
                 cudaEventRecord(s->ev_join, s->side_stream) == cudaSuccess;
            if (!ok) break;
        }
        if (split) {
            // with many replicas some replica rebuilds almost every step: the rebuild kernels are
            // plain nodes of the critical branch (they exit at once when nothing is flagged), so
            // the branch can run beside the step of the other replicas
            ok = do_rebuild(s, q, s->cap_stream, nullptr, s->prio_hi) == cudaSuccess &&
                 do_step(s, q, s->cap_stream, 0, 0, 0, 1) == cudaSuccess &&
                 cudaStreamWaitEvent(s->cap_stream, s->ev_join, 0) == cudaSuccess;
            continue;
        }
        ok = cudaStreamGetCaptureInfo(s->cap_stream, &st, nullptr, &g, &deps, nullptr, &ndeps) ==
             cudaSuccess;
        if (!ok) break;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h[k];
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        ok = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp) == cudaSuccess;
        if (!ok) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamUpdateCaptureDependencies(s->cap_stream, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies) == cudaSuccess;
        ok = ok && cudaStreamBeginCaptureToGraph(s->body_stream, body, nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (!ok) break;
        cudaError_t e1 = do_rebuild(s, q, s->body_stream);
        cudaGraph_t body_out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s->body_stream, &body_out);
        ok = e1 == cudaSuccess && e2 == cudaSuccess;
        ok = ok && do_step(s, q, s->cap_stream, 0, k + 1 < B ? h[k + 1] : 0, k + 1 < B,
                           split ? 1 : -1) == cudaSuccess;
        if (split) ok = ok && cudaStreamWaitEvent(s->cap_stream, s->ev_join, 0) == cudaSuccess;
    }
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &out);
    if (!ok || e != cudaSuccess || out == nullptr) {
        std::fprintf(stderr, "md: graph capture failed: %s\n",
                     cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
        if (out) cudaGraphDestroy(out);
        cudaGetLastError();
        return fail(s, MD_ECUDA);
    }
    cudaGraphExec_t ex = nullptr;
    // the launch priorities captured into the nodes (rebuild branch above the step of the
    // replicas that keep their list) apply only with this flag
    if (cudaGraphInstantiate(&ex, out, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGraphDestroy(out);
        return fail(s, MD_ECUDA);
    }
    s->graph[p] = out;
    s->exec[p] = ex;
    s->graph_len[p] = B;
    s->graph_builds++;
    return MD_OK;
}

int read_ctrl(md_sim *s) {
    if (cudaMemcpyAsync(s->h_ctrl, s->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return fail(s, MD_ECUDA);
    return MD_OK;
}

// After an overflow: double n_max (at least to the largest count seen), rebuild everything.
int recover_overflow(md_sim *s) {
    const int seen = s->h_ctrl->max_count;
    int nm = std::max(2 * s->nmax, seen + seen / 4 + 8);
    s->nmax = round_nmax(s, nm);
    destroy_graphs(s);
    if (alloc_nbl(s)) return MD_ENOMEM;
    Ctrl c = *s->h_ctrl;
    c.overflow = 0;
    c.halt = 0;
    c.max_count = 0;
    c.global_ticket = 0;
    if (cudaMemcpyAsync(s->b.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(s->b.ticket, 0, sizeof(unsigned) * s->R, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->b.disp, 0, sizeof(unsigned) * 2 * s->R, s->stream) != cudaSuccess)
        return fail(s, MD_ECUDA);
    s->overflows++;
    return request_rebuild_all(s);
}

int grow_after_rep_overflow(md_sim *s) {
    const int seen = s->h_ctrl->max_count;
    s->nmax = round_nmax(s, std::max(2 * s->nmax, seen + seen / 4 + 8));
    destroy_graphs(s);
    if (alloc_nbl(s)) return MD_ENOMEM;
    Ctrl c = *s->h_ctrl;
    c.rep_overflow = 0;
    c.max_count = 0;
    if (cudaMemcpyAsync(s->b.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
        return fail(s, MD_ECUDA);
    s->overflows++;
    return request_rebuild_all(s);
}

// Run a plain rebuild pass now (if flagged) and recover from overflow until the list fits.
int ensure_list(md_sim *s) {
    for (int tries = 0; tries < 16; ++tries) {
        if (do_rebuild(s, (int)(s->h_step & 1), s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
        int rc = read_ctrl(s);
        if (rc) return rc;
        if (s->h_ctrl->unstable) return fail(s, MD_EUNSTABLE);
        if (!s->h_ctrl->overflow) {
            // the lists are fresh for the current positions: the next step need not rebuild
            if (cudaMemsetAsync(need_now(s), 0, sizeof(int) * s->R, s->stream) != cudaSuccess)
                return fail(s, MD_ECUDA);
            return MD_OK;
        }
        if ((rc = recover_overflow(s))) return rc;
    }
    return fail(s, MD_ECUDA);
}

int check_replica(md_sim *s, int r) {
    if (!s) return MD_EINVAL;
    if (r < 0 || r >= s->R) return MD_EINVAL;
    return MD_OK;
}

template <typename R> void pack_v4(unsigned char *dst, size_t k, double x, double y, double z,
                                   double w) {
    R v[4] = {(R)x, (R)y, (R)z, (R)w};
    std::memcpy(dst + k * sizeof(v), v, sizeof(v));
}
template <typename R> void pack_v4(std::vector<unsigned char> &dst, size_t k, double x, double y,
                                   double z, double w) {
    pack_v4<R>(dst.data(), k, x, y, z, w);
}

// Mixed precision keeps positions in fixed point (the kernels' layout notes give the units):
// master = round(x / L 2^64) of a coordinate folded into [0, L) (a value that rounds to 2^64,
// i.e. to L, is 0), mirror = the master rounded to 32 bits.  Every step is an IEEE double
// operation or an integer one, so both host architectures give the same bits.
// (Scaling by 2^64 or 2^-64 is exact, and a double of 2^52 or more is already an integer, so the
// rounding call is needed only below 2^52.)
uint64_t to_fixed64(double x, double L) {
    double q = (x / L) * 18446744073709551616.0;   // x / L * 2^64
    if (q < 4503599627370496.0) q = std::nearbyint(q);   // 2^52
    if (!(q < 18446744073709551616.0)) return 0;   // 2^64: the period itself
    return q <= 0.0 ? 0 : (uint64_t)q;
}
// back to a coordinate in [0, L)
double from_fixed64(uint64_t q, double L) {
    const double x = ((double)q * 5.421010862427522170037264e-20) * L;   // q 2^-64 L
    return x < L ? x : std::nextafter(L, 0.0);
}
int32_t mirror32(uint64_t q) { return (int32_t)(uint32_t)((q + 0x80000000ull) >> 32); }

// FP64 mirror: x, y, z and the type's bits in .w
void pack_pos(unsigned char *dst, size_t k, double x, double y, double z, int type) {
    double v[4] = {x, y, z, 0.0};
    long long t = type;
    std::memcpy(&v[3], &t, sizeof(double));
    std::memcpy(dst + k * 32, v, 32);
}
void pack_pos(std::vector<unsigned char> &dst, size_t k, double x, double y, double z, int type) {
    pack_pos(dst.data(), k, x, y, z, type);
}
// fixed-point mirror of a mixed-precision master position
void pack_mirror(unsigned char *dst, size_t k, uint64_t qx, uint64_t qy, uint64_t qz, int type) {
    const int32_t v[4] = {mirror32(qx), mirror32(qy), mirror32(qz), type};
    std::memcpy(dst + k * 16, v, 16);
}
void pack_mirror(std::vector<unsigned char> &dst, size_t k, uint64_t qx, uint64_t qy, uint64_t qz,
                 int type) {
    pack_mirror(dst.data(), k, qx, qy, qz, type);
}

void unpack_v4(const md_sim *s, const unsigned char *src, size_t k, double *out3) {
    if (s->precision == MD_FP64) {
        double v[4];
        std::memcpy(v, src + k * 32, 32);
        out3[0] = v[0]; out3[1] = v[1]; out3[2] = v[2];
    } else {
        float v[4];
        std::memcpy(v, src + k * 16, 16);
        out3[0] = v[0]; out3[1] = v[1]; out3[2] = v[2];
    }
}
void unpack_v4(const md_sim *s, const std::vector<unsigned char> &src, size_t k, double *out3) {
    unpack_v4(s, src.data(), k, out3);
}

// ---- packed state transfers
// md_set_state copies the caller's arrays for a chunk of user indices k0 .. k0 + n - 1 into the
// staging area as they are (positions, velocities, types, images: 64 bytes a particle) and one
// kernel wraps, quantises and packs them into the replica's slots -- the same IEEE steps as the
// host helpers above (explicit roundings, no contraction), so the device holds the same bits.
// md_get_state packs on the device: for a replica that fits one chunk, positions (dequantised),
// velocities and images in user order (60 bytes a particle), so the host only copies them out;
// a larger replica comes out in slot order, chunk by chunk, with its ids (velocity records,
// image counters, the x, y, z masters, ids) and is unpacked on the host.
constexpr int kStageChunk = 1 << 16;
size_t stage_bytes_per_particle(size_t R4) { return 2 * R4 + 48; }

struct StateXfer {
    void *stage;
    int n, k0, o, r4w;
    int mixed, has_image;
    double L;
    int4 *pos, *pos_build, *vel;
    unsigned long long *x, *y, *z;
    int4 *img;
    int *id, *nnb;
};

// wrap of one coordinate into [0, L) with its image shift (the host's steps in md_set_state)
__device__ double wrap_coordinate(double v, double L, double &f) {
    f = 0.0;
    if (!(v > 0.0 && v < L)) {
        f = floor(__ddiv_rn(v, L));
        v = __dsub_rn(v, __dmul_rn(f, L));
        if (v >= L) { v = __dsub_rn(v, L); f = __dadd_rn(f, 1.0); }
        if (v < 0.0) { v = __dadd_rn(v, L); f = __dsub_rn(f, 1.0); }
        if (v >= L) v = 0.0;
    }
    return v;
}
// to_fixed64 / from_fixed64 / mirror32 of the host, on the device
__device__ unsigned long long fixed64_of(double x, double L) {
    double q = __dmul_rn(__ddiv_rn(x, L), 18446744073709551616.0);
    if (q < 4503599627370496.0) q = rint(q);
    if (!(q < 18446744073709551616.0)) return 0ull;
    return q <= 0.0 ? 0ull : __double2ull_rz(q);
}
__device__ double coordinate_of(unsigned long long q, double L) {
    const double x = __dmul_rn(__dmul_rn(__ull2double_rn(q), 5.421010862427522170037264e-20), L);
    return x < L ? x : nextafter(L, 0.0);
}
__device__ int mirror_of(unsigned long long q) {
    return (int)(unsigned)((q + 0x80000000ull) >> 32);
}

__global__ void k_load_state(const StateXfer t) {
    const double *pos = (const double *)t.stage;
    const double *vel = pos + 3 * (size_t)t.n;
    const int *type = (const int *)(vel + 3 * (size_t)t.n);
    const int *image = type + t.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < t.n; k += gridDim.x * blockDim.x) {
        const size_t d = (size_t)t.o + t.k0 + k;
        double w[3], f[3];
        for (int c = 0; c < 3; ++c) w[c] = wrap_coordinate(pos[3 * (size_t)k + c], t.L, f[c]);
        int im[3];
        for (int c = 0; c < 3; ++c)
            im[c] = (int)f[c] + (t.has_image ? image[3 * (size_t)k + c] : 0);
        t.img[d] = make_int4(im[0], im[1], im[2], 0);
        const int ty = type[k];
        const double *v = vel + 3 * (size_t)k;
        if (t.mixed) {
            const unsigned long long q[3] = {fixed64_of(w[0], t.L), fixed64_of(w[1], t.L),
                                             fixed64_of(w[2], t.L)};
            const int4 m = make_int4(mirror_of(q[0]), mirror_of(q[1]), mirror_of(q[2]), ty);
            t.pos[d] = m;
            t.pos_build[d] = m;
            t.x[d] = q[0];
            t.y[d] = q[1];
            t.z[d] = q[2];
            const float4 vf = make_float4(__double2float_rn(v[0]), __double2float_rn(v[1]),
                                          __double2float_rn(v[2]), 0.f);
            t.vel[d] = *(const int4 *)&vf;
        } else {
            const double4_32a m = make_double4_32a(w[0], w[1], w[2],
                                                   __longlong_as_double((long long)ty));
            const double4_32a vd = make_double4_32a(v[0], v[1], v[2], 0.0);
            for (int q = 0; q < 2; ++q) {
                t.pos[2 * d + q] = ((const int4 *)&m)[q];
                t.pos_build[2 * d + q] = ((const int4 *)&m)[q];
                t.vel[2 * d + q] = ((const int4 *)&vd)[q];
            }
            t.x[d] = (unsigned long long)__double_as_longlong(w[0]);
            t.y[d] = (unsigned long long)__double_as_longlong(w[1]);
            t.z[d] = (unsigned long long)__double_as_longlong(w[2]);
        }
        t.id[d] = t.k0 + k;
        t.nnb[d] = 0;
    }
}

// the replica's carry and flags after its particles are loaded: thermostat state, a rebuild
// request for the next step, no displacement since the (pending) build
__global__ void k_load_replica(const Thermo th, Thermo *th_dst, int *need, int *moved,
                               unsigned *disp, Ctrl *ctrl) {
    *th_dst = th;
    *need = 1;
    *moved = 0;
    disp[0] = 0u;
    disp[1] = 0u;
    ctrl->need_any = 1;
}

// a whole replica (t.k0 = 0, t.n = its size) in user order: positions in [0, L), velocities,
// images
__global__ void k_save_user(const StateXfer t) {
    double *pos = (double *)t.stage;
    double *vel = pos + 3 * (size_t)t.n;
    int *image = (int *)(vel + 3 * (size_t)t.n);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < t.n; k += gridDim.x * blockDim.x) {
        const size_t d = (size_t)t.o + k;
        const int u = t.id[d];
        if (u < 0 || u >= t.n) continue;
        double p3[3], v3[3];
        if (t.mixed) {
            p3[0] = coordinate_of(t.x[d], t.L);
            p3[1] = coordinate_of(t.y[d], t.L);
            p3[2] = coordinate_of(t.z[d], t.L);
            const int4 vi = t.vel[d];
            const float4 vf = *(const float4 *)&vi;
            v3[0] = vf.x; v3[1] = vf.y; v3[2] = vf.z;
        } else {
            p3[0] = __longlong_as_double((long long)t.x[d]);
            p3[1] = __longlong_as_double((long long)t.y[d]);
            p3[2] = __longlong_as_double((long long)t.z[d]);
            int4 raw[2] = {t.vel[2 * d], t.vel[2 * d + 1]};
            const double4_32a vd = *(const double4_32a *)raw;
            v3[0] = vd.x; v3[1] = vd.y; v3[2] = vd.z;
        }
        const int4 im = t.img[d];
        for (int c = 0; c < 3; ++c) {
            pos[3 * (size_t)u + c] = p3[c];
            vel[3 * (size_t)u + c] = v3[c];
        }
        image[3 * (size_t)u] = im.x;
        image[3 * (size_t)u + 1] = im.y;
        image[3 * (size_t)u + 2] = im.z;
    }
}

// a chunk of slots k0 .. k0 + n - 1 as stored, with the ids (replicas larger than one chunk)
__global__ void k_save_state(const StateXfer t) {
    int4 *vel = (int4 *)t.stage;
    int4 *img = vel + (size_t)t.n * t.r4w;
    unsigned long long *x = (unsigned long long *)(img + t.n);
    unsigned long long *y = x + t.n, *z = y + t.n;
    int *id = (int *)(z + t.n);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < t.n; k += gridDim.x * blockDim.x) {
        const size_t d = (size_t)t.o + t.k0 + k;
        for (int w = 0; w < t.r4w; ++w) vel[(size_t)k * t.r4w + w] = t.vel[d * t.r4w + w];
        img[k] = t.img[d];
        x[k] = t.x[d];
        y[k] = t.y[d];
        z[k] = t.z[d];
        id[k] = t.id[d];
    }
}

StateXfer state_xfer(md_sim *s, int r, int k0, int n) {
    StateXfer t;
    t.stage = s->stage_d;
    t.n = n;
    t.k0 = k0;
    t.o = s->off[r];
    t.r4w = (int)(s->r4 / 16);
    t.mixed = s->precision == MD_MIXED ? 1 : 0;
    t.has_image = 0;
    t.L = s->L[r];
    t.pos = (int4 *)s->b.pos[s->h_step & 1];
    t.pos_build = (int4 *)s->b.pos_build;
    t.vel = (int4 *)s->b.vel;
    t.x = (unsigned long long *)s->b.xd;
    t.y = (unsigned long long *)s->b.yd;
    t.z = (unsigned long long *)s->b.zd;
    t.img = s->b.img;
    t.id = s->b.id;
    t.nnb = s->b.nnb;
    return t;
}
int xfer_grid(int n) { return std::max(1, std::min((n + 255) / 256, 1024)); }

// Host copy of the device's next_factors (md_step.cuh): the Nose-Hoover friction of the next step
// and its leapfrog factors from the carry; the same IEEE operations in the same order (this file
// is compiled without FMA contraction), so a loaded state steps exactly like a stepped one.
void host_next_factors(const md_sim *s, Thermo &T, double K0) {
    double xi = 0.0;
    if (s->integrator == MD_NVT_NOSE_HOOVER) {
        const double inv_tau2 = 1.0 / (s->tau * s->tau);
        xi = T.xi_prev + (s->dt * (T.K_prev / K0 - 1.0)) * inv_tau2;
    }
    const double h = (0.5 * xi) * s->dt;
    T.xi_next = xi;
    T.A_next = 1.0 - h;
    T.B_next = 1.0 / (1.0 + h);
}

// Interaction range of type pair p: the LJ cutoff, or the Coulomb cutoff if larger.
double pair_range(const md_sim *s, int p) {
    return s->coul ? std::max(s->params[p].rc, s->rcc) : s->params[p].rc;
}

// List thresholds (rc_p + s)^2 of every type pair, then the table upload.
int upload_thresholds(md_sim *s) {
    for (int p = 0; p < s->nt * s->nt; ++p) {
        const double rc = pair_range(s, p), thr2 = (rc + s->skin) * (rc + s->skin);
        s->tab[p].thr2d = thr2;
        s->tab[p].thr2 = (float)thr2;
    }
    return cudaMemcpy(s->b.tab, s->tab.data(), sizeof(PairTab) * MD_MAX_PAIRS,
                      cudaMemcpyHostToDevice) == cudaSuccess ? 0 : 1;
}

}  // namespace

// ================================================================================================
// C ABI
// ================================================================================================
extern "C" {

const char *md_strerror(int status) {
    switch (status) {
    case MD_OK: return "ok";
    case MD_EINVAL: return "invalid argument or violated precondition";
    case MD_ENOMEM: return "out of memory";
    case MD_ECUDA: return "CUDA runtime error";
    case MD_EUNSTABLE: return "unstable: non-finite or runaway displacement";
    case MD_ETIMEOUT: return "bounded device wait timed out";
    case MD_ESTATE: return "call out of order (state not loaded)";
    default: return "unknown md status";
    }
}

void md_destroy(md_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    destroy_graphs(s);
    Buffers &b = s->b;
    void **ptrs[] = {&b.pos[0], &b.pos[1], (void **)&b.xd, (void **)&b.yd, (void **)&b.zd, &b.vel,
                     (void **)&b.img, (void **)&b.id, &b.pos_build, &b.tpos, &b.tkey,
                     (void **)&b.txd, (void **)&b.tyd, (void **)&b.tzd, &b.tvel, (void **)&b.timg,
                     (void **)&b.tid, (void **)&b.cell_of, (void **)&b.rank, (void **)&b.perm,
                     (void **)&b.cell_start, (void **)&b.count, (void **)&b.crep,
                     (void **)&b.prep, (void **)&b.nbl, (void **)&b.nnb, (void **)&b.plan,
                     (void **)&b.plan_arr, (void **)&b.sys,
                     (void **)&b.tab, (void **)&b.th, (void **)&b.ctrl, (void **)&b.moved,
                     (void **)&b.disp, (void **)&b.need, (void **)&b.ticket, (void **)&b.partial,
                     (void **)&b.tile_rep, (void **)&b.log, &b.f_out, &b.w_out};
    for (void **p : ptrs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    if (s->rep_order) cudaFree(s->rep_order);
    if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
    for (int h = 0; h < 2; ++h) {
        if (s->stage_h[h]) cudaFreeHost(s->stage_h[h]);
        if (s->stage_ev[h]) cudaEventDestroy(s->stage_ev[h]);
    }
    if (s->stage_d) cudaFree(s->stage_d);
    for (cudaEvent_t &e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->side_stream) cudaStreamDestroy(s->side_stream);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->body_stream) cudaStreamDestroy(s->body_stream);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int md_create(md_sim **out, int n_replicas, const int *n_particles, const double *box,
              int n_types, const md_pair *params, const double *mass, double skin,
              int cutoff_method, int precision) {
    if (!out) return MD_EINVAL;
    *out = nullptr;
    if (n_replicas < 1 || !n_particles || !box || !params || n_types < 1 ||
        n_types > kMaxTypes || !(skin > 0.0) || !std::isfinite(skin) ||
        (cutoff_method != MD_SHIFTED_POTENTIAL && cutoff_method != MD_SHIFTED_FORCE) ||
        (precision != MD_MIXED && precision != MD_FP64))
        return MD_EINVAL;
    double rc_max = 0.0;
    for (int a = 0; a < n_types; ++a)
        for (int c = 0; c < n_types; ++c) {
            const md_pair &p = params[a * n_types + c], &q = params[c * n_types + a];
            if (!(p.eps >= 0.0) || !(p.sigma > 0.0) || !(p.rc > 0.0) || !std::isfinite(p.eps) ||
                !std::isfinite(p.sigma) || !std::isfinite(p.rc))
                return MD_EINVAL;
            if (p.eps != q.eps || p.sigma != q.sigma || p.rc != q.rc) return MD_EINVAL;
            rc_max = std::max(rc_max, p.rc);
        }
    if (mass)
        for (int t = 0; t < n_types; ++t)
            if (!(mass[t] > 0.0) || !std::isfinite(mass[t])) return MD_EINVAL;
    long long ntot = 0;
    for (int r = 0; r < n_replicas; ++r) {
        if (n_particles[r] < 2) return MD_EINVAL;
        if (!(box[r] > 2.0 * (rc_max + skin)) || !std::isfinite(box[r])) return MD_EINVAL;
        ntot += n_particles[r];
    }
    if (ntot > (1LL << 30)) return MD_EINVAL;

    md_sim *s = new (std::nothrow) md_sim();
    if (!s) return MD_ENOMEM;
    cudaGetDevice(&s->device);
    if (cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        s->nsm < 1) {
        cudaGetLastError();
        s->nsm = 148;
    }
    s->R = n_replicas;
    s->nt = n_types;
    s->precision = precision;
    s->cutoff = cutoff_method;
    s->skin = skin;
    s->rc_max = rc_max;
    s->r4 = precision == MD_FP64 ? 32 : 16;
    s->ntot = (int)ntot;
    s->n.assign(n_particles, n_particles + n_replicas);
    s->L.assign(box, box + n_replicas);
    s->params.assign(params, params + n_types * n_types);
    s->loaded.assign(n_replicas, 0);
    for (int t = 0; t < kMaxTypes; ++t) {
        s->mass[t] = (mass && t < n_types) ? mass[t] : 1.0;
        s->inv_mass[t] = 1.0 / s->mass[t];
    }
    // pair table: u = c12 r^-12 - c6 r^-6 - u(rc), F = r^-2 (12 c12 r^-12 - 6 c6 r^-6) r_ij
    s->tab.resize(MD_MAX_PAIRS);
    std::memset(s->tab.data(), 0, sizeof(PairTab) * MD_MAX_PAIRS);
    for (int p = 0; p < n_types * n_types; ++p) {
        const md_pair &q = params[p];
        const double s6 = std::pow(q.sigma, 6.0), c12 = 4.0 * q.eps * s6 * s6, c6 = 4.0 * q.eps * s6;
        const double rc6 = std::pow(q.rc, 6.0);
        const double ush = c12 / (rc6 * rc6) - c6 / rc6;
        const double thr2 = (q.rc + skin) * (q.rc + skin);
        const double fc = (12.0 * c12 / (rc6 * rc6) - 6.0 * c6 / rc6) / q.rc;   // |F|(rc)
        PairTab &t = s->tab[p];
        t.fcd = fc; t.rcd = q.rc; t.fc = (float)fc; t.rc = (float)q.rc;
        t.rc2d = q.rc * q.rc; t.c12d = c12; t.c6d = c6; t.ushiftd = ush;
        t.a12d = 12.0 * c12; t.a6d = 6.0 * c6; t.thr2d = thr2;
        t.rc2 = (float)t.rc2d; t.c12 = (float)c12; t.c6 = (float)c6; t.ushift = (float)ush;
        t.a12 = (float)t.a12d; t.a6 = (float)t.a6d; t.thr2 = (float)thr2;
    }
    // replicas
    s->off.resize(n_replicas);
    s->sys.resize(n_replicas);
    int off = 0;
    double nmax_est = 0.0;
    int n_big = 0;
    for (int r = 0; r < n_replicas; ++r) {
        SysDesc &d = s->sys[r];
        std::memset(&d, 0, sizeof(d));
        d.off = off;
        d.n = n_particles[r];
        d.L = box[r];
        d.invL = 1.0 / box[r];
        d.Lf = (float)box[r];
        d.invLf = (float)(1.0 / box[r]);
        d.s64 = (float)(18446744073709551616.0 / box[r]);       // 2^64 / L
        const double unit = std::ldexp(box[r], -32);             // L / 2^32 (exact)
        d.ps = (float)unit;
        d.ps_lo = (float)(unit - (double)d.ps);
        d.ps2 = (float)(unit * unit);
        d.ps2_lo = (float)(unit * unit - (double)d.ps2);
        d.K0 = 0.5 * (3.0 * d.n - 3.0) * s->T0;
        s->off[r] = off;
        off += d.n;
        const double rho = d.n / (box[r] * box[r] * box[r]);
        const double rl = rc_max + skin;
        nmax_est = std::max(nmax_est, rho * 4.18879020478639 * rl * rl * rl);
        n_big = std::max(n_big, d.n);
    }
    // Sec. 4: fixed-capacity list; start with headroom and grow x2 on overflow
    s->tp = 1;
    s->nmax = round_nmax(s, estimate_nmax(s));
    s->block = 128;
    s->reach = 2;

    int rc = MD_OK;
    const size_t N = (size_t)ntot, R4 = s->r4;
    Buffers &b = s->b;
    rc |= dallocb(s, &b.pos[0], N * R4);
    rc |= dallocb(s, &b.pos[1], N * R4);
    rc |= dalloc(s, &b.xd, N); rc |= dalloc(s, &b.yd, N); rc |= dalloc(s, &b.zd, N);
    rc |= dallocb(s, &b.vel, N * R4);
    rc |= dalloc(s, &b.img, N);
    rc |= dalloc(s, &b.id, N);
    rc |= dallocb(s, &b.pos_build, N * R4);
    rc |= dallocb(s, &b.tpos, N * R4);
    rc |= dallocb(s, &b.tkey, N * R4);
    rc |= dalloc(s, &b.txd, N); rc |= dalloc(s, &b.tyd, N); rc |= dalloc(s, &b.tzd, N);
    rc |= dallocb(s, &b.tvel, N * R4);
    rc |= dalloc(s, &b.timg, N);
    rc |= dalloc(s, &b.tid, N);
    rc |= dalloc(s, &b.cell_of, N); rc |= dalloc(s, &b.rank, N); rc |= dalloc(s, &b.perm, N);
    rc |= dalloc(s, &b.prep, N);
    rc |= dalloc(s, &b.nnb, N);
    rc |= dalloc(s, &b.plan, 1);
    rc |= dalloc(s, &b.plan_arr, 3 * (size_t)n_replicas + 2);
    rc |= dalloc(s, &b.sys, n_replicas);
    rc |= dalloc(s, &b.tab, MD_MAX_PAIRS);
    rc |= dalloc(s, &b.th, n_replicas);
    rc |= dalloc(s, &b.ctrl, 1);
    rc |= dalloc(s, &b.moved, n_replicas);
    rc |= dalloc(s, &b.disp, 2 * (size_t)n_replicas);
    rc |= dalloc(s, &b.need, 2 * (size_t)n_replicas);   // by step parity: read / written
    rc |= dalloc(s, &b.ticket, n_replicas);
    rc |= dallocb(s, &b.f_out, N * R4);
    rc |= dallocb(s, &b.w_out, N * (R4 / 4));
    if (rc) { md_destroy(s); return MD_ENOMEM; }
    if (alloc_nbl(s)) { md_destroy(s); return MD_ENOMEM; }
    if (cudaMallocHost((void **)&s->h_ctrl, sizeof(Ctrl)) != cudaSuccess) {
        s->h_ctrl = nullptr;
        md_destroy(s);
        return MD_ENOMEM;
    }
    {
        int nbig = 1;
        for (int v : s->n) nbig = std::max(nbig, v);
        s->stage_cap = std::min(nbig, kStageChunk);
        const size_t sb = (size_t)s->stage_cap * stage_bytes_per_particle(R4);
        for (int h = 0; h < 2; ++h)
            if (cudaMallocHost((void **)&s->stage_h[h], sb) != cudaSuccess) {
                s->stage_h[h] = nullptr;
                md_destroy(s);
                return MD_ENOMEM;
            }
        if (dallocb(s, &s->stage_d, sb)) { md_destroy(s); return MD_ENOMEM; }
    }
    std::vector<int> prep(N);
    for (int r = 0; r < n_replicas; ++r)
        for (int k = 0; k < s->n[r]; ++k) prep[s->off[r] + k] = r;
    // replica queue of the replica-resident kernel: descending size (largest jobs first)
    std::vector<int> order(n_replicas);
    for (int r = 0; r < n_replicas; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return s->n[x] > s->n[y]; });
    if (dalloc(s, &s->rep_order, n_replicas)) { md_destroy(s); return MD_ENOMEM; }
    bool ok = cudaMemcpy(b.prep, prep.data(), N * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(s->rep_order, order.data(), n_replicas * sizeof(int),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.tab, s->tab.data(), sizeof(PairTab) * MD_MAX_PAIRS,
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(b.th, 0, sizeof(Thermo) * n_replicas) == cudaSuccess;
    ok = ok && cudaMemset(b.ctrl, 0, sizeof(Ctrl)) == cudaSuccess;
    ok = ok && cudaMemset(b.moved, 0, sizeof(int) * n_replicas) == cudaSuccess;
    ok = ok && cudaMemset(b.disp, 0, sizeof(unsigned) * 2 * n_replicas) == cudaSuccess;
    ok = ok && cudaMemset(b.need, 0, sizeof(int) * 2 * n_replicas) == cudaSuccess;
    ok = ok && cudaMemset(b.ticket, 0, sizeof(unsigned) * n_replicas) == cudaSuccess;
    ok = ok && cudaMemset(b.nnb, 0, sizeof(int) * N) == cudaSuccess;
    ok = ok && cudaMemset(b.plan, 0, sizeof(Plan)) == cudaSuccess;
    ok = ok && cudaMemset(b.img, 0, sizeof(int4) * N) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
    s->own_stream = ok;
    // capture streams: the rebuild branch and the step after it are the critical path of a
    // split step, so they are captured at high priority and the overlapping step at low priority
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    s->prio_lo = prio_lo;
    s->prio_hi = prio_hi;
    ok = ok && cudaStreamCreateWithPriority(&s->cap_stream, cudaStreamNonBlocking, prio_hi) ==
                   cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&s->body_stream, cudaStreamNonBlocking, prio_hi) ==
                   cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&s->side_stream, cudaStreamNonBlocking, prio_lo) ==
                   cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < 3; ++k) ok = cudaEventCreate(&s->ev[k]) == cudaSuccess;
    for (int h = 0; ok && h < 2; ++h)
        ok = cudaEventCreateWithFlags(&s->stage_ev[h], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { md_destroy(s); return MD_ECUDA; }
    rc = configure_layout(s, true);
    if (rc) { md_destroy(s); return rc == MD_ENOMEM ? MD_ENOMEM : MD_ECUDA; }
    *out = s;
    return MD_OK;
}

int md_set_integrator(md_sim *s, int kind, double dt, double T, double tau) {
    if (!s) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (kind != MD_NVE_LEAPFROG && kind != MD_NVT_NOSE_HOOVER) return MD_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return MD_EINVAL;
    if (kind == MD_NVT_NOSE_HOOVER && (!(T > 0.0) || !(tau > 0.0) || !std::isfinite(T) ||
                                       !std::isfinite(tau)))
        return MD_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    s->integrator = kind;
    s->dt = dt;
    s->T0 = kind == MD_NVT_NOSE_HOOVER ? T : (std::isfinite(T) && T > 0 ? T : 1.0);
    s->tau = kind == MD_NVT_NOSE_HOOVER ? tau : 0.2;
    for (auto &d : s->sys) d.K0 = 0.5 * (3.0 * d.n - 3.0) * s->T0;
    if (cudaMemcpy(s->b.sys, s->sys.data(), s->sys.size() * sizeof(SysDesc),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(s, MD_ECUDA);
    // the next step's friction and factors follow the new integrator, dt, T0 and tau
    std::vector<Thermo> th(s->R);
    if (cudaMemcpy(th.data(), s->b.th, sizeof(Thermo) * s->R, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(s, MD_ECUDA);
    for (int r = 0; r < s->R; ++r) host_next_factors(s, th[r], s->sys[r].K0);
    if (cudaMemcpy(s->b.th, th.data(), sizeof(Thermo) * s->R, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(s, MD_ECUDA);
    destroy_graphs(s);
    return MD_OK;
}

int md_set_stream(md_sim *s, void *cuda_stream) {
    if (!s) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    s->own_stream = false;
    s->stream = (cudaStream_t)cuda_stream;
    return MD_OK;
}

int md_set_state(md_sim *s, int r, const double *pos, const int *type, const double *vel,
                 const int *image) {
    int rc = check_replica(s, r);
    if (rc) return rc;
    if (s->sticky) return s->sticky;
    if (!pos || !type || !vel) return MD_EINVAL;
    const int n = s->n[r];
    // validation and the kinetic energy of the FP32 (mixed) or FP64 velocities, in user order
    double K = 0.0;
    for (int k = 0; k < n; ++k) {
        if (type[k] < 0 || type[k] >= s->nt) return MD_EINVAL;
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(pos[3 * k + c]) || !std::isfinite(vel[3 * k + c])) return MD_EINVAL;
        double vs[3];
        for (int c = 0; c < 3; ++c)
            vs[c] = s->precision == MD_FP64 ? vel[3 * k + c] : (double)(float)vel[3 * k + c];
        K += 0.5 * s->mass[type[k]] * (vs[0] * vs[0] + vs[1] * vs[1] + vs[2] * vs[2]);
    }
    // Chunks of the caller's arrays go into a pinned half of the staging area while the other
    // half's copy may still run; each copy and its unpack kernel are ordered on the
    // simulation's stream after the steps already queued, so no step in flight sees a partly
    // written state.
    for (int k0 = 0; k0 < n; k0 += s->stage_cap) {
        const int cn = std::min(s->stage_cap, n - k0);
        const int h = s->stage_k;
        s->stage_k ^= 1;
        if (cudaEventSynchronize(s->stage_ev[h]) != cudaSuccess) return fail(s, MD_ECUDA);
        unsigned char *st = s->stage_h[h];
        std::memcpy(st, pos + 3 * (size_t)k0, 24 * (size_t)cn);
        std::memcpy(st + 24 * (size_t)cn, vel + 3 * (size_t)k0, 24 * (size_t)cn);
        std::memcpy(st + 48 * (size_t)cn, type + k0, 4 * (size_t)cn);
        size_t bytes = 52 * (size_t)cn;
        if (image) {
            std::memcpy(st + bytes, image + 3 * (size_t)k0, 12 * (size_t)cn);
            bytes += 12 * (size_t)cn;
        }
        if (cudaMemcpyAsync(s->stage_d, st, bytes, cudaMemcpyHostToDevice, s->stream) !=
                cudaSuccess ||
            cudaEventRecord(s->stage_ev[h], s->stream) != cudaSuccess)
            return fail(s, MD_ECUDA);
        StateXfer t = state_xfer(s, r, k0, cn);
        t.has_image = image ? 1 : 0;
        k_load_state<<<xfer_grid(cn), 256, 0, s->stream>>>(t);
        if (cudaGetLastError() != cudaSuccess) return fail(s, MD_ECUDA);
    }
    Thermo th;
    std::memset(&th, 0, sizeof(th));
    th.K_prev = K;
    host_next_factors(s, th, s->sys[r].K0);
    Buffers &b = s->b;
    k_load_replica<<<1, 1, 0, s->stream>>>(th, b.th + r, need_now(s) + r, b.moved + r,
                                           b.disp + 2 * r, b.ctrl);
    if (cudaGetLastError() != cudaSuccess) return fail(s, MD_ECUDA);
    s->loaded[r] = 1;
    return MD_OK;
}

int md_step(md_sim *s, long long n_steps) {
    if (!s || n_steps < 0) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    for (char c : s->loaded)
        if (!c) return MD_ESTATE;
    long long remaining = n_steps;
    int guard = 0;
    while (remaining > 0) {
        const long long start = s->h_step;
        while (remaining > 0) {
            const int p = (int)(s->h_step & 1);
            if (s->graph_block > 0 && remaining >= s->graph_block) {
                if (s->exec[p] == nullptr || s->graph_len[p] != s->graph_block) {
                    if (s->exec[p]) {
                        cudaGraphExecDestroy(s->exec[p]);
                        cudaGraphDestroy(s->graph[p]);
                        s->exec[p] = nullptr;
                        s->graph[p] = nullptr;
                    }
                    int rc = build_graph(s, p);
                    if (rc) return rc;
                }
                if (cudaGraphLaunch(s->exec[p], s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
                s->h_step += s->graph_block;
                remaining -= s->graph_block;
            } else {
                if ((!use_rep(s) && do_rebuild(s, p, s->stream) != cudaSuccess) ||
                    do_step(s, p, s->stream, 0) != cudaSuccess)
                    return fail(s, MD_ECUDA);
                s->h_step += 1;
                remaining -= 1;
            }
        }
        int rc = read_ctrl(s);
        if (rc) return rc;
        if (s->h_ctrl->unstable) return fail(s, MD_EUNSTABLE);
        if (s->h_ctrl->overflow) {
            // steps after the overflowing build were skipped on the device; redo them
            const long long done = s->h_ctrl->step;
            remaining += s->h_step - done;
            s->h_step = done;
            if (++guard > 16) return fail(s, MD_ECUDA);
            if ((rc = recover_overflow(s))) return rc;
            (void)start;
            continue;
        }
        if (s->h_ctrl->step != s->h_step) return fail(s, MD_ECUDA);
        if (s->h_ctrl->rep_overflow) {
            // replica-resident builds that overflowed used list-free forces (exact); grow n_max
            if ((rc = grow_after_rep_overflow(s))) return rc;
        }
    }
    return MD_OK;
}

int md_sync(md_sim *s) {
    if (!s) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    return MD_OK;
}

int md_get_state(md_sim *s, int r, double *pos, int *image, double *vel) {
    int rc = check_replica(s, r);
    if (rc) return rc;
    if (s->sticky) return s->sticky;
    if (!s->loaded[r]) return MD_ESTATE;
    const int n = s->n[r];
    const size_t R4 = s->r4;
    if (n <= s->stage_cap) {   // one chunk: packed in user order on the device, copied out
        const int h = s->stage_k;
        k_save_user<<<xfer_grid(n), 256, 0, s->stream>>>(state_xfer(s, r, 0, n));
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(s->stage_h[h], s->stage_d, 60 * (size_t)n, cudaMemcpyDeviceToHost,
                            s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            return fail(s, MD_ECUDA);
        const unsigned char *st = s->stage_h[h];
        if (pos) std::memcpy(pos, st, 24 * (size_t)n);
        if (vel) std::memcpy(vel, st + 24 * (size_t)n, 24 * (size_t)n);
        if (image) std::memcpy(image, st + 48 * (size_t)n, 12 * (size_t)n);
        return MD_OK;
    }
    for (int k0 = 0; k0 < n; k0 += s->stage_cap) {
        const int cn = std::min(s->stage_cap, n - k0);
        // slots k0 .. k0 + cn - 1 packed on the device (after the queued steps), one copy back
        const int h = s->stage_k;
        k_save_state<<<xfer_grid(cn), 256, 0, s->stream>>>(state_xfer(s, r, k0, cn));
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(s->stage_h[h], s->stage_d, (size_t)cn * (R4 + 44),
                            cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            return fail(s, MD_ECUDA);
        const unsigned char *vv = s->stage_h[h];
        const int4 *img = (const int4 *)(vv + (size_t)cn * R4);
        const unsigned char *xs = (const unsigned char *)(img + cn);
        const unsigned char *ys = xs + (size_t)cn * 8, *zs = ys + (size_t)cn * 8;
        const int *ids = (const int *)(zs + (size_t)cn * 8);
        for (int j = 0; j < cn; ++j) {
            const int u = ids[j];
            if (u < 0 || u >= n) return fail(s, MD_ECUDA);
            double p3[3];
            if (s->precision == MD_MIXED) {   // 64-bit fixed-point masters -> [0, L)
                uint64_t q[3];
                std::memcpy(&q[0], xs + 8 * (size_t)j, 8);
                std::memcpy(&q[1], ys + 8 * (size_t)j, 8);
                std::memcpy(&q[2], zs + 8 * (size_t)j, 8);
                for (int c = 0; c < 3; ++c) p3[c] = from_fixed64(q[c], s->L[r]);
            } else {
                std::memcpy(&p3[0], xs + 8 * (size_t)j, 8);
                std::memcpy(&p3[1], ys + 8 * (size_t)j, 8);
                std::memcpy(&p3[2], zs + 8 * (size_t)j, 8);
            }
            if (pos) { pos[3 * u] = p3[0]; pos[3 * u + 1] = p3[1]; pos[3 * u + 2] = p3[2]; }
            if (image) {
                image[3 * u] = img[j].x; image[3 * u + 1] = img[j].y; image[3 * u + 2] = img[j].z;
            }
            if (vel) unpack_v4(s, vv, j, vel + 3 * u);
        }
    }
    return MD_OK;
}

int md_get_energies(md_sim *s, int r, md_energies *out) {
    int rc = check_replica(s, r);
    if (rc) return rc;
    if (!out) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    Thermo th;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
        cudaMemcpy(&th, s->b.th + r, sizeof(th), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(s, MD_ECUDA);
    const double n = s->n[r], L = s->L[r], g = 3.0 * n - 3.0;
    std::memset(out, 0, sizeof(*out));
    out->step = th.step - 1;
    out->n = s->n[r];
    out->V = L * L * L;
    out->U = th.U;
    out->W = th.W;
    out->K_minus = th.K_minus;
    out->K_plus = th.K_plus;
    out->K = 0.5 * (th.K_minus + th.K_plus);
    out->T_kin = 2.0 * out->K / g;
    out->P = (n * out->T_kin + th.W) / out->V;
    out->xi = th.xi;
    out->xi_int = th.xi_int;
    out->H = out->U + out->K;
    if (s->integrator == MD_NVT_NOSE_HOOVER)
        out->H += g * s->T0 * (0.5 * s->tau * s->tau * th.xi * th.xi + th.xi_int);
    out->sum_p[0] = th.px;
    out->sum_p[1] = th.py;
    out->sum_p[2] = th.pz;
    return MD_OK;
}

int md_get_forces(md_sim *s, int r, double *f, double *u, double *w) {
    int rc = check_replica(s, r);
    if (rc) return rc;
    if (s->sticky) return s->sticky;
    for (char c : s->loaded)
        if (!c) return MD_ESTATE;
    if ((rc = ensure_list(s))) return rc;
    const int p = (int)(s->h_step & 1);
    if (do_step(s, p, s->stream, 1) != cudaSuccess) return fail(s, MD_ECUDA);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    const int n = s->n[r], o = s->off[r];
    const size_t R4 = s->r4;
    std::vector<unsigned char> fv((size_t)n * R4), wv((size_t)n * (R4 / 4));
    std::vector<int> ids(n);
    bool ok = cudaMemcpy(fv.data(), (char *)s->b.f_out + o * R4, n * R4, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(wv.data(), (char *)s->b.w_out + o * (R4 / 4), n * (R4 / 4), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(ids.data(), s->b.id + o, n * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return fail(s, MD_ECUDA);
    for (int k = 0; k < n; ++k) {
        const int q = ids[k];
        double v4[4];
        if (s->precision == MD_FP64) {
            std::memcpy(v4, fv.data() + k * 32, 32);
        } else {
            float t[4];
            std::memcpy(t, fv.data() + k * 16, 16);
            for (int c = 0; c < 4; ++c) v4[c] = t[c];
        }
        if (f) { f[3 * q] = v4[0]; f[3 * q + 1] = v4[1]; f[3 * q + 2] = v4[2]; }
        if (u) u[q] = v4[3];
        if (w) {
            if (s->precision == MD_FP64) {
                double t;
                std::memcpy(&t, wv.data() + k * 8, 8);
                w[q] = t;
            } else {
                float t;
                std::memcpy(&t, wv.data() + k * 4, 4);
                w[q] = t;
            }
        }
    }
    return MD_OK;
}

int md_get_neighbors(md_sim *s, int r, int maxp, int *counts, int *nbrs) {
    int rc = check_replica(s, r);
    if (rc) return rc;
    if (!counts || maxp < 0 || (maxp > 0 && !nbrs)) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->list_method == 2) return MD_ESTATE;                  // no list is kept
    const int n = s->n[r], o = s->off[r];
    const int sl0 = o / 32, sl1 = (o + n - 1) / 32;            // slices holding the replica
    const size_t per = (size_t)32 * s->nmax;
    std::vector<int> cnt(n), ids(n), lst((size_t)(sl1 - sl0 + 1) * per);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    bool ok = cudaMemcpy(cnt.data(), s->b.nnb + o, n * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(ids.data(), s->b.id + o, n * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(lst.data(), s->b.nbl + (size_t)sl0 * per, lst.size() * sizeof(int),
                          cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return fail(s, MD_ECUDA);
    for (int k = 0; k < n; ++k) {
        const int q = ids[k], i = o + k;
        counts[q] = cnt[k];
        for (int m = 0; m < maxp; ++m) {
            int v = -1;
            if (m < cnt[k] && m < s->nmax) {
                const size_t off = (((size_t)(i / 32 - sl0) * s->nmax + m) * 32) + (i % 32);
                const int j = lst[off] - o;
                v = (j >= 0 && j < n) ? ids[j] : -2;
            }
            nbrs[(size_t)q * maxp + m] = v;
        }
    }
    return MD_OK;
}

int md_set_tuning(md_sim *s, int tp, int block, int reach, int build_lanes) {
    if (!s) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    const int ntp = tp ? tp : s->tp, nb = block ? block : s->block, nr = reach ? reach : s->reach;
    const int nl = build_lanes ? build_lanes : s->tpb;
    if (!is_pow2_tp(ntp) || nb < 32 || nb > 1024 || (nb % 32) != 0 || nb < ntp || nr < 1 ||
        nr > 3 || !valid_lanes(nl))
        return MD_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    const bool cells_change = nr != s->reach;
    const bool pad_change = ntp != s->tp;   // lists are padded for the force loop's tp
    s->tp = ntp;
    s->block = nb;
    s->reach = nr;
    s->tpb = nl;
    destroy_graphs(s);
    if (pad_change && round_nmax(s, s->nmax) != s->nmax) {
        s->nmax = round_nmax(s, s->nmax);
        if (alloc_nbl(s)) return MD_ENOMEM;
    }
    int rc = configure_layout(s, cells_change);
    if (rc) return rc == MD_ENOMEM ? MD_ENOMEM : fail(s, MD_ECUDA);
    if (cells_change || pad_change) return request_rebuild_all(s);
    return MD_OK;
}

int md_get_tuning(md_sim *s, int *tp, int *block, int *reach, int *build_lanes) {
    if (!s) return MD_EINVAL;
    if (tp) *tp = s->tp;
    if (block) *block = s->block;
    if (reach) *reach = s->reach;
    if (build_lanes) *build_lanes = s->tpb;
    return MD_OK;
}

int md_set_list_method(md_sim *s, int method) {
    if (!s || method < 0 || method > 2) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->list_method = method;
    return method == 2 ? MD_OK : request_rebuild_all(s);
}

int md_set_coulomb(md_sim *s, const double *charge, double rc_coulomb) {
    if (!s) return MD_EINVAL;
    const bool on = charge != nullptr && rc_coulomb > 0.0;
    if (charge && !(rc_coulomb > 0.0 && std::isfinite(rc_coulomb))) return MD_EINVAL;
    if (on)
        for (int t = 0; t < s->nt; ++t)
            if (!std::isfinite(charge[t])) return MD_EINVAL;
    double rc_max = 0.0;
    for (auto &p : s->params) rc_max = std::max(rc_max, p.rc);
    if (on) rc_max = std::max(rc_max, rc_coulomb);
    for (int r = 0; r < s->R; ++r)
        if (!(s->L[r] > 2.0 * (rc_max + s->skin))) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->coul = on;
    s->rcc = on ? rc_coulomb : 0.0;
    s->rc_max = rc_max;
    for (int t = 0; t < kMaxTypes; ++t) s->charge[t] = (on && t < s->nt) ? charge[t] : 0.0;
    for (int a = 0; a < s->nt; ++a)
        for (int c = 0; c < s->nt; ++c) {
            PairTab &t = s->tab[a * s->nt + c];
            const double qq = s->charge[a] * s->charge[c], rcc = s->rcc;
            // an off term gets a zero range, so no pair ever passes r2 < qrc2
            t.qrc2d = on ? rcc * rcc : 0.0;
            t.qqd = qq;
            t.qfd = on ? qq / (rcc * rcc) : 0.0;
            t.qud = on ? 2.0 * qq / rcc : 0.0;
            t.qrc2 = (float)t.qrc2d; t.qq = (float)t.qqd; t.qf = (float)t.qfd; t.qu = (float)t.qud;
        }
    if (upload_thresholds(s)) return fail(s, MD_ECUDA);
    const int need = round_nmax(s, estimate_nmax(s));
    if (need > s->nmax) {
        s->nmax = need;
        if (alloc_nbl(s)) return MD_ENOMEM;
    }
    int rc = configure_layout(s, true);   // cell edge and kernel paths follow the new range
    if (rc) return rc == MD_ENOMEM ? MD_ENOMEM : fail(s, MD_ECUDA);
    return request_rebuild_all(s);
}

int md_set_resort_interval(md_sim *s, int passes) {
    if (!s || passes < 0) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->resort = passes;
    return MD_OK;
}

int md_set_rebuild_batch(md_sim *s, int k) {
    if (!s || k < 1 || k > 64) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->rebuild_batch = k;
    return MD_OK;
}

int md_set_skin(md_sim *s, double skin) {
    if (!s || !(skin > 0.0) || !std::isfinite(skin)) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    for (int r = 0; r < s->R; ++r)
        if (!(s->L[r] > 2.0 * (s->rc_max + skin))) return MD_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->skin = skin;
    if (upload_thresholds(s)) return fail(s, MD_ECUDA);
    const int need = round_nmax(s, estimate_nmax(s));
    if (need > s->nmax) {
        s->nmax = need;
        if (alloc_nbl(s)) return MD_ENOMEM;
    }
    int rc = configure_layout(s, true);   // cell edge follows rc_max + skin
    if (rc) return rc == MD_ENOMEM ? MD_ENOMEM : fail(s, MD_ECUDA);
    return request_rebuild_all(s);
}

int md_get_skin(md_sim *s, double *skin) {
    if (!s || !skin) return MD_EINVAL;
    *skin = s->skin;
    return MD_OK;
}

int md_set_list_capacity(md_sim *s, int n_max) {
    if (!s || n_max < 1) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->nmax = round_nmax(s, n_max);
    if (alloc_nbl(s)) return MD_ENOMEM;
    return request_rebuild_all(s);
}

int md_set_path(md_sim *s, int path) {
    if (!s || path < 0 || path > 4) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (path == 2 && !s->rep_ok) return MD_EINVAL;
    if (path == 3 && !s->staged_ok) return MD_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->path = path;
    return MD_OK;
}

int md_set_graph_block(md_sim *s, int steps) {
    if (!s) return MD_EINVAL;
    if (steps < 0) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    s->graph_block = steps;
    return MD_OK;
}

int md_get_stats(md_sim *s, md_stats *out) {
    if (!s || !out) return MD_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    std::vector<Thermo> th(s->R);
    std::vector<int> nn(s->ntot);
    if (cudaMemcpy(th.data(), s->b.th, sizeof(Thermo) * s->R, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nn.data(), s->b.nnb, sizeof(int) * s->ntot, cudaMemcpyDeviceToHost) != cudaSuccess ||
        read_ctrl(s))
        return fail(s, MD_ECUDA);
    long long reb = 0, ent = 0;
    int mx = 0;
    for (auto &t : th) reb += t.rebuilds;
    for (int v : nn) { ent += v; mx = std::max(mx, v); }
    out->steps = s->h_step;
    out->rebuild_passes = s->h_ctrl->rebuild_passes;
    out->replica_rebuilds = reb;
    out->overflows = s->overflows;
    out->n_max = s->nmax;
    out->max_neighbors = mx;
    out->tp = s->tp;
    out->block = s->block;
    out->reach = s->reach;
    out->build_lanes = s->tpb;
    out->path = use_rep(s) ? 2 : ((s->path == 3 && s->staged_ok) ? 3 : (s->path == 4 ? 4 : 1));
    const int cell_kernels = s->sort_small ? 3 : 7;   // plan, sort (1 or 5 kernels), build
    out->rebuild_kernels = s->list_method == 2   ? 0
                           : s->list_method == 0 ? cell_kernels
                           : s->resort > 0       ? cell_kernels + 1
                                                 : 2;
    out->list_method = s->list_method;
    out->rebuild_batch = s->rebuild_batch;
    out->resort = s->resort;
    out->step_kernels = split_steps(s) ? 2 : 1;     // per graph step
    out->graph_block = s->graph_block;
    out->n_total = s->ntot;
    out->neighbor_entries = ent;
    out->graph_builds = s->graph_builds;
    return MD_OK;
}

int md_profile(md_sim *s, int n_steps, md_timing *out) {
    if (!s || !out || n_steps < 1) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    for (char c : s->loaded)
        if (!c) return MD_ESTATE;
    std::memset(out, 0, sizeof(*out));
    double t_step = 0.0, t_reb = 0.0;
    int n_reb = 0;
    long long entries = 0;
    for (int k = 0; k < n_steps; ++k) {
        int rc = read_ctrl(s);
        if (rc) return rc;
        const bool will = s->h_ctrl->need_any && !s->h_ctrl->halt && !use_rep(s);
        const int p = (int)(s->h_step & 1);
        cudaError_t e;
        if (use_rep(s))
            e = cudaEventRecord(s->ev[0], s->stream) == cudaSuccess &&
                        cudaEventRecord(s->ev[1], s->stream) == cudaSuccess
                    ? cudaSuccess
                    : cudaErrorUnknown;
        else if (s->precision == MD_FP64)
            e = launch_rebuild_timed<double>(rebuild_args<double>(s, p, nullptr), s->stream, s->ev[0], s->ev[1]);
        else
            e = launch_rebuild_timed<float>(rebuild_args<float>(s, p, nullptr), s->stream, s->ev[0], s->ev[1]);
        if (e != cudaSuccess) return fail(s, MD_ECUDA);
        if (do_step(s, p, s->stream, 0) != cudaSuccess || cudaEventRecord(s->ev[2], s->stream) != cudaSuccess)
            return fail(s, MD_ECUDA);
        if ((rc = read_ctrl(s))) return rc;
        if (s->h_ctrl->unstable) return fail(s, MD_EUNSTABLE);
        if (s->h_ctrl->overflow) {
            if ((rc = recover_overflow(s))) return rc;
            --k;
            continue;
        }
        if (s->h_ctrl->rep_overflow && (rc = grow_after_rep_overflow(s))) return rc;
        float a = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, s->ev[0], s->ev[1]);
        cudaEventElapsedTime(&c, s->ev[1], s->ev[2]);
        t_step += c;
        if (will) { t_reb += a; ++n_reb; }
        s->h_step += 1;
    }
    md_stats st;
    if (md_get_stats(s, &st) == MD_OK) entries = st.neighbor_entries;
    out->steps = n_steps;
    out->step_kernel_ms = t_step / n_steps;
    out->rebuild_ms = n_reb ? t_reb / n_reb : 0.0;
    out->rebuild_fraction = (double)n_reb / n_steps;
    out->neighbor_entries = entries;
    return MD_OK;
}

int md_set_log(md_sim *s, int capacity) {
    if (!s || capacity < 0) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    dfree(s->b.log);
    s->log_cap = 0;
    destroy_graphs(s);
    if (capacity == 0) return MD_OK;
    const size_t cnt = (size_t)capacity * s->R * MD_LOG_COLS;
    if (dalloc(s, &s->b.log, cnt)) return MD_ENOMEM;
    if (cudaMemset(s->b.log, 0, cnt * sizeof(double)) != cudaSuccess) return fail(s, MD_ECUDA);
    s->log_cap = capacity;
    return MD_OK;
}

int md_get_log(md_sim *s, int r, int max_rows, double *out, int *rows) {
    int rc = check_replica(s, r);
    if (rc) return rc;
    if (!rows || max_rows < 0 || (max_rows > 0 && !out)) return MD_EINVAL;
    *rows = 0;
    if (s->sticky) return s->sticky;
    if (s->log_cap == 0) return MD_OK;
    Thermo th;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
        cudaMemcpy(&th, s->b.th + r, sizeof(th), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(s, MD_ECUDA);
    const long long done = th.step;
    const long long k = std::min<long long>(std::min<long long>(done, s->log_cap), max_rows);
    std::vector<double> all((size_t)s->log_cap * s->R * MD_LOG_COLS);
    if (cudaMemcpy(all.data(), s->b.log, all.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(s, MD_ECUDA);
    for (long long q = 0; q < k; ++q) {
        const long long step = done - k + q;
        const double *row = all.data() + ((size_t)(step % s->log_cap) * s->R + r) * MD_LOG_COLS;
        std::memcpy(out + q * MD_LOG_COLS, row, sizeof(double) * MD_LOG_COLS);
    }
    *rows = (int)k;
    return MD_OK;
}

// ---------------------------------------------------------------- checkpoints
// Layout: header, then per replica: Thermo, need flag, and per particle (user order):
// x y z (8 bytes each: the master position, double in FP64 mode, 64-bit fixed point in mixed
// precision), image (3 int), type (int), velocity (3 Real), build position (3 x 4 bytes: the
// 32-bit fixed-point mirror in mixed precision; 3 doubles in FP64 mode).
namespace {
struct CkHeader {
    char magic[8];
    int version, R, ntot, precision, nt, pad;
    long long step;
};
size_t ck_bytes(const md_sim *s) {
    size_t b = sizeof(CkHeader) + (size_t)s->R * (sizeof(Thermo) + sizeof(int));
    const size_t rsz = s->precision == MD_FP64 ? 8 : 4;
    b += (size_t)s->ntot * (3 * 8 + 4 * 4 + 6 * rsz);
    return b;
}
}  // namespace

int md_checkpoint_size(md_sim *s, size_t *bytes) {
    if (!s || !bytes) return MD_EINVAL;
    *bytes = ck_bytes(s);
    return MD_OK;
}

int md_save_checkpoint(md_sim *s, void *buf, size_t bytes) {
    if (!s || !buf || bytes < ck_bytes(s)) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    for (char c : s->loaded)
        if (!c) return MD_ESTATE;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    const size_t N = s->ntot, R4 = s->r4, rsz = R4 / 4;
    std::vector<double> x(N), y(N), z(N);
    std::vector<int4> img(N);
    std::vector<int> ids(N), need(s->R);
    std::vector<unsigned char> vel(N * R4), pb(N * R4), cur(N * R4);
    std::vector<Thermo> th(s->R);
    const Buffers &b = s->b;
    bool ok = cudaMemcpy(x.data(), b.xd, N * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(cur.data(), b.pos[s->h_step & 1], N * R4, cudaMemcpyDeviceToHost) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy(y.data(), b.yd, N * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(z.data(), b.zd, N * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(img.data(), b.img, N * sizeof(int4), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(ids.data(), b.id, N * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(vel.data(), b.vel, N * R4, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(pb.data(), b.pos_build, N * R4, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(th.data(), b.th, sizeof(Thermo) * s->R, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(need.data(), b.need + (size_t)(s->h_step & 1) * s->R, sizeof(int) * s->R,
                          cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return fail(s, MD_ECUDA);
    unsigned char *p = (unsigned char *)buf;
    CkHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "MDGB300", 8);
    h.version = 2; h.R = s->R; h.ntot = s->ntot; h.precision = s->precision; h.nt = s->nt;
    h.step = s->h_step;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    for (int r = 0; r < s->R; ++r) {
        std::memcpy(p, &th[r], sizeof(Thermo)); p += sizeof(Thermo);
        std::memcpy(p, &need[r], sizeof(int)); p += sizeof(int);
    }
    // per particle records in user order
    const size_t rec = 3 * 8 + 4 * 4 + 6 * rsz;
    for (int r = 0; r < s->R; ++r) {
        const int o = s->off[r], n = s->n[r];
        for (int k = 0; k < n; ++k) {
            const int q = ids[o + k];
            if (q < 0 || q >= n) return fail(s, MD_ECUDA);
            unsigned char *d = p + (size_t)(o + q) * rec;
            const size_t sl = o + k;
            std::memcpy(d, &x[sl], 8); std::memcpy(d + 8, &y[sl], 8); std::memcpy(d + 16, &z[sl], 8);
            int im[4] = {img[sl].x, img[sl].y, img[sl].z, 0};
            if (s->precision == MD_FP64) {
                long long t;
                std::memcpy(&t, cur.data() + sl * 32 + 24, 8);
                im[3] = (int)t;
            } else {
                std::memcpy(&im[3], cur.data() + sl * 16 + 12, 4);
            }
            std::memcpy(d + 24, im, 16);
            std::memcpy(d + 40, vel.data() + sl * R4, 3 * rsz);
            std::memcpy(d + 40 + 3 * rsz, pb.data() + sl * R4, 3 * rsz);
        }
    }
    return MD_OK;
}

int md_load_checkpoint(md_sim *s, const void *buf, size_t bytes) {
    if (!s || !buf || bytes < ck_bytes(s)) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    const unsigned char *p = (const unsigned char *)buf;
    CkHeader h;
    std::memcpy(&h, p, sizeof(h));
    p += sizeof(h);
    if (std::memcmp(h.magic, "MDGB300", 8) != 0 || h.version != 2 || h.R != s->R ||
        h.ntot != s->ntot || h.precision != s->precision || h.nt != s->nt)
        return MD_EINVAL;
    const size_t N = s->ntot, R4 = s->r4, rsz = R4 / 4;
    std::vector<Thermo> th(s->R);
    std::vector<int> need(s->R);
    for (int r = 0; r < s->R; ++r) {
        std::memcpy(&th[r], p, sizeof(Thermo)); p += sizeof(Thermo);
        std::memcpy(&need[r], p, sizeof(int)); p += sizeof(int);
    }
    std::vector<double> x(N), y(N), z(N);
    std::vector<int4> img(N);
    std::vector<int> ids(N);
    std::vector<unsigned char> mirror(N * R4), vel(N * R4), pb(N * R4);
    std::vector<int> types(N);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
    const size_t rec = 3 * 8 + 4 * 4 + 6 * rsz;
    for (int r = 0; r < s->R; ++r) {
        const int o = s->off[r], n = s->n[r];
        for (int q = 0; q < n; ++q) {
            const unsigned char *d = p + (size_t)(o + q) * rec;
            const size_t sl = o + q;   // load in user order; the restore rebuild sorts
            std::memcpy(&x[sl], d, 8); std::memcpy(&y[sl], d + 8, 8); std::memcpy(&z[sl], d + 16, 8);
            int im[4];
            std::memcpy(im, d + 24, 16);
            img[sl] = make_int4(im[0], im[1], im[2], 0);
            types[sl] = im[3];
            if (im[3] < 0 || im[3] >= s->nt) return MD_EINVAL;
            ids[sl] = q;
            std::memset(vel.data() + sl * R4, 0, R4);
            std::memcpy(vel.data() + sl * R4, d + 40, 3 * rsz);
            if (rsz == 8) {
                pack_pos(mirror, sl, x[sl], y[sl], z[sl], types[sl]);
                double bx[3];
                std::memcpy(bx, d + 40 + 3 * rsz, 24);
                pack_pos(pb, sl, bx[0], bx[1], bx[2], types[sl]);
            } else {
                uint64_t qq[3];
                std::memcpy(&qq[0], &x[sl], 8);
                std::memcpy(&qq[1], &y[sl], 8);
                std::memcpy(&qq[2], &z[sl], 8);
                pack_mirror(mirror, sl, qq[0], qq[1], qq[2], types[sl]);
                int32_t b4[4] = {0, 0, 0, types[sl]};
                std::memcpy(b4, d + 40 + 3 * rsz, 12);
                std::memcpy(pb.data() + sl * 16, b4, 16);
            }
        }
    }
    s->h_step = h.step;
    const int cur = (int)(s->h_step & 1);
    Buffers &b = s->b;
    bool ok = cudaMemcpy(b.pos[cur], mirror.data(), N * R4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.pos_build, pb.data(), N * R4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.xd, x.data(), N * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.yd, y.data(), N * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.zd, z.data(), N * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.vel, vel.data(), N * R4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.img, img.data(), N * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.id, ids.data(), N * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b.th, th.data(), sizeof(Thermo) * s->R, cudaMemcpyHostToDevice) == cudaSuccess;
    Ctrl c;
    std::memset(&c, 0, sizeof(c));
    c.step = h.step;
    c.need_any = 1;
    ok = ok && cudaMemcpy(b.ctrl, &c, sizeof(c), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(b.moved, 0, sizeof(int) * s->R) == cudaSuccess;
    ok = ok && cudaMemset(b.disp, 0, sizeof(unsigned) * 2 * s->R) == cudaSuccess;
    ok = ok && cudaMemset(b.ticket, 0, sizeof(unsigned) * s->R) == cudaSuccess;
    if (!ok) return fail(s, MD_ECUDA);
    int rc = request_rebuild_all(s);
    if (rc) return rc;
    // restore rebuild: cells, order and list from the saved build positions
    for (int tries = 0; tries < 16; ++tries) {
        cudaError_t e = do_rebuild(s, cur, s->stream, s->b.pos_build);
        if (e != cudaSuccess) return fail(s, MD_ECUDA);
        if ((rc = read_ctrl(s))) return rc;
        if (!s->h_ctrl->overflow) break;
        if ((rc = recover_overflow(s))) return rc;
    }
    // pending rebuild flags as saved
    int any = 0;
    for (int v : need) any |= v;
    ok = cudaMemcpy(need_now(s), need.data(), sizeof(int) * s->R, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(&b.ctrl->need_any, &any, sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) return fail(s, MD_ECUDA);
    destroy_graphs(s);
    for (auto &l : s->loaded) l = 1;
    return MD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner (Appendix)
// Short timed runs from one saved state (restored before every trial, so every trial starts from
// the same configuration), a line search over the cell stencil reach, then the double loop of
// the Appendix over block size and threads per particle with its break rules:
//   - the tp loop stops when the time exceeds the best so far three times in a row, or exceeds it
//     by 5%, or the block cannot hold the group;
//   - the block loop stops when its best exceeds the overall best by 10% or more.
// The result is cached in a text file keyed by the "user parameters" (particle counts per type
// and replica, densities, potential, integrator, dt, temperature) and the GPU name.
namespace {

std::string tune_key(md_sim *s) {
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, s->device);
    // FNV-1a over the replica sizes and boxes keeps the key short for large ensembles
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t k = 0; k < n; ++k) { h ^= c[k]; h *= 1099511628211ULL; }
    };
    for (int r = 0; r < s->R; ++r) {
        mix(&s->n[r], sizeof(int));
        const float Lr = (float)s->L[r];   // density within float tolerance
        mix(&Lr, sizeof(float));
    }
    for (auto &p : s->params) {
        const float q[3] = {(float)p.eps, (float)p.sigma, (float)p.rc};
        mix(q, sizeof(q));
    }
    mix(&s->cutoff, sizeof(int));
    if (s->coul) {
        mix(&s->rcc, sizeof(double));
        mix(s->charge, sizeof(double) * s->nt);
    }
    char buf[512];
    std::snprintf(buf, sizeof(buf), "gpu=%s|R=%d|N=%d|nt=%d|prec=%d|skin=%.4g|integ=%d|dt=%.6g|T=%.4g|h=%016llx",
                  prop.name, s->R, s->ntot, s->nt, s->precision, s->skin, s->integrator, s->dt,
                  s->integrator == MD_NVT_NOSE_HOOVER ? s->T0 : 0.0, h);
    std::string k(buf);
    for (char &c : k)
        if (c == ' ') c = '_';
    return k;
}

bool cache_lookup(const char *path, const std::string &key, int *tp, int *block, int *reach,
                  int *lanes, double *skin, int *resort) {
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[900];
        int a, b, c, d, rs = 0;
        double sk = 0.0, ms = 0.0;
        if (std::sscanf(line, "%899s %d %d %d %d %lf %lf %d", k, &a, &b, &c, &d, &sk, &ms, &rs) ==
                8 &&
            key == k) {
            *tp = a; *block = b; *reach = c; *lanes = d; *skin = sk; *resort = rs;
            found = true;   // the last entry for a key wins
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int tp, int block, int reach, int lanes,
                 double skin, double ms, int resort) {
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %.9g %.6f %d\n", key.c_str(), tp, block, reach, lanes, skin, ms,
                 resort);
    std::fclose(f);
}

}  // namespace

extern "C" int md_autotune(md_sim *s, const char *cache_path, int steps, int flags) {
    if (!s || steps < 2 || (flags & ~MD_TUNE_SKIN)) return MD_EINVAL;
    if (s->sticky) return s->sticky;
    for (char c : s->loaded)
        if (!c) return MD_ESTATE;
    const std::string key = tune_key(s) + ((flags & MD_TUNE_SKIN) ? "|skin-tuned" : "") + "|v3";
    int tp = 0, block = 0, reach = 0, lanes = 0, cresort = 0;
    double cskin = 0.0;
    if (cache_lookup(cache_path, key, &tp, &block, &reach, &lanes, &cskin, &cresort) &&
        is_pow2_tp(tp) && cresort >= 0 &&
        block >= tp && block <= 1024 && block % 32 == 0 && reach >= 1 && reach <= 3 &&
        valid_lanes(lanes / 10000) && lanes % 10 <= 4 && (lanes / 10) % 10 <= 2 &&
        (lanes / 100) % 100 >= 1) {
        int e = 0;
        if ((flags & MD_TUNE_SKIN) && cskin > 0.0 && (e = md_set_skin(s, cskin))) return e;
        if ((e = md_set_tuning(s, tp, block, reach, lanes / 10000))) return e;
        if ((e = md_set_list_method(s, (lanes / 10) % 10))) return e;
        if ((e = md_set_rebuild_batch(s, (lanes / 100) % 100))) return e;
        if ((e = md_set_resort_interval(s, cresort))) return e;
        const int path = lanes % 10;
        return md_set_path(s, (path == 2 && s->rep_ok) || (path == 3 && s->staged_ok) || path == 4
                                  ? path : 1);
    }
    size_t bytes = 0;
    md_checkpoint_size(s, &bytes);
    std::vector<unsigned char> ck(bytes);
    int rc = md_save_checkpoint(s, ck.data(), bytes);
    if (rc) return rc;
    const int gb_saved = s->graph_block;
    int trial_block = std::min((steps / 2) * 2, 50);
    if (trial_block < 2) trial_block = 2;
    // time one configuration: restore, warm up (graph capture + first rebuild), restore, time
    // Every trial starts from the stored state and runs the same steps (Appendix).  A restored
    // state rebuilds every list at once, so the first steps after it are unusually quiet; the
    // timed steps follow 2 x steps of warm-up (graph capture included), by which the rebuilds of
    // the replicas have spread out as in a long run.
    const int warm = ((2 * steps + trial_block - 1) / trial_block) * trial_block;
    auto trial = [&](int t, int b, int re, int la, double *ms) -> int {
        int e = md_set_tuning(s, t, b, re, la);
        if (e) return e;
        if ((e = md_set_graph_block(s, trial_block))) return e;
        if ((e = md_load_checkpoint(s, ck.data(), bytes))) return e;
        if ((e = md_step(s, warm))) return e;
        if (cudaEventRecord(s->ev[0], s->stream) != cudaSuccess) return fail(s, MD_ECUDA);
        if ((e = md_step(s, steps))) return e;
        if (cudaEventRecord(s->ev[1], s->stream) != cudaSuccess ||
            cudaEventSynchronize(s->ev[1]) != cudaSuccess)
            return fail(s, MD_ECUDA);
        float f = 0.f;
        cudaEventElapsedTime(&f, s->ev[0], s->ev[1]);
        *ms = f / steps;
        return MD_OK;
    };
    int nmax_part = 0;
    for (int v : s->n) nmax_part = std::max(nmax_part, v);
    // The Appendix tries only t_p = 1 above 10^5 particles, on its GPU with 15 SMs of 2048 resident
    // threads; the size from which one thread per particle fills the GPU grows with its resident
    // threads, so the limit is scaled by this GPU's.
    int max_thr = 2048;
    if (cudaDeviceGetAttribute(&max_thr, cudaDevAttrMaxThreadsPerMultiProcessor, s->device) !=
        cudaSuccess) {
        cudaGetLastError();
        max_thr = 2048;
    }
    const double tp1_limit = 1e5 * (double)s->nsm * (double)max_thr / (15.0 * 2048.0);
    // Appendix defaults: t_p = 4 (p_b = 32) up to 10^4 particles, else t_p = 1 (p_b = 64)
    int best_tp = nmax_part <= 10000 ? 4 : 1, best_block = nmax_part <= 10000 ? 128 : 64;
    int best_reach = 2, best_lanes = 8;
    double best = 1e30, t = 0.0;
    // phase 0: grid path or replica-resident path (when both apply)
    const int path_saved = s->path;
    if (s->rep_ok) {
        double tg = 0.0, tr = 0.0;
        s->path = 1;
        if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &tg))) return rc;
        s->path = 2;
        if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &tr))) return rc;
        s->path = tr < tg ? 2 : 1;
        best = std::min(tg, tr);
    }
    if (best >= 1e30 && (rc = trial(best_tp, best_block, best_reach, best_lanes, &best))) return rc;
    // the register-capped step kernel (path 4) against the chosen one
    if (s->path == 1) {
        double tl = 0.0;
        s->path = 4;
        if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &tl))) return rc;
        if (tl < best) best = tl; else s->path = 1;
    }
    // phase 0b: list method (Appendix phase I: "none" only below 5000 particles, "n2" below 50000)
    {
        int best_m = s->list_method;
        for (int m : {1, 2}) {
            if ((m == 2 && nmax_part > 5000) || (m == 1 && nmax_part > 50000)) continue;
            if ((rc = md_set_list_method(s, m))) return rc;
            if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &t))) return rc;
            if (t < best) { best = t; best_m = m; }
        }
        if ((rc = md_set_list_method(s, best_m))) return rc;
        // Appendix step 5: with the O(N^2) method, a sort by cell every few hundred rebuilds
        // can still pay (near the crossover to the cell method); find the interval
        if (best_m == 1) {
            int best_rs = 0;
            for (int rs : {10, 50, 200}) {
                if ((rc = md_set_resort_interval(s, rs))) return rc;
                if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &t))) return rc;
                if (t < best) { best = t; best_rs = rs; }
            }
            if ((rc = md_set_resort_interval(s, best_rs))) return rc;
        }
    }
    // phase 0c: rebuild slots for batches of replicas (a rebuild pass every K steps serves all
    // replicas due before the next slot; single systems keep K = 1)
    if (s->R >= 8 && s->list_method != 2) {
        int best_k = s->rebuild_batch;
        for (int k : {2, 4, 8}) {
            if ((rc = md_set_rebuild_batch(s, k))) return rc;
            if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &t))) return rc;
            if (t < best) { best = t; best_k = k; }
        }
        if ((rc = md_set_rebuild_batch(s, best_k))) return rc;
    }
    // phase I: cell stencil reach at the default kernel shape
    for (int re : {2, 1, 3}) {
        if ((rc = trial(best_tp, best_block, re, best_lanes, &t))) return rc;
        if (t < best) { best = t; best_reach = re; }
    }
    // phase II: block size x threads per particle with the break rules of the Appendix
    const int blocks[] = {64, 128, 256, 512};
    for (int b : blocks) {
        double best_b = 1e30;
        int worse = 0;
        for (int tpv = 1; tpv <= 32; tpv *= 2) {
            if (tpv > b) break;
            if (nmax_part > tp1_limit && tpv > 1) break;   // Appendix: only t_p = 1 for large N
            if ((rc = trial(tpv, b, best_reach, best_lanes, &t))) return rc;
            if (t < best_b) best_b = t;
            if (t < best) { best = t; best_tp = tpv; best_block = b; worse = 0; continue; }
            if (t > 1.05 * best || ++worse >= 3) break;
        }
        if (best_b >= 1.10 * best) break;
    }
    // the register cap again at the best shape and the blocks beside it (its benefit depends on
    // the block and t_p: the capped kernel fits more CTAs of a given block on an SM)
    if (s->path == 1 || s->path == 4) {
        const int mine = s->path, other = mine == 1 ? 4 : 1;
        const int b0 = best_block;
        int best_path = mine;
        s->path = other;
        for (int b : {b0, b0 / 2, b0 * 2}) {
            if (b < 64 || b > 1024 || b < best_tp) continue;
            if ((rc = trial(best_tp, b, best_reach, best_lanes, &t))) return rc;
            if (t < best) { best = t; best_block = b; best_path = other; }
        }
        s->path = best_path;
    }
    // phase III: lanes per particle of the list build (single minimum: walk down, then up);
    // the replica-resident kernel is built for 8 and 32 lanes
    for (int dir : {-1, 1}) {
        int la = best_lanes;
        for (;;) {
            la = dir < 0 ? la / 2 : la * 2;
            if (la < 1 || la > 32) break;
            if (s->path == 2 && la != 8 && la != 32) continue;
            if ((rc = trial(best_tp, best_block, best_reach, la, &t))) return rc;
            if (t < best) { best = t; best_lanes = la; } else break;
        }
    }
    // ... and the build with one warp per cell (grid kernel paths)
    if (s->path != 2) {
        if ((rc = trial(best_tp, best_block, best_reach, MD_BUILD_CELL, &t))) return rc;
        if (t < best) { best = t; best_lanes = MD_BUILD_CELL; }
    }
    if ((rc = md_set_tuning(s, best_tp, best_block, best_reach, best_lanes))) return rc;
    if ((rc = md_set_graph_block(s, gb_saved))) return rc;
    if ((rc = md_load_checkpoint(s, ck.data(), bytes))) return rc;
    // phase IV (optional): the list skin, 20% steps then 10% steps around the best (Appendix)
    if (flags & MD_TUNE_SKIN) {
        double best_skin = s->skin;
        for (double step : {0.2, 0.1}) {
            for (int dir : {1, -1}) {
                double sk = best_skin;
                for (;;) {
                    sk *= (1.0 + dir * step);
                    if (md_set_skin(s, sk) != MD_OK) break;   // box too small for this skin
                    if ((rc = trial(best_tp, best_block, best_reach, best_lanes, &t))) return rc;
                    if (t < best) { best = t; best_skin = sk; } else break;
                }
            }
        }
        if ((rc = md_set_skin(s, best_skin))) return rc;
        if ((rc = md_set_tuning(s, best_tp, best_block, best_reach, best_lanes))) return rc;
        if ((rc = md_set_graph_block(s, gb_saved))) return rc;
        if ((rc = md_load_checkpoint(s, ck.data(), bytes))) return rc;
    }
    (void)path_saved;
    // lanes, rebuild slots, list method and kernel path share one cache field:
    // lanes * 10000 + K * 100 + method * 10 + path
    cache_store(cache_path, key, best_tp, best_block, best_reach,
                best_lanes * 10000 + s->rebuild_batch * 100 + s->list_method * 10 + s->path,
                s->skin, best, s->resort);
    return MD_OK;
}
