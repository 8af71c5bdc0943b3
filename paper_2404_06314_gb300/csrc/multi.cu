// Uneven batches: many circuits (different n and depth), `batch` samples each,
// forward + adjoint in one persistent kernel launch (qtm_multi_run), or the
// forward alone (qtm_multi_forward, states kept in the workspace) and the
// adjoint alone (qtm_multi_adjoint, consuming them) as two launches.
//
// Work items are (circuit, sample) pairs.  A circuit whose state fits one
// shared-memory tile (n <= 12) runs its forward pass, expectation values,
// costate and reverse pass back to back without leaving shared memory; a
// larger circuit's state lives in a per-item global buffer (L2-resident for
// n <= 16).  Tasks are handed to CTAs by a device counter in list order.  With
// split = 0 a task is a whole item (a tiled item sweeps its tiles pass after
// pass in one CTA); with split = 1 every (item, pass, tile) of a tiled item is
// its own task, listed level by level (pass k of every item before pass k + 1),
// and a task waits (bounded) until all tiles of its item's previous pass are
// done: each task depends only on tasks handed out before it, so the waits
// end, and the largest circuits no longer run on one CTA alone.  The
// run is prep -> counter reset -> persistent kernel -> finalize kernels, and
// can be captured once into a CUDA graph and replayed.  An autotuner picks
// the grid size, the item order and the fusion width by timing candidates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/qtm.h"
#include "../../include/qtm_debug.h"
#include "device.h"
#include "tile.cuh"
#include "tile_cpx.cuh"

namespace qtm {

struct CircDev {
    int n, sq, K, tiles, n_in, P, M, n_runs, n_rots, n_terms;
    int fwd_begin, n_fwd, rev_begin, n_rev;
    int ops_off, diag_off, phases_off, slots_off, runs_off, rots_off, prq_off, ents_off, terms_off,
        amap_off, wptr_off, wrots_off, xptr_off, xrots_off;
    long long x_off, w_off, gE_off, E_off, gx_off, gw_off;   // elements of the packed user buffers
    long long mats_off, tabs_off;                            // complex elements of the workspace
    long long Epart_off, Gpart_off, abar_off, gwws_off;      // doubles
    long long state_off;                                     // complex elements (tiles > 1 only)
};

struct WorkItem {
    int c, b;
};

// One unit of work: a whole item (step < 0) or one tile of one pass of a
// tiled item (step = pass index, forward passes then reverse passes).
struct Task {
    int item, step, tile;
};

// Which passes one launch runs.  MODE_BOTH keeps a one-tile item's state in
// shared memory from its forward into its reverse pass; MODE_FWD stores every
// item's final state in the workspace and MODE_ADJ starts from it.
enum { MODE_BOTH = 0, MODE_FWD = 1, MODE_ADJ = 2 };

struct MultiArgs {
    int n_items, B;
    const WorkItem *items;
    const CircDev *circ;
    const PassDesc *passes;
    const DevOp *ops;
    const DiagPair *diag;
    const DevPhase *phases;
    const int32_t *slot_runs;
    const Run *runs;
    const Rot *rots;
    const int32_t *prq;
    const Ent *ents;
    const Term *terms;
    const MaskTerm *amap;
    const int32_t *w_ptr, *w_rots, *x_ptr, *x_rots;
    const void *x, *w, *gE;
    void *E, *gx, *gw;
    void *mats, *tabs, *state;
    double *Epart, *Gpart, *abar, *gwws;
    unsigned *counter;
    unsigned *status;             // bit 0: deadline hit; bit 1: bad index (both skip work)
    const Task *tasks;
    int n_tasks;
    unsigned long long wait_ns;   // limit of one task's wait for its item's previous pass
    unsigned *abort;              // set when a wait of this run gave up: the others stop waiting
    unsigned *done;               // [n_items] tile tasks completed per item (split schedule)
    int n_circ, n_passes, n_ops_total, n_phases_total;
    int mode;                     // MODE_BOTH, MODE_FWD (forward passes only), MODE_ADJ (reverse only)
    // shared-memory layout bounds (max over all passes of all circuits)
    int max_slots, max_terms, max_M, max_ents, max_sq;
};

namespace {

constexpr unsigned long long kMultiDeadlineNs = 20000000000ull;   // 20 s per CTA
constexpr unsigned long long kMultiWaitNs = 10000000000ull;       // default limit of one task's wait

template <typename R>
__device__ __forceinline__ TileJob make_job(const MultiArgs &m, const CircDev &cd, const PassDesc &pd,
                                            int b, uint32_t base)
{
    TileJob j;
    j.K = pd.K; j.l = pd.l; j.h = pd.h; j.m = pd.m; j.sq = cd.sq;
    j.T = 1 << (pd.K - 4);
    j.base = base;
    j.ops = m.ops + cd.ops_off;
    j.diag = m.diag + cd.diag_off;
    j.phases = m.phases + cd.phases_off;
    j.phase_begin = pd.phase_begin; j.phase_end = pd.phase_end;
    j.slot_runs = m.slot_runs + cd.slots_off + pd.slot_begin;
    j.nslots = pd.slot_end - pd.slot_begin;
    j.mats = static_cast<const Cx<R> *>(m.mats) + cd.mats_off + (size_t)b * cd.n_runs * 4;
    j.tabs = static_cast<const Cx<R> *>(m.tabs) + cd.tabs_off + (size_t)b * ((cd.sq + 3) >> 2) * 16;
    j.prefix_ents = m.ents + cd.ents_off + pd.ents_begin;
    j.analytic_ents = pd.phi_src == SRC_ANALYTIC ? pd.analytic_ents : 0;
    j.amap = m.amap + cd.amap_off + (pd.amap_lin >= 0 ? pd.amap_begin : 0);
    j.amap_lin = pd.phi_src == SRC_ANALYTIC ? pd.amap_lin : -1;
    j.amap_quad = pd.amap_quad;
    j.amap_dlin = pd.amap_dlin;
    j.terms = m.terms + cd.terms_off;
    j.n_terms = cd.n_terms;
    j.M = cd.M;
    j.gE = m.gE ? static_cast<const R *>(m.gE) + cd.gE_off + (size_t)b * cd.M : nullptr;
    j.phi_src = pd.phi_src;
    j.lam_src = pd.lam_src;
    return j;
}

template <typename R>
__device__ __forceinline__ uint32_t tile_base(const PassDesc &pd, int tile)
{
    const int gapbits = pd.h - pd.l;
    const uint32_t gap = tile & ((1u << gapbits) - 1u);
    const uint32_t rest = tile >> gapbits;
    return (gap << pd.l) | (rest << (pd.h + pd.m));
}

__device__ __forceinline__ Cx<float> ld_cg(const Cx<float> *p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ Cx<double> ld_cg(const Cx<double> *p)
{
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}

// global <-> shared tile copies (the item's state is L2-resident).  Loads
// bypass L1: with the split schedule the tile may have been written by a CTA
// on another SM.
template <typename R>
__device__ __forceinline__ void load_tile(const TileJob &j, Cx<R> *dst, const Cx<R> *src)
{
    const int E = 1 << j.K;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint32_t y = j.base | ((uint32_t)e & ((1u << j.l) - 1u)) | (((uint32_t)e >> j.l) << j.h);
        dst[swz<R>(e)] = ld_cg(src + y);
    }
}

template <typename R>
__device__ __forceinline__ void store_tile(const TileJob &j, const Cx<R> *src, Cx<R> *dst)
{
    const int E = 1 << j.K;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint32_t y = j.base | ((uint32_t)e & ((1u << j.l) - 1u)) | (((uint32_t)e >> j.l) << j.h);
        dst[y] = src[swz<R>(e)];
    }
}

template <typename R>
__global__ void k_multi_prep(const MultiArgs m)
{
    __shared__ double2 ufac[2 * 32];
    const WorkItem wi = m.items[blockIdx.x];
    const CircDev cd = m.circ[wi.c];
    prep_sample<R>(m.runs + cd.runs_off, m.rots + cd.rots_off, m.prq + cd.prq_off, cd.n_runs, cd.n, cd.sq,
                   static_cast<const R *>(m.x) + cd.x_off + (size_t)wi.b * cd.n_in,
                   static_cast<const R *>(m.w) + cd.w_off,
                   static_cast<Cx<R> *>(m.mats) + cd.mats_off + (size_t)wi.b * cd.n_runs * 4,
                   static_cast<Cx<R> *>(m.tabs) + cd.tabs_off + (size_t)wi.b * ((cd.sq + 3) >> 2) * 16, ufac,
                   nullptr);
}

// One tile of one pass: load (or generate) phi / lam, run the pass's phases,
// write the partial sums and store the tile.  `resident`: the item's whole
// state is this one tile and stays in shared memory from pass to pass (no
// global loads or stores).  Ends with a barrier.
template <typename R>
__device__ __forceinline__ void run_tile(const MultiArgs &m, const TileSmem<R> &S, const CircDev &cd, const PassDesc &pd,
                                         bool rev, bool resident, int b, int t, Cx<R> *gphi, Cx<R> *glam,
                                         double *Epart_b, double *Gpart_b)
{
    const TileJob j = make_job<R>(m, cd, pd, b, tile_base<R>(pd, t));
    const int nw = (j.T + 31) >> 5;
    if (rev) stage_tables<R, true>(j, S, nw);
    else stage_tables<R, false>(j, S, nw);
    if (!resident) {
        if (pd.phi_src == SRC_LOAD) load_tile<R>(j, S.phi, gphi);
        if (rev && pd.lam_src == SRC_LOAD) load_tile<R>(j, S.lam, glam);
    }
    __syncthreads();
    if (pd.phi_src == SRC_ANALYTIC) fill_analytic<R>(j, S);
    __syncthreads();
    if (rev) {
        run_phases_any<R, true>(j, S, pd.lam_src == SRC_LOAD);
        write_partials<R, true>(j, S, nw, false, nullptr, Gpart_b, cd.tiles, t);
    } else {
        run_phases_any<R, false>(j, S, false);
        write_partials<R, false>(j, S, nw, pd.has_expval != 0, Epart_b + (size_t)t * cd.M, nullptr, cd.tiles, t);
    }
    if (!resident) {
        if (pd.store_phi) store_tile<R>(j, S.phi, gphi);
        if (rev && pd.store_lam) store_tile<R>(j, S.lam, glam);
    }
    __syncthreads();
}

// MINB: CTAs per SM the register budget is compiled for (1: no spills, 2: more
// resident warps); the autotuner's ctas_per_sm picks the variant.
template <typename R, int MINB>
__global__ void __launch_bounds__(256, MINB) k_multi(const MultiArgs m)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ int s_item;
    const Layout L = make_layout(kMaxTileQubits, (int)sizeof(Cx<R>), true, m.max_slots, m.max_terms,
                                 m.max_M, m.max_sq, m.max_ents, 8, (int)sizeof(R));
    const TileSmem<R> S = carve<R>(smem, L);
    const unsigned long long t_start = global_ns();
    for (;;) {
        if (threadIdx.x == 0) {
            int it = (int)atomicAdd(m.counter, 1u);
            if (global_ns() - t_start > kMultiDeadlineNs) {   // self-check: a run never takes this long
                atomicOr(m.status, 1u);
                it = m.n_tasks;
            }
            if (*(volatile unsigned *)m.abort) it = m.n_tasks;   // a wait of this run gave up: drain
            s_item = it;
        }
        __syncthreads();
        const int task = s_item;
        __syncthreads();
        if (task >= m.n_tasks || task < 0) return;
        const Task tk = m.tasks[task];
        if (tk.item < 0 || tk.item >= m.n_items) {
            if (threadIdx.x == 0) atomicOr(m.status, 2u);
            continue;
        }
        const WorkItem wi = m.items[tk.item];
        if (wi.c < 0 || wi.c >= m.n_circ) {
            if (threadIdx.x == 0) atomicOr(m.status, 2u);
            continue;
        }
        const CircDev cd = m.circ[wi.c];
        if (cd.fwd_begin < 0 || cd.rev_begin + cd.n_rev > m.n_passes || cd.tiles < 1 || cd.tiles > (1 << 18) ||
            wi.b < 0 || wi.b >= m.B || tk.step >= cd.n_fwd + cd.n_rev || tk.tile < 0 || tk.tile >= cd.tiles ||
            (tk.step >= 0 && cd.tiles == 1) ||
            (tk.step >= 0 && m.mode == MODE_FWD && tk.step >= cd.n_fwd) ||
            (tk.step >= 0 && m.mode == MODE_ADJ && tk.step < cd.n_fwd)) {
            if (threadIdx.x == 0) atomicOr(m.status, 2u);
            continue;
        }
        const int b = wi.b;
        double *Epart_b = m.Epart + cd.Epart_off + (size_t)b * cd.tiles * cd.M;
        double *Gpart_b = m.Gpart + cd.Gpart_off + (size_t)b * cd.n_runs * cd.tiles * 3;
        Cx<R> *gphi = static_cast<Cx<R> *>(m.state) + cd.state_off + (size_t)b * (2ull << cd.sq);
        Cx<R> *glam = gphi + (1ull << cd.sq);
        if (tk.step >= 0) {
            // one tile of one pass: wait (bounded) for every tile of the item's
            // previous pass, run it, then count it done
            if (threadIdx.x == 0) {
                // the done counters start at zero in every launch: an adjoint-only
                // launch counts its reverse passes from the first one
                const int first = m.mode == MODE_ADJ ? cd.n_fwd : 0;
                const unsigned need = (unsigned)(tk.step - first) * (unsigned)cd.tiles;
                const unsigned long long t0 = global_ns();
                unsigned have;
                bool failed = false;
                for (;;) {
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(have) : "l"(m.done + tk.item) : "memory");
                    if (have >= need) break;
                    // give up after the limit, or at once when another wait already has
                    if (global_ns() - t0 > m.wait_ns || *(volatile unsigned *)m.abort) {
                        failed = true;
                        break;
                    }
                    __nanosleep(64);
                }
                if (failed) {
                    atomicOr(m.status, 1u);
                    atomicExch(m.abort, 1u);
                }
                s_item = failed ? -1 : 0;
            }
            __syncthreads();
            const bool ready = s_item == 0;
            __syncthreads();
            if (!ready) continue;
        }
        // a whole item (the launch's passes, every tile, in order) or one
        // (pass, tile) task.  Only a launch that runs both directions keeps a
        // one-tile item's state in shared memory between its passes; the
        // one-direction launches store it to (forward) or load it from
        // (adjoint) the item's state buffer as the pass descriptors say.
        const bool whole = tk.step < 0;
        const int kb = m.mode == MODE_ADJ ? cd.n_fwd : 0;
        const int ke = m.mode == MODE_FWD ? cd.n_fwd : cd.n_fwd + cd.n_rev;
        const int k0 = whole ? kb : tk.step, k1 = whole ? ke : tk.step + 1;
        const int t0 = whole ? 0 : tk.tile, t1 = whole ? cd.tiles : tk.tile + 1;
        const bool resident = cd.tiles == 1 && m.mode == MODE_BOTH;
        for (int k = k0; k < k1; ++k) {
            const bool rev = k >= cd.n_fwd;
            const PassDesc pd = m.passes[rev ? cd.rev_begin + (k - cd.n_fwd) : cd.fwd_begin + k];
            for (int t = t0; t < t1; ++t)
                run_tile<R>(m, S, cd, pd, rev, resident, b, t, gphi, glam, Epart_b, Gpart_b);
        }
        if (!whole) {
            __threadfence();   // this tile's state writes before the count (release)
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(m.done + tk.item, 1u);
        }
    }
}

template <typename R>
__global__ void k_multi_expval(const MultiArgs m)
{
    const WorkItem wi = m.items[blockIdx.x];
    const CircDev cd = m.circ[wi.c];
    const double *Ep = m.Epart + cd.Epart_off + (size_t)wi.b * cd.tiles * cd.M;
    R *E = static_cast<R *>(m.E) + cd.E_off + (size_t)wi.b * cd.M;
    for (int k = threadIdx.x; k < cd.M; k += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < cd.tiles; ++t) s += Ep[(size_t)t * cd.M + k];
        E[k] = (R)s;
    }
}

template <typename R>
__global__ void k_multi_grad(const MultiArgs m)
{
    const WorkItem wi = m.items[blockIdx.x];
    const CircDev cd = m.circ[wi.c];
    const int b = wi.b;
    grad_finalize_sample<R>(m.runs + cd.runs_off, m.rots + cd.rots_off, cd.n_runs, m.w_ptr + cd.wptr_off,
                            m.w_rots + cd.wrots_off, m.x_ptr + cd.xptr_off, m.x_rots + cd.xrots_off,
                            cd.P, cd.n_in, static_cast<const R *>(m.x) + cd.x_off + (size_t)b * cd.n_in,
                            static_cast<const R *>(m.w) + cd.w_off,
                            m.Gpart + cd.Gpart_off + (size_t)b * cd.n_runs * cd.tiles * 3, cd.tiles,
                            m.abar + cd.abar_off + (size_t)b * cd.n_rots,
                            static_cast<R *>(m.gx) + cd.gx_off + (size_t)b * cd.n_in, nullptr,
                            m.gwws + cd.gwws_off + (size_t)b * cd.P, nullptr);
}

// grad_w of circuit c = sum over its samples, fixed order; one thread per weight
template <typename R>
__global__ void k_multi_gw(const MultiArgs m, const int *wcirc, int total_w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total_w) return;
    const int c = wcirc[i];
    const CircDev cd = m.circ[c];
    const int j = (int)(i - cd.gw_off);
    double s = 0.0;
    for (int b = 0; b < m.B; ++b) s += m.gwws[cd.gwws_off + (size_t)b * cd.P + j];
    static_cast<R *>(m.gw)[i] = (R)s;
}

}  // namespace

}  // namespace qtm

using namespace qtm;

struct qtm_multi {
    int dtype = QTM_C64, B = 1;
    std::vector<std::vector<qtm_gate>> gates;
    std::vector<std::vector<qtm_zterm>> terms;
    std::vector<qtm_circuit> desc;
    std::vector<Plan> plans;
    qtm_multi_config cfg{2, 0, kMaxRunLen, 1};
    // host-side images
    std::vector<CircDev> circ;
    std::vector<WorkItem> items;
    std::vector<Task> tasks;                  // MODE_BOTH (qtm_multi_run)
    std::vector<Task> tasks_fwd, tasks_adj;   // MODE_FWD, MODE_ADJ
    std::vector<PassDesc> passes;
    std::vector<DevOp> ops;
    std::vector<DiagPair> diag;
    std::vector<DevPhase> phases;
    std::vector<int32_t> slots, prq, wptr, wrots, xptr, xrots, wcirc;
    std::vector<Run> runs;
    std::vector<Rot> rots;
    std::vector<Ent> ents;
    std::vector<Term> tms;
    std::vector<MaskTerm> amap;
    std::vector<long long> off[6];
    long long n_mats = 0, n_tabs = 0, n_epart = 0, n_gpart = 0, n_abar = 0, n_gwws = 0, n_state = 0;
    int max_slots = 1, max_terms = 1, max_M = 1, max_ents = 1, max_sq = 4;
    size_t smem = 0;
    unsigned long long wait_ns = kMultiWaitNs;
    bool injected = false;   // task list replaced by qtm_debug_multi_inject
    // device
    int device = -1;
    bool dirty = true;
    void *dev_block = nullptr;      // all tables in one allocation
    void *d_ws = nullptr;           // workspace (mats, tabs, state)
    double *d_dbl = nullptr;        // Epart, Gpart, abar, gwws
    unsigned *d_counter = nullptr;   // [0] status, [1] task counter, [2] abort, [3 ..] per-item done counters
    MultiArgs args{};
    const Task *dev_tasks[3] = {nullptr, nullptr, nullptr};   // per mode
    int n_tasks[3] = {0, 0, 0};
    // graph cache: qtm_multi_run, forward, adjoint, adjoint with recompute
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraph_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    const void *gkey[4][6] = {};
    const int *wcirc_dev = nullptr;
    // the states a qtm_multi_forward left for qtm_multi_adjoint
    bool fwd_valid = false;
    const void *fwd_x = nullptr, *fwd_w = nullptr;
    std::string err;
};

namespace {

void release_graph(qtm_multi *m)
{
    for (int k = 0; k < 4; ++k) {
        if (m->gexec[k]) cudaGraphExecDestroy(m->gexec[k]);
        if (m->graph[k]) cudaGraphDestroy(m->graph[k]);
        m->gexec[k] = nullptr;
        m->graph[k] = nullptr;
        std::fill(std::begin(m->gkey[k]), std::end(m->gkey[k]), nullptr);
    }
}

void release_device(qtm_multi *m)
{
    release_graph(m);
    if (m->dev_block) cudaFree(m->dev_block);
    if (m->d_ws) cudaFree(m->d_ws);
    if (m->d_dbl) cudaFree(m->d_dbl);
    if (m->d_counter) cudaFree(m->d_counter);
    m->dev_block = m->d_ws = nullptr;
    m->d_dbl = nullptr;
    m->d_counter = nullptr;
    m->dirty = true;
    m->fwd_valid = false;
}

// Estimated cost of an item's passes in a launch of the given mode.
double item_cost(const Plan &P, int mode = MODE_BOTH)
{
    double fb, ab, ff, af;
    plan_costs(P, fb, ab, ff, af);
    const double f = ff + 4.0 * fb, a = af + 4.0 * ab;
    return mode == MODE_FWD ? f : mode == MODE_ADJ ? a : f + a;
}

// The task list of one launch mode (MODE_BOTH: every pass; MODE_FWD: the
// forward passes; MODE_ADJ: the reverse passes).  split = 0: one whole task
// per item, in item order.  split = 1: a tiled item becomes one task per
// (pass, tile).  With order 0 the tasks are listed highest level first (a
// list schedule): a task's level is the estimated time from its start to the
// end of its item's chain in this launch, i.e. the item's cost for a whole
// task and (passes left) x (cost of one pass's tile) for a tile task, so the
// long chains of the largest circuits start first and whole small items fill
// in between their passes.  With order 1 they are listed pass by pass: every
// item's first pass (whole items there too), then every item's second pass,
// ...  Either way a tile task comes after every tile of its item's previous
// pass of the launch, which the kernel's waits rely on.
std::vector<Task> build_tasks(const qtm_multi *m, int mode)
{
    std::vector<Task> out;
    const int ni = (int)m->items.size();
    if (m->cfg.split == 0) {
        for (int i = 0; i < ni; ++i) out.push_back({i, -1, 0});
        return out;
    }
    struct Key {
        double level;
        int item, step, tile, rank;   // rank: pass index within this launch
    };
    std::vector<Key> keys;
    for (int i = 0; i < ni; ++i) {
        const Plan &P = m->plans[m->items[i].c];
        const int nf = (int)P.fwd.size(), nr = (int)P.rev.size();
        const int kb = mode == MODE_ADJ ? nf : 0;
        const int ke = mode == MODE_FWD ? nf : nf + nr;
        const int tiles = P.tiles_per_sample, steps = ke - kb;
        const double cost = item_cost(P, mode);
        if (tiles <= 1 || nf + nr < 1) {
            keys.push_back({cost, i, -1, 0, 0});
            continue;
        }
        for (int k = kb; k < ke; ++k)
            for (int t = 0; t < tiles; ++t)
                keys.push_back({(double)(ke - k) * cost / ((double)steps * tiles), i, k, t, k - kb});
    }
    if (m->cfg.order == 0)
        std::sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) {
            if (a.level != b.level) return a.level > b.level;
            if (a.item != b.item) return a.item < b.item;
            if (a.step != b.step) return a.step < b.step;
            return a.tile < b.tile;
        });
    else
        std::stable_sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) { return a.rank < b.rank; });
    for (const Key &k : keys) out.push_back({k.item, k.step, k.tile});
    return out;
}

// (Re)plan every circuit with the current fusion width and lay out the tables.
qtm_status plan_all(qtm_multi *m)
{
    const int nc = (int)m->desc.size();
    m->plans.assign(nc, Plan());
    for (int c = 0; c < nc; ++c) {
        const qtm_circuit &d = m->desc[c];
        std::string err;
        PlanOptions opt;
        opt.max_run = m->cfg.fuse_width;   // greedy phases: the persistent kernel interprets its op records
        qtm_status st = make_plan(d.n_qubits, m->gates[c].data(), (int)m->gates[c].size(), m->terms[c].data(),
                                  (int)m->terms[c].size(), d.n_obs, d.n_weights, d.n_inputs, m->dtype,
                                  QTM_PATH_FUSED, m->plans[c], err, opt);
        if (st != QTM_OK) {
            std::ostringstream s;
            s << "circuit " << c << ": " << err;
            m->err = s.str();
            return st;
        }
    }
    m->circ.assign(nc, CircDev{});
    m->passes.clear(); m->ops.clear(); m->diag.clear(); m->phases.clear(); m->slots.clear();
    m->prq.clear(); m->wptr.clear(); m->wrots.clear(); m->xptr.clear(); m->xrots.clear();
    m->runs.clear(); m->rots.clear(); m->ents.clear(); m->tms.clear(); m->amap.clear(); m->wcirc.clear();
    for (auto &o : m->off) o.assign(nc + 1, 0);
    long long mats = 0, tabs = 0, ep = 0, gp = 0, ab = 0, gw = 0, st = 0;
    m->max_slots = m->max_terms = m->max_M = m->max_ents = 1;
    m->max_sq = 4;
    for (int c = 0; c < nc; ++c) {
        const Plan &P = m->plans[c];
        CircDev &d = m->circ[c];
        d.n = P.n; d.sq = P.state_qubits; d.K = P.K; d.tiles = P.tiles_per_sample;
        d.n_in = P.n_inputs; d.P = P.n_weights; d.M = P.n_obs;
        d.n_runs = (int)P.runs.size(); d.n_rots = (int)P.rots.size(); d.n_terms = (int)P.terms.size();
        d.fwd_begin = (int)m->passes.size(); d.n_fwd = (int)P.fwd.size();
        m->passes.insert(m->passes.end(), P.fwd.begin(), P.fwd.end());
        d.rev_begin = (int)m->passes.size(); d.n_rev = (int)P.rev.size();
        m->passes.insert(m->passes.end(), P.rev.begin(), P.rev.end());
        for (auto *v : {&P.fwd, &P.rev})
            for (const auto &pd : *v) {
                m->max_slots = std::max(m->max_slots, pd.slot_end - pd.slot_begin);
                if (pd.phi_src == SRC_ANALYTIC) m->max_ents = std::max(m->max_ents, pd.analytic_ents);
            }
        m->max_terms = std::max(m->max_terms, (int)P.terms.size());
        m->max_M = std::max(m->max_M, P.n_obs);
        m->max_sq = std::max(m->max_sq, P.state_qubits);
#define APPEND(field, dst, src) d.field = (int)dst.size(); dst.insert(dst.end(), src.begin(), src.end())
        APPEND(ops_off, m->ops, P.ops);
        APPEND(diag_off, m->diag, P.diag_pairs);
        APPEND(phases_off, m->phases, P.phases);
        APPEND(slots_off, m->slots, P.slot_runs);
        APPEND(runs_off, m->runs, P.runs);
        APPEND(rots_off, m->rots, P.rots);
        APPEND(prq_off, m->prq, P.prefix_run_of_q);
        APPEND(ents_off, m->ents, P.pass_ents);
        APPEND(terms_off, m->tms, P.terms);
        APPEND(amap_off, m->amap, P.amap_terms);
        APPEND(wptr_off, m->wptr, P.w_ptr);
        APPEND(wrots_off, m->wrots, P.w_rots);
        APPEND(xptr_off, m->xptr, P.x_ptr);
        APPEND(xrots_off, m->xrots, P.x_rots);
#undef APPEND
        const long long B = m->B;
        d.x_off = m->off[QTM_MULTI_X][c]; m->off[QTM_MULTI_X][c + 1] = d.x_off + B * P.n_inputs;
        d.w_off = m->off[QTM_MULTI_W][c]; m->off[QTM_MULTI_W][c + 1] = d.w_off + P.n_weights;
        d.gE_off = m->off[QTM_MULTI_GE][c]; m->off[QTM_MULTI_GE][c + 1] = d.gE_off + B * P.n_obs;
        d.E_off = m->off[QTM_MULTI_E][c]; m->off[QTM_MULTI_E][c + 1] = d.E_off + B * P.n_obs;
        d.gx_off = m->off[QTM_MULTI_GX][c]; m->off[QTM_MULTI_GX][c + 1] = d.gx_off + B * P.n_inputs;
        d.gw_off = m->off[QTM_MULTI_GW][c]; m->off[QTM_MULTI_GW][c + 1] = d.gw_off + P.n_weights;
        for (int j = 0; j < P.n_weights; ++j) m->wcirc.push_back(c);
        d.mats_off = mats; mats += B * 4 * std::max(1, d.n_runs);
        d.tabs_off = tabs; tabs += B * 16 * ((d.sq + 3) / 4);
        d.Epart_off = ep; ep += B * d.tiles * std::max(1, d.M);
        d.Gpart_off = gp; gp += B * std::max(1, d.n_runs) * d.tiles * 3;
        d.abar_off = ab; ab += B * std::max(1, d.n_rots);
        d.gwws_off = gw; gw += B * std::max(1, d.P);
        d.state_off = st;
        st += B * (2ll << d.sq);   // phi and lam; one-tile items use them between split launches
    }
    m->n_mats = mats; m->n_tabs = tabs; m->n_epart = ep; m->n_gpart = gp; m->n_abar = ab; m->n_gwws = gw;
    m->n_state = st;
    // work items, costliest first (or as given)
    m->items.clear();
    for (int c = 0; c < nc; ++c)
        for (int b = 0; b < m->B; ++b) m->items.push_back({c, b});
    if (m->cfg.order == 0) {
        std::vector<double> cost(nc);
        for (int c = 0; c < nc; ++c) cost[c] = item_cost(m->plans[c]);
        std::stable_sort(m->items.begin(), m->items.end(),
                         [&](const WorkItem &a, const WorkItem &b) { return cost[a.c] > cost[b.c]; });
    }
    m->tasks = build_tasks(m, MODE_BOTH);
    m->tasks_fwd = build_tasks(m, MODE_FWD);
    m->tasks_adj = build_tasks(m, MODE_ADJ);
    m->wait_ns = kMultiWaitNs;
    m->injected = false;
    const int csize = elem_bytes(m->dtype);
    const Layout L = make_layout(kMaxTileQubits, csize, true, m->max_slots, m->max_terms, m->max_M,
                                 m->max_sq, m->max_ents, 8, csize / 2);
    m->smem = (size_t)L.total + 1024;
    if (m->smem > 232448) { m->err = "tables exceed shared memory"; return QTM_EUNSUPPORTED; }
    m->dirty = true;
    return QTM_OK;
}

template <typename T>
size_t put(std::vector<unsigned char> &blob, const std::vector<T> &v)
{
    size_t at = (blob.size() + 255) & ~size_t(255);
    blob.resize(at + sizeof(T) * std::max<size_t>(1, v.size()));
    if (!v.empty()) std::memcpy(blob.data() + at, v.data(), sizeof(T) * v.size());
    return at;
}

qtm_status upload(qtm_multi *m)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { m->err = "no CUDA device"; return QTM_ECUDA; }
    if (!m->dirty && dev == m->device) return QTM_OK;
    release_device(m);
    std::vector<unsigned char> blob;
    const size_t o_tasks = put(blob, m->tasks);
    const size_t o_tasks_fwd = put(blob, m->tasks_fwd), o_tasks_adj = put(blob, m->tasks_adj);
    const size_t o_items = put(blob, m->items), o_circ = put(blob, m->circ), o_passes = put(blob, m->passes),
                 o_ops = put(blob, m->ops), o_diag = put(blob, m->diag), o_phases = put(blob, m->phases),
                 o_slots = put(blob, m->slots), o_runs = put(blob, m->runs), o_rots = put(blob, m->rots),
                 o_prq = put(blob, m->prq), o_ents = put(blob, m->ents), o_terms = put(blob, m->tms),
                 o_amap = put(blob, m->amap), o_wptr = put(blob, m->wptr), o_wrots = put(blob, m->wrots),
                 o_xptr = put(blob, m->xptr), o_xrots = put(blob, m->xrots), o_wcirc = put(blob, m->wcirc);
    const size_t csize = elem_bytes(m->dtype);
    if (cudaMalloc(&m->dev_block, blob.size()) != cudaSuccess ||
        cudaMemcpy(m->dev_block, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        release_device(m);
        m->err = "table upload failed";
        return QTM_ENOMEM;
    }
    const size_t ws = csize * (size_t)(m->n_mats + m->n_tabs + m->n_state);
    const size_t nd = (size_t)(m->n_epart + m->n_gpart + m->n_abar + m->n_gwws);
    if (cudaMalloc(&m->d_ws, ws ? ws : 16) != cudaSuccess || cudaMalloc(&m->d_dbl, 8 * (nd ? nd : 1)) != cudaSuccess ||
        cudaMalloc(&m->d_counter, (3 + m->items.size()) * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(m->d_counter, 0, (3 + m->items.size()) * sizeof(unsigned)) != cudaSuccess) {
        release_device(m);
        m->err = "workspace allocation failed";
        return QTM_ENOMEM;
    }
    unsigned char *db = static_cast<unsigned char *>(m->dev_block);
    MultiArgs &a = m->args;
    a = MultiArgs{};
    a.n_items = (int)m->items.size();
    a.B = m->B;
    a.items = reinterpret_cast<const WorkItem *>(db + o_items);
    m->dev_tasks[MODE_BOTH] = reinterpret_cast<const Task *>(db + o_tasks);
    m->dev_tasks[MODE_FWD] = reinterpret_cast<const Task *>(db + o_tasks_fwd);
    m->dev_tasks[MODE_ADJ] = reinterpret_cast<const Task *>(db + o_tasks_adj);
    m->n_tasks[MODE_BOTH] = (int)m->tasks.size();
    m->n_tasks[MODE_FWD] = (int)m->tasks_fwd.size();
    m->n_tasks[MODE_ADJ] = (int)m->tasks_adj.size();
    a.mode = MODE_BOTH;
    a.tasks = m->dev_tasks[MODE_BOTH];
    a.n_tasks = m->n_tasks[MODE_BOTH];
    a.wait_ns = m->wait_ns;
    a.circ = reinterpret_cast<const CircDev *>(db + o_circ);
    a.passes = reinterpret_cast<const PassDesc *>(db + o_passes);
    a.ops = reinterpret_cast<const DevOp *>(db + o_ops);
    a.diag = reinterpret_cast<const DiagPair *>(db + o_diag);
    a.phases = reinterpret_cast<const DevPhase *>(db + o_phases);
    a.slot_runs = reinterpret_cast<const int32_t *>(db + o_slots);
    a.runs = reinterpret_cast<const Run *>(db + o_runs);
    a.rots = reinterpret_cast<const Rot *>(db + o_rots);
    a.prq = reinterpret_cast<const int32_t *>(db + o_prq);
    a.ents = reinterpret_cast<const Ent *>(db + o_ents);
    a.terms = reinterpret_cast<const Term *>(db + o_terms);
    a.amap = reinterpret_cast<const MaskTerm *>(db + o_amap);
    a.w_ptr = reinterpret_cast<const int32_t *>(db + o_wptr);
    a.w_rots = reinterpret_cast<const int32_t *>(db + o_wrots);
    a.x_ptr = reinterpret_cast<const int32_t *>(db + o_xptr);
    a.x_rots = reinterpret_cast<const int32_t *>(db + o_xrots);
    unsigned char *wsb = static_cast<unsigned char *>(m->d_ws);
    a.mats = wsb;
    a.tabs = wsb + csize * m->n_mats;
    a.state = wsb + csize * (m->n_mats + m->n_tabs);
    a.Epart = m->d_dbl;
    a.Gpart = a.Epart + m->n_epart;
    a.abar = a.Gpart + m->n_gpart;
    a.gwws = a.abar + m->n_abar;
    a.status = m->d_counter;
    a.counter = m->d_counter + 1;
    a.abort = m->d_counter + 2;
    a.done = m->d_counter + 3;
    a.n_circ = (int)m->circ.size();
    a.n_passes = (int)m->passes.size();
    a.n_ops_total = (int)m->ops.size();
    a.n_phases_total = (int)m->phases.size();
    a.max_slots = m->max_slots; a.max_terms = m->max_terms; a.max_M = m->max_M;
    a.max_ents = m->max_ents; a.max_sq = m->max_sq;
    m->wcirc_dev = reinterpret_cast<const int *>(db + o_wcirc);
    m->device = dev;
    m->dirty = false;
    return QTM_OK;
}

}  // namespace

namespace {

// One launch sequence.  MODE_BOTH: prep, forward + reverse passes, expectation
// values (when with_E) and gradients; MODE_FWD: prep, forward passes,
// expectation values; MODE_ADJ: reverse passes from the stored states and
// gradients (the prep tables of the forward are reused).
template <typename R>
cudaError_t enqueue_t(qtm_multi *m, cudaStream_t s, int mode, bool with_E)
{
    MultiArgs a = m->args;
    a.mode = mode;
    a.tasks = m->dev_tasks[mode];
    a.n_tasks = m->n_tasks[mode];
    const int ni = a.n_items;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, (2 + (size_t)ni) * sizeof(unsigned), s);   // counter, abort, done[]
    if (e != cudaSuccess) return e;
    if (mode != MODE_ADJ) k_multi_prep<R><<<ni, 128, 0, s>>>(a);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    const int cps = m->cfg.ctas_per_sm >= 2 ? 2 : 1;
    const int grid = std::max(1, std::min(a.n_tasks, cps * sms));
    if (cps == 2) k_multi<R, 2><<<grid, 256, m->smem, s>>>(a);
    else k_multi<R, 1><<<grid, 256, m->smem, s>>>(a);
    if (mode == MODE_FWD || (mode == MODE_BOTH && with_E)) k_multi_expval<R><<<ni, 32, 0, s>>>(a);
    if (mode != MODE_FWD) {
        k_multi_grad<R><<<ni, 256, 0, s>>>(a);
        const int tw = (int)m->wcirc.size();
        if (tw > 0) k_multi_gw<R><<<(tw + 255) / 256, 256, 0, s>>>(a, m->wcirc_dev, tw);
    }
    return cudaGetLastError();
}

cudaError_t set_smem_attr(qtm_multi *m)
{
    const int v = (int)m->smem;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if (m->dtype == QTM_C128) {
        e = cudaFuncSetAttribute(k_multi<double, 1>, at, v);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_multi<double, 2>, at, v);
    } else {
        e = cudaFuncSetAttribute(k_multi<float, 1>, at, v);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_multi<float, 2>, at, v);
    }
    return e;
}

cudaError_t enqueue(qtm_multi *m, cudaStream_t s, int mode, bool with_E)
{
    return m->dtype == QTM_C128 ? enqueue_t<double>(m, s, mode, with_E) : enqueue_t<float>(m, s, mode, with_E);
}

// Enqueue one launch sequence of `mode` (graph slot: 0 run, 1 forward, 2
// adjoint, 3 adjoint with recompute).  Pointers not used by the mode are NULL.
qtm_status run_impl(qtm_multi *m, const void *x, const void *w, const void *gE, void *E, void *gx, void *gw,
                    int flags, cudaStream_t s, int mode = MODE_BOTH, int slot = 0)
{
    qtm_status st = upload(m);
    if (st != QTM_OK) return st;
    if (set_smem_attr(m) != cudaSuccess) { m->err = "shared-memory attribute"; return QTM_ECUDA; }
    MultiArgs &a = m->args;
    a.x = x; a.w = w; a.gE = gE; a.E = E; a.gx = gx; a.gw = gw;
    const bool with_E = E != nullptr;
    if (!(flags & QTM_MULTI_GRAPH)) {
        cudaError_t e = enqueue(m, s, mode, with_E);
        if (e != cudaSuccess) { m->err = cudaGetErrorString(e); return QTM_ECUDA; }
        return QTM_OK;
    }
    const void *key[6] = {x, w, gE, E, gx, gw};
    if (!m->gexec[slot] || !std::equal(std::begin(key), std::end(key), std::begin(m->gkey[slot]))) {
        if (m->gexec[slot]) cudaGraphExecDestroy(m->gexec[slot]);
        if (m->graph[slot]) cudaGraphDestroy(m->graph[slot]);
        m->gexec[slot] = nullptr;
        m->graph[slot] = nullptr;
        if (!m->cap_stream && cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            m->err = "stream creation failed";
            return QTM_ECUDA;
        }
        cudaError_t e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue(m, m->cap_stream, mode, with_E);
            e = cudaStreamEndCapture(m->cap_stream, &m->graph[slot]);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&m->gexec[slot], m->graph[slot], 0);
        if (e != cudaSuccess) {
            release_graph(m);
            m->err = std::string("graph capture: ") + cudaGetErrorString(e);
            return QTM_ECUDA;
        }
        std::copy(std::begin(key), std::end(key), std::begin(m->gkey[slot]));
    }
    cudaError_t e = cudaGraphLaunch(m->gexec[slot], s);
    if (e != cudaSuccess) { m->err = cudaGetErrorString(e); return QTM_ECUDA; }
    return QTM_OK;
}

std::string signature(const qtm_multi *m)
{
    // FNV-1a over the batch's shape: dtype, batch, every circuit's gates and terms
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](long long v) {
        for (int k = 0; k < 8; ++k) { h ^= (unsigned long long)((v >> (8 * k)) & 0xff); h *= 1099511628211ull; }
    };
    mix(m->dtype); mix(m->B); mix((long long)m->desc.size());
    for (size_t c = 0; c < m->desc.size(); ++c) {
        mix(m->desc[c].n_qubits);
        for (const auto &g : m->gates[c]) { mix(g.kind); mix(g.q0); mix(g.q1); }
        mix((long long)m->terms[c].size());
    }
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &ch : name) if (ch == '"' || ch == '\\') ch = '_';
    std::ostringstream s;
    s << std::hex << h << "@" << name;
    return s.str();
}

bool cache_lookup(const char *path, const std::string &sig, qtm_multi_config &cfg)
{
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    const std::string key = "\"signature\": \"" + sig + "\"";
    while (std::getline(f, line)) {
        if (line.find(key) == std::string::npos) continue;
        auto num = [&](const char *field) -> int {
            const std::string k = std::string("\"") + field + "\": ";
            size_t at = line.find(k);
            return at == std::string::npos ? -1 : std::atoi(line.c_str() + at + k.size());
        };
        qtm_multi_config c{num("ctas_per_sm"), num("order"), num("fuse_width"), num("split")};
        if (c.ctas_per_sm < 1 || c.order < 0 || c.fuse_width < 1 || c.split < 0 || c.split > 1) continue;
        cfg = c;
        return true;
    }
    return false;
}

void cache_store(const char *path, const std::string &sig, const qtm_multi_config &cfg, double ms)
{
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << "{\"signature\": \"" << sig << "\", \"ctas_per_sm\": " << cfg.ctas_per_sm << ", \"order\": " << cfg.order
      << ", \"fuse_width\": " << cfg.fuse_width << ", \"split\": " << cfg.split << ", \"ms\": " << ms
      << "}\n";
}

qtm_status apply_config(qtm_multi *m, const qtm_multi_config &c)
{
    const bool replan = c.fuse_width != m->cfg.fuse_width || c.order != m->cfg.order || c.split != m->cfg.split ||
                        m->injected;
    m->cfg = c;
    m->fwd_valid = false;
    release_graph(m);   // the grid size and the tables are baked into a captured graph
    if (replan) {
        release_device(m);
        return plan_all(m);
    }
    return QTM_OK;
}

}  // namespace

extern "C" {

qtm_status qtm_build_multi(const qtm_circuit *circuits, int n_circuits, int batch, int dtype, qtm_multi **out)
{
    if (!out || !circuits || n_circuits < 1 || batch < 1) return QTM_EINVAL;
    if (dtype != QTM_C64 && dtype != QTM_C128) return QTM_EINVAL;
    *out = nullptr;
    qtm_multi *m = new (std::nothrow) qtm_multi();
    if (!m) return QTM_ENOMEM;
    m->dtype = dtype;
    m->B = batch;
    for (int c = 0; c < n_circuits; ++c) {
        const qtm_circuit &d = circuits[c];
        if (d.n_gates < 0 || d.n_terms < 0 || (d.n_gates > 0 && !d.gates) || (d.n_terms > 0 && !d.terms)) {
            delete m;
            return QTM_EINVAL;
        }
        m->desc.push_back(d);
        m->gates.emplace_back(d.gates, d.gates + d.n_gates);
        m->terms.emplace_back(d.terms, d.terms + d.n_terms);
        m->desc.back().gates = m->gates.back().data();
        m->desc.back().terms = m->terms.back().data();
    }
    qtm_status st = plan_all(m);
    if (st != QTM_OK) { delete m; return st; }
    *out = m;
    return QTM_OK;
}

qtm_status qtm_multi_offsets(const qtm_multi *m, int which, int64_t *offsets)
{
    if (!m || !offsets || which < 0 || which > 5) return QTM_EINVAL;
    for (size_t i = 0; i < m->off[which].size(); ++i) offsets[i] = m->off[which][i];
    return QTM_OK;
}

qtm_status qtm_multi_run(qtm_multi *m, const void *x, const void *w, const void *gE, void *E, void *gx,
                         void *gw, int flags, void *stream)
{
    NvtxRange nvtx_range("qtm_multi_run");
    if (!m || !x || !w || !gE || !E || !gx || !gw) return QTM_EINVAL;
    if (flags & ~QTM_MULTI_GRAPH) return QTM_EINVAL;
    m->fwd_valid = false;   // the run reuses the state buffers
    return run_impl(m, x, w, gE, E, gx, gw, flags, static_cast<cudaStream_t>(stream));
}

qtm_status qtm_multi_forward(qtm_multi *m, const void *x, const void *w, void *E, int flags, void *stream)
{
    NvtxRange nvtx_range("qtm_multi_forward");
    if (!m || !x || !w || !E) return QTM_EINVAL;
    if (flags & ~QTM_MULTI_GRAPH) return QTM_EINVAL;
    m->fwd_valid = false;
    qtm_status st = run_impl(m, x, w, nullptr, E, nullptr, nullptr, flags, static_cast<cudaStream_t>(stream),
                             MODE_FWD, 1);
    if (st != QTM_OK) return st;
    m->fwd_valid = true;
    m->fwd_x = x;
    m->fwd_w = w;
    return QTM_OK;
}

qtm_status qtm_multi_adjoint(qtm_multi *m, const void *x, const void *w, const void *gE, void *gx, void *gw,
                             int flags, void *stream)
{
    NvtxRange nvtx_range("qtm_multi_adjoint");
    if (!m || !x || !w || !gE || !gx || !gw) return QTM_EINVAL;
    if (flags & ~(QTM_MULTI_GRAPH | QTM_MULTI_RECOMPUTE)) return QTM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (flags & QTM_MULTI_RECOMPUTE) {
        m->fwd_valid = false;   // the recompute overwrites the state buffers
        return run_impl(m, x, w, gE, nullptr, gx, gw, flags & QTM_MULTI_GRAPH, s, MODE_BOTH, 3);
    }
    if (!m->fwd_valid || m->fwd_x != x || m->fwd_w != w) {
        m->err = "qtm_multi_adjoint: no stored forward for these x and w (call qtm_multi_forward, or pass "
                 "QTM_MULTI_RECOMPUTE)";
        return QTM_ESTATE;
    }
    qtm_status st = run_impl(m, x, w, gE, nullptr, gx, gw, flags, s, MODE_ADJ, 2);
    m->fwd_valid = false;   // consumed
    return st;
}

qtm_status qtm_multi_tune(qtm_multi *m, const void *x, const void *w, const void *gE, void *E, void *gx,
                          void *gw, void *stream, const char *cache_path)
{
    NvtxRange nvtx_range("qtm_multi_tune");
    if (!m || !x || !w || !gE || !E || !gx || !gw) return QTM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const std::string sig = signature(m);
    qtm_multi_config cached;
    if (cache_lookup(cache_path, sig, cached)) return apply_config(m, cached);
    qtm_multi_config best = m->cfg;
    double best_ms = 1e30;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QTM_ECUDA;
    qtm_status result = QTM_OK;
    for (int fuse : {32, 3, 1})
        for (int order : {0, 1})
            for (int cps : {1, 2})
                for (int split : {0, 1}) {
                qtm_multi_config c{cps, order, fuse, split};
                qtm_status st = apply_config(m, c);
                if (st != QTM_OK) continue;
                std::vector<float> t;
                for (int rep = 0; rep < 7 && st == QTM_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    st = run_impl(m, x, w, gE, E, gx, gw, 0, s);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { st = QTM_ECUDA; break; }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep >= 2) t.push_back(ms);   // two warm-up repetitions
                }
                if (st != QTM_OK) { result = st; continue; }
                std::sort(t.begin(), t.end());
                const double med = t[t.size() / 2];
                if (med < best_ms) { best_ms = med; best = c; }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30) return result != QTM_OK ? result : QTM_ECUDA;
    qtm_status st = apply_config(m, best);
    if (st == QTM_OK) cache_store(cache_path, sig, best, best_ms);
    return st;
}

// Synchronise `stream` and report the persistent kernel's self-checks:
// QTM_ETIMEOUT if a CTA passed its deadline, QTM_EINVAL if an index check
// failed (cleared after reading).
qtm_status qtm_multi_sync(qtm_multi *m, void *stream)
{
    if (!m) return QTM_EINVAL;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return QTM_ECUDA;
    if (!m->d_counter) return QTM_OK;
    unsigned st = 0;
    if (cudaMemcpy(&st, m->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return QTM_ECUDA;
    if (!st) return QTM_OK;
    cudaMemset(m->d_counter, 0, sizeof(unsigned));
    return (st & 1u) ? QTM_ETIMEOUT : QTM_EINVAL;
}

qtm_status qtm_multi_get_config(const qtm_multi *m, qtm_multi_config *cfg)
{
    if (!m || !cfg) return QTM_EINVAL;
    *cfg = m->cfg;
    return QTM_OK;
}

qtm_status qtm_multi_set_config(qtm_multi *m, const qtm_multi_config *cfg)
{
    if (!m || !cfg || cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 8 || cfg->order < 0 || cfg->order > 1 ||
        cfg->fuse_width < 1 || cfg->fuse_width > kMaxRunLen || cfg->split < 0 || cfg->split > 1)
        return QTM_EINVAL;
    return apply_config(m, *cfg);
}

qtm_status qtm_debug_multi_tasks(const qtm_multi *m, int32_t *tasks, int capacity, int *n_tasks, int32_t *items,
                                 int item_capacity, int *n_items)
{
    if (!m || capacity < 0 || item_capacity < 0 || (capacity > 0 && !tasks) || (item_capacity > 0 && !items))
        return QTM_EINVAL;
    for (int i = 0; i < capacity && i < (int)m->tasks.size(); ++i) {
        tasks[3 * i] = m->tasks[i].item;
        tasks[3 * i + 1] = m->tasks[i].step;
        tasks[3 * i + 2] = m->tasks[i].tile;
    }
    for (int i = 0; i < item_capacity && i < (int)m->items.size(); ++i) {
        items[2 * i] = m->items[i].c;
        items[2 * i + 1] = m->items[i].b;
    }
    if (n_tasks) *n_tasks = (int)m->tasks.size();
    if (n_items) *n_items = (int)m->items.size();
    return QTM_OK;
}

qtm_status qtm_debug_multi_mode_tasks(const qtm_multi *m, int which, int32_t *tasks, int capacity, int *n_tasks)
{
    if (!m || which < 0 || which > 2 || capacity < 0 || (capacity > 0 && !tasks)) return QTM_EINVAL;
    const std::vector<Task> &v = which == 0 ? m->tasks : which == 1 ? m->tasks_fwd : m->tasks_adj;
    for (int i = 0; i < capacity && i < (int)v.size(); ++i) {
        tasks[3 * i] = v[i].item;
        tasks[3 * i + 1] = v[i].step;
        tasks[3 * i + 2] = v[i].tile;
    }
    if (n_tasks) *n_tasks = (int)v.size();
    return QTM_OK;
}

const char *qtm_multi_last_error(const qtm_multi *m)
{
    return m ? m->err.c_str() : "";
}

qtm_status qtm_debug_multi_inject(qtm_multi *m, const int32_t *tasks, int n, long long wait_ns)
{
    if (!m || n < 1 || !tasks || wait_ns <= 0) return QTM_EINVAL;
    std::vector<Task> t(n);
    for (int i = 0; i < n; ++i) {
        t[i] = {tasks[3 * i], tasks[3 * i + 1], tasks[3 * i + 2]};
        if (t[i].item < 0 || t[i].item >= (int)m->items.size()) return QTM_EINVAL;
        const Plan &P = m->plans[m->items[t[i].item].c];
        const int steps = (int)(P.fwd.size() + P.rev.size());
        if (t[i].step < -1 || t[i].step >= steps) return QTM_EINVAL;
        if (t[i].step < 0 ? t[i].tile != 0 : (P.tiles_per_sample < 2 || t[i].tile < 0 ||
                                              t[i].tile >= P.tiles_per_sample))
            return QTM_EINVAL;
    }
    if (m->dev_block) cudaDeviceSynchronize();
    m->tasks = t;
    m->fwd_valid = false;
    m->wait_ns = (unsigned long long)wait_ns;
    m->injected = true;
    release_graph(m);
    m->dirty = true;
    return QTM_OK;
}

qtm_status qtm_multi_destroy(qtm_multi *m)
{
    if (!m) return QTM_EINVAL;
    if (m->dev_block) cudaDeviceSynchronize();
    release_device(m);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    delete m;
    return QTM_OK;
}

}  // extern "C"
