// C ABI entry points (include/qtm.h, include/qtm_debug.h).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qtm.h"
#include "../../include/qtm_debug.h"
#include "device.h"
#include "jit.h"
#include "plan.h"

#include <cstdio>
#include <cstdlib>
#include <thread>

namespace qtm {
qtm_status emulate_plan(const Plan &P, int B, const double *x, const double *w, const double *gE,
                        double *E, double *gx, double *gw, std::string &err);
}

using namespace qtm;

namespace {

constexpr size_t kMaxDynSmem = 232448;   // 227 KiB per block on sm_100 / sm_103

struct TmGeom {
    int rank = 0, low_dims = 0, high_dims = 0;
};

}  // namespace

struct qtm_plan {
    Plan P;
    std::string err;
    // the circuit as given, kept for re-planning (qtm_set_schedule, qtm_tune)
    std::vector<qtm_gate> src_gates;
    std::vector<qtm_zterm> src_terms;
    std::vector<PauliTerm> src_pterms;   // strings with X/Y factors of a one-evolution plan
    int src_n = 0, src_n_obs = 0, src_n_weights = 0, src_n_inputs = 0, src_path = QTM_PATH_AUTO;
    PlanOptions opt;
    int minb_f = 3, minb_r = 2;          // CTAs per SM the specialised kernels are compiled for
    int device = -1;
    // device tables
    DevOp *d_ops = nullptr;
    DiagPair *d_diag = nullptr;
    MaskTerm *d_amap = nullptr;
    DevPhase *d_phases = nullptr;
    int32_t *d_slot_runs = nullptr;
    Run *d_runs = nullptr;
    Rot *d_rots = nullptr;
    int32_t *d_prefix_run_of_q = nullptr;
    Ent *d_prefix_ents = nullptr;
    Term *d_terms = nullptr;
    PauliTerm *d_pterms = nullptr;     // terms with X/Y factors (evaluated on the final state)
    int32_t *d_w_ptr = nullptr, *d_w_rots = nullptr, *d_x_ptr = nullptr, *d_x_rots = nullptr;
    unsigned *d_status = nullptr;
    // workspace
    int cap_B = 0;
    void *d_phi = nullptr, *d_lam = nullptr, *d_Escratch = nullptr;
    double *d_Epart = nullptr, *d_Gpart = nullptr, *d_abar = nullptr, *d_gw_ws = nullptr;
    void *d_mats = nullptr, *d_tabs = nullptr;
    double2 *d_cs = nullptr;           // [B][rots] (cos, sin) of half angles (prep -> grad finalize)
    double *d_ppart = nullptr;         // [B][chunks][X/Y terms] expectation-value partial sums
    void *d_onehot = nullptr;          // [B][M] cotangent e_m (qtm_jacobian)
    // qtm_jacobian: the forward's final states [B][2^sq] and the inputs of
    // the pseudo-samples (sample, observable) [B * chunk][n_in]
    void *d_jkeep = nullptr, *d_jx = nullptr;
    size_t jkeep_bytes = 0, jx_bytes = 0;
    int32_t *d_gate_of_rot = nullptr;  // rotation id -> gate index
    int32_t *d_rot_rep = nullptr;      // first rotation with the same angle definition (fused prep)
    double2 *d_cs_shared = nullptr;    // [rots] FP64 (cos, sin) of half angles without an input (one call's)
    std::vector<CUtensorMap> tm_fwd, tm_rev_phi, tm_rev_lam;
    std::vector<TmGeom> g_fwd, g_rev;
    std::vector<size_t> smem_fwd, smem_rev;
    // Pauli-string observables (qtm_build_pauli): one Z-observable plan per
    // group of terms sharing their X/Y qubits, outputs summed in part order
    std::vector<qtm_plan *> parts;
    void *d_tmp = nullptr;             // scratch for the parts' outputs
    size_t tmp_bytes = 0;
    bool needs_lam = false;
    // stored forward
    bool fwd_valid = false;
    int fwd_B = 0;
    const void *fwd_x = nullptr, *fwd_w = nullptr;
    void *fwd_stream = nullptr;
    std::string describe_cache;
    // run-time specialised pass kernels (qtm_compile)
    std::vector<JitKernel> jit_fwd, jit_rev;
    int jit_device = -1;
    std::string jit_src_cache;
    // profiling: events around each launch of the last forward / adjoint
    int profiling = 0;                 // 0 off, 1 every launch, 2 the adjoint's pass kernels only
    struct Rec { cudaEvent_t a, b; int kind; };
    std::vector<Rec> recs[2];
    // one event pool per kind of call, so that an adjoint's records do not
    // re-record the events of the forward before it
    std::vector<cudaEvent_t> ev_pool[2];
    size_t ev_used[2] = {0, 0};
    int cur_which = 0;
    cudaStream_t cur_stream = nullptr;
};

namespace {

qtm_status fail(qtm_plan *p, qtm_status st, const std::string &msg)
{
    if (p) p->err = msg;
    return st;
}

qtm_status cuda_fail(qtm_plan *p, cudaError_t e, const char *where)
{
    return fail(p, QTM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &v)
{
    *dst = nullptr;
    size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

void free_tables(qtm_plan *p)
{
    void *ptrs[] = {p->d_gate_of_rot, p->d_ops, p->d_diag, p->d_amap, p->d_phases, p->d_slot_runs, p->d_runs, p->d_rots,
                    p->d_prefix_run_of_q, p->d_prefix_ents, p->d_terms, p->d_pterms, p->d_w_ptr,
                    p->d_w_rots, p->d_x_ptr, p->d_x_rots, p->d_status, p->d_rot_rep, p->d_cs_shared};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    p->d_gate_of_rot = nullptr;
    p->d_rot_rep = nullptr; p->d_cs_shared = nullptr;
    p->d_ops = nullptr; p->d_diag = nullptr; p->d_amap = nullptr; p->d_phases = nullptr; p->d_slot_runs = nullptr; p->d_runs = nullptr;
    p->d_rots = nullptr; p->d_prefix_run_of_q = nullptr; p->d_prefix_ents = nullptr;
    p->d_terms = nullptr; p->d_pterms = nullptr; p->d_w_ptr = p->d_w_rots = p->d_x_ptr = p->d_x_rots = nullptr;
    p->d_status = nullptr;
}

void free_workspace(qtm_plan *p)
{
    void *ptrs[] = {p->d_phi, p->d_lam, p->d_Escratch, p->d_Epart, p->d_Gpart, p->d_abar, p->d_gw_ws,
                    p->d_mats, p->d_tabs, p->d_onehot, p->d_cs, p->d_ppart, p->d_jkeep, p->d_jx};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    p->d_jkeep = p->d_jx = nullptr;
    p->jkeep_bytes = p->jx_bytes = 0;
    p->d_phi = p->d_lam = p->d_Escratch = p->d_mats = p->d_tabs = p->d_onehot = nullptr;
    p->d_cs = nullptr;
    p->d_Epart = p->d_Gpart = p->d_abar = p->d_gw_ws = p->d_ppart = nullptr;
    p->cap_B = 0;
    p->fwd_valid = false;
}

bool fault_alloc_injected()
{
    const char *v = std::getenv("QTM_FAULT_ALLOC");
    return v && v[0] == '1';
}

cudaError_t dmalloc(void **p, size_t bytes)
{
    if (fault_alloc_injected()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMalloc(p, bytes ? bytes : 16);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// Tensor map over the batched state [B][2^sq] for a pass's tile geometry.
// Dimensions (innermost first): 16 eight-byte words (128 bytes: 16 complex64
// or 8 complex128 = the low tile bits), the rest of the low block in chunks of
// <= 8 bits, the gap [l, h) (box 1), the high block [h, h+m), and everything
// above h+m together with the sample index (box 1).  128-byte swizzle.
bool make_tmap(CUtensorMap *tm, void *base, const PassDesc &pd, int sq, int B, int dtype, TmGeom &g)
{
    const int es = elem_bytes(dtype);
    const int d0bits = dtype == QTM_C128 ? 3 : 4;
    cuuint64_t dim[8], stride[8];
    cuuint32_t box[8], estr[8];
    int r = 0;
    dim[r] = 16; box[r] = 16; ++r;
    g.low_dims = 1;
    for (int bit = d0bits; bit < pd.l; bit += 8) {
        int cnt = std::min(8, pd.l - bit);
        dim[r] = 1ull << cnt; box[r] = 1u << cnt; stride[r - 1] = (cuuint64_t)es << bit; ++r;
        g.low_dims++;
    }
    if (pd.h > pd.l) {
        dim[r] = 1ull << (pd.h - pd.l); box[r] = 1; stride[r - 1] = (cuuint64_t)es << pd.l; ++r;
    }
    g.high_dims = 0;
    for (int bit = pd.h; bit < pd.h + pd.m; bit += 8) {
        int cnt = std::min(8, pd.h + pd.m - bit);
        dim[r] = 1ull << cnt; box[r] = 1u << cnt; stride[r - 1] = (cuuint64_t)es << bit; ++r;
        g.high_dims++;
    }
    const int rb = pd.h + pd.m;
    dim[r] = (1ull << (sq - rb)) * (cuuint64_t)B; box[r] = 1; stride[r - 1] = (cuuint64_t)es << rb; ++r;
    if (r > 5) return false;
    g.rank = r;
    for (int i = 0; i < r; ++i) estr[i] = 1;
    auto fn = encode_fn();
    if (!fn) return false;
    CUresult res = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)r, base, dim, stride, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return res == CUDA_SUCCESS;
}

qtm_status ensure_device(qtm_plan *p)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(p, e, "no CUDA device");
    int count = 0;
    e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) return fail(p, QTM_ECUDA, "no CUDA device");
    if (p->device == dev && p->d_status) return QTM_OK;
    if (p->d_status) {
        free_workspace(p);
        free_tables(p);
    }
    const Plan &P = p->P;
    std::vector<unsigned> zero(1, 0u);
#define UP(dst, vec)                                               \
    do {                                                           \
        e = upload(&(dst), vec);                                   \
        if (e != cudaSuccess) { free_tables(p); return cuda_fail(p, e, "upload"); } \
    } while (0)
    UP(p->d_ops, P.ops);
    UP(p->d_diag, P.diag_pairs);
    UP(p->d_amap, P.amap_terms);
    UP(p->d_phases, P.phases);
    UP(p->d_slot_runs, P.slot_runs);
    UP(p->d_runs, P.runs);
    UP(p->d_rots, P.rots);
    UP(p->d_prefix_run_of_q, P.prefix_run_of_q);
    UP(p->d_prefix_ents, P.pass_ents);   // per-pass entangler subsets (ents_begin offsets)
    UP(p->d_terms, P.terms);
    UP(p->d_pterms, P.pterms);
    UP(p->d_w_ptr, P.w_ptr);
    UP(p->d_w_rots, P.w_rots);
    UP(p->d_x_ptr, P.x_ptr);
    UP(p->d_x_rots, P.x_rots);
    UP(p->d_status, zero);
    {
        std::vector<int32_t> gor(P.rots.size());
        for (size_t r = 0; r < P.rots.size(); ++r) gor[r] = P.rots[r].gate;
        UP(p->d_gate_of_rot, gor);
        // rotations with the same angle definition share one sine and cosine
        std::vector<int32_t> rep(P.rots.size());
        for (size_t i = 0; i < P.rots.size(); ++i) {
            const Rot &a = P.rots[i];
            size_t k = 0;
            while (k < i && !(P.rots[k].coef == a.coef && P.rots[k].w_idx == a.w_idx && P.rots[k].x_idx == a.x_idx)) ++k;
            rep[i] = (int32_t)k;
        }
        UP(p->d_rot_rep, rep);
        UP(p->d_cs_shared, std::vector<double2>(P.rots.size()));
    }
#undef UP
    p->device = dev;
    return QTM_OK;
}

// Specialised kernels are loaded for the current device (all passes).
bool jit_active(const qtm_plan *p)
{
    return p->jit_device >= 0 && p->jit_device == p->device;
}



cudaError_t launch_any(qtm_plan *p, bool rev, size_t i, PassArgs a, const CUtensorMap &t0, const CUtensorMap &t1,
                       cudaStream_t s, bool pdl = false)
{
    const auto &v = rev ? p->jit_rev : p->jit_fwd;
    if (jit_active(p) && i < v.size() && v[i].fn) {
        a.smem_bytes = v[i].smem;
        return jit_launch(v[i], a, t0, t1, s, pdl);
    }
    return launch_pass(p->P.dtype, rev, a, t0, t1, s, pdl);
}

qtm_status ensure_workspace(qtm_plan *p, int B)
{
    if (B <= p->cap_B && p->d_phi) return QTM_OK;
    free_workspace(p);
    const Plan &P = p->P;
    const size_t csize = elem_bytes(P.dtype);
    const size_t rsize = csize / 2;
    const size_t NS = P.path == QTM_PATH_NAIVE ? (1ull << P.n) : (1ull << P.state_qubits);
    const size_t runs = P.runs.size() ? P.runs.size() : 1;
    const size_t rots = P.rots.size() ? P.rots.size() : 1;
    const size_t tiles = P.tiles_per_sample;
    cudaError_t e;
#define AL(ptr, bytes)                                                                  \
    do {                                                                                \
        e = dmalloc(reinterpret_cast<void **>(&(ptr)), bytes);                          \
        if (e != cudaSuccess) { free_workspace(p); return fail(p, QTM_ENOMEM, "workspace allocation failed"); } \
    } while (0)
    AL(p->d_phi, csize * NS * B);
    if (p->needs_lam || P.path == QTM_PATH_NAIVE) AL(p->d_lam, csize * NS * B);
    AL(p->d_Escratch, rsize * (size_t)B * P.n_obs);
    AL(p->d_Epart, sizeof(double) * (size_t)B * tiles * P.n_obs);
    AL(p->d_Gpart, sizeof(double) * (size_t)B * runs * tiles * 3);
    AL(p->d_abar, sizeof(double) * (size_t)B * rots * 3);   // naive path keeps cos/sin in the tail
    AL(p->d_gw_ws, sizeof(double) * (size_t)B * (P.n_weights ? P.n_weights : 1));
    AL(p->d_mats, csize * 4 * (size_t)B * runs);
    AL(p->d_tabs, csize * 16 * (size_t)B * ((P.state_qubits + 3) / 4));
    AL(p->d_onehot, rsize * (size_t)B * P.n_obs);
    AL(p->d_cs, sizeof(double2) * (size_t)B * rots);
    if (!P.pterms.empty())
        AL(p->d_ppart, sizeof(double) * (size_t)B * pauli_chunks(P.state_qubits) * P.pterms.size());
#undef AL
    p->cap_B = B;
    if (P.path == QTM_PATH_FUSED) {
        const int mdtype = P.dtype, mB = B;
        p->tm_fwd.assign(P.fwd.size(), CUtensorMap{});
        p->g_fwd.assign(P.fwd.size(), TmGeom{});
        p->tm_rev_phi.assign(P.rev.size(), CUtensorMap{});
        p->tm_rev_lam.assign(P.rev.size(), CUtensorMap{});
        p->g_rev.assign(P.rev.size(), TmGeom{});
        for (size_t i = 0; i < P.fwd.size(); ++i)
            if (!make_tmap(&p->tm_fwd[i], p->d_phi, P.fwd[i], P.state_qubits, mB, mdtype, p->g_fwd[i])) {
                free_workspace(p);
                return fail(p, QTM_ECUDA, "cuTensorMapEncodeTiled failed (forward)");
            }
        for (size_t i = 0; i < P.rev.size(); ++i) {
            if (!make_tmap(&p->tm_rev_phi[i], p->d_phi, P.rev[i], P.state_qubits, mB, mdtype, p->g_rev[i])) {
                free_workspace(p);
                return fail(p, QTM_ECUDA, "cuTensorMapEncodeTiled failed (reverse)");
            }
            TmGeom gl;
            void *lb = p->d_lam ? p->d_lam : p->d_phi;
            if (!make_tmap(&p->tm_rev_lam[i], lb, P.rev[i], P.state_qubits, mB, mdtype, gl)) {
                free_workspace(p);
                return fail(p, QTM_ECUDA, "cuTensorMapEncodeTiled failed (costate)");
            }
        }
    }
    return QTM_OK;
}

// ---- profiling hooks: events around launches (no-ops unless enabled) ----
void prof_begin_call(qtm_plan *p, int which, cudaStream_t s)
{
    p->cur_which = which;
    p->cur_stream = s;
    if (!p->profiling) return;
    p->recs[which].clear();
    p->ev_used[which] = 0;
}

cudaEvent_t prof_event(qtm_plan *p)
{
    std::vector<cudaEvent_t> &pool = p->ev_pool[p->cur_which];
    size_t &used = p->ev_used[p->cur_which];
    if (used == pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
    }
    return pool[used++];
}

struct ProfScope {
    qtm_plan *p;
    qtm_plan::Rec r{};
    bool on = false;
    ProfScope(qtm_plan *p_, int kind) : p(p_)
    {
        if (!p->profiling) return;
        if (p->profiling == 2 && (p->cur_which != 1 || kind != 0)) return;   // reverse passes only
        r.a = prof_event(p);
        r.b = prof_event(p);
        r.kind = kind;
        on = r.a && r.b;
        if (on) cudaEventRecord(r.a, p->cur_stream);
    }
    ~ProfScope()
    {
        if (!on) return;
        cudaEventRecord(r.b, p->cur_stream);
        p->recs[p->cur_which].push_back(r);
    }
};

PassArgs pass_args(qtm_plan *p, const PassDesc &pd, const TmGeom &g, size_t smem, int B,
                   const void *x, const void *w, const void *gE)
{
    const Plan &P = p->P;
    PassArgs a{};
    a.K = pd.K; a.l = pd.l; a.h = pd.h; a.m = pd.m;
    a.state_qubits = P.state_qubits; a.n = P.n;
    a.tiles = P.tiles_per_sample;
    a.log_tiles = 0;
    while ((1 << a.log_tiles) < a.tiles) ++a.log_tiles;
    a.B = B;
    a.rank = g.rank; a.low_dims = g.low_dims; a.high_dims = g.high_dims;
    a.gap_dim = pd.h > pd.l ? 1 : 0;
    a.ops = p->d_ops; a.diag = p->d_diag; a.phases = p->d_phases;
    a.phase_begin = pd.phase_begin; a.phase_end = pd.phase_end;
    a.slot_runs = p->d_slot_runs; a.slot_begin = pd.slot_begin; a.nslots = pd.slot_end - pd.slot_begin;
    a.n_runs = (int)P.runs.size();
    a.mats = p->d_mats; a.tabs = p->d_tabs;
    a.prefix_ents = p->d_prefix_ents + pd.ents_begin;
    a.analytic_ents = pd.phi_src == SRC_ANALYTIC ? pd.analytic_ents : 0;
    a.amap = p->d_amap + (pd.amap_lin >= 0 ? pd.amap_begin : 0);
    a.amap_lin = pd.phi_src == SRC_ANALYTIC ? pd.amap_lin : -1;
    a.amap_quad = pd.amap_quad; a.amap_dlin = pd.amap_dlin;
    a.phi_src = pd.phi_src; a.lam_src = pd.lam_src;
    a.store_phi = pd.store_phi; a.store_lam = pd.store_lam; a.has_expval = pd.has_expval;
    a.terms = p->d_terms; a.n_terms = (int)P.terms.size(); a.M = P.n_obs;
    a.x = x; a.w = w; a.gE = gE; a.n_in = P.n_inputs;
    a.Epart = p->d_Epart; a.Gpart = p->d_Gpart;
    a.status = p->d_status;
    a.smem_bytes = (int)smem;
    return a;
}

qtm_status run_prep(qtm_plan *p, int B, const void *x, const void *w, cudaStream_t s)
{
    const Plan &P = p->P;
    PrepArgs a{};
    a.B = B; a.n = P.n; a.state_qubits = P.state_qubits; a.n_runs = (int)P.runs.size();
    a.n_in = P.n_inputs; a.runs = p->d_runs; a.rots = p->d_rots;
    a.prefix_run_of_q = p->d_prefix_run_of_q; a.x = x; a.w = w; a.mats = p->d_mats; a.tabs = p->d_tabs;
    a.cs = p->d_cs; a.n_rots = (int)P.rots.size();
    ProfScope ps(p, 1);
    cudaError_t e = launch_prep(P.dtype, a, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "prep launch");
    return QTM_OK;
}

// Plans of one tile per sample run the per-sample prep inside their first
// forward pass and the gradient finalize inside their last reverse pass (one
// CTA holds a whole sample); the two-samples-per-CTA kernels keep them apart.
// QTM_FUSE_SAMPLE_STEPS=0 (a tuning switch) keeps them apart always.
bool fuse_sample_steps(const qtm_plan *p)
{
    const char *e = std::getenv("QTM_FUSE_SAMPLE_STEPS");
    if (e && *e == '0') return false;
    return p->P.path == QTM_PATH_FUSED && p->P.tiles_per_sample == 1;
}

// Fused prep with shared sines and cosines (prep_sample_shared): the first
// forward pass of a one-tile plan starts from the analytic state, so its idle
// tile holds the per-sample pairs.  QTM_PREP_SHARED=0 (a tuning switch)
// computes every rotation's pair per sample.
bool prep_shared(const qtm_plan *p)
{
    const Plan &P = p->P;
    const char *e = std::getenv("QTM_PREP_SHARED");
    return fuse_sample_steps(p) && !P.fwd.empty() && !(e && *e == '0') && P.fwd[0].phi_src == SRC_ANALYTIC &&
           P.rots.size() * sizeof(double2) <= ((size_t)elem_bytes(P.dtype) << P.fwd[0].K);
}

// ... which launches one per-call kernel when some rotation has no input.
bool prep_shared_launches(const qtm_plan *p)
{
    if (!prep_shared(p)) return false;
    for (const Rot &r : p->P.rots)
        if (r.x_idx < 0) return true;
    return false;
}

void set_prep_fields(qtm_plan *p, PassArgs &a)
{
    const Plan &P = p->P;
    a.runs = p->d_runs; a.rots = p->d_rots; a.prq = p->d_prefix_run_of_q;
    a.cs = p->d_cs; a.n_rots = (int)P.rots.size(); a.n_weights = P.n_weights;
    a.w_ptr = p->d_w_ptr; a.w_rots = p->d_w_rots; a.x_ptr = p->d_x_ptr; a.x_rots = p->d_x_rots;
    a.abar = p->d_abar;
}

// expvals (may be null): where a plan of one tile per sample writes its
// expectation values straight from the measuring pass (returns true if so).
qtm_status run_forward_passes(qtm_plan *p, int B, const void *x, const void *w, cudaStream_t s,
                              void *expvals = nullptr, bool *wrote_expvals = nullptr)
{
    const Plan &P = p->P;
    const bool fused = fuse_sample_steps(p) && !P.fwd.empty();
    if (wrote_expvals) *wrote_expvals = fused && expvals;
    if (!fused) {
        qtm_status st = run_prep(p, B, x, w, s);
        if (st != QTM_OK) return st;
    }
    const bool shared = prep_shared(p);
    const bool after_shared = shared && prep_shared_launches(p);   // the first pass follows k_prep_shared
    if (shared) {
        if (after_shared) {
            ProfScope ps(p, 1);
            cudaError_t e = launch_prep_shared(P.dtype, p->d_rots, p->d_rot_rep, (int)P.rots.size(), w,
                                               p->d_cs_shared, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "shared prep launch");
        }
    }
    for (size_t i = 0; i < P.fwd.size(); ++i) {
        PassArgs a = pass_args(p, P.fwd[i], p->g_fwd[i], p->smem_fwd[i], B, x, w, nullptr);
        if (fused && i == 0) {
            set_prep_fields(p, a);
            a.prep_fused = 1;
            if (shared) { a.rot_rep = p->d_rot_rep; a.cs_shared = p->d_cs_shared; }
        }
        if (fused) a.E_out = expvals;
        ProfScope ps(p, 0);
        // the first pass may overlap k_prep_shared (it waits before reading its pairs)
        cudaError_t e = launch_any(p, false, i, a, p->tm_fwd[i], p->tm_fwd[i], s, i == 0 && after_shared);
        if (e != cudaSuccess) return cuda_fail(p, e, "forward pass launch");
    }
    return QTM_OK;
}

FinalizeArgs finalize_args(qtm_plan *p, int B, const void *x, const void *w)
{
    const Plan &P = p->P;
    FinalizeArgs f{};
    f.B = B; f.M = P.n_obs; f.tiles = P.tiles_per_sample; f.n_runs = (int)P.runs.size();
    f.n_rots = (int)P.rots.size(); f.P = P.n_weights; f.n_in = P.n_inputs;
    f.runs = p->d_runs; f.rots = p->d_rots;
    f.w_ptr = p->d_w_ptr; f.w_rots = p->d_w_rots; f.x_ptr = p->d_x_ptr; f.x_rots = p->d_x_rots;
    f.x = x; f.w = w; f.Epart = p->d_Epart; f.Gpart = p->d_Gpart; f.abar = p->d_abar;
    f.cs = p->d_cs;
    return f;
}

NaiveArgs naive_args(qtm_plan *p, int B, const void *x, const void *w, const void *gE)
{
    const Plan &P = p->P;
    NaiveArgs a{};
    a.n = P.n; a.B = B; a.n_in = P.n_inputs; a.M = P.n_obs; a.n_terms = (int)P.terms.size();
    a.n_rots = (int)P.rots.size(); a.P = P.n_weights;
    a.gates_host = P.gates.data(); a.n_gates = (int)P.gates.size();
    a.terms = p->d_terms; a.rot_of_gate_host = P.rot_of_gate.data(); a.rots = p->d_rots;
    a.w_ptr = p->d_w_ptr; a.w_rots = p->d_w_rots; a.x_ptr = p->d_x_ptr; a.x_rots = p->d_x_rots;
    a.x = x; a.w = w; a.gE = gE; a.phi = p->d_phi; a.lam = p->d_lam; a.abar = p->d_abar;
    a.gw_ws = p->d_gw_ws;
    return a;
}

}  // namespace

bool qtm_internal_is_composite(const qtm_plan *plan) { return plan && !plan->parts.empty(); }

const qtm::Plan *qtm_internal_plan(const qtm_plan *plan) { return &plan->P; }

extern "C" {

const char *qtm_status_str(int st)
{
    switch (st) {
    case QTM_OK: return "ok";
    case QTM_EINVAL: return "invalid argument";
    case QTM_ENOMEM: return "out of memory";
    case QTM_ECUDA: return "CUDA error";
    case QTM_EUNSUPPORTED: return "unsupported";
    case QTM_ETIMEOUT: return "device wait timed out";
    case QTM_ESTATE: return "call order violated";
    default: return "unknown status";
    }
}

const char *qtm_version(void) { return "qtm 0.1 sm_103a"; }

const char *qtm_last_error(const qtm_plan *plan) { return plan ? plan->err.c_str() : ""; }


namespace {

bool is_composite(const qtm_plan *p) { return !p->parts.empty(); }

qtm_status part_fail(qtm_plan *p, qtm_plan *part, qtm_status st)
{
    return fail(p, st, part->err);
}

// device scratch of at least `bytes` for the parts' outputs
qtm_status ensure_tmp(qtm_plan *p, size_t bytes)
{
    if (bytes <= p->tmp_bytes && p->d_tmp) return QTM_OK;
    if (p->d_tmp) cudaFree(p->d_tmp);
    p->d_tmp = nullptr;
    p->tmp_bytes = 0;
    cudaError_t e = cudaMalloc(&p->d_tmp, bytes ? bytes : 16);
    if (e != cudaSuccess) return fail(p, QTM_ENOMEM, "composite scratch allocation failed");
    p->tmp_bytes = bytes;
    return QTM_OK;
}

// (Re)build p->P from the circuit as given with p->opt: the schedule, the
// costate buffer it needs and every pass's shared memory.  Host only; p->P
// is replaced only on success.
qtm_status plan_from_source(qtm_plan *p, int dtype)
{
    Plan P;
    std::string err;
    qtm_status st = make_plan(p->src_n, p->src_gates.data(), (int)p->src_gates.size(), p->src_terms.data(),
                              (int)p->src_terms.size(), p->src_n_obs, p->src_n_weights, p->src_n_inputs, dtype,
                              p->src_path, P, err, p->opt);
    if (st != QTM_OK) { p->err = err; return st; }
    if (!p->src_pterms.empty()) attach_pauli_terms(P, p->src_pterms);
    bool needs_lam = !p->src_pterms.empty();
    std::vector<size_t> sf, sr;
    if (P.path == QTM_PATH_FUSED) {
        for (const auto &pd : P.rev)
            if (pd.lam_src == SRC_LOAD || pd.store_lam) needs_lam = true;
        auto sm = [&](const PassDesc &pd, bool rev) {
            return pass_smem_bytes(pd.K, P.dtype, rev, pd.slot_end - pd.slot_begin, (int)P.terms.size(),
                                   P.n_obs, P.state_qubits,
                                   pd.phi_src == SRC_ANALYTIC ? pd.analytic_ents : 0);
        };
        for (const auto &pd : P.fwd) sf.push_back(sm(pd, false));
        for (const auto &pd : P.rev) sr.push_back(sm(pd, true));
        for (size_t v : sf)
            if (v > kMaxDynSmem) { p->err = "a pass needs more shared memory than a CTA has"; return QTM_EUNSUPPORTED; }
        for (size_t v : sr)
            if (v > kMaxDynSmem) { p->err = "a pass needs more shared memory than a CTA has"; return QTM_EUNSUPPORTED; }
    }
    p->P = std::move(P);
    p->needs_lam = needs_lam;
    p->smem_fwd = std::move(sf);
    p->smem_rev = std::move(sr);
    return QTM_OK;
}

// Key of a tuned schedule: the circuit as given, the observables, dtype,
// batch size and device name (FNV-1a).
std::string tune_signature(const qtm_plan *p, int B)
{
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](unsigned long long v) {
        for (int k = 0; k < 8; ++k) { h ^= (v >> (8 * k)) & 0xffull; h *= 1099511628211ull; }
    };
    mix((unsigned long long)p->src_n); mix((unsigned long long)p->P.dtype); mix((unsigned long long)B);
    mix((unsigned long long)p->src_n_obs);
    for (const auto &g : p->src_gates) {
        mix((unsigned long long)(uint32_t)g.kind); mix((unsigned long long)(uint32_t)g.q0);
        mix((unsigned long long)(uint32_t)g.q1); mix((unsigned long long)(uint32_t)g.w_idx);
        mix((unsigned long long)(uint32_t)g.x_idx);
    }
    for (const auto &t : p->src_terms) { mix(t.zmask); mix((unsigned long long)(uint32_t)t.obs); }
    for (const auto &t : p->src_pterms) { mix(t.xmask); mix(t.zmask); mix((unsigned long long)(uint32_t)t.obs); }
    std::string name = "unknown";
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &ch : name) if (ch == '"' || ch == '\\') ch = '_';
    char buf[32];
    std::snprintf(buf, sizeof(buf), "%016llx", h);
    return std::string(buf) + "@" + name;
}

bool tune_cache_lookup(const char *path, const std::string &sig, qtm_schedule &out)
{
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    const std::string key = "\"signature\": \"" + sig + "\"";
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        const std::string l(line);
        if (l.find(key) == std::string::npos) continue;
        auto num = [&](const char *field) -> int {
            const std::string k = std::string("\"") + field + "\": ";
            const size_t at = l.find(k);
            return at == std::string::npos ? -1 : std::atoi(l.c_str() + at + k.size());
        };
        qtm_schedule c{num("phase_mode"), num("tile_qubits"), num("low_min"), num("kernels"), num("minb_fwd"),
                       num("minb_rev")};
        if (c.phase_mode < 0 || c.tile_qubits < 0 || c.low_min < 0 || c.kernels < 0 || c.minb_fwd < 1 || c.minb_rev < 1)
            continue;
        out = c;
        found = true;   // the last matching line wins
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(const char *path, const std::string &sig, const qtm_schedule &c, double ms)
{
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"signature\": \"%s\", \"phase_mode\": %d, \"tile_qubits\": %d, \"low_min\": %d, \"kernels\": %d, "
                 "\"minb_fwd\": %d, \"minb_rev\": %d, \"ms\": %.6f}\n",
                 sig.c_str(), c.phase_mode, c.tile_qubits, c.low_min, c.kernels, c.minb_fwd, c.minb_rev, ms);
    std::fclose(f);
}

// A device buffer of at least `bytes` (kept across calls; freed with the workspace).
cudaError_t ensure_buffer(void *&ptr, size_t &cap, size_t bytes)
{
    if (ptr && bytes <= cap) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    cudaError_t e = dmalloc(&ptr, bytes);
    if (e == cudaSuccess) cap = bytes ? bytes : 16;
    return e;
}

}  // namespace

namespace {

// Observables with X/Y factors as one plan per measurement group (circuit +
// basis change, Z strings), summed: the naive path always; fused plans with
// QTM_PAULI_GROUPS=1 (a comparison switch).
bool pauli_groups_forced()
{
    const char *v = std::getenv("QTM_PAULI_GROUPS");
    return v && *v == '1';
}

}  // namespace

qtm_status qtm_build_pauli(int n_qubits, const qtm_gate *gates, int n_gates, const qtm_pauli_term *terms,
                           int n_terms, int n_obs, int n_weights, int n_inputs, int dtype, int path,
                           qtm_plan **out)
{
    if (!out) return QTM_EINVAL;
    *out = nullptr;
    if (n_terms < 0 || (n_terms > 0 && !terms)) return QTM_EINVAL;
    if (n_qubits < 1 || n_qubits > kMaxQubits) return QTM_EINVAL;
    if (n_gates < 0 || (n_gates > 0 && !gates)) return QTM_EINVAL;
    const uint64_t all = n_qubits >= 64 ? ~0ull : ((1ull << n_qubits) - 1ull);
    for (int t = 0; t < n_terms; ++t) {
        const qtm_pauli_term &T = terms[t];
        if (T.reserved != 0 || (T.xmask & ~all) || (T.zmask & ~all) || T.obs < 0 || T.obs >= n_obs ||
            !std::isfinite(T.coef))
            return QTM_EINVAL;
    }
    // group by the basis change: X qubits (xmask & ~zmask) and Y qubits (xmask & zmask)
    std::vector<std::pair<uint64_t, uint64_t>> keys;
    std::vector<std::vector<qtm_zterm>> zterms;
    for (int t = 0; t < n_terms; ++t) {
        const qtm_pauli_term &T = terms[t];
        const std::pair<uint64_t, uint64_t> key{T.xmask & ~T.zmask, T.xmask & T.zmask};
        size_t g = 0;
        while (g < keys.size() && keys[g] != key) ++g;
        if (g == keys.size()) { keys.push_back(key); zterms.emplace_back(); }
        // after the basis change the string is Z on its whole support
        zterms[g].push_back(qtm_zterm{T.zmask | T.xmask, T.coef, T.obs, 0});
    }
    if (keys.empty()) { keys.push_back({0, 0}); zterms.emplace_back(); }
    if (keys.size() == 1 && keys[0].first == 0 && keys[0].second == 0)   // Z strings only: an ordinary plan
        return qtm_build(n_qubits, gates, n_gates, zterms[0].data(), (int)zterms[0].size(), n_obs, n_weights,
                         n_inputs, dtype, path, out);
    if (path != QTM_PATH_NAIVE && !pauli_groups_forced()) {   // AUTO plans are fused
        // one evolution: Z strings in the pass kernels, X/Y strings on the final state
        std::vector<qtm_zterm> zs;
        std::vector<PauliTerm> ps;
        for (int t = 0; t < n_terms; ++t) {
            const qtm_pauli_term &T = terms[t];
            if (T.xmask == 0) zs.push_back(qtm_zterm{T.zmask, T.coef, T.obs, 0});
            else ps.push_back(PauliTerm{T.xmask, T.zmask, T.coef, T.obs, __builtin_popcountll(T.xmask & T.zmask)});
        }
        qtm_plan *p = nullptr;
        qtm_status st = qtm_build(n_qubits, gates, n_gates, zs.data(), (int)zs.size(), n_obs, n_weights, n_inputs,
                                  dtype, path, &p);
        if (st != QTM_OK) return st;
        p->src_pterms = ps;
        st = plan_from_source(p, dtype);   // the same schedule, with the X/Y strings attached
        if (st != QTM_OK) { qtm_destroy(p); return st; }
        *out = p;
        return QTM_OK;
    }
    qtm_plan *p = new (std::nothrow) qtm_plan();
    if (!p) return QTM_ENOMEM;
    constexpr double kPi = 3.14159265358979323846264338327950288;
    for (size_t g = 0; g < keys.size(); ++g) {
        // V = RY(-pi/2) on X qubits (V X V^dagger = Z), RX(pi/2) on Y qubits (V Y V^dagger = Z)
        std::vector<qtm_gate> gl(gates, gates + n_gates);
        for (int q = 0; q < n_qubits; ++q) {
            if ((keys[g].first >> q) & 1ull) gl.push_back({QTM_RY, q, -1, -1, -1, 0, -0.5 * kPi});
            if ((keys[g].second >> q) & 1ull) gl.push_back({QTM_RX, q, -1, -1, -1, 0, 0.5 * kPi});
        }
        qtm_plan *part = nullptr;
        qtm_status st = qtm_build(n_qubits, gl.data(), (int)gl.size(), zterms[g].data(), (int)zterms[g].size(),
                                  n_obs, n_weights, n_inputs, dtype, path, &part);
        if (st != QTM_OK) {
            for (qtm_plan *q : p->parts) qtm_destroy(q);
            p->parts.clear();
            delete p;
            return st;
        }
        p->parts.push_back(part);
    }
    p->P = p->parts[0]->P;            // shape fields (n, dtype, n_obs, n_weights, n_inputs, path)
    p->P.n_user_gates = n_gates;      // Jacobian columns: the gates as given
    *out = p;
    return QTM_OK;
}

int qtm_plan_parts(const qtm_plan *p) { return p ? (p->parts.empty() ? 1 : (int)p->parts.size()) : 0; }

namespace {

qtm_status composite_forward(qtm_plan *p, int B, const void *x, const void *w, void *expvals, void *stream)
{
    const Plan &P = p->P;
    const size_t n = (size_t)B * P.n_obs, es = elem_bytes(P.dtype) / 2;
    if (p->parts.size() > 1) {
        qtm_status st = ensure_tmp(p, n * es);
        if (st != QTM_OK) return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < p->parts.size(); ++i) {
        qtm_plan *part = p->parts[i];
        qtm_status st = qtm_forward(part, B, x, w, i == 0 ? expvals : p->d_tmp, stream);
        if (st != QTM_OK) return part_fail(p, part, st);
        if (i > 0) {
            cudaError_t e = launch_accumulate(P.dtype, p->d_tmp, expvals, n, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "composite accumulate");
        }
    }
    return QTM_OK;
}

qtm_status composite_adjoint(qtm_plan *p, int B, const void *gE, const void *x, const void *w, void *gx, void *gw,
                             int flags, void *stream)
{
    const Plan &P = p->P;
    const size_t es = elem_bytes(P.dtype) / 2;
    const size_t ngx = gx ? (size_t)B * P.n_inputs : 0;
    const size_t ngw = gw ? ((flags & QTM_ADJ_GW_PER_SAMPLE) ? (size_t)B : 1) * P.n_weights : 0;
    if (p->parts.size() > 1) {
        qtm_status st = ensure_tmp(p, (ngx + ngw) * es + 256);
        if (st != QTM_OK) return st;
    }
    char *tgx = static_cast<char *>(p->d_tmp);
    char *tgw = tgx + ((ngx * es + 255) & ~size_t(255));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < p->parts.size(); ++i) {
        qtm_plan *part = p->parts[i];
        qtm_status st = qtm_adjoint(part, B, gE, x, w, gx ? (i == 0 ? gx : (void *)tgx) : nullptr,
                                    gw ? (i == 0 ? gw : (void *)tgw) : nullptr, flags, stream);
        if (st != QTM_OK) return part_fail(p, part, st);
        if (i > 0) {
            cudaError_t e = cudaSuccess;
            if (gx) e = launch_accumulate(P.dtype, tgx, gx, ngx, s);
            if (e == cudaSuccess && gw) e = launch_accumulate(P.dtype, tgw, gw, ngw, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "composite accumulate");
        }
    }
    return QTM_OK;
}

// Observables per reverse sweep of qtm_jacobian: all of them, so that a
// single reverse launch covers every (sample, observable), unless the
// pseudo-samples' states (phi and lam) would pass kJacobianStateBudget; then
// as many as fit (at least one).  The passes are ALU-bound even with the
// states in HBM: at 16 qubits, B = 96 and 16 observables one chunk of 16
// took 5.99 ms against 6.32 (chunks of 4) and 7.94 ms (one per sweep).
// QTM_JAC_CHUNK=<c> (a tuning switch) sets it.
constexpr double kJacobianStateBudget = 8.0 * (1ull << 30);

int jacobian_chunk(const qtm_plan *p, int B)
{
    const Plan &P = p->P;
    const int M = std::max(1, P.n_obs);
    int c = M;
    if (const char *e = std::getenv("QTM_JAC_CHUNK")) {
        const int v = std::atoi(e);
        if (v >= 1) c = std::min(v, M);
    } else {
        const double per = (double)B * std::ldexp((double)elem_bytes(P.dtype), P.state_qubits) * (p->needs_lam ? 2 : 1);
        c = std::max(1, std::min(M, (int)(kJacobianStateBudget / per)));
    }
    // the pseudo-batch stays within the batch sizes the kernels index with int
    while (c > 1 && (long long)B * c > (1LL << 24)) c = (c + 1) / 2;
    return c;
}

qtm_status composite_jacobian(qtm_plan *p, int B, const void *x, const void *w, void *jac, void *stream)
{
    const Plan &P = p->P;
    const size_t es = elem_bytes(P.dtype) / 2;
    const int G = P.n_user_gates;
    size_t need = 0;
    for (qtm_plan *part : p->parts) need = std::max(need, (size_t)B * P.n_obs * (size_t)std::max(1, part->P.n_user_gates) * es);
    qtm_status st = ensure_tmp(p, need);
    if (st != QTM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(jac, 0, es * (size_t)B * P.n_obs * (G > 0 ? G : 1), s);
    if (e != cudaSuccess) return cuda_fail(p, e, "jacobian clear");
    for (qtm_plan *part : p->parts) {
        // a part's columns: the gates as given, then its basis-change rotations (dropped)
        st = qtm_jacobian(part, B, x, w, p->d_tmp, stream);
        if (st != QTM_OK) return part_fail(p, part, st);
        e = launch_accumulate_cols(P.dtype, p->d_tmp, part->P.n_user_gates, jac, G, (size_t)B * P.n_obs, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "composite accumulate");
    }
    return QTM_OK;
}

}  // namespace

qtm_status qtm_build(int n_qubits, const qtm_gate *gates, int n_gates, const qtm_zterm *terms,
                     int n_terms, int n_obs, int n_weights, int n_inputs, int dtype, int path,
                     qtm_plan **out)
{
    if (!out) return QTM_EINVAL;
    *out = nullptr;
    if (n_gates < 0 || (n_gates > 0 && !gates) || n_terms < 0 || (n_terms > 0 && !terms)) return QTM_EINVAL;
    qtm_plan *p = new (std::nothrow) qtm_plan();
    if (!p) return QTM_ENOMEM;
    p->src_gates.assign(gates, gates + n_gates);
    p->src_terms.assign(terms, terms + n_terms);
    p->src_n = n_qubits; p->src_n_obs = n_obs; p->src_n_weights = n_weights; p->src_n_inputs = n_inputs;
    p->src_path = path;
    p->P.dtype = dtype;
    // phase grouping: automatic (default), or QTM_PHASES=greedy / rr (a tuning switch)
    const char *pm = std::getenv("QTM_PHASES");
    p->opt.phase_mode = !pm                              ? PHASES_AUTO
                        : std::strcmp(pm, "rr") == 0     ? PHASES_ROUND_ROBIN
                        : std::strcmp(pm, "greedy") == 0 ? PHASES_GREEDY
                                                         : PHASES_AUTO;
    qtm_status st = plan_from_source(p, dtype);
    if (st != QTM_OK) { delete p; return st; }
    *out = p;
    return QTM_OK;
}

qtm_status qtm_get_plan_info(const qtm_plan *p, qtm_plan_info *info)
{
    if (!p || !info) return QTM_EINVAL;
    const Plan &P = p->P;
    std::memset(info, 0, sizeof(*info));
    info->n_qubits = P.n;
    info->dtype = P.dtype;
    info->path = P.path;
    info->tile_qubits = P.K;
    info->fwd_passes = (int)P.fwd.size();
    info->adj_passes = (int)P.rev.size();
    if (P.path == QTM_PATH_FUSED) {
        // one-sample kernels: plans of one tile per sample run the prep in the
        // first forward pass, write E from the measuring pass and run the
        // gradient finalize in the last reverse pass; otherwise k_prep,
        // k_expval_finalize and k_grad_finalize launch on their own.  X/Y
        // strings add two launches forward and one to the adjoint.
        const bool one_tile = P.tiles_per_sample == 1 && !P.fwd.empty();
        const int xy = P.pterms.empty() ? 0 : 1;
        info->fwd_launches = (int)P.fwd.size() + (one_tile ? 0 : 2) + 2 * xy + (prep_shared_launches(p) ? 1 : 0);
        info->adj_launches = (int)P.rev.size() + (one_tile ? 0 : 1) + xy;
    } else {
        int nrot = 0;
        for (const auto &g : P.gates) nrot += (g.kind <= QTM_RZ);
        info->fwd_launches = (int)P.gates.size() + 2 + (nrot > 0);
        info->adj_launches = 1 + (int)P.gates.size() + nrot + 1;
    }
    info->n_runs = (int)P.runs.size();
    int np = 0;
    for (const auto &r : P.runs) np += r.prefix;
    info->n_prefix_runs = np;
    info->n_prefix_ents = (int)P.prefix_ents.size();
    plan_costs(P, info->fwd_state_bytes, info->adj_state_bytes, info->fwd_flops, info->adj_flops);
    return QTM_OK;
}

namespace {

// B = 0 is an empty batch: nothing is computed, but a CUDA device is still
// required (a missing GPU fails the same way at every batch size).  B < 0 is
// an argument error, caught before the composite dispatch.
qtm_status check_batch(qtm_plan *p, int B)
{
    if (B < 0) return fail(p, QTM_EINVAL, "B must be >= 0");
    if (B == 0) {
        int count = 0;
        const cudaError_t e = cudaGetDeviceCount(&count);
        if (e != cudaSuccess || count == 0) return fail(p, QTM_ECUDA, "no CUDA device");
    }
    return QTM_OK;
}

void drop_stored_forward(qtm_plan *p)
{
    p->fwd_valid = false;
    for (qtm_plan *part : p->parts) drop_stored_forward(part);
}

}  // namespace

qtm_status qtm_forward(qtm_plan *p, int B, const void *x, const void *w, void *expvals, void *stream)
{
    NvtxRange nvtx_range("qtm_forward");
    if (!p) return QTM_EINVAL;
    qtm_status bs = check_batch(p, B);
    if (bs != QTM_OK) return bs;
    if (B == 0) {   // nothing to evolve; an earlier stored forward is no longer the last one
        drop_stored_forward(p);
        return QTM_OK;
    }
    if (is_composite(p)) return composite_forward(p, B, x, w, expvals, stream);
    const Plan &P = p->P;
    if ((P.n_inputs > 0 && !x) || (P.n_weights > 0 && !w) || !expvals)
        return fail(p, QTM_EINVAL, "null pointer");
    qtm_status st = ensure_device(p);
    if (st != QTM_OK) return st;
    st = ensure_workspace(p, B);
    if (st != QTM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->fwd_valid = false;
    prof_begin_call(p, 0, s);
    if (P.path == QTM_PATH_NAIVE) {
        NaiveArgs a = naive_args(p, B, x, w, nullptr);
        a.E = expvals;
        cudaError_t e = naive_forward(P.dtype, a, s, nullptr);
        if (e != cudaSuccess) return cuda_fail(p, e, "naive forward");
    } else {
        bool direct = false;
        st = run_forward_passes(p, B, x, w, s, expvals, &direct);
        if (st != QTM_OK) return st;
        if (!direct) {
            FinalizeArgs f = finalize_args(p, B, x, w);
            f.E = expvals;
            ProfScope ps(p, 1);
            cudaError_t e = launch_expval_finalize(P.dtype, f, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "expval finalize");
        }
        if (!P.pterms.empty()) {   // X/Y strings on the final state
            ProfScope ps(p, 1);
            cudaError_t e = launch_pauli_expval(P.dtype, p->d_phi, P.state_qubits, p->d_pterms, (int)P.pterms.size(),
                                                B, P.n_obs, p->d_ppart, expvals, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "pauli expectation values");
        }
    }
    p->fwd_valid = true;
    p->fwd_B = B; p->fwd_x = x; p->fwd_w = w; p->fwd_stream = stream;
    return QTM_OK;
}

qtm_status qtm_adjoint(qtm_plan *p, int B, const void *gE, const void *x, const void *w, void *gx,
                       void *gw, int flags, void *stream)
{
    NvtxRange nvtx_range("qtm_adjoint");
    if (!p) return QTM_EINVAL;
    qtm_status bs = check_batch(p, B);
    if (bs != QTM_OK) return bs;
    if (B == 0) {   // empty batch: a batch-summed grad_w is the zero vector
        if (flags & ~(QTM_ADJ_GW_PER_SAMPLE | QTM_ADJ_RECOMPUTE)) return fail(p, QTM_EINVAL, "unknown flags");
        drop_stored_forward(p);
        if (gw && !(flags & QTM_ADJ_GW_PER_SAMPLE) && p->P.n_weights > 0) {
            const cudaError_t e = cudaMemsetAsync(gw, 0, elem_bytes(p->P.dtype) / 2 * (size_t)p->P.n_weights,
                                                  static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return cuda_fail(p, e, "grad_w clear");
        }
        return QTM_OK;
    }
    if (is_composite(p)) return composite_adjoint(p, B, gE, x, w, gx, gw, flags, stream);
    const Plan &P = p->P;
    if (!gE || (P.n_inputs > 0 && !x) || (P.n_weights > 0 && !w))
        return fail(p, QTM_EINVAL, "null pointer");
    if (flags & ~(QTM_ADJ_GW_PER_SAMPLE | QTM_ADJ_RECOMPUTE)) return fail(p, QTM_EINVAL, "unknown flags");
    const bool recompute = (flags & QTM_ADJ_RECOMPUTE) != 0;
    const bool per_sample = (flags & QTM_ADJ_GW_PER_SAMPLE) != 0;
    if (!recompute && !(p->fwd_valid && p->fwd_B == B && p->fwd_x == x && p->fwd_w == w))
        return fail(p, QTM_ESTATE, "no stored forward for these (B, x, w); pass QTM_ADJ_RECOMPUTE");
    qtm_status st = ensure_device(p);
    if (st != QTM_OK) return st;
    st = ensure_workspace(p, B);
    if (st != QTM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    prof_begin_call(p, 1, s);
    if (P.path == QTM_PATH_NAIVE) {
        NaiveArgs a = naive_args(p, B, x, w, gE);
        if (recompute) {
            a.E = nullptr;
            e = naive_forward(P.dtype, a, s, nullptr);
            if (e != cudaSuccess) return cuda_fail(p, e, "naive forward");
        }
        a.gx = gx; a.gw_out = gw;
        e = naive_adjoint(P.dtype, a, per_sample, s, nullptr);
        if (e != cudaSuccess) return cuda_fail(p, e, "naive adjoint");
        p->fwd_valid = false;
        return QTM_OK;
    }
    if (recompute) {
        st = run_forward_passes(p, B, x, w, s);
        if (st != QTM_OK) return st;
    }
    if (!P.pterms.empty()) {   // the costate's X/Y part, which the first reverse pass loads
        ProfScope ps(p, 1);
        e = launch_pauli_costate(P.dtype, p->d_phi, P.state_qubits, p->d_pterms, (int)P.pterms.size(), gE, P.n_obs,
                                 B, p->d_lam, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "pauli costate");
    }
    bool consumes = false;
    const bool fused = fuse_sample_steps(p) && !P.rev.empty();
    for (size_t i = 0; i < P.rev.size(); ++i) {
        PassArgs a = pass_args(p, P.rev[i], p->g_rev[i], p->smem_rev[i], B, x, w, gE);
        if (fused && i + 1 == P.rev.size()) {
            set_prep_fields(p, a);
            a.finalize_fused = 1;
            a.gx = gx;
            a.gw_out = per_sample ? gw : nullptr;
            a.gw_ws = (!per_sample && gw) ? p->d_gw_ws : nullptr;
        }
        if (P.rev[i].store_phi) consumes = true;
        ProfScope ps(p, 0);
        e = launch_any(p, true, i, a, p->tm_rev_phi[i], p->tm_rev_lam[i], s);
        if (e != cudaSuccess) return cuda_fail(p, e, "reverse pass launch");
    }
    if (!fused) {
        FinalizeArgs f = finalize_args(p, B, x, w);
        f.gx = gx;
        f.gw_out = per_sample ? gw : nullptr;
        f.gw_ws = (!per_sample && gw) ? p->d_gw_ws : nullptr;
        {
            ProfScope ps(p, 1);
            e = launch_grad_finalize(P.dtype, f, s);
        }
        if (e != cudaSuccess) return cuda_fail(p, e, "gradient finalize");
    }
    if (!per_sample && gw) {
        ProfScope ps(p, 1);
        e = launch_gw_reduce(P.dtype, p->d_gw_ws, B, P.n_weights, gw, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "gw reduce");
    }
    // the smem path leaves the stored state untouched; HBM sweeps consume it
    p->fwd_valid = !consumes && (recompute ? true : p->fwd_valid);
    if (recompute && !consumes) { p->fwd_B = B; p->fwd_x = x; p->fwd_w = w; p->fwd_stream = stream; }
    return QTM_OK;
}

qtm_status qtm_debug_fma_rate(int dtype, double *flops_per_s)
{
    if (!flops_per_s || (dtype != QTM_C64 && dtype != QTM_C128)) return QTM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QTM_ECUDA;
    const int blocks = sms * 16;
    void *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * 256 * elem_bytes(dtype)) != cudaSuccess) return QTM_ENOMEM;
    const int iters = dtype == QTM_C128 ? 1 << 11 : 1 << 14;
    cudaError_t e = probe_fma_rate(dtype, out, blocks, iters, nullptr, flops_per_s);
    cudaFree(out);
    return e == cudaSuccess ? QTM_OK : QTM_ECUDA;
}

qtm_status qtm_debug_gate_rate(double *flops_per_s)
{
    if (!flops_per_s) return QTM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QTM_ECUDA;
    const int blocks = sms * 2 * 4;   // four waves of two CTAs per SM
    // an SU(2) matrix a = 0.6 + 0.48i, b = 0.64 (|a|^2 + |b|^2 = 1) in the
    // broadcast form of the complex-pair tables, then 16 amplitude pairs
    float tab[44] = {0.6f, 0.6f, -0.48f, 0.48f, 0.64f, 0.64f, -0.f, 0.f, -0.64f, -0.64f, 0.48f, -0.48f};
    for (int j = 0; j < 16; ++j) { tab[12 + 2 * j] = 0.25f; tab[13 + 2 * j] = 0.125f * (float)((j & 3) - 1); }
    float *out = nullptr, *dtab = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float)) != cudaSuccess) return QTM_ENOMEM;
    if (cudaMalloc(&dtab, sizeof(tab)) != cudaSuccess) { cudaFree(out); return QTM_ENOMEM; }
    cudaError_t e = cudaMemcpy(dtab, tab, sizeof(tab), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = probe_gate_rate(out, dtab, blocks, 1 << 11, nullptr, flops_per_s);
    cudaFree(dtab);
    cudaFree(out);
    return e == cudaSuccess ? QTM_OK : QTM_ECUDA;
}

qtm_status qtm_jacobian(qtm_plan *p, int B, const void *x, const void *w, void *jac, void *stream)
{
    NvtxRange nvtx_range("qtm_jacobian");
    if (!p) return QTM_EINVAL;
    qtm_status bs = check_batch(p, B);
    if (bs != QTM_OK) return bs;
    if (B == 0) {   // the Jacobian of an empty batch has no elements
        drop_stored_forward(p);
        return QTM_OK;
    }
    if (is_composite(p)) return composite_jacobian(p, B, x, w, jac, stream);
    const Plan &P = p->P;
    if ((P.n_inputs > 0 && !x) || (P.n_weights > 0 && !w) || !jac) return fail(p, QTM_EINVAL, "null pointer");
    if (P.path != QTM_PATH_FUSED) return fail(p, QTM_EUNSUPPORTED, "qtm_jacobian runs on the fused path");
    qtm_status st = ensure_device(p);
    if (st != QTM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t csize = elem_bytes(P.dtype), rsize = csize / 2;
    const size_t row = csize << P.state_qubits;   // one sample's state
    const int M = P.n_obs;
    const int G = P.n_user_gates;   // Jacobian columns: the gates as given
    // One costate per observable (Sec. II-B's (B, M, |Theta|) output), all of
    // a chunk of observables in one reverse sweep: pseudo-sample b * cc + k
    // is sample b with cotangent e_(m0 + k), starting from b's final state.
    // The forward runs once; its states are kept and expanded per chunk.
    const int c = jacobian_chunk(p, B);
    st = ensure_workspace(p, B * c);
    if (st != QTM_OK) return st;
    if (ensure_buffer(p->d_jkeep, p->jkeep_bytes, row * (size_t)B) != cudaSuccess ||
        ensure_buffer(p->d_jx, p->jx_bytes, rsize * (size_t)B * c * std::max(1, P.n_inputs)) != cudaSuccess)
        return fail(p, QTM_ENOMEM, "jacobian buffer allocation failed");
    cudaError_t e = cudaMemsetAsync(jac, 0, rsize * (size_t)B * M * (G > 0 ? G : 1), s);
    if (e != cudaSuccess) return cuda_fail(p, e, "jacobian clear");
    p->fwd_valid = false;
    prof_begin_call(p, 1, s);
    st = run_forward_passes(p, B, x, w, s);
    if (st != QTM_OK) return st;
    e = cudaMemcpyAsync(p->d_jkeep, p->d_phi, row * (size_t)B, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "jacobian state copy");
    for (int m0 = 0; m0 < M; m0 += c) {
        const int cc = std::min(c, M - m0), Bp = B * cc;
        e = launch_expand_rows(p->d_jkeep, p->d_phi, row, Bp, cc, s);
        if (e == cudaSuccess && P.n_inputs > 0) e = launch_expand_x(P.dtype, x, p->d_jx, P.n_inputs, Bp, cc, s);
        if (e == cudaSuccess) e = launch_onehot(P.dtype, p->d_onehot, Bp, M, m0, cc, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "jacobian pseudo-samples");
        const void *xp = P.n_inputs > 0 ? p->d_jx : x;
        st = run_prep(p, Bp, xp, w, s);   // run matrices and tables of the pseudo-samples
        if (st != QTM_OK) return st;
        if (!P.pterms.empty()) {
            e = launch_pauli_costate(P.dtype, p->d_phi, P.state_qubits, p->d_pterms, (int)P.pterms.size(),
                                     p->d_onehot, M, Bp, p->d_lam, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "pauli costate");
        }
        for (size_t i = 0; i < P.rev.size(); ++i) {
            PassArgs a = pass_args(p, P.rev[i], p->g_rev[i], p->smem_rev[i], Bp, xp, w, p->d_onehot);
            ProfScope ps(p, 0);
            e = launch_any(p, true, i, a, p->tm_rev_phi[i], p->tm_rev_lam[i], s);
            if (e != cudaSuccess) return cuda_fail(p, e, "reverse pass launch");
        }
        FinalizeArgs f = finalize_args(p, Bp, xp, w);
        e = launch_grad_finalize(P.dtype, f, s);
        if (e == cudaSuccess)
            e = launch_jac_scatter(P.dtype, p->d_abar, p->d_gate_of_rot, (int)P.rots.size(), Bp, M, m0, cc, G, jac, s);
        if (e != cudaSuccess) return cuda_fail(p, e, "gradient finalize / jacobian scatter");
    }
    return QTM_OK;
}

namespace {

bool applies_udagger(const Plan &P, const PassDesc &pd)
{
    for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph)
        for (int o = P.phases[ph].op_begin; o < P.phases[ph].op_end; ++o)
            if (P.ops[o].type == OP_GRAD && !(P.ops[o].flags & OPF_SKIP_APPLY)) return true;
    return false;
}

// Generate and compile every pass (host only; NVRTC, no device).
qtm_status compile_all(qtm_plan *p, std::vector<std::vector<char>> &fwd_bin, std::vector<std::vector<char>> &rev_bin)
{
    const Plan &P = p->P;
    if (P.path != QTM_PATH_FUSED) return fail(p, QTM_EUNSUPPORTED, "specialised kernels exist for fused plans");
    if (!jit_nvrtc_available()) return fail(p, QTM_EUNSUPPORTED, "NVRTC not found");
    struct Job { const PassDesc *pd; std::vector<char> *out; int minb; };
    std::vector<Job> jobs;
    fwd_bin.assign(P.fwd.size(), {});
    rev_bin.assign(P.rev.size(), {});
    // CTAs per SM the register budget is compiled for (forward, reverse)
    int minb_f = p->minb_f, minb_r = p->minb_r;
    if (const char *e = std::getenv("QTM_JIT_MINB")) {   // tuning: "<forward>,<reverse>"
        int f = 0, r = 0;
        if (std::sscanf(e, "%d,%d", &f, &r) == 2 && f >= 1 && f <= 8 && r >= 1 && r <= 8) { minb_f = f; minb_r = r; }
    }
    for (size_t i = 0; i < P.fwd.size(); ++i) {
        if (!jit_eligible(P, P.fwd[i])) return fail(p, QTM_EUNSUPPORTED, "plan has passes the specialiser does not cover");
        jobs.push_back({&P.fwd[i], &fwd_bin[i], minb_f});
    }
    for (size_t i = 0; i < P.rev.size(); ++i) {
        if (!jit_eligible(P, P.rev[i])) return fail(p, QTM_EUNSUPPORTED, "plan has passes the specialiser does not cover");
        // a reverse pass that applies no U^dagger (every gradient is its qubit's
        // last) holds no second register state: the forward budget, more CTAs
        jobs.push_back({&P.rev[i], &rev_bin[i], applies_udagger(P, P.rev[i]) ? minb_r : std::max(minb_r, minb_f)});
    }
    std::vector<std::string> logs(jobs.size());
    std::vector<char> ok(jobs.size(), 0);
    std::vector<std::thread> th;
    for (size_t k = 0; k < jobs.size(); ++k)
        th.emplace_back([&, k] {
            ok[k] = jit_compile(jit_source(P, *jobs[k].pd, jobs[k].minb), *jobs[k].out, logs[k]) ? 1 : 0;
        });
    for (auto &t : th) t.join();
    for (size_t k = 0; k < jobs.size(); ++k)
        if (!ok[k]) return fail(p, QTM_EINVAL, "generated kernel failed to compile: " + logs[k].substr(0, 4000));
    return QTM_OK;
}

}  // namespace

qtm_status qtm_compile(qtm_plan *p, int flags)
{
    NvtxRange nvtx_range("qtm_compile");
    if (!p) return QTM_EINVAL;
    if (is_composite(p)) {
        for (qtm_plan *part : p->parts) {
            qtm_status st = qtm_compile(part, flags);
            if (st != QTM_OK) return part_fail(p, part, st);
        }
        return QTM_OK;
    }
    if (flags != 0) return fail(p, QTM_EINVAL, "flags must be 0");
    if (!jit_available()) return fail(p, QTM_EUNSUPPORTED, "NVRTC or driver entry points not available");
    qtm_status st = ensure_device(p);
    if (st != QTM_OK) return st;
    std::vector<std::vector<char>> fb, rb;
    st = compile_all(p, fb, rb);
    if (st != QTM_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();   // no launch of the old kernels or layout is in flight
    if (e != cudaSuccess) return cuda_fail(p, e, "synchronize before loading kernels");
    auto unload_all = [p] {
        for (auto *v : {&p->jit_fwd, &p->jit_rev})
            for (auto &k : *v) jit_unload(k);
        p->jit_device = -1;
    };
    unload_all();
    // the state layout in HBM changes with the kernels: drop the workspace and
    // any stored forward state
    free_workspace(p);
    p->cap_B = 0;
    p->fwd_valid = false;
    const Plan &P = p->P;
    p->jit_fwd.assign(P.fwd.size(), JitKernel{});
    p->jit_rev.assign(P.rev.size(), JitKernel{});
    std::string err;
    for (int rev = 0; rev < 2; ++rev) {
        const auto &pds = rev ? P.rev : P.fwd;
        auto &ks = rev ? p->jit_rev : p->jit_fwd;
        const auto &bins = rev ? rb : fb;
        for (size_t i = 0; i < pds.size(); ++i) {
            const int smem = (int)jit_smem_bytes_cpx(P, pds[i]);
            if ((size_t)smem > kMaxDynSmem) {
                unload_all();
                return fail(p, QTM_EUNSUPPORTED, "specialised kernel needs more shared memory than a CTA has");
            }
            if (!jit_load(bins[i], smem, ks[i], err)) {
                unload_all();
                return fail(p, QTM_ECUDA, err);
            }
        }
    }
    p->jit_device = p->device;
    return QTM_OK;
}

qtm_status qtm_get_schedule(const qtm_plan *p, qtm_schedule *sched)
{
    if (!p || !sched) return QTM_EINVAL;
    if (is_composite(p) || p->P.path != QTM_PATH_FUSED) return QTM_EUNSUPPORTED;
    sched->phase_mode = p->P.phase_mode;
    sched->tile_qubits = p->P.K;
    sched->low_min = p->P.low_min;
    sched->kernels = jit_active(p) ? 1 : 0;
    sched->minb_fwd = p->minb_f;
    sched->minb_rev = p->minb_r;
    return QTM_OK;
}

qtm_status qtm_set_schedule(qtm_plan *p, const qtm_schedule *sched)
{
    NvtxRange nvtx_range("qtm_set_schedule");
    if (!p || !sched) return QTM_EINVAL;
    if (is_composite(p) || p->P.path != QTM_PATH_FUSED)
        return fail(p, QTM_EUNSUPPORTED, "schedules apply to single fused plans");
    const qtm_schedule &q = *sched;
    const int kmax = p->P.dtype == QTM_C128 ? kMaxTileQubits128 : kMaxTileQubits;
    if (q.phase_mode < 0 || q.phase_mode > 2 || q.kernels < 0 || q.kernels > 1 || q.minb_fwd < 1 || q.minb_fwd > 4 ||
        q.minb_rev < 1 || q.minb_rev > 4 || (q.tile_qubits != 0 && (q.tile_qubits < kRegBits || q.tile_qubits > kMaxTileQubits)) ||
        q.low_min < kRegBits || q.low_min > kMaxTileQubits)
        return fail(p, QTM_EINVAL, "schedule field out of range");
    PlanOptions opt = p->opt;
    opt.phase_mode = q.phase_mode == 1 ? PHASES_ROUND_ROBIN : q.phase_mode == 2 ? PHASES_AUTO : PHASES_GREEDY;
    // a one-tile state reports its own width; only multi-tile states take the field
    const bool multi = p->P.state_qubits > kMaxTileQubits;
    if (multi && q.tile_qubits != 0 && q.tile_qubits < 9)
        return fail(p, QTM_EINVAL, "tiles of a multi-tile state have 9 .. 12 qubits");
    opt.tile_qubits = multi ? std::min(q.tile_qubits ? q.tile_qubits : kmax, kmax) : 0;
    opt.low_min = q.low_min;
    if (q.kernels == 1 && p->P.dtype != QTM_C64)
        return fail(p, QTM_EUNSUPPORTED, "specialised kernels exist for complex64 plans");
    // nothing of the old schedule may still run: tables, workspace and kernels go
    if (p->d_status) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (p->device >= 0) cudaSetDevice(p->device);
        cudaError_t e = cudaDeviceSynchronize();
        if (cur >= 0) cudaSetDevice(cur);
        if (e != cudaSuccess) return cuda_fail(p, e, "synchronize before re-planning");
    }
    const Plan old_P = p->P;
    const PlanOptions old_opt = p->opt;
    const int old_f = p->minb_f, old_r = p->minb_r;
    p->opt = opt;
    qtm_status st = plan_from_source(p, p->P.dtype);
    if (st != QTM_OK) { p->opt = old_opt; return st; }
    for (auto *v : {&p->jit_fwd, &p->jit_rev})
        for (auto &k : *v) jit_unload(k);
    p->jit_fwd.clear();
    p->jit_rev.clear();
    p->jit_device = -1;
    free_workspace(p);
    free_tables(p);
    p->device = -1;
    p->fwd_valid = false;
    p->minb_f = q.minb_fwd;
    p->minb_r = q.minb_rev;
    if (q.kernels == 1) {
        st = qtm_compile(p, 0);
        if (st != QTM_OK) {   // back to the old schedule on the general kernel
            const std::string why = p->err;
            p->P = old_P;
            p->opt = old_opt;
            p->minb_f = old_f;
            p->minb_r = old_r;
            plan_from_source(p, p->P.dtype);
            free_workspace(p);
            free_tables(p);
            p->device = -1;
            p->err = why;
            return st;
        }
    }
    return QTM_OK;
}

qtm_status qtm_tune(qtm_plan *p, int B, const void *x, const void *w, const void *gE, void *stream,
                    const char *cache_path)
{
    NvtxRange nvtx_range("qtm_tune");
    if (!p) return QTM_EINVAL;
    if (is_composite(p) || p->P.path != QTM_PATH_FUSED)
        return fail(p, QTM_EUNSUPPORTED, "schedules apply to single fused plans");
    const Plan &P0 = p->P;
    if (B < 1 || (P0.n_inputs > 0 && !x) || (P0.n_weights > 0 && !w) || !gE) return fail(p, QTM_EINVAL, "bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const std::string sig = tune_signature(p, B);
    qtm_schedule best{};
    qtm_status st = qtm_get_schedule(p, &best);
    if (st != QTM_OK) return st;
    if (tune_cache_lookup(cache_path, sig, best)) return qtm_set_schedule(p, &best);
    const size_t rsize = elem_bytes(P0.dtype) / 2;
    void *E = nullptr, *gx = nullptr, *gw = nullptr;
    if (cudaMalloc(&E, rsize * (size_t)B * std::max(1, P0.n_obs)) != cudaSuccess ||
        cudaMalloc(&gx, rsize * (size_t)B * std::max(1, P0.n_inputs)) != cudaSuccess ||
        cudaMalloc(&gw, rsize * std::max(1, P0.n_weights)) != cudaSuccess) {
        cudaFree(E); cudaFree(gx); cudaFree(gw);
        return fail(p, QTM_ENOMEM, "tuning scratch allocation failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // median time (ms) of forward + adjoint under schedule c; < 0 if c does not apply
    auto time_of = [&](const qtm_schedule &c) -> double {
        if (qtm_set_schedule(p, &c) != QTM_OK) return -1.0;
        std::vector<float> t;
        for (int rep = 0; rep < 7; ++rep) {
            cudaEventRecord(e0, s);
            if (qtm_forward(p, B, x, w, E, s) != QTM_OK ||
                qtm_adjoint(p, B, gE, x, w, P0.n_inputs > 0 ? gx : nullptr, P0.n_weights > 0 ? gw : nullptr, 0, s) !=
                    QTM_OK)
                return -1.0;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 2) t.push_back(ms);   // two warm-up steps
        }
        std::sort(t.begin(), t.end());
        return t[t.size() / 2];
    };
    if (P0.dtype == QTM_C64 && best.kernels == 0) {   // start from the specialised kernels where they apply
        qtm_schedule c = best;
        c.kernels = 1;
        if (qtm_set_schedule(p, &c) == QTM_OK) best = c;
    }
    double best_ms = time_of(best);
    if (best_ms < 0) {
        cudaFree(E); cudaFree(gx); cudaFree(gw);
        cudaEventDestroy(e0); cudaEventDestroy(e1);
        return fail(p, QTM_ECUDA, "timing the current schedule failed: " + p->err);
    }
    const bool multi = p->P.state_qubits > kMaxTileQubits;
    const int kmax = p->P.dtype == QTM_C128 ? kMaxTileQubits128 : kMaxTileQubits;
    // one knob at a time, each alternative against the best so far
    std::vector<std::vector<qtm_schedule>> rounds;
    auto with = [&](auto set) {
        std::vector<qtm_schedule> v;
        set(v);
        rounds.push_back(v);
    };
    with([&](std::vector<qtm_schedule> &v) { for (int m : {0, 1}) { qtm_schedule c{}; c.phase_mode = m; v.push_back(c); } });
    if (multi) {
        with([&](std::vector<qtm_schedule> &v) { for (int k = kmax; k >= std::max(9, kmax - 2); --k) { qtm_schedule c{}; c.tile_qubits = k; v.push_back(c); } });
        with([&](std::vector<qtm_schedule> &v) { for (int l : {4, 6, 8}) { qtm_schedule c{}; c.low_min = l; v.push_back(c); } });
    }
    if (p->P.dtype == QTM_C64) {
        with([&](std::vector<qtm_schedule> &v) {
            for (auto fr : {std::pair<int, int>{3, 2}, {2, 2}, {4, 2}, {3, 1}}) {
                qtm_schedule c{}; c.minb_fwd = fr.first; c.minb_rev = fr.second; v.push_back(c);
            }
        });
        with([&](std::vector<qtm_schedule> &v) { for (int k : {0, 1}) { qtm_schedule c{}; c.kernels = k; v.push_back(c); } });
    }
    for (size_t r = 0; r < rounds.size(); ++r)
        for (const qtm_schedule &alt : rounds[r]) {
            qtm_schedule c = best;
            if (r == 0) c.phase_mode = alt.phase_mode;
            else if (multi && r == 1) c.tile_qubits = alt.tile_qubits;
            else if (multi && r == 2) c.low_min = alt.low_min;
            else if (alt.minb_fwd) { c.minb_fwd = alt.minb_fwd; c.minb_rev = alt.minb_rev; }
            else c.kernels = alt.kernels;
            if (std::memcmp(&c, &best, sizeof(c)) == 0) continue;
            if (c.kernels == 0 && (c.minb_fwd != best.minb_fwd || c.minb_rev != best.minb_rev)) continue;
            const double ms = time_of(c);
            if (ms > 0 && ms < 0.99 * best_ms) { best = c; best_ms = ms; }
        }
    cudaFree(E); cudaFree(gx); cudaFree(gw);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    st = qtm_set_schedule(p, &best);
    if (st == QTM_OK) tune_cache_store(cache_path, sig, best, best_ms);
    return st;
}

int qtm_compiled_passes(const qtm_plan *p)
{
    if (!p) return 0;
    if (is_composite(p)) {
        int n = 0;
        for (const qtm_plan *part : p->parts) n += qtm_compiled_passes(part);
        return n;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->jit_device) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    for (const auto *v : {&p->jit_fwd, &p->jit_rev})
        for (const auto &k : *v) n += k.fn != nullptr;
    return n;
}

const char *qtm_debug_jit_source(const qtm_plan *p, int which, int index, int flags)
{
    if (!p) return "";
    const Plan &P = p->P;
    const auto &v = which ? P.rev : P.fwd;
    if (index < 0 || index >= (int)v.size()) return "";
    qtm_plan *m = const_cast<qtm_plan *>(p);
    m->jit_src_cache = flags == 0 && jit_eligible(P, v[index])
                           ? jit_source(P, v[index], which && applies_udagger(P, v[index]) ? 2 : 3)
                           : std::string();
    return m->jit_src_cache.c_str();
}

qtm_status qtm_debug_jit_compile(qtm_plan *p, int flags)
{
    if (!p) return QTM_EINVAL;
    if (flags != 0) return fail(p, QTM_EINVAL, "flags must be 0");
    std::vector<std::vector<char>> fb, rb;
    return compile_all(p, fb, rb);
}

qtm_status qtm_sync(qtm_plan *p, void *stream)
{
    if (!p) return QTM_EINVAL;
    if (is_composite(p)) {
        for (qtm_plan *part : p->parts) {
            qtm_status st = qtm_sync(part, stream);
            if (st != QTM_OK) return part_fail(p, part, st);
        }
        return QTM_OK;
    }
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(p, e, "stream synchronize");
    if (!p->d_status) return QTM_OK;
    unsigned st = 0;
    e = cudaMemcpy(&st, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "status read");
    if (st) {
        unsigned zero = 0;
        cudaMemcpy(p->d_status, &zero, sizeof(unsigned), cudaMemcpyHostToDevice);
        return fail(p, QTM_ETIMEOUT, "a device-side wait gave up");
    }
    return QTM_OK;
}

qtm_status qtm_set_profiling(qtm_plan *p, int enable)
{
    if (!p) return QTM_EINVAL;
    if (enable < 0 || enable > 2) return QTM_EINVAL;
    p->profiling = enable;
    return QTM_OK;
}

qtm_status qtm_get_launch_times(qtm_plan *p, int which, float *ms, int *kinds, int cap, int *count)
{
    if (!p || which < 0 || which > 1 || cap < 0) return QTM_EINVAL;
    const auto &v = p->recs[which];
    if (count) *count = (int)v.size();
    for (int i = 0; i < (int)v.size() && i < cap; ++i) {
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, v[i].a, v[i].b);
        if (e != cudaSuccess) return cuda_fail(p, e, "event elapsed time");
        if (ms) ms[i] = t;
        if (kinds) kinds[i] = v[i].kind;
    }
    return QTM_OK;
}

qtm_status qtm_destroy(qtm_plan *p)
{
    if (!p) return QTM_EINVAL;
    for (qtm_plan *part : p->parts) qtm_destroy(part);
    p->parts.clear();
    if (p->d_tmp) cudaFree(p->d_tmp);
    p->d_tmp = nullptr;
    for (const auto &pool : p->ev_pool)
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    for (auto *v : {&p->jit_fwd, &p->jit_rev})
        for (auto &k : *v) jit_unload(k);
    if (p->d_status) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(p->device);
        cudaDeviceSynchronize();
        free_workspace(p);
        free_tables(p);
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete p;
    return QTM_OK;
}

const char *qtm_debug_describe(const qtm_plan *p)
{
    if (!p) return "";
    qtm_plan *m = const_cast<qtm_plan *>(p);
    m->describe_cache = p->P.describe();
    return m->describe_cache.c_str();
}

qtm_status qtm_debug_emulate(const qtm_plan *p, int B, const double *x, const double *w,
                             const double *gE, double *E, double *gx, double *gw)
{
    if (!p || B < 1) return QTM_EINVAL;
    if (is_composite(p)) {   // sum of the parts, in part order
        const Plan &P = p->P;
        std::vector<double> e((size_t)B * P.n_obs), a((size_t)B * P.n_inputs), b((size_t)B * P.n_weights);
        if (E) std::fill(E, E + e.size(), 0.0);
        if (gx) std::fill(gx, gx + a.size(), 0.0);
        if (gw) std::fill(gw, gw + b.size(), 0.0);
        for (const qtm_plan *part : p->parts) {
            qtm_status st = qtm_debug_emulate(part, B, x, w, gE, E ? e.data() : nullptr, gx ? a.data() : nullptr,
                                              gw ? b.data() : nullptr);
            if (st != QTM_OK) { const_cast<qtm_plan *>(p)->err = part->err; return st; }
            for (size_t i = 0; E && i < e.size(); ++i) E[i] += e[i];
            for (size_t i = 0; gx && i < a.size(); ++i) gx[i] += a[i];
            for (size_t i = 0; gw && i < b.size(); ++i) gw[i] += b[i];
        }
        return QTM_OK;
    }
    std::string err;
    qtm_status st = emulate_plan(p->P, B, x, w, gE, E, gx, gw, err);
    if (st != QTM_OK) const_cast<qtm_plan *>(p)->err = err;
    return st;
}

}  // extern "C"
