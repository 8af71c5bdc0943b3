// qtm_forward_noalloc: expectation values without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into a CUDA graph (allocation is not a capturable operation and may
// synchronise the device), programs whose GPU memory belongs to another
// allocator with a fixed budget, and latency-critical loops where a first-call
// allocation would stall.  For them this entry point runs the same fused
// forward kernels as qtm_forward (per-sample FP64 prep, one shared-memory pass,
// fixed-order reduction) but takes every device-side table and every scratch
// buffer from one file-scope device array, g_scratch, that the library holds
// on each GPU it is loaded on until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qtm.h"
#include "device.h"
#include "plan.h"

using namespace qtm;

namespace {

static __device__ __align__(256) unsigned char g_scratch[QTM_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_ptr[256] = {nullptr};   // device address of g_scratch, per device ordinal

// Resolve g_scratch's device address for the current device (once per device).
cudaError_t scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t at = (off + 255) & ~size_t(255);
        off = at + (bytes ? bytes : 1);
        return at;
    }
};

}  // namespace

// Host-side description of the plan, reachable without the plan's own device
// tables (defined in capi.cu).
const qtm::Plan *qtm_internal_plan(const qtm_plan *plan);
bool qtm_internal_is_composite(const qtm_plan *plan);

extern "C" qtm_status qtm_forward_noalloc(qtm_plan *plan, int B, const void *x, const void *w,
                                          void *expvals, void *stream)
{
    if (!plan) return QTM_EINVAL;
    if (qtm_internal_is_composite(plan)) return QTM_EUNSUPPORTED;   // Pauli-string observables: several plans
    const Plan &P = *qtm_internal_plan(plan);
    if (!P.pterms.empty()) return QTM_EUNSUPPORTED;   // X/Y observables need the state in memory
    if (B < 1) return QTM_EINVAL;
    if ((P.n_inputs > 0 && !x) || (P.n_weights > 0 && !w) || !expvals) return QTM_EINVAL;
    if (P.path != QTM_PATH_FUSED || P.fwd.size() != 1 || P.tiles_per_sample != 1)
        return QTM_EUNSUPPORTED;   // whole state in one shared-memory tile only (n <= 12)
    const PassDesc &pd = P.fwd[0];
    if (pd.phi_src != SRC_ANALYTIC) return QTM_EUNSUPPORTED;

    const size_t csize = elem_bytes(P.dtype);
    const int ntab = (P.state_qubits + 3) / 4;
    const size_t nruns = P.runs.empty() ? 1 : P.runs.size();
    Carve c;
    const size_t o_ops = c.take(sizeof(DevOp) * P.ops.size());
    const size_t o_diag = c.take(sizeof(DiagPair) * P.diag_pairs.size());
    const size_t o_phases = c.take(sizeof(DevPhase) * P.phases.size());
    const size_t o_slots = c.take(sizeof(int32_t) * P.slot_runs.size());
    const size_t o_runs = c.take(sizeof(Run) * P.runs.size());
    const size_t o_rots = c.take(sizeof(Rot) * P.rots.size());
    const size_t o_prq = c.take(sizeof(int32_t) * P.prefix_run_of_q.size());
    const size_t o_ents = c.take(sizeof(Ent) * P.pass_ents.size());
    const size_t o_terms = c.take(sizeof(Term) * P.terms.size());
    const size_t o_amap = c.take(sizeof(MaskTerm) * P.amap_terms.size());
    const size_t o_status = c.take(sizeof(unsigned));
    const size_t o_mats = c.take(csize * 4 * nruns * (size_t)B);
    const size_t o_tabs = c.take(csize * 16 * ntab * (size_t)B);
    const size_t o_epart = c.take(sizeof(double) * (size_t)B * P.n_obs);
    if (c.off > (size_t)QTM_NOALLOC_SCRATCH_BYTES) return QTM_EINVAL;   // batch too large for the array

    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return QTM_ECUDA;
    unsigned char *sb = static_cast<unsigned char *>(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes == 0 || e != cudaSuccess) return;
        e = cudaMemcpyAsync(sb + off, src, bytes, cudaMemcpyHostToDevice, s);
    };
    put(o_ops, P.ops.data(), sizeof(DevOp) * P.ops.size());
    put(o_diag, P.diag_pairs.data(), sizeof(DiagPair) * P.diag_pairs.size());
    put(o_phases, P.phases.data(), sizeof(DevPhase) * P.phases.size());
    put(o_slots, P.slot_runs.data(), sizeof(int32_t) * P.slot_runs.size());
    put(o_runs, P.runs.data(), sizeof(Run) * P.runs.size());
    put(o_rots, P.rots.data(), sizeof(Rot) * P.rots.size());
    put(o_prq, P.prefix_run_of_q.data(), sizeof(int32_t) * P.prefix_run_of_q.size());
    put(o_ents, P.pass_ents.data(), sizeof(Ent) * P.pass_ents.size());
    put(o_terms, P.terms.data(), sizeof(Term) * P.terms.size());
    put(o_amap, P.amap_terms.data(), sizeof(MaskTerm) * P.amap_terms.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(sb + o_status, 0, sizeof(unsigned), s);   // starts at zero
    if (e != cudaSuccess) return QTM_ECUDA;

    PrepArgs pa{};
    pa.B = B; pa.n = P.n; pa.state_qubits = P.state_qubits; pa.n_runs = (int)P.runs.size();
    pa.n_in = P.n_inputs;
    pa.runs = reinterpret_cast<const Run *>(sb + o_runs);
    pa.rots = reinterpret_cast<const Rot *>(sb + o_rots);
    pa.prefix_run_of_q = reinterpret_cast<const int32_t *>(sb + o_prq);
    pa.x = x; pa.w = w; pa.mats = sb + o_mats; pa.tabs = sb + o_tabs;
    e = launch_prep(P.dtype, pa, s);
    if (e != cudaSuccess) return QTM_ECUDA;

    PassArgs a{};
    a.K = pd.K; a.l = pd.l; a.h = pd.h; a.m = pd.m;
    a.state_qubits = P.state_qubits; a.n = P.n;
    a.tiles = 1; a.log_tiles = 0; a.B = B;
    a.rank = 0; a.low_dims = 0; a.gap_dim = 0; a.high_dims = 0;   // no TMA: nothing loaded or stored
    a.ops = reinterpret_cast<const DevOp *>(sb + o_ops);
    a.diag = reinterpret_cast<const DiagPair *>(sb + o_diag);
    a.phases = reinterpret_cast<const DevPhase *>(sb + o_phases);
    a.phase_begin = pd.phase_begin; a.phase_end = pd.phase_end;
    a.slot_runs = reinterpret_cast<const int32_t *>(sb + o_slots);
    a.slot_begin = pd.slot_begin; a.nslots = pd.slot_end - pd.slot_begin;
    a.n_runs = (int)P.runs.size();
    a.mats = sb + o_mats; a.tabs = sb + o_tabs;
    a.prefix_ents = reinterpret_cast<const Ent *>(sb + o_ents) + pd.ents_begin;
    a.analytic_ents = pd.analytic_ents;
    a.amap = reinterpret_cast<const MaskTerm *>(sb + o_amap) + (pd.amap_lin >= 0 ? pd.amap_begin : 0);
    a.amap_lin = pd.amap_lin; a.amap_quad = pd.amap_quad; a.amap_dlin = pd.amap_dlin;
    a.phi_src = SRC_ANALYTIC; a.lam_src = SRC_NONE;
    a.store_phi = 0; a.store_lam = 0; a.has_expval = 1;
    a.terms = reinterpret_cast<const Term *>(sb + o_terms);
    a.n_terms = (int)P.terms.size(); a.M = P.n_obs;
    a.x = x; a.w = w; a.gE = nullptr; a.n_in = P.n_inputs;
    a.Epart = reinterpret_cast<double *>(sb + o_epart);
    a.Gpart = nullptr;
    a.status = reinterpret_cast<unsigned *>(sb + o_status);
    a.smem_bytes = (int)pass_smem_bytes(pd.K, P.dtype, false, a.nslots, a.n_terms, a.M,
                                        P.state_qubits, a.analytic_ents);
    CUtensorMap unused;
    std::memset(&unused, 0, sizeof(unused));
    e = launch_pass(P.dtype, false, a, unused, unused, s);
    if (e != cudaSuccess) return QTM_ECUDA;

    FinalizeArgs f{};
    f.B = B; f.M = P.n_obs; f.tiles = 1;
    f.Epart = a.Epart;
    f.E = expvals;
    e = launch_expval_finalize(P.dtype, f, s);
    return e == cudaSuccess ? QTM_OK : QTM_ECUDA;
}
