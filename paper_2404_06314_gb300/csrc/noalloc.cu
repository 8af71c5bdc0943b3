// qtm_forward_noalloc: expectation values without any device allocation.
//
// Some callers cannot call cudaMalloc: a host program whose GPU memory is
// owned by another allocator with a fixed budget (a framework that reserves
// the device's memory up front, an embedding application that forbids its
// plugins to allocate), and loops that must not stall on an allocation, which
// can synchronise the device.  For them this entry point runs the same fused
// forward kernels as qtm_forward (per-sample FP64 prep, one shared-memory pass,
// fixed-order reduction) but takes every device-side table and every scratch
// buffer from one file-scope device array, g_scratch, that the library holds
// on each GPU it is loaded on until the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>
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
// Device address of g_scratch per device ordinal, and the context it was
// resolved in: a device reset (cudaDeviceReset, or a primary-context reset by
// another library) unloads the module, and the array may come back at another
// address, so a cached address is only used in the context that produced it.
struct ScratchAddr {
    void *ptr = nullptr;
    unsigned long long ctx_id = 0;
};
ScratchAddr g_scratch_addr[256];

// Unique id of the current context (0 if the driver entry points are missing).
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// g_scratch's device address on the current device.  Set-up, once per device
// (and again after that device's context was replaced): cudaGetSymbolAddress
// with the device current.  The first call on a device also loads the
// library's device code there.
cudaError_t scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();   // 0 before the device's first use
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr &a = g_scratch_addr[dev];
    if (!a.ptr || ctx == 0 || a.ctx_id != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);   // makes the device's primary context current
        if (e != cudaSuccess) return e;
        a.ptr = p;
        a.ctx_id = current_context_id();
    }
    *out = a.ptr;
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

    // The plan's tables (a few KB) are copied from its host vectors on every
    // call: cudaMemcpyAsync from pageable memory returns once the bytes have
    // been staged, so the call does not depend on the plan after it returns.
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
    // The pass takes a status word, but this path loads no tiles (no TMA, rank
    // 0 below), so it runs no bounded device wait and never sets the word;
    // it is zeroed only so that the kernel never sees a stale value.
    if (e == cudaSuccess) e = cudaMemsetAsync(sb + o_status, 0, sizeof(unsigned), s);
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
