// Kernel argument blocks and launch declarations (CUDA side, internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "plan.h"

namespace qtm {

// An NVTX range around one C-ABI call (named by the entry point), so that
// profilers that read NVTX (ncu --nvtx, nsys) attribute kernels to calls;
// without such a tool attached the calls do nothing measurable.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


struct FinalizeArgs {
    int B, M, tiles, n_runs, n_rots, P, n_in;
    const Run *runs;
    const Rot *rots;
    const int32_t *w_ptr, *w_rots, *x_ptr, *x_rots;
    const void *x, *w;            // plan real type
    const double *Epart;
    double *Gpart;                // [B][n_runs][tiles][3]; the finalize sums tiles in place
    void *E;                      // [B][M] real type (may be null)
    double *abar;                 // [B][n_rots] workspace
    void *gx;                     // [B][n_in] real (may be null)
    void *gw_out;                 // per-sample [B][P] real (may be null)
    double *gw_ws;                // per-sample [B][P] double workspace (may be null)
    const double2 *cs;            // [B][n_rots] (cos, sin) of half angles from the prep (may be null)
};

struct PrepArgs {
    int B, n, state_qubits, n_runs, n_in;
    const Run *runs;
    const Rot *rots;
    const int32_t *prefix_run_of_q;
    const void *x, *w;            // plan real type
    void *mats;                   // out: [B][n_runs][4] complex
    void *tabs;                   // out: [B][ntab][16] complex
    double2 *cs;                  // out: [B][n_rots] (cos, sin) of half angles (may be null)
    int n_rots;
};

// Per-sample run matrices and product-state tables, computed in FP64 and
// rounded once to the plan's complex type.
cudaError_t launch_prep(int dtype, const PrepArgs &a, cudaStream_t s);

// Shared memory a pass kernel needs (bytes), for K tile qubits.
size_t pass_smem_bytes(int K, int dtype, bool reverse, int nslots, int n_terms, int M,
                       int state_qubits, int n_prefix_ents);

cudaError_t launch_pass(int dtype, bool reverse, const PassArgs &a, const CUtensorMap &tm_phi,
                        const CUtensorMap &tm_lam, cudaStream_t s, bool pdl = false);
cudaError_t launch_expval_finalize(int dtype, const FinalizeArgs &f, cudaStream_t s);
cudaError_t launch_grad_finalize(int dtype, const FinalizeArgs &f, cudaStream_t s);
// FP64 (cos, sin) of the half angles of the rotations without an input,
// at cs_shared[i] for each i with rep[i] == i.
cudaError_t launch_prep_shared(int dtype, const Rot *rots, const int32_t *rep, int n_rots, const void *w,
                               double2 *cs_shared, cudaStream_t s);
cudaError_t launch_gw_reduce(int dtype, const double *gw_ws, int B, int P, void *gw,
                             cudaStream_t s);

// composite plans: dst[i] += src[i]; dst[r][g] += src[r][g] for g < Gd
cudaError_t launch_accumulate(int dtype, const void *src, void *dst, size_t n, cudaStream_t s);
cudaError_t launch_accumulate_cols(int dtype, const void *src, int Gs, void *dst, int Gd, size_t rows, cudaStream_t s);

// Jacobian pseudo-samples (b' = b * cc + k stands for sample b, observable
// m0 + k): one-hot cotangents, the scatter of per-rotation gradients into
// J [B][M][G], and the expansion of per-sample rows (states, inputs).
cudaError_t launch_onehot(int dtype, void *gE, int Bp, int M, int m0, int cc, cudaStream_t s);
cudaError_t probe_fma_rate(int dtype, void *out, int blocks, int iters, cudaStream_t s, double *flops_per_s);
cudaError_t probe_gate_rate(float *out, const float *tab, int blocks, int iters, cudaStream_t s, double *flops_per_s);
cudaError_t launch_expand_rows(const void *src, void *dst, size_t row_bytes, int Bp, int cc, cudaStream_t s);
cudaError_t launch_expand_x(int dtype, const void *x, void *xp, int n_in, int Bp, int cc, cudaStream_t s);

// Pauli strings with X/Y factors on the final state phi [B][2^sq] (pauli.cu):
// E[b][m] += their expectation values (Ppart: [B][pauli_chunks(sq)][T] FP64
// scratch), and lam = their part of the costate for cotangents gE [B][M].
int pauli_chunks(int sq);
cudaError_t launch_pauli_expval(int dtype, const void *phi, int sq, const PauliTerm *terms, int T, int B, int M,
                                double *Ppart, void *E, cudaStream_t s);
cudaError_t launch_pauli_costate(int dtype, const void *phi, int sq, const PauliTerm *terms, int T, const void *gE,
                                 int M, int B, void *lam, cudaStream_t s);
cudaError_t launch_jac_scatter(int dtype, const double *abar, const int32_t *gate_of_rot, int n_rots, int Bp,
                               int M, int m0, int cc, int G, void *J, cudaStream_t s);

// naive one-gate-per-kernel path
struct NaiveArgs {
    int n, B, n_in, M, n_terms, n_rots, P;
    const qtm_gate *gates_host;   // host copy (launch loop)
    int n_gates;
    const Term *terms;
    const int32_t *rot_of_gate_host;
    const Rot *rots;
    const int32_t *w_ptr, *w_rots, *x_ptr, *x_rots;
    const void *x, *w, *gE;
    void *phi, *lam;              // [B][2^n] complex
    double *abar;                 // [B][n_rots]
    void *E, *gx, *gw_out;
    double *gw_ws;
};
cudaError_t naive_forward(int dtype, const NaiveArgs &a, cudaStream_t s, int *launches);
cudaError_t naive_adjoint(int dtype, const NaiveArgs &a, bool gw_per_sample, cudaStream_t s,
                          int *launches);

}  // namespace qtm
