// Run-time specialised pass kernels (see jit.cpp).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "plan.h"

namespace qtm {

struct JitKernel {
    void *mod = nullptr;   // CUmodule
    void *fn = nullptr;    // CUfunction
    int smem = 0;          // dynamic shared memory per CTA
};

// Passes worth specialising: fused complex64 passes whose tile has >= 9 qubits
// (full warps).
bool jit_eligible(const Plan &P, const PassDesc &pd);
bool jit_available();
bool jit_nvrtc_available();
// Generated source of one pass: one sample per CTA, each complex amplitude
// one f32x2 register pair (tile_cpx.cuh), compiled for min_blocks CTAs per SM.
std::string jit_source(const Plan &P, const PassDesc &pd, int min_blocks);
size_t jit_smem_bytes_cpx(const Plan &P, const PassDesc &pd);
bool jit_compile(const std::string &body, std::vector<char> &cubin, std::string &log);
bool jit_load(const std::vector<char> &cubin, int smem, JitKernel &k, std::string &err);
void jit_unload(JitKernel &k);
// pdl: a programmatic dependent launch (the kernel may start while the
// stream's previous kernel runs; it waits with griddepcontrol.wait before
// reading what that kernel writes).
cudaError_t jit_launch(const JitKernel &k, const PassArgs &a, const CUtensorMap &tm_phi, const CUtensorMap &tm_lam,
                       cudaStream_t s, bool pdl = false);

}  // namespace qtm
