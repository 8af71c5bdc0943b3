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
    int pairs = 0;         // 1: two samples per CTA (tile_x2.cuh)
};

// Passes worth specialising: fused complex64 passes whose tile has >= 9 qubits
// (full warps).
bool jit_eligible(const Plan &P, const PassDesc &pd);
bool jit_available();
bool jit_nvrtc_available();
// Kinds of specialised kernel: two samples per CTA on f32x2 register pairs
// (tile_x2.cuh); one sample per CTA with scalar registers (tile.cuh); one
// sample per CTA with amplitudes paired in f32x2 registers (tile_lanes.cuh);
// one sample per CTA with each complex amplitude one f32x2 pair (tile_cpx.cuh).
enum JitMode { JIT_PAIRS = 0, JIT_ONE = 1, JIT_LANES = 2, JIT_CPX = 3 };

// Generated source of one pass.
std::string jit_source(const Plan &P, const PassDesc &pd, int min_blocks, JitMode mode);
size_t jit_smem_bytes_x2(const Plan &P, const PassDesc &pd);
size_t jit_smem_bytes_lanes(const Plan &P, const PassDesc &pd);
size_t jit_smem_bytes_cpx(const Plan &P, const PassDesc &pd);
bool jit_compile(const std::string &body, std::vector<char> &cubin, std::string &log);
bool jit_load(const std::vector<char> &cubin, int smem, JitKernel &k, std::string &err);
void jit_unload(JitKernel &k);
cudaError_t jit_launch(const JitKernel &k, const PassArgs &a, const CUtensorMap &tm_phi, const CUtensorMap &tm_lam,
                       cudaStream_t s);

}  // namespace qtm
