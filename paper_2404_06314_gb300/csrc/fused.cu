// Fused pass kernel, expectation/gradient finalize kernels (sm_103a).
//
// One CTA processes one tile of 2^K amplitudes of one sample (the whole state
// when n <= 12).  The tile is staged in shared memory by TMA (bulk tensor
// copies with the 128-byte swizzle) or generated analytically from the folded
// product-state prefix, then the pass's phases run: each thread holds 16
// amplitudes (tile bits [lo, lo+4)) in registers and applies every op of the
// phase there; between phases the tile goes through shared memory.  The
// forward applies fused run matrices U (Eq. (qnn)); the reverse applies U^dagger
// to the state phi and the costate lam and accumulates v = Im<lam|sigma phi>
// per run (Sec. II-A adjoint method).  Partial sums per tile are written to
// global memory and reduced in fixed order by the finalize kernels.
#include <algorithm>
#include <cstdint>

#include "device.h"
#include "tile.cuh"
#include "tile_cpx.cuh"

namespace qtm {

namespace {

template <typename R>
__global__ void k_prep(const PrepArgs a)
{
    __shared__ double2 ufac[2 * 32];
    const int b = blockIdx.x;
    const int ntab = (a.state_qubits + 3) >> 2;
    prep_sample<R>(a.runs, a.rots, a.prefix_run_of_q, a.n_runs, a.n, a.state_qubits,
                   static_cast<const R *>(a.x) + (size_t)b * a.n_in, static_cast<const R *>(a.w),
                   static_cast<Cx<R> *>(a.mats) + (size_t)b * a.n_runs * 4,
                   static_cast<Cx<R> *>(a.tabs) + (size_t)b * ntab * 16, ufac,
                   a.cs ? a.cs + (size_t)b * a.n_rots : nullptr);
}

// FP64 (cos, sin) of the half angles of the rotations without an input (the
// same for every sample of a call), one thread per distinct angle.
template <typename R>
__global__ void k_prep_shared(const Rot *rots, const int32_t *rep, int n_rots, const R *w, double2 *cs_shared)
{
    // the forward pass after this kernel may start now; it waits for these
    // pairs before reading them
    asm volatile("griddepcontrol.launch_dependents;");
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rots || rep[i] != i) return;
    const Rot ro = rots[i];
    if (ro.x_idx >= 0) return;
    double t = ro.coef;
    if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
    double s, c;
    sincos(0.5 * t, &s, &c);
    cs_shared[i] = double2{c, s};
}


template <typename R, bool REV>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 1 : (REV ? 2 : 3)) k_pass(const __grid_constant__ PassArgs a,
                                              const __grid_constant__ CUtensorMap tm_phi,
                                              const __grid_constant__ CUtensorMap tm_lam)
{
    pass_body<R, REV>(a, &tm_phi, &tm_lam, [](const TileJob &j, const TileSmem<R> &S, bool lam_valid) {
        run_phases_any<R, REV>(j, S, lam_valid);
    });
}

// One warp per (sample, observable): lanes take every 32nd tile, then a
// fixed butterfly (deterministic order).
template <typename R>
__global__ void k_expval_finalize(const double *Epart, int B, int tiles, int M, R *E)
{
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= B * M) return;   // whole warps leave together
    const int b = i / M, m = i % M;
    double s = 0.0;
    for (int t = lane; t < tiles; t += 32) s += Epart[((size_t)b * tiles + t) * M + m];
    s = warp_sum(s, 32, 0xffffffffu);
    if (lane == 0) E[i] = (R)s;
}

template <typename R>
__global__ void k_grad_finalize(const FinalizeArgs f)
{
    const int b = blockIdx.x;
    grad_finalize_sample<R>(f.runs, f.rots, f.n_runs, f.w_ptr, f.w_rots, f.x_ptr, f.x_rots, f.P, f.n_in,
                            static_cast<const R *>(f.x) + (size_t)b * f.n_in, static_cast<const R *>(f.w),
                            f.Gpart + (size_t)b * f.n_runs * f.tiles * 3, f.tiles,
                            f.abar + (size_t)b * f.n_rots,
                            f.gx ? static_cast<R *>(f.gx) + (size_t)b * f.n_in : nullptr,
                            f.gw_out ? static_cast<R *>(f.gw_out) + (size_t)b * f.P : nullptr,
                            f.gw_ws ? f.gw_ws + (size_t)b * f.P : nullptr,
                            f.cs ? f.cs + (size_t)b * f.n_rots : nullptr);
}

// dst[i] += src[i] (composite plans: sum of the parts' outputs, part order)
template <typename R>
__global__ void k_accumulate(const R *src, R *dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

// dst[r][g] += src[r][g] for g < Gd (src rows have Gs >= Gd columns)
template <typename R>
__global__ void k_accumulate_cols(const R *src, int Gs, R *dst, int Gd, size_t rows)
{
    const size_t n = rows * (size_t)Gd;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / Gd, g = i % Gd;
        dst[i] += src[r * Gs + g];
    }
}

// grad_w[j] = sum_b gw_ws[b][j]: one CTA per weight; each thread sums a fixed
// strided subset of the samples, each warp a fixed shuffle butterfly, and the
// first thread the warps' sums in warp order: the same order on every run.
template <typename R>
__global__ void k_gw_reduce(const double *gw_ws, int B, int P, R *gw)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the per-sample sums of the kernel before
    __shared__ double red[32];
    const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += gw_ws[(size_t)b * P + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        gw[j] = (R)t;
    }
}

// Jacobian pseudo-samples: row b' = b * cc + k of a chunk stands for sample
// b and observable m0 + k.  Cotangent e_(m0 + k): gE[b'][j] = (j == m0 + b' % cc).
template <typename R>
__global__ void k_onehot(R *gE, int Bp, int M, int m0, int cc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Bp * M) gE[i] = (i % M) == m0 + (i / M) % cc ? (R)1 : (R)0;
}

// J[b][m0 + k][gate_of_rot[r]] = abar[b * cc + k][r]  (gates that are not
// rotations stay 0)
template <typename R>
__global__ void k_jac_scatter(const double *abar, const int32_t *gate_of_rot, int n_rots, int Bp, int M,
                              int m0, int cc, int G, R *J)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * n_rots) return;
    const int bp = i / n_rots, r = i % n_rots;
    const int b = bp / cc, m = m0 + bp % cc;
    const int g = gate_of_rot[r];   // -1: a constant rotation from a lowered H (no column)
    if (g >= 0) J[((size_t)b * M + m) * G + g] = (R)abar[(size_t)bp * n_rots + r];
}

// dst[b'][i] = src[b' / cc][i] over rows of `row` 16-byte words (a state
// row, 2^sq complex amplitudes, is a whole number of them for sq >= 4 (c64)).
__global__ void k_expand_rows16(const uint4 *src, uint4 *dst, size_t row, int Bp, int cc)
{
    const size_t n = row * (size_t)Bp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bp = i / row, k = i % row;
        dst[i] = src[(bp / cc) * row + k];
    }
}

// x'[b'][j] = x[b' / cc][j]
template <typename R>
__global__ void k_expand_x(const R *x, R *xp, int n_in, int Bp, int cc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * n_in) return;
    xp[i] = x[(size_t)(i / n_in / cc) * n_in + i % n_in];
}

}  // namespace

cudaError_t launch_onehot(int dtype, void *gE, int Bp, int M, int m0, int cc, cudaStream_t s)
{
    const int n = Bp * M, blk = 256, grd = (n + blk - 1) / blk;
    if (n <= 0) return cudaSuccess;
    if (dtype == QTM_C128) k_onehot<double><<<grd, blk, 0, s>>>(static_cast<double *>(gE), Bp, M, m0, cc);
    else k_onehot<float><<<grd, blk, 0, s>>>(static_cast<float *>(gE), Bp, M, m0, cc);
    return cudaGetLastError();
}

cudaError_t launch_jac_scatter(int dtype, const double *abar, const int32_t *gate_of_rot, int n_rots, int Bp,
                               int M, int m0, int cc, int G, void *J, cudaStream_t s)
{
    if (n_rots <= 0 || Bp <= 0) return cudaSuccess;
    const int n = Bp * n_rots, blk = 256, grd = (n + blk - 1) / blk;
    if (dtype == QTM_C128)
        k_jac_scatter<double><<<grd, blk, 0, s>>>(abar, gate_of_rot, n_rots, Bp, M, m0, cc, G,
                                                   static_cast<double *>(J));
    else
        k_jac_scatter<float><<<grd, blk, 0, s>>>(abar, gate_of_rot, n_rots, Bp, M, m0, cc, G,
                                                  static_cast<float *>(J));
    return cudaGetLastError();
}

// Register-only FMA loop for a throughput probe: 8 independent chains per
// thread, `iters` rounds; one store per thread keeps the chains live.
template <typename R>
__global__ void k_fma_probe(R *out, int iters, R a, R b)
{
    R v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (R)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = v[k] * a + b;
    }
    R t = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += v[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// The complex-pair kernels' reverse arithmetic on registers only: per round
// and register bit, a run's gradient sums (grad_cpx) and its gate on phi and
// lam (su2_apply), 256 threads with the register budget of two CTAs per SM,
// as the 12-qubit reverse pass runs.  `tab` holds six f32x2 table pairs
// (an SU(2) matrix in broadcast form) and 16 amplitude pairs; one store per
// thread keeps everything live.
__global__ void __launch_bounds__(256, 2) k_gate_probe(float *out, int iters, const float *tab)
{
    f2 p[kRegs], q[kRegs], t[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = pack2(tab[2 * k], tab[2 * k + 1]);
    const float d = 1e-3f * (float)(threadIdx.x & 31);
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        p[j] = pack2(tab[12 + 2 * j] + d, tab[13 + 2 * j]);
        q[j] = pack2(tab[13 + 2 * j], tab[12 + 2 * j] - d);
    }
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float vx, vy, vz;
        grad_cpx<3>(p, q, vx, vy, vz); acc += vx + vy + vz;
        su2_apply<3>(p, t[0], t[1], t[2], t[3], t[4], t[5]); su2_apply<3>(q, t[0], t[1], t[2], t[3], t[4], t[5]);
        grad_cpx<2>(p, q, vx, vy, vz); acc += vx + vy + vz;
        su2_apply<2>(p, t[0], t[1], t[2], t[3], t[4], t[5]); su2_apply<2>(q, t[0], t[1], t[2], t[3], t[4], t[5]);
        grad_cpx<1>(p, q, vx, vy, vz); acc += vx + vy + vz;
        su2_apply<1>(p, t[0], t[1], t[2], t[3], t[4], t[5]); su2_apply<1>(q, t[0], t[1], t[2], t[3], t[4], t[5]);
        grad_cpx<0>(p, q, vx, vy, vz); acc += vx + vy + vz;
        su2_apply<0>(p, t[0], t[1], t[2], t[3], t[4], t[5]); su2_apply<0>(q, t[0], t[1], t[2], t[3], t[4], t[5]);
    }
#pragma unroll
    for (int j = 0; j < kRegs; ++j) acc += lane0(p[j]) + lane1(q[j]);
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_expand_rows(const void *src, void *dst, size_t row_bytes, int Bp, int cc, cudaStream_t s)
{
    if (Bp <= 0 || row_bytes == 0) return cudaSuccess;
    if (row_bytes % 16) return cudaErrorInvalidValue;
    const size_t row = row_bytes / 16, n = row * (size_t)Bp;
    const int blk = 256;
    const int grd = (int)std::min<size_t>((n + blk - 1) / blk, 152 * 16);
    k_expand_rows16<<<grd, blk, 0, s>>>(static_cast<const uint4 *>(src), static_cast<uint4 *>(dst), row, Bp, cc);
    return cudaGetLastError();
}

cudaError_t launch_expand_x(int dtype, const void *x, void *xp, int n_in, int Bp, int cc, cudaStream_t s)
{
    const int n = Bp * n_in, blk = 256, grd = (n + blk - 1) / blk;
    if (n <= 0) return cudaSuccess;
    if (dtype == QTM_C128)
        k_expand_x<double><<<grd, blk, 0, s>>>(static_cast<const double *>(x), static_cast<double *>(xp), n_in, Bp, cc);
    else
        k_expand_x<float><<<grd, blk, 0, s>>>(static_cast<const float *>(x), static_cast<float *>(xp), n_in, Bp, cc);
    return cudaGetLastError();
}

size_t pass_smem_bytes(int K, int dtype, bool reverse, int nslots, int n_terms, int M,
                       int state_qubits, int n_prefix_ents)
{
    const int csize = dtype == QTM_C128 ? 16 : 8;
    const int rsize = csize / 2;
    const int T = K >= 4 ? (1 << (K - 4)) : 1;
    const int nwarps = (T + 31) / 32;
    Layout L = make_layout(K, csize, reverse, nslots, n_terms, M, state_qubits, n_prefix_ents,
                           nwarps, rsize);
    return (size_t)L.total + 1024;
}

// Launch, as a programmatic dependent launch when pdl is set (the kernel
// may start while the stream's previous kernel runs and waits with
// griddepcontrol.wait before reading what that kernel writes).
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                             Args... args)
{
    if (!pdl) {
        fn<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, args...);
}

cudaError_t launch_pass(int dtype, bool reverse, const PassArgs &a, const CUtensorMap &tm_phi,
                        const CUtensorMap &tm_lam, cudaStream_t s, bool pdl)
{
    // a tile below 9 qubits has fewer than 32 threads' worth of registers; the
    // CTA still takes a full warp, whose other lanes share the staging, the
    // per-sample prep and the finalize but skip the phases (pass_body)
    const int T = 1 << (a.K - 4);
    const dim3 grid((unsigned)a.B * (unsigned)a.tiles), block((unsigned)(T < 32 ? 32 : T));
    const size_t smem = (size_t)a.smem_bytes;
    cudaError_t e;
#define QTM_LAUNCH(R, REV)                                                                     \
    do {                                                                                       \
        auto fn = k_pass<R, REV>;                                                              \
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        if (e != cudaSuccess) return e;                                                        \
        e = launch_maybe_pdl(fn, grid, block, smem, s, pdl, a, tm_phi, tm_lam);                \
        if (e != cudaSuccess) return e;                                                        \
    } while (0)
    if (dtype == QTM_C128) {
        if (reverse) QTM_LAUNCH(double, true); else QTM_LAUNCH(double, false);
    } else {
        if (reverse) QTM_LAUNCH(float, true); else QTM_LAUNCH(float, false);
    }
#undef QTM_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_prep(int dtype, const PrepArgs &a, cudaStream_t s)
{
    if (dtype == QTM_C128) k_prep<double><<<a.B, 128, 0, s>>>(a);
    else k_prep<float><<<a.B, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prep_shared(int dtype, const Rot *rots, const int32_t *rep, int n_rots, const void *w,
                               double2 *cs_shared, cudaStream_t s)
{
    if (n_rots <= 0) return cudaSuccess;
    const int blk = 64, grd = (n_rots + blk - 1) / blk;   // a few warps on as many SMs
    if (dtype == QTM_C128)
        k_prep_shared<double><<<grd, blk, 0, s>>>(rots, rep, n_rots, static_cast<const double *>(w), cs_shared);
    else
        k_prep_shared<float><<<grd, blk, 0, s>>>(rots, rep, n_rots, static_cast<const float *>(w), cs_shared);
    return cudaGetLastError();
}

cudaError_t launch_expval_finalize(int dtype, const FinalizeArgs &f, cudaStream_t s)
{
    const int n = f.B * f.M;
    const int blk = 256, grd = (n + 7) / 8;   // 8 warps per block, one per output
    if (dtype == QTM_C128)
        k_expval_finalize<double><<<grd, blk, 0, s>>>(f.Epart, f.B, f.tiles, f.M, static_cast<double *>(f.E));
    else
        k_expval_finalize<float><<<grd, blk, 0, s>>>(f.Epart, f.B, f.tiles, f.M, static_cast<float *>(f.E));
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(int dtype, const FinalizeArgs &f, cudaStream_t s)
{
    if (dtype == QTM_C128) k_grad_finalize<double><<<f.B, 256, 0, s>>>(f);
    else k_grad_finalize<float><<<f.B, 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(int dtype, const void *src, void *dst, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 1216);
    if (dtype == QTM_C128)
        k_accumulate<double><<<grid, 256, 0, s>>>(static_cast<const double *>(src), static_cast<double *>(dst), n);
    else
        k_accumulate<float><<<grid, 256, 0, s>>>(static_cast<const float *>(src), static_cast<float *>(dst), n);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_cols(int dtype, const void *src, int Gs, void *dst, int Gd, size_t rows, cudaStream_t s)
{
    if (rows == 0 || Gd <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<size_t>((rows * Gd + 255) / 256, 1216);
    if (dtype == QTM_C128)
        k_accumulate_cols<double><<<grid, 256, 0, s>>>(static_cast<const double *>(src), Gs,
                                                        static_cast<double *>(dst), Gd, rows);
    else
        k_accumulate_cols<float><<<grid, 256, 0, s>>>(static_cast<const float *>(src), Gs,
                                                       static_cast<float *>(dst), Gd, rows);
    return cudaGetLastError();
}

cudaError_t launch_gw_reduce(int dtype, const double *gw_ws, int B, int P, void *gw, cudaStream_t s)
{
    if (P <= 0) return cudaSuccess;
    // launched while the kernel that writes gw_ws (always one of this
    // library's) finishes; it waits for it before reading
    if (dtype == QTM_C128)
        return launch_maybe_pdl(k_gw_reduce<double>, dim3(P), dim3(256), 0, s, true, gw_ws, B, P,
                                static_cast<double *>(gw));
    return launch_maybe_pdl(k_gw_reduce<float>, dim3(P), dim3(256), 0, s, true, gw_ws, B, P, static_cast<float *>(gw));
}

}  // namespace qtm

namespace qtm {

// FMA throughput (flop/s, an FMA counted as 2) of a register-only loop in the
// plan real type of `dtype`, timed with CUDA events on `s`; `out` holds one
// element per thread of the grid (blocks x 256).
cudaError_t probe_fma_rate(int dtype, void *out, int blocks, int iters, cudaStream_t s, double *flops_per_s)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        if (dtype == QTM_C128) k_fma_probe<double><<<blocks, 256, 0, s>>>(static_cast<double *>(out), iters, 0.999999, 1e-7);
        else k_fma_probe<float><<<blocks, 256, 0, s>>>(static_cast<float *>(out), iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.f) best = std::min(best, ms);   // the first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * 256.0 / (best * 1e-3);
    return e;
}


// Throughput of k_gate_probe (flop/s counted as the plans count a gradient
// op with its two gates: 40 flop per amplitude) over `blocks` CTAs; `out`
// holds one float per thread, `tab` the 44 floats the kernel reads.
cudaError_t probe_gate_rate(float *out, const float *tab, int blocks, int iters, cudaStream_t s, double *flops_per_s)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        k_gate_probe<<<blocks, 256, 0, s>>>(out, iters, tab);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.f) best = std::min(best, ms);   // the first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // per round and thread: 4 gradient ops of 16 amplitudes at 40 flop each
    if (e == cudaSuccess) *flops_per_s = 4.0 * 16.0 * 40.0 * (double)iters * blocks * 256.0 / (best * 1e-3);
    return e;
}

}  // namespace qtm
