// Pauli strings with X or Y factors on the final state (sm_103a).
//
// The pass kernels measure Z strings inside the evolution (diagonal: a sign
// per amplitude).  A string with X or Y factors pairs amplitude x with
// x ^ xmask, P|x> = i^ny (-1)^popcount(x & zmask) |x ^ xmask>, so it is
// evaluated on the final state that the last forward pass leaves in memory:
//   expectation value   <psi|P|psi> = sum_y conj(psi_y) (P psi)_y
//   costate part        lam_y = sum_t gE[obs_t] coef_t (P_t psi)_y
// (Sec. II-A: every observable from the one evolved state; the adjoint's
// costate is the cotangent-weighted observable applied to it).  The first
// reverse pass loads this costate part and adds the Z part.
#include <algorithm>
#include <cstdint>

#include "device.h"
#include "tile.cuh"

namespace qtm {

namespace {

constexpr int kChunkBits = 12;   // amplitudes per expectation-value CTA: 2^12

// Ppart[b][chunk][t] = Re sum over the chunk's y of conj(psi_y) (P_t psi)_y;
// one CTA per (sample, chunk of 2^12 amplitudes).  A thread sums its (up to 16)
// products in the plan's real type, the 256 thread sums are added in FP64 in
// a fixed order.
template <typename R>
__global__ void k_pauli_partial(const Cx<R> *phi, int sq, const PauliTerm *terms, int T, int chunks,
                                double *Ppart)
{
    __shared__ double red[8];
    const int b = blockIdx.x / chunks, c = blockIdx.x % chunks;
    const uint64_t NS = 1ull << sq;
    const uint64_t lo = (uint64_t)c << kChunkBits;
    const uint64_t len = NS < (1ull << kChunkBits) ? NS : (1ull << kChunkBits);
    const Cx<R> *psi = phi + (size_t)b * NS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = 0; t < T; ++t) {
        const PauliTerm pt = terms[t];
        R st = 0;
        for (uint64_t k = threadIdx.x; k < len; k += blockDim.x) {
            const uint64_t y = lo + k, x = y ^ pt.xmask;
            const Cx<R> a = psi[y];
            Cx<R> v = psi[x];
            if (__popcll(x & pt.zmask) & 1) { v.x = -v.x; v.y = -v.y; }
            switch (pt.ny & 3) {   // times i^ny
            case 1: v = Cx<R>{-v.y, v.x}; break;
            case 2: v = Cx<R>{-v.x, -v.y}; break;
            case 3: v = Cx<R>{v.y, -v.x}; break;
            default: break;
            }
            st += a.x * v.x + a.y * v.y;   // Re(conj(psi_y) v)
        }
        double s = warp_sum((double)st, 32, 0xffffffffu);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0.0;
            for (int w2 = 0; w2 < nw; ++w2) acc += red[w2];
            Ppart[((size_t)b * chunks + c) * T + t] = acc;
        }
        __syncthreads();
    }
}

// E[b][m] += sum_t [obs_t == m] coef_t sum_chunks Ppart[b][chunk][t], in fixed order.
template <typename R>
__global__ void k_pauli_finalize(const double *Ppart, const PauliTerm *terms, int T, int chunks, int B, int M,
                                 R *E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * M) return;
    const int b = i / M, m = i % M;
    double e = 0.0;
    for (int t = 0; t < T; ++t) {
        if (terms[t].obs != m) continue;
        double s = 0.0;
        for (int c = 0; c < chunks; ++c) s += Ppart[((size_t)b * chunks + c) * T + t];
        e += terms[t].coef * s;
    }
    E[i] = (R)((double)E[i] + e);
}

// lam_y = sum_t gE[b][obs_t] coef_t (P_t psi)_y for every amplitude of every sample.
template <typename R>
__global__ void k_pauli_costate(const Cx<R> *phi, int sq, const PauliTerm *terms, int T, const R *gE, int M,
                                int B, Cx<R> *lam)
{
    const uint64_t NS = 1ull << sq, total = NS * (uint64_t)B;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = i >> sq, y = i & (NS - 1);
        const Cx<R> *psi = phi + b * NS;
        R lr = 0, li = 0;   // a sum over the terms: the plan's real type suffices
        for (int t = 0; t < T; ++t) {
            const PauliTerm pt = terms[t];
            const R k = (R)((double)gE[b * M + pt.obs] * pt.coef);
            if (k == (R)0) continue;
            const uint64_t x = y ^ pt.xmask;
            Cx<R> a = psi[x];
            if (__popcll(x & pt.zmask) & 1) { a.x = -a.x; a.y = -a.y; }
            switch (pt.ny & 3) {   // times i^ny
            case 1: a = Cx<R>{-a.y, a.x}; break;
            case 2: a = Cx<R>{-a.x, -a.y}; break;
            case 3: a = Cx<R>{a.y, -a.x}; break;
            default: break;
            }
            lr += k * a.x;
            li += k * a.y;
        }
        lam[i] = Cx<R>{lr, li};
    }
}

}  // namespace

int pauli_chunks(int sq) { return sq > kChunkBits ? 1 << (sq - kChunkBits) : 1; }

cudaError_t launch_pauli_expval(int dtype, const void *phi, int sq, const PauliTerm *terms, int T, int B, int M,
                                double *Ppart, void *E, cudaStream_t s)
{
    if (T <= 0 || B <= 0) return cudaSuccess;
    const int chunks = pauli_chunks(sq);
    const unsigned grid = (unsigned)B * (unsigned)chunks;
    const int n = B * M, fgrid = (n + 255) / 256;
    if (dtype == QTM_C128) {
        k_pauli_partial<double><<<grid, 256, 0, s>>>(static_cast<const Cx<double> *>(phi), sq, terms, T, chunks, Ppart);
        k_pauli_finalize<double><<<fgrid, 256, 0, s>>>(Ppart, terms, T, chunks, B, M, static_cast<double *>(E));
    } else {
        k_pauli_partial<float><<<grid, 256, 0, s>>>(static_cast<const Cx<float> *>(phi), sq, terms, T, chunks, Ppart);
        k_pauli_finalize<float><<<fgrid, 256, 0, s>>>(Ppart, terms, T, chunks, B, M, static_cast<float *>(E));
    }
    return cudaGetLastError();
}

cudaError_t launch_pauli_costate(int dtype, const void *phi, int sq, const PauliTerm *terms, int T, const void *gE,
                                 int M, int B, void *lam, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    const uint64_t total = (1ull << sq) * (uint64_t)B;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 152ull * 16);
    if (dtype == QTM_C128)
        k_pauli_costate<double><<<grid, 256, 0, s>>>(static_cast<const Cx<double> *>(phi), sq, terms, T,
                                                     static_cast<const double *>(gE), M, B,
                                                     static_cast<Cx<double> *>(lam));
    else
        k_pauli_costate<float><<<grid, 256, 0, s>>>(static_cast<const Cx<float> *>(phi), sq, terms, T,
                                                    static_cast<const float *>(gE), M, B,
                                                    static_cast<Cx<float> *>(lam));
    return cudaGetLastError();
}

}  // namespace qtm
