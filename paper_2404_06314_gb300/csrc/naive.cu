// Naive GPU path: one kernel launch per gate over the whole batch, the state
// in HBM, a separate reduction kernel per observable and per adjoint inner
// product.  It is the plain baseline the fused path is measured against, and
// a second, independent route through the same math (Eq. (qnn); Sec. II-A
// adjoint method with one inner product per gate).
#include <cstdint>
#include <vector>

#include "device.h"

namespace qtm {

namespace {

template <typename R>
struct Cx { R x, y; };

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename R>
__global__ void k_init(Cx<R> *s, long long total, int n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        s[i] = ((i & ((1ll << n) - 1)) == 0) ? Cx<R>{1, 0} : Cx<R>{0, 0};
}

// cos/sin of half angles for every (sample, rotation)
template <typename R>
__global__ void k_halfangles(const Rot *rots, int n_rots, const R *x, const R *w, int n_in, int B,
                             Cx<R> *cs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * n_rots) return;
    const int b = i / n_rots, r = i % n_rots;
    const Rot ro = rots[r];
    double t = ro.coef;
    if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
    if (ro.x_idx >= 0) t *= (double)x[(size_t)b * n_in + ro.x_idx];
    double s, c;
    sincos(0.5 * t, &s, &c);   // FP64, rounded once: cos^2 + sin^2 stays unbiased
    cs[i] = {(R)c, (R)s};
}

// one rotation (or its adjoint) on qubit q, applied to s1 and (optionally) s2
template <typename R>
__global__ void k_rot(Cx<R> *s1, Cx<R> *s2, int B, int n, int q, int kind, const Cx<R> *cs,
                      int rot, int n_rots, int dagger)
{
    const long long half = 1ll << (n - 1);
    const long long total = half * B;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / half, p = i % half;
        const long long lowm = (1ll << q) - 1;
        const long long x0 = ((p & ~lowm) << 1) | (p & lowm);
        const long long x1 = x0 | (1ll << q);
        const Cx<R> c = cs[b * n_rots + rot];
        const R co = c.x, si = dagger ? -c.y : c.y;   // R(-t) = R(t)^dagger
        Cx<R> *arrs[2] = {s1, s2};
        for (int k = 0; k < 2; ++k) {
            Cx<R> *s = arrs[k];
            if (!s) continue;
            Cx<R> *st = s + b * (half << 1);
            const Cx<R> a0 = st[x0], a1 = st[x1];
            Cx<R> r0, r1;
            if (kind == QTM_RX) {        // [[c, -i s], [-i s, c]]
                r0 = {co * a0.x + si * a1.y, co * a0.y - si * a1.x};
                r1 = {co * a1.x + si * a0.y, co * a1.y - si * a0.x};
            } else if (kind == QTM_RY) { // [[c, -s], [s, c]]
                r0 = {co * a0.x - si * a1.x, co * a0.y - si * a1.y};
                r1 = {si * a0.x + co * a1.x, si * a0.y + co * a1.y};
            } else {                     // diag(c - i s, c + i s)
                r0 = cmul(Cx<R>{co, -si}, a0);
                r1 = cmul(Cx<R>{co, si}, a1);
            }
            st[x0] = r0;
            st[x1] = r1;
        }
    }
}

template <typename R>
__global__ void k_cz(Cx<R> *s1, Cx<R> *s2, long long total, int a, int b)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        if (((i >> a) & 1) && ((i >> b) & 1)) {
            s1[i] = {-s1[i].x, -s1[i].y};
            if (s2) s2[i] = {-s2[i].x, -s2[i].y};
        }
}

template <typename R>
__global__ void k_cnot(Cx<R> *s1, Cx<R> *s2, long long total, int c, int t)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        if (((i >> c) & 1) && !((i >> t) & 1)) {
            const long long j = i | (1ll << t);
            Cx<R> tmp = s1[i]; s1[i] = s1[j]; s1[j] = tmp;
            if (s2) { tmp = s2[i]; s2[i] = s2[j]; s2[j] = tmp; }
        }
}

__device__ double block_sum(double v)
{
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;   // valid on thread 0
}

// E[b][m], one CTA per sample, one observable at a time
template <typename R>
__global__ void k_expval(const Cx<R> *s, int n, const Term *terms, int n_terms, int M, R *E)
{
    const int b = blockIdx.x;
    const long long N = 1ll << n;
    const Cx<R> *st = s + (size_t)b * N;
    for (int m = 0; m < M; ++m) {
        double acc = 0.0;
        for (long long x = threadIdx.x; x < N; x += blockDim.x) {
            const double p = (double)st[x].x * st[x].x + (double)st[x].y * st[x].y;
            double d = 0.0;
            for (int t = 0; t < n_terms; ++t)
                if (terms[t].obs == m)
                    d += (__popcll((unsigned long long)x & terms[t].zmask) & 1) ? -terms[t].coef : terms[t].coef;
            acc += p * d;
        }
        acc = block_sum(acc);
        if (threadIdx.x == 0) E[(size_t)b * M + m] = (R)acc;
    }
}

template <typename R>
__global__ void k_costate(const Cx<R> *phi, Cx<R> *lam, int n, const Term *terms, int n_terms,
                          int M, const R *gE)
{
    const int b = blockIdx.y;
    const long long N = 1ll << n;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N;
         x += (long long)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int t = 0; t < n_terms; ++t) {
            const double k = (double)gE[(size_t)b * M + terms[t].obs] * terms[t].coef;
            d += (__popcll((unsigned long long)x & terms[t].zmask) & 1) ? -k : k;
        }
        const Cx<R> a = phi[(size_t)b * N + x];
        lam[(size_t)b * N + x] = {(R)(d * a.x), (R)(d * a.y)};
    }
}

// abar[b][rot] = Im<lam| P_q |phi>, one CTA per sample
template <typename R>
__global__ void k_inner(const Cx<R> *phi, const Cx<R> *lam, int n, int q, int kind, double *abar,
                        int rot, int n_rots)
{
    const int b = blockIdx.x;
    const long long N = 1ll << n;
    const Cx<R> *ph = phi + (size_t)b * N, *la = lam + (size_t)b * N;
    double acc = 0.0;
    for (long long x = threadIdx.x; x < N; x += blockDim.x) {
        const Cx<R> l = la[x];
        const int bit = (int)((x >> q) & 1);
        Cx<R> pa;   // (P phi)_x
        if (kind == QTM_RZ) {
            const Cx<R> a = ph[x];
            pa = bit ? Cx<R>{-a.x, -a.y} : a;
        } else {
            const Cx<R> a = ph[x ^ (1ll << q)];
            if (kind == QTM_RX) pa = a;
            else pa = bit ? Cx<R>{-a.y, a.x} : Cx<R>{a.y, -a.x};   // Y: (i a) or (-i a)
        }
        acc += (double)l.x * pa.y - (double)l.y * pa.x;          // Im(conj(l) pa)
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) abar[(size_t)b * n_rots + rot] = acc;
}

template <typename R>
__global__ void k_chain(const NaiveArgs a, R *gx, R *gw_out, double *gw_ws)
{
    const int b = blockIdx.x;
    const R *xb = static_cast<const R *>(a.x) + (size_t)b * a.n_in;
    const R *w = static_cast<const R *>(a.w);
    const double *ab = a.abar + (size_t)b * a.n_rots;
    for (int j = threadIdx.x; j < a.P; j += blockDim.x) {
        double s = 0.0;
        for (int k = a.w_ptr[j]; k < a.w_ptr[j + 1]; ++k) {
            const Rot ro = a.rots[a.w_rots[k]];
            s += ab[a.w_rots[k]] * ro.coef * (ro.x_idx >= 0 ? (double)xb[ro.x_idx] : 1.0);
        }
        if (gw_out) gw_out[(size_t)b * a.P + j] = (R)s;
        if (gw_ws) gw_ws[(size_t)b * a.P + j] = s;
    }
    if (gx)
        for (int k = threadIdx.x; k < a.n_in; k += blockDim.x) {
            double s = 0.0;
            for (int i = a.x_ptr[k]; i < a.x_ptr[k + 1]; ++i) {
                const Rot ro = a.rots[a.x_rots[i]];
                s += ab[a.x_rots[i]] * ro.coef * (ro.w_idx >= 0 ? (double)w[ro.w_idx] : 1.0);
            }
            gx[(size_t)b * a.n_in + k] = (R)s;
        }
}

inline int grid_for(long long work)
{
    long long g = (work + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

template <typename R>
cudaError_t fwd_impl(const NaiveArgs &a, cudaStream_t s, int *launches, Cx<R> *cs)
{
    Cx<R> *phi = static_cast<Cx<R> *>(a.phi);
    const long long total = (long long)a.B << a.n;
    int L = 0;
    k_init<R><<<grid_for(total), 256, 0, s>>>(phi, total, a.n); ++L;
    if (a.n_rots > 0) {
        k_halfangles<R><<<(a.B * a.n_rots + 255) / 256, 256, 0, s>>>(
            a.rots, a.n_rots, static_cast<const R *>(a.x), static_cast<const R *>(a.w), a.n_in, a.B, cs);
        ++L;
    }
    for (int g = 0; g < a.n_gates; ++g) {
        const qtm_gate &G = a.gates_host[g];
        if (G.kind == QTM_CZ) k_cz<R><<<grid_for(total), 256, 0, s>>>(phi, nullptr, total, G.q0, G.q1);
        else if (G.kind == QTM_CNOT) k_cnot<R><<<grid_for(total), 256, 0, s>>>(phi, nullptr, total, G.q0, G.q1);
        else
            k_rot<R><<<grid_for(total / 2), 256, 0, s>>>(phi, nullptr, a.B, a.n, G.q0, G.kind, cs,
                                                         a.rot_of_gate_host[g], a.n_rots, 0);
        ++L;
    }
    if (a.E) { k_expval<R><<<a.B, 256, 0, s>>>(phi, a.n, a.terms, a.n_terms, a.M, static_cast<R *>(a.E)); ++L; }
    if (launches) *launches = L;
    return cudaGetLastError();
}

template <typename R>
cudaError_t adj_impl(const NaiveArgs &a, bool per_sample, cudaStream_t s, int *launches, Cx<R> *cs)
{
    Cx<R> *phi = static_cast<Cx<R> *>(a.phi), *lam = static_cast<Cx<R> *>(a.lam);
    const long long total = (long long)a.B << a.n;
    const long long N = 1ll << a.n;
    int L = 0;
    dim3 cg((unsigned)grid_for(N > 4096 ? 4096 : N), (unsigned)a.B);
    k_costate<R><<<cg, 256, 0, s>>>(phi, lam, a.n, a.terms, a.n_terms, a.M, static_cast<const R *>(a.gE));
    ++L;
    for (int g = a.n_gates - 1; g >= 0; --g) {
        const qtm_gate &G = a.gates_host[g];
        if (G.kind == QTM_CZ) { k_cz<R><<<grid_for(total), 256, 0, s>>>(phi, lam, total, G.q0, G.q1); ++L; }
        else if (G.kind == QTM_CNOT) { k_cnot<R><<<grid_for(total), 256, 0, s>>>(phi, lam, total, G.q0, G.q1); ++L; }
        else {
            const int r = a.rot_of_gate_host[g];
            k_inner<R><<<a.B, 256, 0, s>>>(phi, lam, a.n, G.q0, G.kind, a.abar, r, a.n_rots);
            k_rot<R><<<grid_for(total / 2), 256, 0, s>>>(phi, lam, a.B, a.n, G.q0, G.kind, cs, r, a.n_rots, 1);
            L += 2;
        }
    }
    R *gx = static_cast<R *>(a.gx);
    R *gwo = per_sample ? static_cast<R *>(a.gw_out) : nullptr;
    double *gws = per_sample ? nullptr : a.gw_ws;
    k_chain<R><<<a.B, 256, 0, s>>>(a, gx, gwo, gws);
    ++L;
    if (!per_sample && a.gw_out && a.P > 0) {
        cudaError_t e = launch_gw_reduce(sizeof(R) == 8 ? QTM_C128 : QTM_C64, a.gw_ws, a.B, a.P, a.gw_out, s);
        if (e != cudaSuccess) return e;
        ++L;
    }
    if (launches) *launches = L;
    return cudaGetLastError();
}

}  // namespace

// the half-angle table lives in the abar workspace's tail (see capi.cu)
cudaError_t naive_forward(int dtype, const NaiveArgs &a, cudaStream_t s, int *launches)
{
    void *cs = a.abar + (size_t)a.B * (a.n_rots > 0 ? a.n_rots : 1);
    if (dtype == QTM_C128) return fwd_impl<double>(a, s, launches, static_cast<Cx<double> *>(cs));
    return fwd_impl<float>(a, s, launches, static_cast<Cx<float> *>(cs));
}

cudaError_t naive_adjoint(int dtype, const NaiveArgs &a, bool gw_per_sample, cudaStream_t s,
                          int *launches)
{
    void *cs = a.abar + (size_t)a.B * (a.n_rots > 0 ? a.n_rots : 1);
    if (dtype == QTM_C128) return adj_impl<double>(a, gw_per_sample, s, launches, static_cast<Cx<double> *>(cs));
    return adj_impl<float>(a, gw_per_sample, s, launches, static_cast<Cx<float> *>(cs));
}

}  // namespace qtm
