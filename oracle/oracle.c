/*
 * FP64 CPU oracle for batched, noise-free statevector evaluation of a
 * parameterised quantum circuit: expectation values of Pauli-Z strings and
 * their gradients (adjoint method, parameter-shift rule, full Jacobian).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file.  It is used by tests/, by __graft_entry__.smoke() and by
 * bench.py's timed CPU baseline.  It shares no code, header or constant table
 * with the CUDA path; only the circuit description (gate list, observables)
 * and the seeded inputs are common.
 *
 * Everything is complex128 (C99 double complex), one gate at a time, in the
 * order of the gate list, with no fusion, tiling or reordering.
 *
 * Conventions (paper Sec. II, built on Qiskit):
 *   - qubit q is bit q of the amplitude index (little endian);
 *   - a rotation about Pauli P by angle t is R_P(t) = exp(-i t P / 2)
 *     = cos(t/2) I - i sin(t/2) P;
 *   - H is the Hadamard gate (|0> + |1>)/sqrt2 <- |0>; RZZ(t) = exp(-i t Z_a Z_b / 2)
 *     multiplies amplitude x by exp(-i t/2) when bits a and b of x agree and by
 *     exp(+i t/2) when they differ;
 *   - the angle of gate g for sample b is
 *       theta = coef[g] * (w_idx >= 0 ? w[w_idx] : 1) * (x_idx >= 0 ? x[b][x_idx] : 1)
 *     (trainable variational weights and trainable input scaling, Sec. II-C,
 *     Eq. (concrete_ansatz));
 *   - observable m is a real combination of Pauli strings,
 *       O_m = sum_{t : obs_t = m} c_t P_t,
 *     P_t = prod_q sigma_q with sigma_q = X where only xmask_t has bit q,
 *     Y where both xmask_t and zmask_t have it, Z where only zmask_t has it;
 *     Z strings (xmask = 0, or no xmask array) are diagonal:
 *       P|x> = i^(#Y) (-1)^popcount(x & zmask) |x ^ xmask>.
 *
 * Parity is pinned by tests/test_oracle_pins.py (closed forms, dense
 * Kronecker-product unitaries, product-state Bloch rotations, parameter shift
 * and finite differences).  No function here is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double OR_PI = 3.14159265358979323846264338327950288;

/* Gate kinds of the circuit description. */
enum { OR_RX = 0, OR_RY = 1, OR_RZ = 2, OR_CZ = 3, OR_CNOT = 4, OR_H = 5, OR_RZZ = 6 };

typedef struct {
    int32_t n;          /* qubits */
    int32_t G;          /* gates */
    const int32_t *kind, *q0, *q1, *widx, *xidx;
    const double *coef;
    int32_t T;          /* Z-string terms */
    const uint64_t *zmask;
    const double *zcoef;
    const int32_t *zobs;
    int32_t M;          /* observables */
    int32_t P;          /* weights */
    int32_t n_in;       /* inputs per sample */
    const uint64_t *xmask;   /* per term X/Y qubits, or NULL: all terms are Z strings */
} or_circuit;

/* ------------------------------------------------------------------ */
/* batch partition (Sec. II-B, Eq. (qnn_batched)): B samples over T    */
/* workers, the first B - T*floor(B/T) workers take one extra sample. */
/* ------------------------------------------------------------------ */
void oracle_partition(int B, int T, int t, int *start, int *count)
{
    int base = B / T;
    int extra = B - T * base;
    *count = base + (t < extra ? 1 : 0);
    *start = t * base + (t < extra ? t : extra);
}

static int is_rotation(int k) { return k == OR_RX || k == OR_RY || k == OR_RZ; }
/* gates with an angle (rotations and RZZ) */
static int has_angle(int k) { return is_rotation(k) || k == OR_RZZ; }

static double gate_angle(const or_circuit *c, int g, const double *xb, const double *w)
{
    double th = c->coef[g];
    if (c->widx[g] >= 0) th *= w[c->widx[g]];
    if (c->xidx[g] >= 0) th *= xb[c->xidx[g]];
    return th;
}

/* Pauli matrices, row-major m[r][col]. */
static void pauli(int kind, cplx m[2][2])
{
    m[0][0] = m[0][1] = m[1][0] = m[1][1] = 0;
    if (kind == OR_RX) { m[0][1] = 1; m[1][0] = 1; }
    else if (kind == OR_RY) { m[0][1] = -I; m[1][0] = I; }
    else { m[0][0] = 1; m[1][1] = -1; }
}

/* R_P(t) = cos(t/2) I - i sin(t/2) P */
static void rotation(int kind, double t, cplx m[2][2])
{
    cplx p[2][2];
    pauli(kind, p);
    double co = cos(0.5 * t), si = sin(0.5 * t);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k)
            m[r][k] = (r == k ? co : 0.0) - I * si * p[r][k];
}

/* dR_P/dt = -(1/2) sin(t/2) I - (i/2) cos(t/2) P */
static void rotation_derivative(int kind, double t, cplx m[2][2])
{
    cplx p[2][2];
    pauli(kind, p);
    double co = cos(0.5 * t), si = sin(0.5 * t);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k)
            m[r][k] = (r == k ? -0.5 * si : 0.0) - I * 0.5 * co * p[r][k];
}

static void dagger(cplx m[2][2])
{
    cplx t01 = m[0][1];
    m[0][0] = conj(m[0][0]);
    m[1][1] = conj(m[1][1]);
    m[0][1] = conj(m[1][0]);
    m[1][0] = conj(t01);
}

/* Apply a 2x2 matrix to qubit q of an n-qubit state. */
static void apply_1q(cplx *psi, int n, int q, cplx m[2][2])
{
    uint64_t N = 1ull << n, bit = 1ull << q;
    for (uint64_t x = 0; x < N; ++x) {
        if (x & bit) continue;
        cplx a0 = psi[x], a1 = psi[x | bit];
        psi[x] = m[0][0] * a0 + m[0][1] * a1;
        psi[x | bit] = m[1][0] * a0 + m[1][1] * a1;
    }
}

/* Gate g (or its adjoint) at angle t.  CZ and CNOT are self-inverse. */
static void apply_gate(const or_circuit *c, int g, double t, int adjoint, cplx *psi)
{
    int n = c->n, k = c->kind[g];
    uint64_t N = 1ull << n;
    if (is_rotation(k)) {
        cplx m[2][2];
        rotation(k, t, m);
        if (adjoint) dagger(m);
        apply_1q(psi, n, c->q0[g], m);
    } else if (k == OR_H) {    /* self-inverse */
        const double r = 1.0 / sqrt(2.0);
        cplx m[2][2] = {{r, r}, {r, -r}};
        apply_1q(psi, n, c->q0[g], m);
    } else if (k == OR_RZZ) {  /* diagonal phase by the parity of bits q0, q1 */
        uint64_t ba = 1ull << c->q0[g], bb = 1ull << c->q1[g];
        cplx same = cexp(-I * 0.5 * t), diff = cexp(I * 0.5 * t);
        if (adjoint) { same = conj(same); diff = conj(diff); }
        for (uint64_t x = 0; x < N; ++x)
            psi[x] *= (((x & ba) != 0) == ((x & bb) != 0)) ? same : diff;
    } else if (k == OR_CZ) {
        uint64_t ba = 1ull << c->q0[g], bb = 1ull << c->q1[g];
        for (uint64_t x = 0; x < N; ++x)
            if ((x & ba) && (x & bb)) psi[x] = -psi[x];
    } else { /* CNOT: control q0, target q1 */
        uint64_t bc = 1ull << c->q0[g], bt = 1ull << c->q1[g];
        for (uint64_t x = 0; x < N; ++x)
            if ((x & bc) && !(x & bt)) {
                cplx tmp = psi[x];
                psi[x] = psi[x | bt];
                psi[x | bt] = tmp;
            }
    }
}

/* mu <- (dU_g/dtheta) mu for an angle gate g at angle t (mu holds the state
 * before gate g on entry). */
static void apply_gate_derivative(const or_circuit *c, int g, double t, cplx *mu)
{
    int n = c->n, k = c->kind[g];
    if (is_rotation(k)) {
        cplx dm[2][2];
        rotation_derivative(k, t, dm);
        apply_1q(mu, n, c->q0[g], dm);
    } else { /* RZZ: d/dt exp(-i t z / 2) = (-i z / 2) exp(-i t z / 2), z = +-1 */
        uint64_t N = 1ull << n, ba = 1ull << c->q0[g], bb = 1ull << c->q1[g];
        for (uint64_t x = 0; x < N; ++x) {
            double z = (((x & ba) != 0) == ((x & bb) != 0)) ? 1.0 : -1.0;
            mu[x] *= -I * 0.5 * z * cexp(-I * 0.5 * t * z);
        }
    }
}

static int popcount64(uint64_t v)
{
    int s = 0;
    while (v) { s += (int)(v & 1ull); v >>= 1; }
    return s;
}

/* Diagonal of observable m: d_m(x) = sum_t c_t (-1)^{popcount(x & mask_t)}. */
static double obs_diag(const or_circuit *c, int m, uint64_t x)
{
    double d = 0.0;
    for (int t = 0; t < c->T; ++t)
        if (c->zobs[t] == m)
            d += c->zcoef[t] * ((popcount64(x & c->zmask[t]) & 1) ? -1.0 : 1.0);
    return d;
}

static int has_xy(const or_circuit *c)
{
    if (!c->xmask) return 0;
    for (int t = 0; t < c->T; ++t)
        if (c->xmask[t]) return 1;
    return 0;
}

/* out += s * P_t in, for one Pauli string (see the conventions above). */
static void add_pauli(const or_circuit *c, int t, double s, const cplx *in, cplx *out)
{
    uint64_t N = 1ull << c->n, xm = c->xmask ? c->xmask[t] : 0, zm = c->zmask[t];
    int ny = popcount64(xm & zm);
    cplx ph = 1;
    for (int k = 0; k < (ny & 3); ++k) ph *= I;       /* i^(#Y) */
    for (uint64_t y = 0; y < N; ++y) {
        uint64_t x = y ^ xm;                            /* <y|P|x> != 0 only for x = y ^ xmask */
        double sg = (popcount64(x & zm) & 1) ? -1.0 : 1.0;
        out[y] += s * ph * sg * in[x];
    }
}

/* out = (sum_m g_m O_m) in, g = NULL: observable m_only alone. */
static void apply_observables(const or_circuit *c, const double *g, int m_only, const cplx *in, cplx *out)
{
    uint64_t N = 1ull << c->n;
    for (uint64_t y = 0; y < N; ++y) out[y] = 0;
    for (int t = 0; t < c->T; ++t) {
        int m = c->zobs[t];
        if (g) add_pauli(c, t, g[m] * c->zcoef[t], in, out);
        else if (m == m_only) add_pauli(c, t, c->zcoef[t], in, out);
    }
}

/* |psi> = U_{G-1} ... U_0 |0>, with the angles given per gate. */
static void evolve(const or_circuit *c, const double *theta, cplx *psi)
{
    uint64_t N = 1ull << c->n;
    for (uint64_t x = 0; x < N; ++x) psi[x] = 0;
    psi[0] = 1;
    for (int g = 0; g < c->G; ++g) apply_gate(c, g, theta[g], 0, psi);
}

/* Eq. (qnn): <O_m> = <psi|O_m|psi>, all M from one evolved state (Sec. II-A).
 * scratch (2^n, used only with X/Y terms) receives O_m psi. */
static void expvals_general(const or_circuit *c, const cplx *psi, double *E, cplx *scratch)
{
    uint64_t N = 1ull << c->n;
    for (int m = 0; m < c->M; ++m) {
        apply_observables(c, NULL, m, psi, scratch);
        double s = 0.0;
        for (uint64_t x = 0; x < N; ++x) s += creal(conj(psi[x]) * scratch[x]);
        E[m] = s;
    }
}

static void expvals(const or_circuit *c, const cplx *psi, double *E)
{
    uint64_t N = 1ull << c->n;
    if (has_xy(c)) {
        cplx *scratch = malloc(sizeof(cplx) * N);
        if (scratch) expvals_general(c, psi, E, scratch);
        free(scratch);
        return;
    }
    for (int m = 0; m < c->M; ++m) {
        double s = 0.0;
        for (uint64_t x = 0; x < N; ++x) {
            double p = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
            s += p * obs_diag(c, m, x);
        }
        E[m] = s;
    }
}

static double inner_re(const cplx *a, const cplx *b, uint64_t N) /* Re <a|b> */
{
    double s = 0.0;
    for (uint64_t x = 0; x < N; ++x) s += creal(conj(a[x]) * b[x]);
    return s;
}

/* Chain rule: theta_g = coef * W * X  =>  dW += dtheta * coef * X,  dX += dtheta * coef * W. */
static void chain_rule(const or_circuit *c, const double *xb, const double *w,
                       const double *dtheta, double *gx_b, double *gw_b)
{
    if (gx_b) for (int i = 0; i < c->n_in; ++i) gx_b[i] = 0.0;
    if (gw_b) for (int j = 0; j < c->P; ++j) gw_b[j] = 0.0;
    for (int g = 0; g < c->G; ++g) {
        if (!has_angle(c->kind[g])) continue;
        double W = c->widx[g] >= 0 ? w[c->widx[g]] : 1.0;
        double X = c->xidx[g] >= 0 ? xb[c->xidx[g]] : 1.0;
        if (gw_b && c->widx[g] >= 0) gw_b[c->widx[g]] += dtheta[g] * c->coef[g] * X;
        if (gx_b && c->xidx[g] >= 0) gx_b[c->xidx[g]] += dtheta[g] * c->coef[g] * W;
    }
}

static int nthreads_or_default(int threads)
{
    if (threads > 0) return threads;
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* public entry points                                                 */
/* ------------------------------------------------------------------ */

/* Angles of every gate for one sample (0 for CZ, CNOT and H). */
void oracle_angles(const or_circuit *c, const double *xb, const double *w, double *theta)
{
    for (int g = 0; g < c->G; ++g)
        theta[g] = has_angle(c->kind[g]) ? gate_angle(c, g, xb, w) : 0.0;
}

/* Final state of one sample, interleaved (re, im), length 2 * 2^n. */
int oracle_state(const or_circuit *c, const double *xb, const double *w, double *psi_out)
{
    uint64_t N = 1ull << c->n;
    double *theta = malloc(sizeof(double) * (c->G > 0 ? c->G : 1));
    cplx *psi = malloc(sizeof(cplx) * N);
    if (!theta || !psi) { free(theta); free(psi); return 1; }
    oracle_angles(c, xb, w, theta);
    evolve(c, theta, psi);
    for (uint64_t x = 0; x < N; ++x) { psi_out[2 * x] = creal(psi[x]); psi_out[2 * x + 1] = cimag(psi[x]); }
    free(theta); free(psi);
    return 0;
}

/* Expectation values E[B][M] (Eq. (qnn_batched)); workers split the batch by the
 * partition rule above. */
int oracle_forward(const or_circuit *c, int B, const double *x, const double *w,
                   double *E, int threads)
{
    int T = nthreads_or_default(threads);
    int err = 0;
    uint64_t N = 1ull << c->n;
#pragma omp parallel num_threads(T) reduction(| : err)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
        int Tr = omp_get_num_threads();
#else
        int Tr = 1;
#endif
        int start, count;
        oracle_partition(B, Tr, t, &start, &count);
        double *theta = malloc(sizeof(double) * (c->G > 0 ? c->G : 1));
        cplx *psi = malloc(sizeof(cplx) * N);
        if (!theta || !psi) err = 1;
        else
            for (int b = start; b < start + count; ++b) {
                const double *xb = x + (size_t)b * c->n_in;
                oracle_angles(c, xb, w, theta);
                evolve(c, theta, psi);
                expvals(c, psi, E + (size_t)b * c->M);
            }
        free(theta); free(psi);
    }
    return err;
}

/*
 * Vector-Jacobian product by the adjoint ("reverse") method of Jones & Gacon,
 * Algorithm 1, as extended in Sec. II-A to M observables: the cotangent gE[b][m]
 * weights the observables into one costate, lambda = (sum_m gE_m O_m) psi.
 * Steps per gate g = G-1 ... 0:
 *     phi    <- U_g^dagger phi            (phi is now the state before gate g)
 *     mu     <- (dU_g/dtheta) phi
 *     dtheta <- 2 Re <lambda|mu>
 *     lambda <- U_g^dagger lambda
 * Outputs (any may be NULL): dtheta[B][G], gx[B][n_in], gw[B][P] (per sample).
 */
int oracle_adjoint(const or_circuit *c, int B, const double *gE, const double *x,
                   const double *w, double *dtheta_out, double *gx, double *gw, int threads)
{
    int T = nthreads_or_default(threads);
    int err = 0;
    uint64_t N = 1ull << c->n;
#pragma omp parallel num_threads(T) reduction(| : err)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
        int Tr = omp_get_num_threads();
#else
        int Tr = 1;
#endif
        int start, count;
        oracle_partition(B, Tr, t, &start, &count);
        int Gs = c->G > 0 ? c->G : 1;
        double *theta = malloc(sizeof(double) * Gs);
        double *dth = malloc(sizeof(double) * Gs);
        cplx *phi = malloc(sizeof(cplx) * N);
        cplx *lam = malloc(sizeof(cplx) * N);
        cplx *mu = malloc(sizeof(cplx) * N);
        if (!theta || !dth || !phi || !lam || !mu) err = 1;
        else
            for (int b = start; b < start + count; ++b) {
                const double *xb = x + (size_t)b * c->n_in;
                const double *gEb = gE + (size_t)b * c->M;
                oracle_angles(c, xb, w, theta);
                evolve(c, theta, phi);
                if (has_xy(c)) {
                    apply_observables(c, gEb, -1, phi, lam);   /* lambda = (sum_m gE_m O_m) phi */
                } else
                for (uint64_t xx = 0; xx < N; ++xx) {
                    double d = 0.0;
                    for (int m = 0; m < c->M; ++m) d += gEb[m] * obs_diag(c, m, xx);
                    lam[xx] = d * phi[xx];
                }
                for (int g = c->G - 1; g >= 0; --g) {
                    apply_gate(c, g, theta[g], 1, phi);
                    dth[g] = 0.0;
                    if (has_angle(c->kind[g])) {
                        memcpy(mu, phi, sizeof(cplx) * N);
                        apply_gate_derivative(c, g, theta[g], mu);
                        dth[g] = 2.0 * inner_re(lam, mu, N);
                    }
                    apply_gate(c, g, theta[g], 1, lam);
                }
                if (dtheta_out) memcpy(dtheta_out + (size_t)b * c->G, dth, sizeof(double) * c->G);
                chain_rule(c, xb, w, dth, gx ? gx + (size_t)b * c->n_in : NULL,
                           gw ? gw + (size_t)b * c->P : NULL);
            }
        free(theta); free(dth); free(phi); free(lam); free(mu);
    }
    return err;
}

/*
 * Full Jacobian J[B][M][G] = d<O_m>/d theta_g (the (B, M, |Theta|) output of
 * Sec. II-B), with one costate lambda_m = O_m psi per observable, each run
 * through the same reverse recursion as oracle_adjoint.
 */
int oracle_jacobian(const or_circuit *c, int B, const double *x, const double *w,
                    double *J, int threads)
{
    int T = nthreads_or_default(threads);
    int err = 0;
    uint64_t N = 1ull << c->n;
#pragma omp parallel num_threads(T) reduction(| : err)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
        int Tr = omp_get_num_threads();
#else
        int Tr = 1;
#endif
        int start, count;
        oracle_partition(B, Tr, t, &start, &count);
        int Gs = c->G > 0 ? c->G : 1;
        double *theta = malloc(sizeof(double) * Gs);
        cplx *psi = malloc(sizeof(cplx) * N);
        cplx *phi = malloc(sizeof(cplx) * N);
        cplx *lam = malloc(sizeof(cplx) * N);
        cplx *mu = malloc(sizeof(cplx) * N);
        if (!theta || !psi || !phi || !lam || !mu) err = 1;
        else
            for (int b = start; b < start + count; ++b) {
                const double *xb = x + (size_t)b * c->n_in;
                oracle_angles(c, xb, w, theta);
                evolve(c, theta, psi);
                for (int m = 0; m < c->M; ++m) {
                    double *Jbm = J + ((size_t)b * c->M + m) * c->G;
                    memcpy(phi, psi, sizeof(cplx) * N);
                    if (has_xy(c)) apply_observables(c, NULL, m, phi, lam);   /* lambda_m = O_m phi */
                    else
                        for (uint64_t xx = 0; xx < N; ++xx) lam[xx] = obs_diag(c, m, xx) * phi[xx];
                    for (int g = c->G - 1; g >= 0; --g) {
                        apply_gate(c, g, theta[g], 1, phi);
                        Jbm[g] = 0.0;
                        if (has_angle(c->kind[g])) {
                            memcpy(mu, phi, sizeof(cplx) * N);
                            apply_gate_derivative(c, g, theta[g], mu);
                            Jbm[g] = 2.0 * inner_re(lam, mu, N);
                        }
                        apply_gate(c, g, theta[g], 1, lam);
                    }
                }
            }
        free(theta); free(psi); free(phi); free(lam); free(mu);
    }
    return err;
}

/*
 * Parameter-shift rule (Crooks, cited in Sec. II-A): for each angle gate
 * (rotations and RZZ, generators with eigenvalues +-1),
 *     d<O_m>/d theta_g = ( <O_m>(theta_g + pi/2) - <O_m>(theta_g - pi/2) ) / 2,
 * shifting the gate angle (never a weight shared by several gates), then the
 * cotangent gE and the chain rule.  2 |Theta| evolutions per sample.
 */
int oracle_param_shift(const or_circuit *c, int B, const double *gE, const double *x,
                       const double *w, double *dtheta_out, double *gx, double *gw, int threads)
{
    int T = nthreads_or_default(threads);
    int err = 0;
    uint64_t N = 1ull << c->n;
#pragma omp parallel num_threads(T) reduction(| : err)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
        int Tr = omp_get_num_threads();
#else
        int Tr = 1;
#endif
        int start, count;
        oracle_partition(B, Tr, t, &start, &count);
        int Gs = c->G > 0 ? c->G : 1;
        int Ms = c->M > 0 ? c->M : 1;
        double *theta = malloc(sizeof(double) * Gs);
        double *dth = malloc(sizeof(double) * Gs);
        double *Ep = malloc(sizeof(double) * Ms);
        double *Em = malloc(sizeof(double) * Ms);
        cplx *psi = malloc(sizeof(cplx) * N);
        if (!theta || !dth || !Ep || !Em || !psi) err = 1;
        else
            for (int b = start; b < start + count; ++b) {
                const double *xb = x + (size_t)b * c->n_in;
                const double *gEb = gE + (size_t)b * c->M;
                oracle_angles(c, xb, w, theta);
                for (int g = 0; g < c->G; ++g) {
                    dth[g] = 0.0;
                    if (!has_angle(c->kind[g])) continue;   /* generators with eigenvalues +-1 */
                    double t0 = theta[g];
                    theta[g] = t0 + 0.5 * OR_PI;
                    evolve(c, theta, psi);
                    expvals(c, psi, Ep);
                    theta[g] = t0 - 0.5 * OR_PI;
                    evolve(c, theta, psi);
                    expvals(c, psi, Em);
                    theta[g] = t0;
                    for (int m = 0; m < c->M; ++m) dth[g] += gEb[m] * 0.5 * (Ep[m] - Em[m]);
                }
                if (dtheta_out) memcpy(dtheta_out + (size_t)b * c->G, dth, sizeof(double) * c->G);
                chain_rule(c, xb, w, dth, gx ? gx + (size_t)b * c->n_in : NULL,
                           gw ? gw + (size_t)b * c->P : NULL);
            }
        free(theta); free(dth); free(Ep); free(Em); free(psi);
    }
    return err;
}

/* Max worker count the oracle would use by default (for reporting). */
int oracle_max_threads(void) { return nthreads_or_default(0); }
