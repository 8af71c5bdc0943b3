// Gradients of the rotations of one fused run from a single 3-vector.
//
// For a run R_m ... R_1 on qubit q (R_i = exp(-i t_i P_i / 2), applied in the
// order 1..m), let phi and lam be the state and costate just after the run.
// The adjoint gradient of rotation i is Im<lam_i|P_i phi_i> (Sec. II-A; Jones
// & Gacon Alg. 1), with lam_i, phi_i the states after rotation i.  Because
// W = R_m ... R_{i+1} acts on qubit q only,
//     Im<lam_i|P_i phi_i> = Im<lam| W P_i W^dagger |phi> = (Ad_W^T v)[P_i],
// where v_s = Im<lam|s_q phi> for s in {X, Y, Z} and Ad_R is the SO(3) matrix
// with R s R^dagger = sum_s' Ad_R[s'][s] s'.  So one reduction of v per run
// gives every gradient of the run: u <- v; for i = m..1: grad_i = u[P_i];
// u <- Ad_{R_i}^T u.
#pragma once

#ifndef __CUDACC_RTC__
#include <cmath>
#endif

#ifdef __CUDACC__
#define QTM_HD __host__ __device__ __forceinline__
#else
#define QTM_HD inline
#endif

namespace qtm {

// axis index of a rotation kind: X = 0, Y = 1, Z = 2 (QTM_RX/RY/RZ = 0/1/2);
// c = cos(t), s = sin(t)
QTM_HD void adjoint_transpose_apply_cs(int kind, double c, double s, double u[3])
{
    double u0 = u[0], u1 = u[1], u2 = u[2];
    if (kind == 0) {        // Ad_RX = [[1,0,0],[0,c,-s],[0,s,c]]
        u[1] = c * u1 + s * u2;
        u[2] = -s * u1 + c * u2;
    } else if (kind == 1) { // Ad_RY = [[c,0,s],[0,1,0],[-s,0,c]]
        u[0] = c * u0 - s * u2;
        u[2] = s * u0 + c * u2;
    } else {                // Ad_RZ = [[c,-s,0],[s,c,0],[0,0,1]]
        u[0] = c * u0 + s * u1;
        u[1] = -s * u0 + c * u1;
    }
}

QTM_HD void adjoint_transpose_apply(int kind, double t, double u[3])
{
    adjoint_transpose_apply_cs(kind, cos(t), sin(t), u);
}

// kinds[i], theta[i]: the run's rotations in forward order; v = (vx, vy, vz).
QTM_HD void run_angle_grads(int m, const int *kinds, const double *theta, const double v[3],
                            double *grad)
{
    double u[3] = {v[0], v[1], v[2]};
    for (int i = m - 1; i >= 0; --i) {
        grad[i] = u[kinds[i]];
        adjoint_transpose_apply(kinds[i], theta[i], u);
    }
}

}  // namespace qtm
