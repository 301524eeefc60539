// Kirchhoff stresses and plastic return maps of the full-order step, in
// float64 (paper App. F), with a float64 3x3 singular value decomposition.
//
// SVD: F = U diag(s) V^T from the eigen-decomposition of F^T F by cyclic
// Jacobi rotations (Jacobi's method for symmetric matrices, as in Golub & Van
// Loan, "Matrix Computations", §8.5), singular values sorted in decreasing
// order, det V = +1, U = [u0, u1, u0 x u1] from F V (Gram-Schmidt on the first
// two columns), so det U = +1 and the smallest singular value carries the sign
// of det F.
//
// Models (the same readings as the FP64 oracle):
//   fixed corotated (F.1)  tau = 2 mu (F - R) F^T + lambda (J - 1) J I,  R = U V^T
//   Hencky / StVK (F.2)    tau = U diag(2 mu eps + lambda sum(eps)) U^T,  eps = log|s|
//   von Mises (F.4)        dgamma = ||dev eps|| - tau_y / (2 mu) > 0:
//                          eps <- eps - dgamma dev(eps) / ||dev eps||
//   Drucker-Prager (F.3)   sum(eps) > 0: s <- 1; otherwise dgamma = ||dev eps||
//                          + alpha (3 lambda + 2 mu) sum(eps) / (2 mu) > 0:
//                          eps <- eps - dgamma dev(eps) / ||dev eps||,
//                          alpha = sqrt(2/3) 2 sin(phi) / (3 - sin(phi))
// The plastic models return F^E = U diag(s_new) V^T and the Hencky stress of it.
#pragma once

#include "device_common.cuh"

namespace nsf {

// Eigen-decomposition of a symmetric 3x3 matrix S = V diag(l) V^T by cyclic
// Jacobi sweeps (rotation zeroing S_pq, t = sgn(th) / (|th| + sqrt(th^2 + 1)),
// th = (S_qq - S_pp) / (2 S_pq)).
__device__ inline void jacobi_eig3(double S[3][3], double V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 8; ++sweep) {
        const double off = fabs(S[0][1]) + fabs(S[0][2]) + fabs(S[1][2]);
        const double dia = fabs(S[0][0]) + fabs(S[1][1]) + fabs(S[2][2]);
        if (off <= 1e-17 * dia || off == 0.0) break;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int p = P[k], q = Q[k];
            const double spq = S[p][q];
            if (spq == 0.0) continue;
            const double th = (S[q][q] - S[p][p]) / (2.0 * spq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            const int m = 3 - p - q;             // the third index
            const double smp = S[m][p], smq = S[m][q];
            S[m][p] = S[p][m] = c * smp - s * smq;
            S[m][q] = S[q][m] = s * smp + c * smq;
            S[p][p] -= t * spq;
            S[q][q] += t * spq;
            S[p][q] = S[q][p] = 0.0;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double vp = V[r][p], vq = V[r][q];
                V[r][p] = c * vp - s * vq;
                V[r][q] = s * vp + c * vq;
            }
        }
    }
}

// F (row-major) = U diag(s) V^T with the conventions above.
__device__ inline void svd3(const double F[9], double U[9], double s[3], double V[9]) {
    double S[3][3], E[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];   // F^T F
    jacobi_eig3(S, E);
    double l[3] = {S[0][0], S[1][1], S[2][2]};
    int ord[3] = {0, 1, 2};
    // sort eigenvalues decreasing
    if (l[ord[0]] < l[ord[1]]) { int t = ord[0]; ord[0] = ord[1]; ord[1] = t; }
    if (l[ord[1]] < l[ord[2]]) { int t = ord[1]; ord[1] = ord[2]; ord[2] = t; }
    if (l[ord[0]] < l[ord[1]]) { int t = ord[0]; ord[0] = ord[1]; ord[1] = t; }
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) V[3 * i + c] = E[i][ord[c]];
    const double detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                        V[2] * (V[3] * V[7] - V[4] * V[6]);
    if (detV < 0.0)
        for (int i = 0; i < 3; ++i) V[3 * i + 2] = -V[3 * i + 2];
    // columns of F V
    double FV[3][3];
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < 3; ++i)
            FV[c][i] = F[3 * i] * V[c] + F[3 * i + 1] * V[3 + c] + F[3 * i + 2] * V[6 + c];
    double u0[3], u1[3], u2[3];
    double n0 = sqrt(FV[0][0] * FV[0][0] + FV[0][1] * FV[0][1] + FV[0][2] * FV[0][2]);
    if (n0 > 1e-300) {
        for (int i = 0; i < 3; ++i) u0[i] = FV[0][i] / n0;
    } else {
        u0[0] = 1.0; u0[1] = 0.0; u0[2] = 0.0;
    }
    const double d01 = u0[0] * FV[1][0] + u0[1] * FV[1][1] + u0[2] * FV[1][2];
    for (int i = 0; i < 3; ++i) u1[i] = FV[1][i] - d01 * u0[i];
    double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    if (n1 > 1e-300) {
        for (int i = 0; i < 3; ++i) u1[i] /= n1;
    } else {
        // any unit vector orthogonal to u0
        const double a[3] = {fabs(u0[0]) < 0.9 ? 1.0 : 0.0, fabs(u0[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        const double d = a[0] * u0[0] + a[1] * u0[1];
        for (int i = 0; i < 3; ++i) u1[i] = a[i] - d * u0[i];
        n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
        for (int i = 0; i < 3; ++i) u1[i] /= n1;
    }
    u2[0] = u0[1] * u1[2] - u0[2] * u1[1];
    u2[1] = u0[2] * u1[0] - u0[0] * u1[2];
    u2[2] = u0[0] * u1[1] - u0[1] * u1[0];
    for (int i = 0; i < 3; ++i) {
        U[3 * i] = u0[i];
        U[3 * i + 1] = u1[i];
        U[3 * i + 2] = u2[i];
    }
    s[0] = u0[0] * FV[0][0] + u0[1] * FV[0][1] + u0[2] * FV[0][2];
    s[1] = u1[0] * FV[1][0] + u1[1] * FV[1][1] + u1[2] * FV[1][2];
    s[2] = u2[0] * FV[2][0] + u2[1] * FV[2][1] + u2[2] * FV[2][2];
}

// tau = U diag(d) U^T  (symmetric, Voigt order xx, yy, zz, yz, xz, xy)
__device__ inline void udut(const double U[9], const double d[3], double t6[6]) {
    double T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j)
            T[i][j] = U[3 * i] * d[0] * U[3 * j] + U[3 * i + 1] * d[1] * U[3 * j + 1] +
                      U[3 * i + 2] * d[2] * U[3 * j + 2];
    t6[0] = T[0][0]; t6[1] = T[1][1]; t6[2] = T[2][2];
    t6[3] = T[1][2]; t6[4] = T[0][2]; t6[5] = T[0][1];
}

__device__ inline void hencky_diag(const double s[3], double mu, double lam, double d[3],
                                   double eps[3]) {
    for (int i = 0; i < 3; ++i) eps[i] = log(fmax(fabs(s[i]), 1e-12));
    const double tr = eps[0] + eps[1] + eps[2];
    for (int i = 0; i < 3; ++i) d[i] = 2.0 * mu * eps[i] + lam * tr;
}

// Return map (plastic models, when apply_return) and Kirchhoff stress of one
// particle in float64.  F: F^trial (row-major) on entry, F^E on return; tau6
// receives the stress of F^E.
__device__ inline void return_map_and_stress(int model, double F[9], double mu, double lam,
                                             double tau_y, double friction_deg,
                                             bool apply_return, double tau6[6]) {
    double U[9], s[3], V[9];
    svd3(F, U, s, V);
    if (model == NSF_FIXED_COROTATED) {
        double R[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                R[3 * i + j] = U[3 * i] * V[3 * j] + U[3 * i + 1] * V[3 * j + 1] + U[3 * i + 2] * V[3 * j + 2];
        const double J = s[0] * s[1] * s[2];
        double T[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0.0;
                for (int k = 0; k < 3; ++k) a += (F[3 * i + k] - R[3 * i + k]) * F[3 * j + k];
                T[i][j] = 2.0 * mu * a + (i == j ? lam * (J - 1.0) * J : 0.0);
            }
        tau6[0] = T[0][0]; tau6[1] = T[1][1]; tau6[2] = T[2][2];
        tau6[3] = 0.5 * (T[1][2] + T[2][1]); tau6[4] = 0.5 * (T[0][2] + T[2][0]);
        tau6[5] = 0.5 * (T[0][1] + T[1][0]);
        return;
    }
    double eps[3], d[3];
    hencky_diag(s, mu, lam, d, eps);
    bool changed = false;
    double snew[3] = {s[0], s[1], s[2]};
    if (apply_return && (model == NSF_VON_MISES || model == NSF_DRUCKER_PRAGER)) {
        const double tr = eps[0] + eps[1] + eps[2];
        double eh[3] = {eps[0] - tr / 3.0, eps[1] - tr / 3.0, eps[2] - tr / 3.0};
        const double nrm = sqrt(eh[0] * eh[0] + eh[1] * eh[1] + eh[2] * eh[2]);
        const double safe = nrm > 0.0 ? nrm : 1.0;
        if (model == NSF_VON_MISES) {
            const double dg = nrm - tau_y / (2.0 * mu);
            if (dg > 0.0) {
                for (int i = 0; i < 3; ++i) snew[i] = exp(eps[i] - dg / safe * eh[i]);
                changed = true;
            }
        } else {
            const double sphi = sin(friction_deg * 3.14159265358979323846 / 180.0);
            const double alpha = sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi);
            if (tr > 0.0) {
                snew[0] = snew[1] = snew[2] = 1.0;
                changed = true;
            } else {
                const double dg = nrm + alpha * (3.0 * lam + 2.0 * mu) * tr / (2.0 * mu);
                if (dg > 0.0) {
                    for (int i = 0; i < 3; ++i) snew[i] = exp(eps[i] - dg / safe * eh[i]);
                    changed = true;
                }
            }
        }
    }
    if (changed) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                F[3 * i + j] = U[3 * i] * snew[0] * V[3 * j] + U[3 * i + 1] * snew[1] * V[3 * j + 1] +
                               U[3 * i + 2] * snew[2] * V[3 * j + 2];
        hencky_diag(snew, mu, lam, d, eps);
    }
    udut(U, d, tau6);
}

}  // namespace nsf
