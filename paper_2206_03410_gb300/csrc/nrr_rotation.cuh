// Closest rotation proj_R(A) of Sec. 3.2 (the rotation nearest to A in the
// Frobenius norm) and the 3x3 symmetric eigen-decomposition it rests on, in
// FP64. Shared by the energy kernel and the unrolled backward.
#pragma once

#include <cuda_runtime.h>

namespace nrr_rot {

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (Golub & Van
// Loan, Sec. 8.5). A is destroyed; eigenvectors are the columns of Q.
__device__ inline void jacobi3(double A[9], double Q[9]) {
    for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 16; ++sweep) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-34 * dia || off == 0.0) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0;
            const int q = pq == 0 ? 1 : 2;
            const double apq = A[3 * p + q];
            if (apq == 0.0) continue;
            const double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            for (int k = 0; k < 3; ++k) {
                const double akp = A[3 * k + p], akq = A[3 * k + q];
                A[3 * k + p] = c * akp - s * akq;
                A[3 * k + q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                const double apk = A[3 * p + k], aqk = A[3 * q + k];
                A[3 * p + k] = c * apk - s * aqk;
                A[3 * q + k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                const double qkp = Q[3 * k + p], qkq = Q[3 * k + q];
                Q[3 * k + p] = c * qkp - s * qkq;
                Q[3 * k + q] = s * qkp + c * qkq;
            }
        }
    }
}

// proj_R(A): the rotation closest to A in the Frobenius norm (Sec. 3.2).
// With A^T A = V diag(l) V^T (l descending, det V = +1) and A = U S V^T,
// the closest rotation is U diag(1, 1, det(U V^T)) V^T = [u1, u2, u1 x u2] V^T
// where u1 = A v1 / |A v1|, u2 = the unit part of A v2 orthogonal to u1.
// This form needs only the two largest singular values to be non-zero.
__device__ inline void closest_rotation(const double A[9], double R[9]) {
    double M[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            M[3 * a + b] = A[0 * 3 + a] * A[0 * 3 + b] + A[1 * 3 + a] * A[1 * 3 + b] +
                           A[2 * 3 + a] * A[2 * 3 + b];
    double V[9];
    jacobi3(M, V);
    double l[3] = {M[0], M[4], M[8]};
    int o[3] = {0, 1, 2};
    // sort eigenpairs by descending eigenvalue (stable 3-element sort)
    if (l[o[1]] > l[o[0]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    if (l[o[2]] > l[o[1]]) { int t = o[1]; o[1] = o[2]; o[2] = t; }
    if (l[o[1]] > l[o[0]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    double v1[3], v2[3], v3[3];
    for (int k = 0; k < 3; ++k) { v1[k] = V[3 * k + o[0]]; v2[k] = V[3 * k + o[1]]; v3[k] = V[3 * k + o[2]]; }
    const double det = v1[0] * (v2[1] * v3[2] - v2[2] * v3[1]) - v1[1] * (v2[0] * v3[2] - v2[2] * v3[0]) +
                       v1[2] * (v2[0] * v3[1] - v2[1] * v3[0]);
    if (det < 0) for (int k = 0; k < 3; ++k) v3[k] = -v3[k];
    double a1[3], a2[3];
    for (int k = 0; k < 3; ++k) {
        a1[k] = A[3 * k + 0] * v1[0] + A[3 * k + 1] * v1[1] + A[3 * k + 2] * v1[2];
        a2[k] = A[3 * k + 0] * v2[0] + A[3 * k + 1] * v2[1] + A[3 * k + 2] * v2[2];
    }
    double n1 = sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
    if (!(n1 > 0)) {
        for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
        return;
    }
    double u1[3] = {a1[0] / n1, a1[1] / n1, a1[2] / n1};
    const double pr = u1[0] * a2[0] + u1[1] * a2[1] + u1[2] * a2[2];
    double w2[3] = {a2[0] - pr * u1[0], a2[1] - pr * u1[1], a2[2] - pr * u1[2]};
    double n2 = sqrt(w2[0] * w2[0] + w2[1] * w2[1] + w2[2] * w2[2]);
    if (!(n2 > 1e-300)) {
        // rank-one A: any unit vector orthogonal to u1
        const int k = fabs(u1[0]) < 0.9 ? 0 : 1;
        double e[3] = {0, 0, 0};
        e[k] = 1.0;
        const double pe = u1[k];
        w2[0] = e[0] - pe * u1[0]; w2[1] = e[1] - pe * u1[1]; w2[2] = e[2] - pe * u1[2];
        n2 = sqrt(w2[0] * w2[0] + w2[1] * w2[1] + w2[2] * w2[2]);
    }
    double u2[3] = {w2[0] / n2, w2[1] / n2, w2[2] / n2};
    double u3[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[3 * a + b] = u1[a] * v1[b] + u2[a] * v2[b] + u3[a] * v3[b];
}

// Closest rotation for det(A) > 0: the orthogonal polar factor of A, by
// Newton's iteration X <- (X + X^{-T}) / 2 (Higham, "Computing the polar
// decomposition - with applications", SIAM J. Sci. Stat. Comput. 1986),
// with X^{-T} = cof(X) / det(X). Quadratic convergence; near-orthogonal A
// (the usual case) takes 4-6 steps. Returns false if it did not converge,
// in which case the SVD route is used.
__device__ inline bool polar_rotation(const double A[9], double R[9]) {
    double X[9];
    for (int k = 0; k < 9; ++k) X[k] = A[k];
    for (int iter = 0; iter < 30; ++iter) {
        const double c0 = X[4] * X[8] - X[5] * X[7];
        const double c1 = X[5] * X[6] - X[3] * X[8];
        const double c2 = X[3] * X[7] - X[4] * X[6];
        const double det = X[0] * c0 + X[1] * c1 + X[2] * c2;
        if (!(det > 0)) return false;
        const double id = 1.0 / det;
        double C[9];
        C[0] = c0; C[1] = c1; C[2] = c2;
        C[3] = X[2] * X[7] - X[1] * X[8];
        C[4] = X[0] * X[8] - X[2] * X[6];
        C[5] = X[1] * X[6] - X[0] * X[7];
        C[6] = X[1] * X[5] - X[2] * X[4];
        C[7] = X[2] * X[3] - X[0] * X[5];
        C[8] = X[0] * X[4] - X[1] * X[3];
        double diff = 0.0;
        for (int k = 0; k < 9; ++k) {
            const double nx = 0.5 * (X[k] + C[k] * id);
            diff += (nx - X[k]) * (nx - X[k]);
            X[k] = nx;
        }
        if (diff < 1e-30) {
            for (int k = 0; k < 9; ++k) R[k] = X[k];
            return true;
        }
    }
    return false;
}

// proj_R(A) for A [9] row-major: the polar route when it converges (det A
// > 0), else the singular-vector route.
__device__ inline void proj_rotation(const double A[9], double R[9]) {
    if (!polar_rotation(A, R)) closest_rotation(A, R);
}

}  // namespace nrr_rot
