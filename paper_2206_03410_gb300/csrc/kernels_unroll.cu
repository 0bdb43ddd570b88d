// Reverse-mode derivative of one plain MM step X' = K(X^k)^-1 B(X^k)
// (Sec. 3.3.1-3.3.2, Eq. surr_solution) for the unrolled backward.
//
// With lambda = K^-1 g_bar (the adjoint solve, run by the PCG kernels) and
// the solve taken as exact, dL/dB = lambda and dL/dK = -lambda X'^T. K and B
// depend on X^k through the Welsch weights w^a_i (of d_i), w^r_ij (of D_ij)
// and the rotation targets proj_R(A_j); they depend on the source positions
// v_i through the rows f_i = [w_ij (v_i - p_j)^T, w_ij]_j of F. Closest
// points, node positions p_j and skinning weights w_ij are held constant.
//
// Per point i (adj_point_kernel), with a_i = lambda^T f_i, v'_i the deformed
// point under X', u_i the closest target point:
//   dL/dw^a_i = a_i . (u_i - v'_i)
//   e_i       = dL/dv_hat_i = 2 (dL/dw^a_i) w'(d_i^2) (v_hat_i - u_i)
//   dL/dv_i  += w^a_i sum_j w_ij (Lambda_j (u_i - v'_i) - A'_j^T a_i)
//             + sum_j w_ij A_j^T e_i
// (Lambda_j: rows 0..2 of lambda's block j, in the layout of X).
// Per node n (adj_node_kernel), the new cotangent dL/dX^k_n collects
//   sum_i w_in [v_i - p_n; 1] e_i^T                       (alignment weights)
//   h D_ij(X^k)^T scaled by 2 (dL/dw^r_ij) w'(|D_ij|^2),
//     dL/dw^r_ij = -alpha (h^T lambda) . D_ij(X')         (regularisation weights)
//   the derivative of proj_R at A_n applied to beta Lambda_n^T (rotation targets).
// The slope w' of a weight is -w / (2 nu^2) for Welsch's function and 0 for
// the squared norm and its truncation (almost everywhere).
// The derivative of proj_R: with R = proj_R(A) and S = R^T A (symmetric),
// A = R S gives R^T dR = Omega with Omega S + S Omega = R^T dA - dA^T R; in
// the eigenbasis of S the adjoint is Gamma_kl = skew(R^T Rbar)_kl /
// (s_k + s_l) and dL/dA = 2 R Gamma.
// Groups of 8 lanes own one node and sum its contribution list in a fixed
// order: deterministic, no atomics.
#include "nrr_device.cuh"
#include "nrr_rotation.cuh"

namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads)
    adj_point_kernel(DevProblem<T> d, const T* __restrict__ lam, const T* __restrict__ Xn,
                     const int* __restrict__ order, T* __restrict__ ebuf, double* __restrict__ gv) {
    const NrrState* st = d.st;
    const int P = d.P;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const T* vh = d.vhat + (size_t)(st->vk ^ 1) * 3 * P;   // v_hat at X^k (evaluation buffer)
    const T* Xk = d.Xeval;
    const T vx = d.v[i], vy = d.v[P + i], vz = d.v[2 * P + i];
    const T ux = d.u[i], uy = d.u[P + i], uz = d.u[2 * P + i];
    T a[3] = {0, 0, 0}, vn[3] = {0, 0, 0};
    const int s0 = d.infl_ptr[i], s1 = d.infl_ptr[i + 1];
    for (int s = s0; s < s1; ++s) {
        const int j = d.infl_node[s];
        const T w = d.infl_w[s];
        const T px = d.p[3 * j], py = d.p[3 * j + 1], pz = d.p[3 * j + 2];
        const T dx = vx - px, dy = vy - py, dz = vz - pz;
        const T* L = lam + 12 * j;
        const T* N = Xn + 12 * j;
        const T pj[3] = {px, py, pz};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c] += w * (L[c] * dx + L[3 + c] * dy + L[6 + c] * dz + L[9 + c]);
            vn[c] += w * (N[c] * dx + N[3 + c] * dy + N[6 + c] * dz + N[9 + c] + pj[c]);
        }
    }
    const T rq[3] = {ux - vn[0], uy - vn[1], uz - vn[2]};
    const T wai = d.wa[i];
    const T ia = (T)(1.0 / (2.0 * st->nu_a * st->nu_a));
    const T wbar = a[0] * rq[0] + a[1] * rq[1] + a[2] * rq[2];
    // dw/d(d^2): -w / (2 nu_a^2) for Welsch's function, 0 for the l2 variants
    const T c2 = d.robust == NRR_WELSCH ? (T)-2 * wbar * wai * ia : (T)0;
    const T e[3] = {c2 * (vh[i] - ux), c2 * (vh[P + i] - uy), c2 * (vh[2 * P + i] - uz)};
    ebuf[i] = e[0];
    ebuf[P + i] = e[1];
    ebuf[2 * P + i] = e[2];
    T g[3] = {0, 0, 0};
    for (int s = s0; s < s1; ++s) {
        const int j = d.infl_node[s];
        const T w = d.infl_w[s];
        const T* L = lam + 12 * j;
        const T* N = Xn + 12 * j;
        const T* K = Xk + 12 * j;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const T lr = L[3 * r] * rq[0] + L[3 * r + 1] * rq[1] + L[3 * r + 2] * rq[2];
            const T nr = N[3 * r] * a[0] + N[3 * r + 1] * a[1] + N[3 * r + 2] * a[2];
            const T kr = K[3 * r] * e[0] + K[3 * r + 1] * e[1] + K[3 * r + 2] * e[2];
            g[r] += w * (wai * (lr - nr) + kr);
        }
    }
    const int ci = order[i];
    gv[3 * ci + 0] += (double)g[0];
    gv[3 * ci + 1] += (double)g[1];
    gv[3 * ci + 2] += (double)g[2];
}

// dL/dA of proj_R at A for dL/dR = Rb (row-major 3x3, FP64).
__device__ void proj_rotation_adjoint(const double A[9], const double Rb[9], double Ab[9]) {
    double R[9];
    nrr_rot::proj_rotation(A, R);
    double S[9], M[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0, m = 0.0;
            for (int k = 0; k < 3; ++k) {
                s += R[3 * k + a] * A[3 * k + b];
                m += R[3 * k + a] * Rb[3 * k + b];
            }
            S[3 * a + b] = s;
            M[3 * a + b] = m;
        }
    // symmetrise S (it is symmetric up to rounding) and diagonalise it
    double Ss[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Ss[3 * a + b] = 0.5 * (S[3 * a + b] + S[3 * b + a]);
    double V[9];
    nrr_rot::jacobi3(Ss, V);
    const double ev[3] = {Ss[0], Ss[4], Ss[8]};
    // skew part of R^T Rb in the eigenbasis: Vt K V
    double Kk[9], KV[9], Gt[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Kk[3 * a + b] = 0.5 * (M[3 * a + b] - M[3 * b + a]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            KV[3 * a + b] = Kk[3 * a] * V[b] + Kk[3 * a + 1] * V[3 + b] + Kk[3 * a + 2] * V[6 + b];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            const double t = V[k] * KV[l] + V[3 + k] * KV[3 + l] + V[6 + k] * KV[6 + l];
            const double den = ev[k] + ev[l];
            Gt[3 * k + l] = (k != l && den != 0.0) ? t / den : 0.0;
        }
    // Gamma = V Gt V^T, dL/dA = 2 R Gamma
    double GV[9], Gm[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            GV[3 * a + b] = Gt[3 * a] * V[3 * b] + Gt[3 * a + 1] * V[3 * b + 1] + Gt[3 * a + 2] * V[3 * b + 2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Gm[3 * a + b] = V[3 * a] * GV[b] + V[3 * a + 1] * GV[3 + b] + V[3 * a + 2] * GV[6 + b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Ab[3 * a + b] = 2.0 * (R[3 * a] * Gm[b] + R[3 * a + 1] * Gm[3 + b] + R[3 * a + 2] * Gm[6 + b]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    adj_node_kernel(DevProblem<T> d, const T* __restrict__ lam, const T* __restrict__ Xn,
                    const T* __restrict__ ebuf, double* __restrict__ gd, T* __restrict__ gt) {
    const NrrState* st = d.st;
    const int lane8 = threadIdx.x & 7;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int P = d.P;
    const T alpha = (T)st->alpha;
    const double beta = st->beta;
    const T ir = (T)(1.0 / (2.0 * st->nu_r * st->nu_r));
    const T* Xk = d.Xeval;
    for (int n0 = gwarp * 4; n0 < d.N; n0 += nwarps * 4) {
        const int n = min(n0 + ((threadIdx.x & 31) >> 3), d.N - 1);
        const bool active = (n0 + ((threadIdx.x & 31) >> 3)) < d.N;
        int bdg = d.bsr_ptr[n];
        while (d.bsr_col[bdg] != n) ++bdg;
        const T pnx = d.p[3 * n], pny = d.p[3 * n + 1], pnz = d.p[3 * n + 2];
        T g[12];
#pragma unroll
        for (int t = 0; t < 12; ++t) g[t] = 0;
        // alignment weights: sum_i w_in [v_i - p_n; 1] e_i^T
        const int e_end = active ? d.ent_ptr[bdg + 1] : 0;
        for (int e = d.ent_ptr[bdg] + lane8; e < e_end; e += 8) {
            const int i = d.ent[e] >> 6;
            const T wn = d.ent_q[e];   // diagonal block: w_in
            const T an[4] = {d.v[i] - pnx, d.v[P + i] - pny, d.v[2 * P + i] - pnz, (T)1};
            const T ex = ebuf[i], ey = ebuf[P + i], ez = ebuf[2 * P + i];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const T ca = wn * an[a];
                g[3 * a + 0] += ca * ex;
                g[3 * a + 1] += ca * ey;
                g[3 * a + 2] += ca * ez;
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
            for (int t = 0; t < 12; ++t) g[t] += __shfl_xor_sync(0xffffffffu, g[t], o);
        }
        if (lane8 != 0 || !active) continue;
        // regularisation weights: pairs (n, j) (n first: h = [0,0,0,-r] at X_n)
        // and reverse pairs (j, n) (n second: h = r [(p_j - p_n)^T, 1] at X_n)
        for (int e = d.adj_ptr[n]; e < d.adj_ptr[n + 1]; ++e) {
            for (int side = 0; side < 2; ++side) {
                const int ee = side == 0 ? e : d.e_rev[e];
                const int a_ = d.e_i[ee], b_ = d.e_j[ee];
                const T r = d.e_r[ee];
                const T dx = d.p[3 * a_] - d.p[3 * b_];
                const T dy = d.p[3 * a_ + 1] - d.p[3 * b_ + 1];
                const T dz = d.p[3 * a_ + 2] - d.p[3 * b_ + 2];
                const T dd[3] = {dx, dy, dz};
                const T* Ka = Xk + 12 * a_;
                const T* Kb = Xk + 12 * b_;
                const T* Na = Xn + 12 * a_;
                const T* Nb = Xn + 12 * b_;
                const T* La = lam + 12 * a_;
                const T* Lb = lam + 12 * b_;
                T Dk[3];
                T wbar = 0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Dk[c] = r * ((Kb[c] * dx + Kb[3 + c] * dy + Kb[6 + c] * dz - dd[c]) + (Kb[9 + c] - Ka[9 + c]));
                    const T Dn = r * ((Nb[c] * dx + Nb[3 + c] * dy + Nb[6 + c] * dz - dd[c]) + (Nb[9 + c] - Na[9 + c]));
                    const T hl = r * ((Lb[c] * dx + Lb[3 + c] * dy + Lb[6 + c] * dz) + (Lb[9 + c] - La[9 + c]));
                    wbar -= hl * Dn;
                }
                wbar *= alpha;
                const T coef = d.robust == NRR_WELSCH ? (T)-2 * wbar * d.wr[ee] * ir : (T)0;
                if (side == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) g[9 + c] -= coef * r * Dk[c];
                } else {
                    const T h[4] = {r * dx, r * dy, r * dz, r};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) g[3 * a + c] += coef * h[a] * Dk[c];
                }
            }
        }
        // rotation targets: dL/dR_n[a][b] = beta lambda_n[3b + a]
        {
            const T* Kn = Xk + 12 * n;
            const T* Ln = lam + 12 * n;
            double A[9], Rb[9], Ab[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    A[3 * a + b] = (double)Kn[3 * b + a];
                    Rb[3 * a + b] = beta * (double)Ln[3 * b + a];
                }
            proj_rotation_adjoint(A, Rb, Ab);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) g[3 * b + a] += (T)Ab[3 * a + b];
        }
#pragma unroll
        for (int t = 0; t < 12; ++t) {
            gd[12 * n + t] = (double)g[t];
            gt[12 * n + t] = g[t];
        }
    }
}

template <typename T>
__global__ void to_t_kernel(const double* __restrict__ in, T* __restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_adjoint(const DevProblem<T>& d, const T* lam, const T* Xn, const int* order, T* ebuf,
                               double* gv, double* gd, T* gt, cudaStream_t s) {
    if (d.P > 0) adj_point_kernel<T><<<(d.P + kThreads - 1) / kThreads, kThreads, 0, s>>>(d, lam, Xn, order, ebuf, gv);
    const int grid = (d.N + 31) / 32 > 0 ? (d.N + 31) / 32 : 1;
    adj_node_kernel<T><<<grid, kThreads, 0, s>>>(d, lam, Xn, ebuf, gd, gt);
    return cudaGetLastError();
}

template <typename T>
cudaError_t nrr_launch_to_t(const double* in, T* out, int n, cudaStream_t s) {
    if (n > 0) to_t_kernel<T><<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_adjoint<float>(const DevProblem<float>&, const float*, const float*, const int*,
                                               float*, double*, double*, float*, cudaStream_t);
template cudaError_t nrr_launch_adjoint<double>(const DevProblem<double>&, const double*, const double*, const int*,
                                                double*, double*, double*, double*, cudaStream_t);
template cudaError_t nrr_launch_to_t<float>(const double*, float*, int, cudaStream_t);
template cudaError_t nrr_launch_to_t<double>(const double*, double*, int, cudaStream_t);
