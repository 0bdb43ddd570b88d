// Energy (Eq. objective_func), Welsch weights of the surrogate (Sec. 3.3.1),
// rotation projections, the safeguard test of Algorithm 2, and assembly of
// the normal equations K X = B of Eq. (surr_solution) (Sec. 3.3.2).
#include "nrr_device.cuh"
#include "nrr_rotation.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double x, double* sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    return s;   // valid in thread 0
}

template <typename T>
__device__ __forceinline__ T t_exp(T x);
template <>
__device__ __forceinline__ float t_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double t_exp<double>(double x) { return exp(x); }
template <typename T>
__device__ __forceinline__ T t_expm1(T x);
template <>
__device__ __forceinline__ float t_expm1<float>(float x) { return expm1f(x); }
template <>
__device__ __forceinline__ double t_expm1<double>(double x) { return expm1(x); }

// |D_ab|^2 of the regularisation residual of directed edge e (Eq. RegTerm):
// D_ab = r_ab (A_b (p_a - p_b) + p_b + t_b - p_a - t_a). One definition for
// both kernels that form the weights, so that they agree bit for bit.
template <typename T>
__device__ __forceinline__ T reg_d2(const DevProblem<T>& d, const T* X, int e) {
    const int a = d.e_i[e], b = d.e_j[e];
    const T r = d.e_r[e];
    const T* Xb = X + 12 * b;
    const T* Xa = X + 12 * a;
    const T dx = d.p[3 * a] - d.p[3 * b];
    const T dy = d.p[3 * a + 1] - d.p[3 * b + 1];
    const T dz = d.p[3 * a + 2] - d.p[3 * b + 2];
    // p_b - p_a = -(p_a - p_b)
    const T Dx = r * ((Xb[0] * dx + Xb[3] * dy + Xb[6] * dz - dx) + (Xb[9] - Xa[9]));
    const T Dy = r * ((Xb[1] * dx + Xb[4] * dy + Xb[7] * dz - dy) + (Xb[10] - Xa[10]));
    const T Dz = r * ((Xb[2] * dx + Xb[5] * dy + Xb[8] * dz - dz) + (Xb[11] - Xa[11]));
    return Dx * Dx + Dy * Dy + Dz * Dz;
}

// 1 / (2 nu^2) in T, the scale of the Welsch weights and energy terms
template <typename T>
__device__ __forceinline__ T welsch_scale(double nu) { return (T)(1.0 / (2.0 * nu * nu)); }

// Terms of Eq. (objective_func) that depend on X only, not on the closest
// points: the regularisation term (Eq. RegTerm) with its surrogate weights
// w^r_ij, and the rotation term with the projections proj_R(A_n). A pass
// runs this kernel on a parallel branch of its graph, beside the
// closest-point search, whose last CTA may end the stage (Algorithm 2) and
// halve nu_r while this kernel runs. So each CTA records the nu_r it read
// and sums the regularisation term at that nu_r and at half of it;
// energy_kernel, which runs after both, takes the sum at the stage's nu_r
// and re-forms the weights if a CTA read the previous stage's value.
// Per CTA: d.xpartials[4 b ..] = {E_reg at nu, E_reg at nu / 2, E_rot, nu}.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) xterm_kernel(DevProblem<T> d) {
    __shared__ double sh[kThreads / 32];
    NrrState* st = d.st;
    if (MODE == NRR_MODE_PASS && st->done) return;
    const T* X = (MODE == NRR_MODE_EVAL) ? d.Xeval : d.X;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gstride = gridDim.x * blockDim.x;
    __shared__ double s_nu;
    if (threadIdx.x == 0) s_nu = *reinterpret_cast<volatile const double*>(&st->nu_r);
    __syncthreads();
    const double nur = s_nu;
    const T ir = welsch_scale<T>(nur), irh = welsch_scale<T>(0.5 * nur);
    double er = 0.0, erh = 0.0, eo = 0.0;
    // regularisation term (Eq. RegTerm) over directed pairs, weights w^r_ij
    for (int e = gtid; e < d.E2; e += gstride) {
        const T D2 = reg_d2(d, X, e);
        if (d.robust == NRR_WELSCH) {
            er += (double)(-t_expm1<T>(-D2 * ir));
            erh += (double)(-t_expm1<T>(-D2 * irh));
            d.wr[e] = t_exp<T>(-D2 * ir) * ir;
        } else {
            // squared norm: energy |D|^2, weight 1
            er += (double)D2;
            erh += (double)D2;
            d.wr[e] = (T)1;
        }
    }
    // rotation term: |A_n - proj_R(A_n)|_F^2
    // nodes are spread CTA-major so that the double-precision SVDs use every SM
    for (int n = blockIdx.x + threadIdx.x * gridDim.x; n < d.N; n += gstride) {
        const T* Xn = X + 12 * n;
        double A[9], R[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[3 * a + b] = (double)Xn[3 * b + a];
        nrr_rot::proj_rotation(A, R);
        double s = 0.0;
        for (int k = 0; k < 9; ++k) {
            const double df = A[k] - R[k];
            s += df * df;
            d.Rm[9 * n + k] = (T)R[k];
        }
        eo += s;
    }
    const double sr = block_sum(er, sh);
    const double srh = block_sum(erh, sh);
    const double so = block_sum(eo, sh);
    if (threadIdx.x == 0) {
        d.xpartials[4 * blockIdx.x + 0] = sr;
        d.xpartials[4 * blockIdx.x + 1] = srh;
        d.xpartials[4 * blockIdx.x + 2] = so;
        d.xpartials[4 * blockIdx.x + 3] = nur;
    }
}

// The alignment term (Eq. AlignmentTerm) and its surrogate weights w^a_i
// from the closest-point distances, the sum of all terms (FP64, fixed
// order: the last CTA adds every CTA's partial sums and xterm_kernel's), and
// in a pass the safeguard test of Algorithm 2.
// The assembly's row of point i (pts, 8 values of T): v_i, w^a_i, and
// Q_i = u_rho(i) - pbar_i (the same float operations the assembly did on its
// gathers), stored as two 16-byte vectors (float) or four (double).
template <typename T>
__device__ __forceinline__ void store_pt(T* pts, int i, T vx, T vy, T vz, T wa, T qx, T qy, T qz);
template <>
__device__ __forceinline__ void store_pt<float>(float* pts, int i, float vx, float vy, float vz, float wa, float qx,
                                                float qy, float qz) {
    float4* p = reinterpret_cast<float4*>(pts) + 2 * (size_t)i;
    p[0] = make_float4(vx, vy, vz, wa);
    p[1] = make_float4(qx, qy, qz, 0.f);
}
template <>
__device__ __forceinline__ void store_pt<double>(double* pts, int i, double vx, double vy, double vz, double wa,
                                                 double qx, double qy, double qz) {
    double2* p = reinterpret_cast<double2*>(pts) + 4 * (size_t)i;
    p[0] = make_double2(vx, vy);
    p[1] = make_double2(vz, wa);
    p[2] = make_double2(qx, qy);
    p[3] = make_double2(qz, 0.0);
}
template <typename T>
__device__ __forceinline__ void load_pt_v(const T* pts, int i, T& vx, T& vy, T& vz, T& wa);
template <>
__device__ __forceinline__ void load_pt_v<float>(const float* pts, int i, float& vx, float& vy, float& vz, float& wa) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(pts) + 2 * (size_t)i);
    vx = a.x; vy = a.y; vz = a.z; wa = a.w;
}
template <>
__device__ __forceinline__ void load_pt_v<double>(const double* pts, int i, double& vx, double& vy, double& vz,
                                                  double& wa) {
    const double2* p = reinterpret_cast<const double2*>(pts) + 4 * (size_t)i;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    vx = a.x; vy = a.y; vz = b.x; wa = b.y;
}
template <typename T>
__device__ __forceinline__ void load_pt_q(const T* pts, int i, T& qx, T& qy, T& qz);
template <>
__device__ __forceinline__ void load_pt_q<float>(const float* pts, int i, float& qx, float& qy, float& qz) {
    const float4 b = __ldg(reinterpret_cast<const float4*>(pts) + 2 * (size_t)i + 1);
    qx = b.x; qy = b.y; qz = b.z;
}
template <>
__device__ __forceinline__ void load_pt_q<double>(const double* pts, int i, double& qx, double& qy, double& qz) {
    const double2* p = reinterpret_cast<const double2*>(pts) + 4 * (size_t)i + 2;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    qx = a.x; qy = a.y; qz = b.x;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) energy_kernel(DevProblem<T> d) {
    __shared__ double sh[kThreads / 32];
    __shared__ int s_last, s_reject;
    NrrState* st = d.st;
    if (MODE == NRR_MODE_PASS && st->done) return;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gstride = gridDim.x * blockDim.x;
    const double nua = st->nu_a;
    const T ia = welsch_scale<T>(nua);
    double ea = 0.0;
    // did a CTA of xterm_kernel read the nu_r of the previous stage (the
    // closest-point search ended the stage while it ran)? Then the weights
    // w^r are formed again here at the stage's nu_r.
    const double nur = st->nu_r;
    int mine = 0;
    for (int b = threadIdx.x; b < d.n_xpart; b += blockDim.x) mine |= __ldcg(d.xpartials + 4 * b + 3) != nur;
    const int stale = __syncthreads_or(mine);
    if (stale && d.robust == NRR_WELSCH) {
        const T* X = (MODE == NRR_MODE_EVAL) ? d.Xeval : d.X;
        const T ir = welsch_scale<T>(nur);
        for (int e = gtid; e < d.E2; e += gstride) d.wr[e] = t_exp<T>(-reg_d2(d, X, e) * ir) * ir;
    }
    // alignment term (Eq. AlignmentTerm) and its surrogate weights w^a_i;
    // the l2 variants: d^2 with weight 1, or min(d^2, 9 nu_a^2) with weight
    // 1 below 3 nu_a and 0 from there on
    const int P = d.P;
    auto put_row = [&](int i, T w) {
        d.wa[i] = w;
        store_pt<T>(d.pts, i, d.v[i], d.v[P + i], d.v[2 * P + i], w, d.u[i] - d.pbar[i],
                    d.u[P + i] - d.pbar[P + i], d.u[2 * P + i] - d.pbar[2 * P + i]);
    };
    if (d.robust == NRR_WELSCH) {
        for (int i = gtid; i < P; i += gstride) {
            const T x = d.d2[i] * ia;
            ea += (double)(-t_expm1<T>(-x));
            put_row(i, t_exp<T>(-x) * ia);
        }
    } else {
        const T cut = (T)(9.0 * nua * nua);
        const bool trunc = d.robust == NRR_L2_TRUNCATED;
        for (int i = gtid; i < P; i += gstride) {
            const T d2 = d.d2[i];
            const bool in = !trunc || d2 < cut;
            ea += (double)(in ? d2 : cut);
            put_row(i, in ? (T)1 : (T)0);
        }
    }
    const double sa = block_sum(ea, sh);
    if (threadIdx.x == 0) {
        d.partials[blockIdx.x * NRR_PARTIAL_STRIDE + 0] = sa;
        __threadfence();
        const unsigned t = atomicAdd(&st->cnt_energy, 1u);
        s_last = (t == gridDim.x - 1);
        s_reject = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    {
        // the last CTA adds all partials: thread-strided, then a fixed-order tree
        double pa = 0.0, pr = 0.0, po = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            pa += __ldcg(d.partials + b * NRR_PARTIAL_STRIDE + 0);
        for (int b = threadIdx.x; b < d.n_xpart; b += blockDim.x) {
            // a CTA that read the previous stage's nu_r (twice the current
            // one, exactly) summed the term at the current nu_r second
            const bool same = __ldcg(d.xpartials + 4 * b + 3) == nur;
            pr += __ldcg(d.xpartials + 4 * b + (same ? 0 : 1));
            po += __ldcg(d.xpartials + 4 * b + 2);
        }
        const double ta = block_sum(pa, sh);
        const double tr = block_sum(pr, sh);
        const double to = block_sum(po, sh);
        if (threadIdx.x == 0) { sh[0] = ta; sh[1] = tr; sh[2] = to; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double A = sh[0], Rg = sh[1], O = sh[2];
        st->cnt_energy = 0;
        const double E = A + st->alpha * Rg + st->beta * O;
        if (MODE == NRR_MODE_EVAL) {
            st->E_eval[0] = E; st->E_eval[1] = A; st->E_eval[2] = Rg; st->E_eval[3] = O;
        } else {
            st->E = E; st->E_align = A; st->E_reg = Rg; st->E_rot = O;
            st->n_passes += 1;
            st->solved = 0;
            st->n_singular = 0;
            if (E > st->E_prev && !st->just_reverted) {
                // Anderson iterate rejected: revert to the last MM result
                st->kept = 0;
                st->skip = 1;
                st->just_reverted = 1;
                st->n_rejected += 1;
                s_reject = 1;
            } else {
                st->kept = 1;
                st->just_reverted = 0;
                st->vk = st->vlast;
                st->have_vk = 1;
                const double Ep = st->E_prev;
                if (st->rel_tol > 0 && isfinite(Ep) && fabs(Ep - E) < st->rel_tol * fabs(Ep)) {
                    st->skip = 1;
                    nrr_end_stage(st);
                } else {
                    st->E_prev = E;
                    st->skip = 0;
                }
            }
        }
    }
    __syncthreads();
    if (MODE == NRR_MODE_PASS && s_reject) {
        const int n12 = d.N * 12;
        for (int k = threadIdx.x; k < n12; k += blockDim.x) d.X[k] = d.Gprev[k];
    }
}

// ---------------------------------------------------------------------------
// Assembly of K = F^T W_a F + alpha H^T W_r H + beta J^T J and
// B = F^T W_a Q + alpha H^T W_r Y + beta J^T J Z (Sec. 3.3.2).
// Every 4x4 block sums its precomputed list of point contributions in a
// fixed order, then adds its regularisation and rotation parts:
// deterministic, no atomics. A diagonal block (node n, n) collects every
// point that n influences (about |I|-times more than an off-diagonal block)
// and the node's row of B: a whole warp owns it and accumulates the 10
// entries of its symmetric upper triangle. Off-diagonal blocks go four to a
// warp, 8 lanes each. Warps with diagonal blocks come first.
// ---------------------------------------------------------------------------
// entries per lane loaded together (independent gather chains in flight)
constexpr int kU = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 1) assemble_kernel(DevProblem<T> d) {
    NrrState* st = d.st;
    if (st->done || st->skip) return;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int P = d.P;
    const int N = d.N;
    const int n_off = d.nblk - N;
    const int n_work = N + (n_off + 3) / 4;
    const T alpha = (T)st->alpha, beta = (T)st->beta;
    // the loop is warp-uniform so that the shuffles see all 32 lanes
    for (int wk = gwarp; wk < n_work; wk += nwarps) {
        if (wk < N) {
            // ---- diagonal block of node n and row n of B: one warp ----
            const int n = wk;
            const int4 desc = __ldg(d.asm_diag + n);   // {block, entries, first edge}
            const int b = desc.x;
            const int adj1 = __ldg(d.adj_ptr + n + 1);
            const T pnx = d.p[3 * n], pny = d.p[3 * n + 1], pnz = d.p[3 * n + 2];
            T acc[10];
            T accB[12];
#pragma unroll
            for (int t = 0; t < 10; ++t) acc[t] = 0;
#pragma unroll
            for (int t = 0; t < 12; ++t) accB[t] = 0;
            // kU entries per lane at a time (e, e + 32, ...): every gather of
            // the batch is issued before the first is used; each lane still
            // adds its entries in increasing order
            const int e_end = desc.z;
            for (int e0 = desc.y + lane; e0 < e_end; e0 += 32 * kU) {
                int ii[kU];
                T wq[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int e = e0 + 32 * u;
                    ii[u] = e < e_end ? __ldg(d.ent + e) >> 6 : -1;
                    wq[u] = e < e_end ? __ldg(d.ent_q + e) : (T)0;
                }
                T vx[kU], vy[kU], vz[kU], wa[kU], qx[kU], qy[kU], qz[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    // v_i, w^a_i and Q_i = u_rho(i) - sum_j w_ij p_j, one row
                    const int i = ii[u] < 0 ? 0 : ii[u];
                    load_pt_v<T>(d.pts, i, vx[u], vy[u], vz[u], wa[u]);
                    load_pt_q<T>(d.pts, i, qx[u], qy[u], qz[u]);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    if (ii[u] < 0) break;
                    const T an[4] = {vx[u] - pnx, vy[u] - pny, vz[u] - pnz, (T)1};
                    const T cb = wa[u] * wq[u];
                    const T c = cb * wq[u];
                    int t = 0;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const T cr = c * an[r];
#pragma unroll
                        for (int s2 = r; s2 < 4; ++s2) acc[t++] += cr * an[s2];
                        const T br = cb * an[r];
                        accB[3 * r + 0] += br * qx[u];
                        accB[3 * r + 1] += br * qy[u];
                        accB[3 * r + 2] += br * qz[u];
                    }
                }
            }
            // the alignment part of the (t, t) entry, summed apart: 0 when no
            // point that node n influences has alignment weight (singular K,
            // kernels_solve.cu)
            T a33 = acc[9];
            // regularisation part, one edge of node n per lane (all lanes'
            // loads in flight together). Pair (n, j): its H row is
            // [0,0,0,-r] at X_n, so r^2 on entry (3,3) and B row 3 gets
            // -r y with y = r (p_n - p_j); reverse pair (j, n): h = r'[(p_j -
            // p_n)^T, 1] at X_n adds h h^T and h y'^T with y' = r'(p_j - p_n)
            for (int e = desc.w + lane; e < adj1; e += 32) {
                const int j = d.e_j[e];
                const int er = d.e_rev[e];
                const T r = d.e_r[e], w = alpha * d.wr[e];
                const T r2 = d.e_r[er], w2 = alpha * d.wr[er];
                const T dj[3] = {d.p[3 * j] - pnx, d.p[3 * j + 1] - pny, d.p[3 * j + 2] - pnz};
                const T wrr = w * r * r;
                acc[9] += wrr;
                accB[9] += wrr * dj[0];
                accB[10] += wrr * dj[1];
                accB[11] += wrr * dj[2];
                const T h[4] = {r2 * dj[0], r2 * dj[1], r2 * dj[2], r2};
                int t = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const T wh = w2 * h[a];
#pragma unroll
                    for (int cc = a; cc < 4; ++cc) acc[t++] += wh * h[cc];
                    accB[3 * a + 0] += wh * h[0];
                    accB[3 * a + 1] += wh * h[1];
                    accB[3 * a + 2] += wh * h[2];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int t = 0; t < 10; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
#pragma unroll
                for (int t = 0; t < 12; ++t) accB[t] += __shfl_xor_sync(0xffffffffu, accB[t], o);
                a33 += __shfl_xor_sync(0xffffffffu, a33, o);
            }
            if (lane != 0) continue;
            d.anode[n] = a33;
            T K16[16];
            {
                int t = 0;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int s2 = r; s2 < 4; ++s2) {
                        K16[4 * r + s2] = acc[t];
                        K16[4 * s2 + r] = acc[t];
                        ++t;
                    }
            }
            // rotation term: beta on A-rows, B rows 0..2 += beta R_n^T
            K16[0] += beta; K16[5] += beta; K16[10] += beta;
            const T* R = d.Rm + 9 * n;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) accB[3 * a + cc] += beta * R[3 * cc + a];
#pragma unroll
            for (int t = 0; t < 12; ++t) d.Bv[12 * n + t] = accB[t];
#pragma unroll
            for (int t = 0; t < 16; ++t) d.Kv[16 * b + t] = K16[t];
        } else {
            // ---- four off-diagonal blocks, 8 lanes each ----
            const int q = (wk - N) * 4 + (lane >> 3);
            const bool active = q < n_off;
            const int lane8 = lane & 7;
            const int4 desc = __ldg(d.asm_off + (active ? q : n_off - 1));   // {block, entries, pair}
            const int4 nk = __ldg(d.asm_off2 + (active ? q : n_off - 1));    // {n, k, reverse pair}
            const int b = desc.x;
            const int n = nk.x, k = nk.y;
            const T pnx = d.p[3 * n], pny = d.p[3 * n + 1], pnz = d.p[3 * n + 2];
            const T pkx = d.p[3 * k], pky = d.p[3 * k + 1], pkz = d.p[3 * k + 2];
            T acc[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) acc[t] = 0;
            const int e_end = active ? desc.z : 0;
            for (int e0 = desc.y + lane8; e0 < e_end; e0 += 8 * kU) {
                int ii[kU];
                T wq[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int e = e0 + 8 * u;
                    ii[u] = e < e_end ? __ldg(d.ent + e) >> 6 : -1;
                    wq[u] = e < e_end ? __ldg(d.ent_q + e) : (T)0;
                }
                T vx[kU], vy[kU], vz[kU], wa[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int i = ii[u] < 0 ? 0 : ii[u];
                    load_pt_v<T>(d.pts, i, vx[u], vy[u], vz[u], wa[u]);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    if (ii[u] < 0) break;
                    const T an[4] = {vx[u] - pnx, vy[u] - pny, vz[u] - pnz, (T)1};
                    const T ak[4] = {vx[u] - pkx, vy[u] - pky, vz[u] - pkz, (T)1};
                    const T c = wa[u] * wq[u];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const T cr = c * an[r];
#pragma unroll
                        for (int s2 = 0; s2 < 4; ++s2) acc[4 * r + s2] += cr * ak[s2];
                    }
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
                for (int t = 0; t < 16; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
            }
            if (lane8 != 0 || !active) continue;
            // pair (n, k): block (n, k) gets -r w h_k^T on row 3,
            // h_k = r [(p_n - p_k)^T, 1]
            const int e = desc.w;
            const T r = d.e_r[e], w = alpha * d.wr[e];
            const T hk[4] = {r * (pnx - pkx), r * (pny - pky), r * (pnz - pkz), r};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[12 + cc] -= w * r * hk[cc];
            // pair (k, n): block (n, k) gets -r' w' h_n on column 3,
            // h_n = r' [(p_k - p_n)^T, 1]
            const int er = nk.z;
            const T r2 = d.e_r[er], w2 = alpha * d.wr[er];
            const T hn[4] = {r2 * (pkx - pnx), r2 * (pky - pny), r2 * (pkz - pnz), r2};
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[4 * a + 3] -= w2 * r2 * hn[a];
#pragma unroll
            for (int t = 0; t < 16; ++t) d.Kv[16 * b + t] = acc[t];
        }
    }
}


// ---------------------------------------------------------------------------
// Gradient of E (Eq. objective_func) at the evaluated iterate (Xeval), with
// the closest points fixed at their values there (piecewise-constant rho):
//   dE/dX_n = sum_i 2 w^a_i w_in [v_i - p_n; 1] (v_hat_i - u_i)^T
//           + 2 alpha sum_{pairs with n} w^r h D^T + 2 beta [(A_n - R_n)^T; 0]
// (the surrogate of Sec. 3.3.1 touches E with the same gradient). A group of
// 8 lanes owns one node and sums the contribution list of its diagonal
// block in a fixed order; deterministic.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) gradient_kernel(DevProblem<T> d, double* __restrict__ gX) {
    NrrState* st = d.st;
    const int lane8 = threadIdx.x & 7;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int P = d.P;
    const T alpha = (T)st->alpha, beta = (T)st->beta;
    const T* vh = d.vhat + (size_t)(st->vk ^ 1) * 3 * P;   // written by the evaluation
    const T* X = d.Xeval;
    for (int n0 = gwarp * 4; n0 < d.N; n0 += nwarps * 4) {
        const int n = min(n0 + ((threadIdx.x & 31) >> 3), d.N - 1);
        const bool active = (n0 + ((threadIdx.x & 31) >> 3)) < d.N;
        int bdg = d.bsr_ptr[n];
        while (d.bsr_col[bdg] != n) ++bdg;
        const T pnx = d.p[3 * n], pny = d.p[3 * n + 1], pnz = d.p[3 * n + 2];
        T g[12];
#pragma unroll
        for (int t = 0; t < 12; ++t) g[t] = 0;
        const int e_end = active ? d.ent_ptr[bdg + 1] : 0;
        for (int e = d.ent_ptr[bdg] + lane8; e < e_end; e += 8) {
            const int i = d.ent[e] >> 6;
            const T wn = d.ent_q[e];   // diagonal block: w_in
            const T c = (T)2 * d.wa[i] * wn;
            const T an[4] = {d.v[i] - pnx, d.v[P + i] - pny, d.v[2 * P + i] - pnz, (T)1};
            const T rx = vh[i] - d.u[i], ry = vh[P + i] - d.u[P + i], rz = vh[2 * P + i] - d.u[2 * P + i];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const T ca = c * an[a];
                g[3 * a + 0] += ca * rx;
                g[3 * a + 1] += ca * ry;
                g[3 * a + 2] += ca * rz;
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
            for (int t = 0; t < 12; ++t) g[t] += __shfl_xor_sync(0xffffffffu, g[t], o);
        }
        if (lane8 != 0 || !active) continue;
        // regularisation: pairs (n, j) with h_i = [0,0,0,-r] at X_n, and the
        // reverse pairs (j, n) with h_j = r [(p_j - p_n)^T, 1] at X_n
        const T* Xn = X + 12 * n;
        for (int e = d.adj_ptr[n]; e < d.adj_ptr[n + 1]; ++e) {
            for (int side = 0; side < 2; ++side) {
                const int ee = side == 0 ? e : d.e_rev[e];
                const int a_ = d.e_i[ee], b_ = d.e_j[ee];   // D_ab: a = first node, b = second
                const T r = d.e_r[ee];
                const T* Xa = X + 12 * a_;
                const T* Xb = X + 12 * b_;
                const T dx = d.p[3 * a_] - d.p[3 * b_];
                const T dy = d.p[3 * a_ + 1] - d.p[3 * b_ + 1];
                const T dz = d.p[3 * a_ + 2] - d.p[3 * b_ + 2];
                const T D[3] = {r * ((Xb[0] * dx + Xb[3] * dy + Xb[6] * dz - dx) + (Xb[9] - Xa[9])),
                                r * ((Xb[1] * dx + Xb[4] * dy + Xb[7] * dz - dy) + (Xb[10] - Xa[10])),
                                r * ((Xb[2] * dx + Xb[5] * dy + Xb[8] * dz - dz) + (Xb[11] - Xa[11]))};
                const T w2 = (T)2 * alpha * d.wr[ee];
                if (side == 0) {
                    // n is the first node of the pair: h at X_n = [0,0,0,-r]
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) g[9 + cc] -= w2 * r * D[cc];
                } else {
                    // n is the second node: h at X_n = r [(p_a - p_n)^T, 1]
                    const T h[4] = {r * dx, r * dy, r * dz, r};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) g[3 * a + cc] += w2 * h[a] * D[cc];
                }
            }
        }
        // rotation term: 2 beta (A_n - R_n)^T in rows 0..2
        const T* R = d.Rm + 9 * n;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) g[3 * a + cc] += (T)2 * beta * (Xn[3 * a + cc] - R[3 * cc + a]);
#pragma unroll
        for (int t = 0; t < 12; ++t) gX[12 * n + t] = (double)g[t];
    }
}

// dE/dv_i = 2 w^a_i (sum_j w_ij A_j)^T (v_hat_i - u_i), written in the
// caller's point order (order[internal] = caller index).
template <typename T>
__global__ void __launch_bounds__(kThreads) src_gradient_kernel(DevProblem<T> d, const int* __restrict__ order,
                                                                double* __restrict__ gv) {
    NrrState* st = d.st;
    const int P = d.P;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const T* vh = d.vhat + (size_t)(st->vk ^ 1) * 3 * P;
    const T rx = vh[i] - d.u[i], ry = vh[P + i] - d.u[P + i], rz = vh[2 * P + i] - d.u[2 * P + i];
    const T c = (T)2 * d.wa[i];
    T o[3] = {0, 0, 0};
    for (int s = d.infl_ptr[i]; s < d.infl_ptr[i + 1]; ++s) {
        const T* Xj = d.Xeval + 12 * d.infl_node[s];
        const T w = d.infl_w[s];
        // (A_j^T r): A_j[b][a] = Xj[3a + b], so (A^T r)_a = sum_b Xj[3a + b] r_b
#pragma unroll
        for (int a = 0; a < 3; ++a) o[a] += w * (Xj[3 * a] * rx + Xj[3 * a + 1] * ry + Xj[3 * a + 2] * rz);
    }
    const int ci = order[i];
    gv[3 * ci + 0] = (double)(c * o[0]);
    gv[3 * ci + 1] = (double)(c * o[1]);
    gv[3 * ci + 2] = (double)(c * o[2]);
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_energy(const DevProblem<T>& d, int mode, int grid, cudaStream_t s) {
    if (mode == NRR_MODE_EVAL) energy_kernel<T, NRR_MODE_EVAL><<<grid, kThreads, 0, s>>>(d);
    else energy_kernel<T, NRR_MODE_PASS><<<grid, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t nrr_launch_xterm(const DevProblem<T>& d, int mode, cudaStream_t s) {
    if (mode == NRR_MODE_EVAL) xterm_kernel<T, NRR_MODE_EVAL><<<d.n_xpart, kThreads, 0, s>>>(d);
    else xterm_kernel<T, NRR_MODE_PASS><<<d.n_xpart, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_xterm<float>(const DevProblem<float>&, int, cudaStream_t);
template cudaError_t nrr_launch_xterm<double>(const DevProblem<double>&, int, cudaStream_t);

template <typename T>
cudaError_t nrr_launch_assemble(const DevProblem<T>& d, int grid, cudaStream_t s) {
    assemble_kernel<T><<<grid, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_energy<float>(const DevProblem<float>&, int, int, cudaStream_t);
template cudaError_t nrr_launch_energy<double>(const DevProblem<double>&, int, int, cudaStream_t);
template cudaError_t nrr_launch_assemble<float>(const DevProblem<float>&, int, cudaStream_t);
template cudaError_t nrr_launch_assemble<double>(const DevProblem<double>&, int, cudaStream_t);

template <typename T>
cudaError_t nrr_launch_gradient(const DevProblem<T>& d, double* grad_X, double* grad_v, const int* order,
                                int grid, cudaStream_t s) {
    if (grad_X) gradient_kernel<T><<<grid, kThreads, 0, s>>>(d, grad_X);
    if (grad_v) src_gradient_kernel<T><<<(d.P + kThreads - 1) / kThreads, kThreads, 0, s>>>(d, order, grad_v);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_gradient<float>(const DevProblem<float>&, double*, double*, const int*, int, cudaStream_t);
template cudaError_t nrr_launch_gradient<double>(const DevProblem<double>&, double*, double*, const int*, int, cudaStream_t);
