// Solve of the surrogate normal equations K X = B (Eq. surr_solution) by
// block-Jacobi preconditioned conjugate gradients, followed by the Anderson
// mix of Sec. 3.3.4 (Eq. AA_solution), in one persistent kernel.
//
// K is the same 4N x 4N matrix for the three columns of X, so the kernel
// runs three CG recurrences (one per column) that share every SpMV and every
// grid-wide reduction. A thread owns one (node, column) pair: 4 unknowns.
// Each CTA owns a contiguous range of nodes. Per CG iteration there are two
// grid-wide reductions, and the SpMV is applied to z (whose values are made
// visible by the first reduction's barrier) using q = K z + beta q, so no
// third barrier is needed. Reductions are deterministic: each CTA writes its
// partial sums, and after the barrier every CTA adds all partials in the same
// fixed order. The barrier is bounded: after about two seconds of waiting it
// records NRR_E_TIMEOUT in the state and the kernel returns.
#include "nrr_device.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kMaxRed = 2 * NRR_AA_MMAX;   // values per reduction
constexpr long long kSpinLimit = 4000000000LL;   // clock64 cycles

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct Barrier {
    NrrState* st;
    unsigned gen;
    unsigned nblocks;
    int* s_flag;

    // Returns false if the wait timed out or another CTA reported a failure.
    __device__ bool sync() {
        __syncthreads();
        if (threadIdx.x == 0) {
            int fail = 0;
            __threadfence();
            const unsigned arrived = atomicAdd(&st->bar_count, 1u);
            if (arrived == nblocks - 1) {
                atomicExch(&st->bar_count, 0u);
                __threadfence();
                atomicExch(&st->bar_gen, gen + 1);
            } else {
                const long long t0 = clock64();
                while (ld_acquire(&st->bar_gen) == gen) {
                    if (clock64() - t0 > kSpinLimit) {
                        atomicExch(&st->status, (int)NRR_E_TIMEOUT);
                        fail = 1;
                        break;
                    }
                }
            }
            __threadfence();
            gen += 1;
            *s_flag = fail || (*(volatile int*)&st->status != 0);
        }
        __syncthreads();
        return *s_flag == 0;
    }
};

struct Red {
    double* partials;
    int buf;
    // Sums K per-thread values over the whole grid; out[] valid in all threads.
    // Every CTA adds the partials of all CTAs in the same fixed order, so the
    // result is identical everywhere and deterministic.
    template <int K>
    __device__ bool run(Barrier& bar, const double (&v)[K], double* s_tmp, double (&out)[K]) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double x = v[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) s_tmp[w * kMaxRed + j] = x;
        }
        __syncthreads();
        if (threadIdx.x < K) {
            double s = 0.0;
#pragma unroll
            for (int ww = 0; ww < kThreads / 32; ++ww) s += s_tmp[ww * kMaxRed + threadIdx.x];
            partials[((size_t)buf * gridDim.x + blockIdx.x) * NRR_PARTIAL_STRIDE + threadIdx.x] = s;
        }
        if (!bar.sync()) return false;
        if (w == 0) {
            double s[K];
#pragma unroll
            for (int j = 0; j < K; ++j) s[j] = 0.0;
            for (unsigned b = lane; b < gridDim.x; b += 32) {
                const double* src = partials + ((size_t)buf * gridDim.x + b) * NRR_PARTIAL_STRIDE;
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] += __ldcg(src + j);
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
            }
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < K; ++j) s_tmp[j] = s[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K; ++j) out[j] = s_tmp[j];
        __syncthreads();
        buf ^= 1;
        return true;
    }
};

// 4x4 SPD inverse by Cholesky, in double. Returns false if not positive definite.
__device__ bool spd_inverse4(const double A[16], double Inv[16]) {
    double L[16] = {0};
    for (int j = 0; j < 4; ++j) {
        double s = A[4 * j + j];
        for (int k = 0; k < j; ++k) s -= L[4 * j + k] * L[4 * j + k];
        if (!(s > 0)) return false;
        L[4 * j + j] = sqrt(s);
        for (int i = j + 1; i < 4; ++i) {
            double t = A[4 * i + j];
            for (int k = 0; k < j; ++k) t -= L[4 * i + k] * L[4 * j + k];
            L[4 * i + j] = t / L[4 * j + j];
        }
    }
    // columns of inv(L), then Inv = inv(L)^T inv(L)
    double Li[16] = {0};
    for (int c = 0; c < 4; ++c) {
        for (int i = 0; i < 4; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= L[4 * i + k] * Li[4 * k + c];
            Li[4 * i + c] = t / L[4 * i + i];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += Li[4 * k + i] * Li[4 * k + j];
            Inv[4 * i + j] = s;
        }
    return true;
}

// y[a] = sum over blocks of row n of K[b][a][t] * vec[col(b)][t][c], a = 0..3
template <typename T, bool CG_LOAD>
__device__ __forceinline__ void spmv_pair(const DevProblem<T>& d, const T* vec, int n, int c, T y[4]) {
    y[0] = y[1] = y[2] = y[3] = 0;
#pragma unroll 4
    for (int b = d.bsr_ptr[n], be = d.bsr_ptr[n + 1]; b < be; ++b) {
        const int k = d.bsr_col[b];
        const T* Kb = d.Kv + 16 * b;
        T x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) x[t] = CG_LOAD ? __ldcg(vec + 12 * k + 3 * t + c) : vec[12 * k + 3 * t + c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
            y[a] += Kb[4 * a + 0] * x[0] + Kb[4 * a + 1] * x[1] + Kb[4 * a + 2] * x[2] + Kb[4 * a + 3] * x[3];
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) solve_kernel(DevProblem<T> d) {
    __shared__ double s_tmp[(kThreads / 32) * kMaxRed];
    __shared__ int s_flag;
    __shared__ double s_theta[NRR_AA_MMAX];
    NrrState* st = d.st;
    if (st->done || st->skip) return;
    const int N = d.N;
    const int G = gridDim.x;
    const int per = (N + G - 1) / G;
    const int n0 = min(N, (int)blockIdx.x * per), n1 = min(N, n0 + per);
    const int npairs = (n1 - n0) * 3;
    Barrier bar{st, *(volatile unsigned*)&st->bar_gen, (unsigned)G, &s_flag};
    Red red{d.partials, 0};
    const int first_solve = st->n_solves_stage == 0;
    const int aa_m = d.aa_m;
    const int aa_count = st->aa_count, aa_head = st->aa_head;
    const double tol = (double)d.pcg_tol;

    // block-Jacobi preconditioner: inverse of each node's diagonal block
    for (int n = n0 + (int)threadIdx.x; n < n1; n += kThreads) {
        int bd = d.bsr_ptr[n];
        while (d.bsr_col[bd] != n) ++bd;
        double A[16], I[16];
        for (int t = 0; t < 16; ++t) A[t] = (double)d.Kv[16 * bd + t];
        if (!spd_inverse4(A, I)) {
            // fall back to the inverse diagonal
            for (int t = 0; t < 16; ++t) I[t] = 0.0;
            for (int t = 0; t < 4; ++t) I[5 * t] = A[5 * t] > 0 ? 1.0 / A[5 * t] : 1.0;
        }
        for (int t = 0; t < 16; ++t) d.Minv[16 * n + t] = (T)I[t];
    }
    __syncthreads();

    // initial residual with the warm start X^(k)
    double acc[9];
    double sums[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) acc[j] = 0.0;
    for (int idx = threadIdx.x; idx < npairs; idx += kThreads) {
        const int n = n0 + idx / 3, c = idx % 3;
        T y[4];
        spmv_pair<T, false>(d, d.X, n, c, y);
        T rr[4];
        for (int a = 0; a < 4; ++a) {
            const T b = d.Bv[12 * n + 3 * a + c];
            rr[a] = b - y[a];
            d.r[12 * n + 3 * a + c] = rr[a];
            d.G[12 * n + 3 * a + c] = d.X[12 * n + 3 * a + c];
            acc[6 + c] += (double)b * (double)b;
        }
        const T* Mi = d.Minv + 16 * n;
        for (int a = 0; a < 4; ++a) {
            const T zz = Mi[4 * a] * rr[0] + Mi[4 * a + 1] * rr[1] + Mi[4 * a + 2] * rr[2] + Mi[4 * a + 3] * rr[3];
            d.z[12 * n + 3 * a + c] = zz;
            acc[c] += (double)rr[a] * (double)zz;
            acc[3 + c] += (double)rr[a] * (double)rr[a];
        }
    }
    if (!red.run<9>(bar, acc, s_tmp, sums)) return;
    double rz[3] = {sums[0], sums[1], sums[2]};
    double bb[3] = {sums[6], sums[7], sums[8]};
    double rel = 0.0;
    for (int c = 0; c < 3; ++c) rel = fmax(rel, sqrt(sums[3 + c] / fmax(bb[c], 1e-300)));
    int it = 0;
    double beta_c[3] = {0, 0, 0};
    while (rel > tol && it < d.pcg_max) {
        // w = K z; p = z + beta p; q = w + beta q
        double a3[3] = {0.0, 0.0, 0.0}, s3[3];
        for (int idx = threadIdx.x; idx < npairs; idx += kThreads) {
            const int n = n0 + idx / 3, c = idx % 3;
            T w[4];
            spmv_pair<T, true>(d, d.z, n, c, w);
            const T bt = (T)beta_c[c];
            for (int a = 0; a < 4; ++a) {
                const int e = 12 * n + 3 * a + c;
                const T zz = d.z[e];
                const T pn = (it == 0) ? zz : zz + bt * d.pv[e];
                const T qn = (it == 0) ? w[a] : w[a] + bt * d.q[e];
                d.pv[e] = pn;
                d.q[e] = qn;
                a3[c] += (double)pn * (double)qn;
            }
        }
        if (!red.run<3>(bar, a3, s_tmp, s3)) return;
        double al[3];
        for (int c = 0; c < 3; ++c) al[c] = s3[c] != 0.0 ? rz[c] / s3[c] : 0.0;
        double a6[6] = {0, 0, 0, 0, 0, 0}, s6[6];
        for (int idx = threadIdx.x; idx < npairs; idx += kThreads) {
            const int n = n0 + idx / 3, c = idx % 3;
            const T a_ = (T)al[c];
            T rr[4];
            for (int a = 0; a < 4; ++a) {
                const int e = 12 * n + 3 * a + c;
                d.G[e] += a_ * d.pv[e];
                rr[a] = d.r[e] - a_ * d.q[e];
                d.r[e] = rr[a];
            }
            const T* Mi = d.Minv + 16 * n;
            for (int a = 0; a < 4; ++a) {
                const T zz = Mi[4 * a] * rr[0] + Mi[4 * a + 1] * rr[1] + Mi[4 * a + 2] * rr[2] + Mi[4 * a + 3] * rr[3];
                d.z[12 * n + 3 * a + c] = zz;
                a6[c] += (double)rr[a] * (double)zz;
                a6[3 + c] += (double)rr[a] * (double)rr[a];
            }
        }
        if (!red.run<6>(bar, a6, s_tmp, s6)) return;
        ++it;
        rel = 0.0;
        for (int c = 0; c < 3; ++c) {
            beta_c[c] = rz[c] != 0.0 ? s6[c] / rz[c] : 0.0;
            rz[c] = s6[c];
            rel = fmax(rel, sqrt(s6[3 + c] / fmax(bb[c], 1e-300)));
        }
    }

    // ---- Anderson acceleration (Eq. AA_solution) ---------------------------
    const bool insert = !first_solve && aa_m > 0;
    const int slot = aa_head;
    const int mk = insert ? min(aa_count + 1, aa_m) : 0;
    const size_t n12 = (size_t)N * 12;
    if (mk > 0) {
        double aa[kMaxRed], sa[kMaxRed];
#pragma unroll
        for (int j = 0; j < kMaxRed; ++j) aa[j] = 0.0;
        for (int idx = threadIdx.x; idx < npairs; idx += kThreads) {
            const int n = n0 + idx / 3, c = idx % 3;
            for (int a = 0; a < 4; ++a) {
                const int e = 12 * n + 3 * a + c;
                const T g = d.G[e];
                const T f = g - d.X[e];
                const T dfn = f - d.Fprev[e];
                d.dF[slot * n12 + e] = dfn;
                d.dG[slot * n12 + e] = g - d.Gprev[e];
                for (int b = 0; b < mk; ++b) {
                    const T dfb = (b == slot) ? dfn : d.dF[b * n12 + e];
                    aa[b] += (double)dfb * (double)dfn;                 // Gram row of the new slot
                    aa[NRR_AA_MMAX + b] += (double)dfb * (double)f;     // right-hand side
                }
            }
        }
        if (!red.run<kMaxRed>(bar, aa, s_tmp, sa)) return;
        if (threadIdx.x == 0) {
            double Gm[NRR_AA_MMAX * NRR_AA_MMAX], rhs[NRR_AA_MMAX], th[NRR_AA_MMAX];
            double tr = 0.0;
            for (int a = 0; a < mk; ++a) {
                for (int b = 0; b < mk; ++b) {
                    double v;
                    if (a == slot) v = sa[b];
                    else if (b == slot) v = sa[a];
                    else v = st->gram[a * NRR_AA_MMAX + b];
                    Gm[a * NRR_AA_MMAX + b] = v;
                }
                rhs[a] = sa[NRR_AA_MMAX + a];
                tr += Gm[a * NRR_AA_MMAX + a];
            }
            const double lam = 1e-10 * tr / mk;
            for (int a = 0; a < mk; ++a) Gm[a * NRR_AA_MMAX + a] += lam;
            // Cholesky solve in place
            bool ok = true;
            for (int j = 0; j < mk && ok; ++j) {
                double s = Gm[j * NRR_AA_MMAX + j];
                for (int k = 0; k < j; ++k) s -= Gm[j * NRR_AA_MMAX + k] * Gm[j * NRR_AA_MMAX + k];
                if (!(s > 0)) { ok = false; break; }
                const double l = sqrt(s);
                Gm[j * NRR_AA_MMAX + j] = l;
                for (int i = j + 1; i < mk; ++i) {
                    double t = Gm[i * NRR_AA_MMAX + j];
                    for (int k = 0; k < j; ++k) t -= Gm[i * NRR_AA_MMAX + k] * Gm[j * NRR_AA_MMAX + k];
                    Gm[i * NRR_AA_MMAX + j] = t / l;
                }
            }
            double nrm = 0.0;
            if (ok) {
                for (int i = 0; i < mk; ++i) {
                    double t = rhs[i];
                    for (int k = 0; k < i; ++k) t -= Gm[i * NRR_AA_MMAX + k] * th[k];
                    th[i] = t / Gm[i * NRR_AA_MMAX + i];
                }
                for (int i = mk - 1; i >= 0; --i) {
                    double t = th[i];
                    for (int k = i + 1; k < mk; ++k) t -= Gm[k * NRR_AA_MMAX + i] * th[k];
                    th[i] = t / Gm[i * NRR_AA_MMAX + i];
                }
                for (int i = 0; i < mk; ++i) nrm += th[i] * th[i];
                ok = isfinite(nrm) && sqrt(nrm) <= 1e4;
            }
            for (int i = 0; i < NRR_AA_MMAX; ++i) s_theta[i] = (ok && i < mk) ? th[i] : 0.0;
            if (blockIdx.x == 0) {
                for (int b = 0; b < mk; ++b) {
                    st->gram[slot * NRR_AA_MMAX + b] = sa[b];
                    st->gram[b * NRR_AA_MMAX + slot] = sa[b];
                }
                st->aa_mk = ok ? mk : 0;
                for (int i = 0; i < NRR_AA_MMAX; ++i) st->theta[i] = s_theta[i];
            }
        }
        __syncthreads();
    } else if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->aa_mk = 0;
    }
    // X^(k+1) = G - sum theta_b dG_b; keep F and G for the next differences
    for (int idx = threadIdx.x; idx < npairs; idx += kThreads) {
        const int n = n0 + idx / 3, c = idx % 3;
        for (int a = 0; a < 4; ++a) {
            const int e = 12 * n + 3 * a + c;
            const T g = d.G[e];
            const T f = g - d.X[e];
            T xn = g;
            for (int b = 0; b < mk; ++b) xn -= (T)s_theta[b] * d.dG[b * n12 + e];
            d.X[e] = xn;
            d.Fprev[e] = f;
            d.Gprev[e] = g;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->aa_count = mk;
        st->aa_head = insert ? (aa_head + 1) % aa_m : aa_head;
        st->n_solves_stage += 1;
        st->n_solves += 1;
        st->pending_stop = 1;
        st->solved = 1;
        st->pcg_iters = it;
        st->pcg_res = rel;
    }
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_solve(const DevProblem<T>& d, int grid, cudaStream_t s, bool cooperative) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cooperative ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, solve_kernel<T>, d);
}

int nrr_solve_threads() { return kThreads; }

template <typename T>
int nrr_solve_max_blocks_per_sm() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<T>, kThreads, 0);
    return nb;
}

template cudaError_t nrr_launch_solve<float>(const DevProblem<float>&, int, cudaStream_t, bool);
template cudaError_t nrr_launch_solve<double>(const DevProblem<double>&, int, cudaStream_t, bool);
template int nrr_solve_max_blocks_per_sm<float>();
template int nrr_solve_max_blocks_per_sm<double>();
