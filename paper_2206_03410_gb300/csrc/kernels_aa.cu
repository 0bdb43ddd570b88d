// Anderson acceleration of the MM map (Sec. 3.3.4, Eq. AA_solution), after
// the solve of K X = B has left G = G(X^(k)) in d.G:
//   F^(k) = G^(k) - X^(k);  dF, dG = differences with the previous solve
//   theta = argmin |F^(k) - sum_j theta_j dF_j|^2 (+ ridge)
//   X^(k+1) = G^(k) - sum_j theta_j dG_j
// Two grid-wide kernels: aa_dots (differences, Gram row and right-hand side,
// then in its last CTA the FP64 Gram solve and the bookkeeping) and aa_mix.
// Products and per-warp sums in T, CTA and grid sums in double, fixed order.
#include "nrr_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kM = NRR_AA_MMAX;
constexpr int kGroups = kThreads / (2 * kM);
static_assert(2 * kM == 16 && kThreads >= kM * kM, "thread mapping of the grid sums");

template <typename T>
__global__ void __launch_bounds__(kThreads) aa_dots_kernel(DevProblem<T> d) {
    __shared__ double sh[kThreads / 32][2 * kM];
    __shared__ double gsum[kGroups][2 * kM];
    __shared__ double tot[2 * kM];
    __shared__ double s_gram[kM * kM];
    __shared__ int s_last;
    NrrState* st = d.st;
    if (st->done || st->skip || st->status != 0) return;
    const int aa_m = d.aa_m;
    const bool insert = st->n_solves_stage > 0 && aa_m > 0;
    const int slot = st->aa_head;
    const int mk = insert ? min(st->aa_count + 1, aa_m) : 0;
    const size_t n12 = (size_t)d.N * 12;
    T acc[2 * kM];
#pragma unroll
    for (int j = 0; j < 2 * kM; ++j) acc[j] = 0;
    if (mk > 0) {
        for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n12; e += (size_t)gridDim.x * blockDim.x) {
            const T g = d.G[e];
            const T f = g - d.X[e];
            const T dfn = f - d.Fprev[e];
            T dfo[kM];
#pragma unroll
            for (int b = 0; b < kM; ++b) dfo[b] = (b < mk && b != slot) ? d.dF[b * n12 + e] : T(0);
            d.dF[slot * n12 + e] = dfn;
            d.dG[slot * n12 + e] = g - d.Gprev[e];
#pragma unroll
            for (int b = 0; b < kM; ++b) {
                const T dfb = (b == slot) ? dfn : dfo[b];
                acc[b] += dfb * dfn;          // Gram row of the new slot
                acc[kM + b] += dfb * f;       // right-hand side
            }
        }
    }
    // CTA sums: shuffle tree per warp in T, then the warps in double
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = 0; j < 2 * kM; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 2 * kM; ++j) sh[w][j] = (double)acc[j];
    }
    __syncthreads();
    if (threadIdx.x < 2 * kM) {
        double s = 0.0;
        for (int ww = 0; ww < kThreads / 32; ++ww) s += sh[ww][threadIdx.x];
        d.partials[(size_t)blockIdx.x * NRR_PARTIAL_STRIDE + threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&st->cnt_energy, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // grid sums in the last CTA: kGroups groups of 16 threads take every
    // kGroups-th CTA's partials, then a fixed-order sum over the groups
    {
        const int j = threadIdx.x & 15, grp = threadIdx.x >> 4;
        double s = 0.0;
        for (unsigned b = grp; b < gridDim.x; b += kGroups)
            s += __ldcg(d.partials + (size_t)b * NRR_PARTIAL_STRIDE + j);
        gsum[grp][j] = s;
        if (threadIdx.x < kM * kM) s_gram[threadIdx.x] = st->gram[threadIdx.x];
        __syncthreads();
        if (threadIdx.x < 2 * kM) {
            double t = 0.0;
            for (int g2 = 0; g2 < kGroups; ++g2) t += gsum[g2][threadIdx.x];
            tot[threadIdx.x] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    st->cnt_energy = 0;
    double th[kM];
    nrr_aa_finish(st, s_gram, tot, mk, slot, insert, aa_m, th, true);
}

// X^(k+1) = G - sum_b theta_b dG_b; F and G kept for the next differences.
template <typename T>
__global__ void __launch_bounds__(kThreads) aa_mix_kernel(DevProblem<T> d) {
    NrrState* st = d.st;
    // the same decision as the dots kernel (which changes none of the three)
    if (st->done || st->skip || st->status != 0) return;
    const int mk = st->aa_mk;
    T th[kM];
#pragma unroll
    for (int b = 0; b < kM; ++b) th[b] = (T)st->theta[b];
    const size_t n12 = (size_t)d.N * 12;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n12; e += (size_t)gridDim.x * blockDim.x) {
        const T g = d.G[e];
        const T f = g - d.X[e];
        T xn = g;
#pragma unroll
        for (int b = 0; b < kM; ++b)
            if (b < mk) xn -= th[b] * d.dG[b * n12 + e];
        d.X[e] = xn;
        d.Fprev[e] = f;
        d.Gprev[e] = g;
    }
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_aa(const DevProblem<T>& d, int grid, cudaStream_t s) {
    aa_dots_kernel<T><<<grid, kThreads, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    aa_mix_kernel<T><<<grid, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_aa<float>(const DevProblem<float>&, int, cudaStream_t);
template cudaError_t nrr_launch_aa<double>(const DevProblem<double>&, int, cudaStream_t);
