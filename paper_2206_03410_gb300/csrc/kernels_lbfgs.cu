// Vector kernels of the preliminary version's solver (Sec. 3.3.4, the
// Remark on the preliminary version; Sec. 4.3): an inner L-BFGS that
// minimises the energy with the closest points held. The vectors have n =
// 12 N entries (the node transforms); they are small, so each step is one
// CTA of 1024 threads whose sums run in double in a fixed order (per-thread
// strided sums, then a shuffle tree and the 32 warps in order):
// deterministic. The line search's trial point and the updates of the
// iterate are grid-wide element-wise kernels.
#include "nrr_device.cuh"

namespace {

constexpr int kLb = 1024;

// sum over the CTA of one double per thread; valid in every thread
__device__ __forceinline__ double cta_sum(double x, double* sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < kLb / 32; ++k) s += sh[k];
    return s;
}

__device__ __forceinline__ double dot(int n, const double* a, const double* b, double* sh) {
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kLb) s += a[k] * b[k];
    return cta_sum(s, sh);
}

// d = -H g by the two-loop recursion (Nocedal and Wright, Algorithm 7.4):
// H0 = gamma I with gamma = s.y / y.y of the newest pair, or 1 / |g| without
// pairs. The pairs are visited newest to oldest, then oldest to newest.
__global__ void __launch_bounds__(kLb) lbfgs_dir_kernel(int n, const double* __restrict__ g, const double* S,
                                                        const double* Y, int mk, int head, int m, double* dvec,
                                                        double* scal) {
    __shared__ double sh[kLb / 32];
    __shared__ double s_alpha[NRR_AA_MMAX], s_rho[NRR_AA_MMAX];
    for (int k = threadIdx.x; k < n; k += kLb) dvec[k] = g[k];   // q = g (held in dvec)
    __syncthreads();
    const double gn = sqrt(dot(n, g, g, sh));
    for (int j = 0; j < mk; ++j) {
        const int slot = ((head - 1 - j) % m + m) % m;   // newest first
        const double* s = S + (size_t)slot * n;
        const double* y = Y + (size_t)slot * n;
        const double rho = 1.0 / dot(n, y, s, sh);
        const double a = rho * dot(n, s, dvec, sh);
        if (threadIdx.x == 0) { s_alpha[j] = a; s_rho[j] = rho; }
        for (int k = threadIdx.x; k < n; k += kLb) dvec[k] -= a * y[k];
        __syncthreads();
    }
    double gamma = 1.0 / gn;
    if (mk > 0) {
        const int slot = ((head - 1) % m + m) % m;
        const double* s = S + (size_t)slot * n;
        const double* y = Y + (size_t)slot * n;
        gamma = dot(n, s, y, sh) / dot(n, y, y, sh);
    }
    for (int k = threadIdx.x; k < n; k += kLb) dvec[k] *= gamma;
    __syncthreads();
    for (int j = mk - 1; j >= 0; --j) {   // oldest first
        const int slot = ((head - 1 - j) % m + m) % m;
        const double* s = S + (size_t)slot * n;
        const double* y = Y + (size_t)slot * n;
        const double b = s_rho[j] * dot(n, y, dvec, sh);
        const double a = s_alpha[j];
        for (int k = threadIdx.x; k < n; k += kLb) dvec[k] += (a - b) * s[k];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < n; k += kLb) dvec[k] = -dvec[k];
    __syncthreads();
    const double gd = dot(n, g, dvec, sh);
    if (threadIdx.x == 0) { scal[0] = gd; scal[1] = gn; }
}

template <typename T>
__global__ void lbfgs_axpy_kernel(int n, const T* __restrict__ Xk, double t, const double* __restrict__ dvec,
                                  T* __restrict__ Xout) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        Xout[k] = (T)((double)Xk[k] + t * dvec[k]);
}

template <typename T>
__global__ void __launch_bounds__(kLb) lbfgs_pair_kernel(int n, T* Xk, const T* __restrict__ Xt, double* g,
                                                         const double* __restrict__ gn, double* S, double* Y,
                                                         int slot, double* scal) {
    __shared__ double sh[kLb / 32];
    double* s = S + (size_t)slot * n;
    double* y = Y + (size_t)slot * n;
    double ys = 0.0, yy = 0.0, ss = 0.0, gg = 0.0;
    for (int k = threadIdx.x; k < n; k += kLb) {
        const double sk = (double)Xt[k] - (double)Xk[k];
        const double yk = gn[k] - g[k];
        s[k] = sk;
        y[k] = yk;
        ys += yk * sk;
        yy += yk * yk;
        ss += sk * sk;
        gg += gn[k] * gn[k];
        Xk[k] = Xt[k];
        g[k] = gn[k];
    }
    ys = cta_sum(ys, sh);
    yy = cta_sum(yy, sh);
    ss = cta_sum(ss, sh);
    gg = cta_sum(gg, sh);
    if (threadIdx.x == 0) { scal[2] = ys; scal[3] = sqrt(yy); scal[4] = sqrt(ss); scal[5] = sqrt(gg); }
}

// largest squared displacement, as the bits of a non-negative double (which
// order like the values) by an atomic max; scal[6] must start at 0
template <typename T>
__global__ void max_disp_kernel(int P, const T* __restrict__ a, const T* __restrict__ b, double* scal) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const double dx = (double)a[i] - (double)b[i];
        const double dy = (double)a[P + i] - (double)b[P + i];
        const double dz = (double)a[2 * P + i] - (double)b[2 * P + i];
        m = fmax(m, dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(scal + 6), (unsigned long long)__double_as_longlong(m));
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_lbfgs_dir(int n, const double* g, const double* S, const double* Y, int mk, int head, int m,
                                 double* dvec, double* scal, cudaStream_t s) {
    lbfgs_dir_kernel<<<1, kLb, 0, s>>>(n, g, S, Y, mk, head, m, dvec, scal);
    return cudaGetLastError();
}

template <typename T>
cudaError_t nrr_launch_lbfgs_axpy(int n, const T* Xk, double t, const double* dvec, T* Xout, cudaStream_t s) {
    lbfgs_axpy_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(n, Xk, t, dvec, Xout);
    return cudaGetLastError();
}

template <typename T>
cudaError_t nrr_launch_lbfgs_pair(int n, T* Xk, const T* Xt, double* g, const double* gn, double* S, double* Y,
                                  int slot, double* scal, cudaStream_t s) {
    lbfgs_pair_kernel<T><<<1, kLb, 0, s>>>(n, Xk, Xt, g, gn, S, Y, slot, scal);
    return cudaGetLastError();
}

template <typename T>
cudaError_t nrr_launch_max_disp(int P, const T* a, const T* b, double* scal, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scal + 6, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(1024, (P + 255) / 256);
    max_disp_kernel<T><<<grid, 256, 0, s>>>(P, a, b, scal);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_lbfgs_dir<float>(int, const double*, const double*, const double*, int, int, int,
                                                  double*, double*, cudaStream_t);
template cudaError_t nrr_launch_lbfgs_dir<double>(int, const double*, const double*, const double*, int, int, int,
                                                   double*, double*, cudaStream_t);
template cudaError_t nrr_launch_lbfgs_axpy<float>(int, const float*, double, const double*, float*, cudaStream_t);
template cudaError_t nrr_launch_lbfgs_axpy<double>(int, const double*, double, const double*, double*, cudaStream_t);
template cudaError_t nrr_launch_lbfgs_pair<float>(int, float*, const float*, double*, const double*, double*,
                                                   double*, int, double*, cudaStream_t);
template cudaError_t nrr_launch_lbfgs_pair<double>(int, double*, const double*, double*, const double*, double*,
                                                    double*, int, double*, cudaStream_t);
template cudaError_t nrr_launch_max_disp<float>(int, const float*, const float*, double*, cudaStream_t);
template cudaError_t nrr_launch_max_disp<double>(int, const double*, const double*, double*, cudaStream_t);
