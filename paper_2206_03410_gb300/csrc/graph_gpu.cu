// Algorithm 1 (Sec. 3.1) on the GPU, with Euclidean distances in place of
// geodesics (the point-cloud reading: the ball B(v_j) is {q : |v_j - q| < R},
// strict), followed by the weights of Eq. (weight_data), the edges of the
// capped influence sets and r_ij of Sec. 3.2. It builds the same graph as the
// host code (graph_build.cpp) and the FP64 oracle: every distance is formed
// in double as dx*dx + dy*dy + dz*dz with separate roundings (no fused
// multiply-adds), and so is every projection on the PCA axis.
//
// Steps (all on the device; the host only sequences them and reads the
// final arrays back):
//  1. PCA: mean and covariance by fixed-order reductions, the 3x3 symmetric
//     eigenproblem by cyclic Jacobi in one thread; the axis of the largest
//     eigenvalue with its largest-magnitude entry made positive.
//  2. The visiting order: projections sorted by a stable radix sort (ties
//     keep the lower index).
//  3. The greedy sampling, node by node as Algorithm 1 states it: the next
//     point in visiting order that no node covers becomes a node and covers
//     every point strictly within R of it. One CTA runs it: its threads share
//     the forward scan for the next uncovered point and the covering of each
//     ball, so the sequential steps are the N node creations, not the P
//     points.
//  4. Influence sets (the K nearest nodes within R, ties to the lower node
//     id), weights, the edges between the nodes of each set (sorted, unique)
//     and r_ij.
// Neighbours come from a uniform grid of cell size R (points sorted by cell
// key; cells found through a dense table of each cell's first entry, or by
// binary search of the sorted keys when the grid has too many cells).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <chrono>
#include <string>
#include <vector>

#include "nrr_device.cuh"

namespace {

constexpr int kT = 256;
constexpr int kBadCap = 4096;   // l-bar: points searched by brute force at most
constexpr int kRed = 256;   // CTAs of the fixed-order reductions

int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kT - 1) / kT, 4096)); }

__device__ __forceinline__ double sqd(double ax, double ay, double az, double bx, double by, double bz) {
    const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// order-preserving map of a double to an unsigned key (-0 taken as +0)
__device__ __forceinline__ unsigned long long dkey(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x + 0.0);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Float prefilter of the nearest-neighbour searches. The source
// points are floats, so the float copies of the coordinates are exact, and
// a squared distance formed in float (round to nearest, no contraction)
// is within a relative 4e-7 of the exact one, except below 1e-36 where
// subnormal rounding adds an absolute error. So if t is the kk-th smallest
// float squared distance of a point's candidates, each of its kk nearest
// (by the double distance) has a float squared distance of at most
// t (1 + 1e-5) + 1e-36: only those candidates are measured in double.
__device__ __forceinline__ float sqdf(float4 a, float4 b) {
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}
__device__ __forceinline__ float knn_filter(float t) { return __fadd_ru(__fmul_ru(t, 1.00001f), 1e-36f); }
// the K smallest values seen, ascending (registers: compile-time indices)
template <int K, typename V>
__device__ __forceinline__ void topk_insert(V (&best)[K], V d2) {
    if (d2 < best[K - 1]) {
        best[K - 1] = d2;
#pragma unroll
        for (int p = K - 1; p > 0; --p)
            if (best[p] < best[p - 1]) {
                const V t = best[p];
                best[p] = best[p - 1];
                best[p - 1] = t;
            }
    }
}

__global__ void to_double_kernel(const float* __restrict__ src, double* __restrict__ V, int64_t n3) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
        V[k] = (double)src[k];
}

// per-CTA partial sums over a contiguous range of points (thread-strided,
// then a fixed shuffle tree and the warps in order) of: mode 0 the
// coordinates and their min/max; mode 1 the products (v - mu)(v - mu)^T
__global__ void __launch_bounds__(kT) moments_kernel(const double* __restrict__ V, int64_t P, int mode,
                                                     const double* __restrict__ mu, double* __restrict__ part) {
    __shared__ double sh[kT / 32][12];
    const int64_t per = (P + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = blockIdx.x * per, i1 = min(P, i0 + per);
    double a[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) a[k] = 0.0;
    if (mode == 0) {
        for (int k = 3; k < 6; ++k) a[k] = INFINITY;
        for (int k = 6; k < 9; ++k) a[k] = -INFINITY;
    }
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kT) {
        const double x = V[3 * i], y = V[3 * i + 1], z = V[3 * i + 2];
        if (mode == 0) {
            a[0] += x; a[1] += y; a[2] += z;
            a[3] = fmin(a[3], x); a[4] = fmin(a[4], y); a[5] = fmin(a[5], z);
            a[6] = fmax(a[6], x); a[7] = fmax(a[7], y); a[8] = fmax(a[8], z);
        } else {
            const double c[3] = {x - mu[0], y - mu[1], z - mu[2]};
            a[0] += c[0] * c[0]; a[1] += c[0] * c[1]; a[2] += c[0] * c[2];
            a[3] += c[1] * c[1]; a[4] += c[1] * c[2]; a[5] += c[2] * c[2];
        }
    }
    const int nv = mode == 0 ? 9 : 6;
    for (int k = 0; k < nv; ++k) {
        double v = a[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, v, o);
            v = (mode == 0 && k >= 3) ? (k < 6 ? fmin(v, u) : fmax(v, u)) : v + u;
        }
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < kT / 32; ++w)
            v = (mode == 0 && k >= 3) ? (k < 6 ? fmin(v, sh[w][k]) : fmax(v, sh[w][k])) : v + sh[w][k];
        part[blockIdx.x * 12 + k] = v;
    }
}

// cyclic Jacobi for a symmetric 3x3 matrix (Golub and Van Loan, Sec. 8.5):
// eigenvalues in ev, eigenvectors as the columns of Q
__device__ void jacobi3(const double Ain[9], double ev[3], double Q[9]) {
    double A[9];
    for (int i = 0; i < 9; ++i) { A[i] = Ain[i]; Q[i] = (i % 4 == 0) ? 1.0 : 0.0; }
    for (int sweep = 0; sweep < 50; ++sweep) {
        // off-diagonal mass below (1e-18 of the diagonal)^2: further
        // rotations move no eigenvector by a unit in the last place
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        if (off <= 1e-36 * (A[0] * A[0] + A[4] * A[4] + A[8] * A[8])) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
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
    ev[0] = A[0]; ev[1] = A[4]; ev[2] = A[8];
}

// single thread: the CTA partials added in order; mode 0 leaves the mean
// (sc[0..2]) and the bounding box (sc[3..8]); mode 1 the covariance, its
// eigen-decomposition and the axis (sc[9..11])
__global__ void finish_moments_kernel(const double* __restrict__ part, int nb, int64_t P, int mode, double* sc) {
    if (mode == 0) {
        double a[9] = {0, 0, 0, INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 9; ++k)
                a[k] = k < 3 ? a[k] + part[12 * b + k] : (k < 6 ? fmin(a[k], part[12 * b + k]) : fmax(a[k], part[12 * b + k]));
        for (int k = 0; k < 3; ++k) sc[k] = a[k] / (double)P;
        for (int k = 3; k < 9; ++k) sc[k] = a[k];
        return;
    }
    double s6[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 6; ++k) s6[k] += part[12 * b + k];
    double C[9] = {s6[0], s6[1], s6[2], s6[1], s6[3], s6[4], s6[2], s6[4], s6[5]};
    for (int k = 0; k < 9; ++k) C[k] /= (double)P;
    double ev[3], Q[9];
    jacobi3(C, ev, Q);
    int top = 0;
    for (int i = 1; i < 3; ++i) if (ev[i] > ev[top]) top = i;
    double ax[3] = {Q[top], Q[3 + top], Q[6 + top]};
    int big = 0;
    for (int i = 1; i < 3; ++i) if (fabs(ax[i]) > fabs(ax[big])) big = i;
    if (ax[big] < 0) for (int i = 0; i < 3; ++i) ax[i] = -ax[i];
    for (int i = 0; i < 3; ++i) sc[9 + i] = ax[i];
}

// projections on the axis as sort keys; grid cell keys of the points
__global__ void keys_kernel(const double* __restrict__ V, int64_t P, const double* __restrict__ sc, double h,
                            long long d1, long long d2, unsigned long long* __restrict__ pkey,
                            unsigned long long* __restrict__ ckey, int* __restrict__ idx) {
    const double a0 = sc[9], a1 = sc[10], a2 = sc[11];
    const double lo[3] = {sc[3], sc[4], sc[5]};
    const long long dims[3] = {0, d1, d2};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = V[3 * i], y = V[3 * i + 1], z = V[3 * i + 2];
        pkey[i] = dkey(__dadd_rn(__dadd_rn(__dmul_rn(x, a0), __dmul_rn(y, a1)), __dmul_rn(z, a2)));
        long long c[3];
        const double p[3] = {x, y, z};
        for (int d = 0; d < 3; ++d) {
            long long v = (long long)floor((p[d] - lo[d]) / h);
            const long long dm = d == 0 ? (long long)sc[12] : dims[d];
            c[d] = v < 0 ? 0 : (v > dm - 1 ? dm - 1 : v);
        }
        ckey[i] = (unsigned long long)((c[0] * d1 + c[1]) * d2 + c[2]);
        idx[i] = (int)i;
    }
}

// the grid's point coordinates in cell order
__global__ void grid_data_kernel(int64_t P, const int* __restrict__ gitem, const double* __restrict__ V,
                                 double* __restrict__ gxyz, float4* __restrict__ gf) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < P; s += (int64_t)gridDim.x * blockDim.x) {
        const int i = gitem[s];
        gxyz[3 * s] = V[3 * (int64_t)i];
        gxyz[3 * s + 1] = V[3 * (int64_t)i + 1];
        gxyz[3 * s + 2] = V[3 * (int64_t)i + 2];
        gf[s] = make_float4((float)V[3 * (int64_t)i], (float)V[3 * (int64_t)i + 1], (float)V[3 * (int64_t)i + 2], 0.f);
    }
}

// [first, last) of the sorted keys equal to k
__device__ __forceinline__ void cell_range(const unsigned long long* keys, int n, unsigned long long k, int* s0,
                                           int* s1) {
    int lo = 0, hi = n;
    while (lo < hi) { const int m = (lo + hi) >> 1; if (keys[m] < k) lo = m + 1; else hi = m; }
    *s0 = lo;
    hi = n;
    while (lo < hi) { const int m = (lo + hi) >> 1; if (keys[m] <= k) lo = m + 1; else hi = m; }
    *s1 = lo;
}

struct GridView {
    const unsigned long long* keys;   // sorted cell keys [n]
    const double* xyz;                // coordinates in that order [n][3]
    int n;
    double lo[3];
    double h;
    long long dims[3];
    const int* cstart;                // [cells + 1]: first entry of each cell key, or NULL (binary search)
    __device__ __forceinline__ void range(unsigned long long k, int* s0, int* s1) const {
        if (cstart) { *s0 = cstart[k]; *s1 = cstart[k + 1]; }
        else cell_range(keys, n, k, s0, s1);
    }
    __device__ void cell(double x, double y, double z, long long c[3]) const {
        const double p[3] = {x, y, z};
        for (int d = 0; d < 3; ++d) {
            long long v = (long long)floor((p[d] - lo[d]) / h);
            c[d] = v < 0 ? 0 : (v > dims[d] - 1 ? dims[d] - 1 : v);
        }
    }
};

// first entry of every cell key in the sorted keys (a dense table over all
// cells of the grid)
__global__ void cell_start_kernel(const unsigned long long* __restrict__ keys, int n, long long cells,
                                  int* __restrict__ cstart) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k <= cells; k += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (keys[m] < (unsigned long long)k) lo = m + 1; else hi = m; }
        cstart[k] = lo;
    }
}

// l-bar (the mean distance of every point to its kk = 6 nearest others) on
// the grid of cell size h = R: per point the kk smallest squared distances
// among the points of its 27 cells (ascending; a float pass, then the
// double distances of the candidates the filter keeps), certified when the
// kk-th is at most h^2 (every point outside the 27 cells is at least h
// away); the sum of their square roots in ascending order, as the host
// computes it. Uncertified points are listed (at most bad_cap; beyond that
// the host computes l-bar itself) for spacing_fallback_kernel.
template <int KK>
__global__ void spacing_kernel(GridView g, const float4* __restrict__ gf, const int* __restrict__ gitem,
                               const double* __restrict__ V, int P, double* __restrict__ per_point,
                               int* __restrict__ n_bad, int* __restrict__ bad, int bad_cap) {
    // points in grid-cell order (slot sl holds point gitem[sl]): the lanes
    // of a warp share their cells, so their candidate loads coincide
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < P; sl += gridDim.x * blockDim.x) {
        const int i = gitem[sl];
        const double x = g.xyz[3 * (int64_t)sl], y = g.xyz[3 * (int64_t)sl + 1], z = g.xyz[3 * (int64_t)sl + 2];
        const float4 pf = gf[sl];
        long long c[3];
        g.cell(x, y, z, c);
        int rs0[27], rs1[27];
        int nc = 0;
        for (long long a = c[0] - 1; a <= c[0] + 1; ++a) {
            for (long long b = c[1] - 1; b <= c[1] + 1; ++b) {
                for (long long d = c[2] - 1; d <= c[2] + 1; ++d) {
                    if (a < 0 || a >= g.dims[0] || b < 0 || b >= g.dims[1] || d < 0 || d >= g.dims[2]) continue;
                    g.range((unsigned long long)((a * g.dims[1] + b) * g.dims[2] + d), &rs0[nc], &rs1[nc]);
                    ++nc;
                }
            }
        }
        float bf[KK];
#pragma unroll
        for (int t = 0; t < KK; ++t) bf[t] = INFINITY;
        for (int k = 0; k < nc; ++k)
            for (int s = rs0[k]; s < rs1[k]; ++s)
                if (s != sl) topk_insert(bf, sqdf(pf, gf[s]));
        const float thr = knn_filter(bf[KK - 1]);
        double best[KK];
#pragma unroll
        for (int t = 0; t < KK; ++t) best[t] = INFINITY;
        for (int k = 0; k < nc; ++k)
            for (int s = rs0[k]; s < rs1[k]; ++s)
                if (sqdf(pf, gf[s]) <= thr && s != sl)
                    topk_insert(best, sqd(x, y, z, g.xyz[3 * s], g.xyz[3 * s + 1], g.xyz[3 * s + 2]));
        if (!(best[KK - 1] <= g.h * g.h)) {
            const int k = atomicAdd(n_bad, 1);
            if (k < bad_cap) bad[k] = i;
        }
        double sp = 0.0;
#pragma unroll
        for (int t = 0; t < KK; ++t) sp += sqrt(best[t]);
        per_point[i] = sp;
    }
}

// The points whose kk nearest others are not all within R: brute force
// over every point, one CTA per listed point: the kk smallest float squared
// distances of each thread's share, merged by thread 0 into the filter
// bound, then the same for the double distances of the candidates the
// filter keeps; the same sum.
template <int KK>
__global__ void __launch_bounds__(256) spacing_fallback_kernel(const double* __restrict__ V,
                                                               const float* __restrict__ fsrc, int P,
                                                               const int* __restrict__ n_bad,
                                                               const int* __restrict__ bad, int bad_cap,
                                                               double* __restrict__ per_point) {
    __shared__ double cand[256 * KK];
    __shared__ float s_thr;
    const int nb = min(*n_bad, bad_cap);
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int i = bad[b];
        const double x = V[3 * (int64_t)i], y = V[3 * (int64_t)i + 1], z = V[3 * (int64_t)i + 2];
        const float4 pf = make_float4(fsrc[3 * (int64_t)i], fsrc[3 * (int64_t)i + 1], fsrc[3 * (int64_t)i + 2], 0.f);
        float bf[KK];
#pragma unroll
        for (int t = 0; t < KK; ++t) bf[t] = INFINITY;
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            if (j == i) continue;
            topk_insert(bf, sqdf(pf, make_float4(fsrc[3 * (int64_t)j], fsrc[3 * (int64_t)j + 1],
                                                 fsrc[3 * (int64_t)j + 2], 0.f)));
        }
#pragma unroll
        for (int t = 0; t < KK; ++t) cand[threadIdx.x * KK + t] = (double)bf[t];
        __syncthreads();
        if (threadIdx.x == 0) {
            float m[KK];
#pragma unroll
            for (int t = 0; t < KK; ++t) m[t] = INFINITY;
            for (int q = 0; q < (int)blockDim.x * KK; ++q) topk_insert(m, (float)cand[q]);
            s_thr = knn_filter(m[KK - 1]);
        }
        __syncthreads();
        const float thr = s_thr;
        double best[KK];
#pragma unroll
        for (int t = 0; t < KK; ++t) best[t] = INFINITY;
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            if (j == i) continue;
            const float4 qf = make_float4(fsrc[3 * (int64_t)j], fsrc[3 * (int64_t)j + 1], fsrc[3 * (int64_t)j + 2], 0.f);
            if (sqdf(pf, qf) <= thr)
                topk_insert(best, sqd(x, y, z, V[3 * (int64_t)j], V[3 * (int64_t)j + 1], V[3 * (int64_t)j + 2]));
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < KK; ++t) cand[threadIdx.x * KK + t] = best[t];
        __syncthreads();
        if (threadIdx.x == 0) {
            double m[KK];
#pragma unroll
            for (int t = 0; t < KK; ++t) m[t] = INFINITY;
            for (int q = 0; q < (int)blockDim.x * KK; ++q) topk_insert(m, cand[q]);
            double sp = 0.0;
#pragma unroll
            for (int t = 0; t < KK; ++t) sp += sqrt(m[t]);
            per_point[i] = sp;
        }
        __syncthreads();
    }
}

template <int KK>
void launch_spacing(const GridView& gv, const float4* gf, const int* gitem, const double* V, const float* fsrc,
                    int n, double* pp, int* d_bad, int* d_badlist, cudaStream_t s) {
    spacing_kernel<KK><<<blocks_for(n), kT, 0, s>>>(gv, gf, gitem, V, n, pp, d_bad, d_badlist, kBadCap);
    spacing_fallback_kernel<KK><<<256, 256, 0, s>>>(V, fsrc, n, d_bad, d_badlist, kBadCap, pp);
}

// Fixed-order sum of x[0..n): per CTA a contiguous share reduced by a
// shared-memory tree, then the CTAs' partials in order by one thread.
__global__ void sum_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
    __shared__ double sh[kT];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b = blockIdx.x * per, e = b + per < n ? b + per : n;
    double acc = 0.0;
    for (int64_t k = b + threadIdx.x; k < e; k += blockDim.x) acc += x[k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void finish_sum_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t += part[k];
    *out = t * scale;
}

// The greedy sampling, node by node, in one CTA: the next rank (in visiting
// order) that no node covers becomes a node, and every point strictly within
// R of it is marked covered (state by visiting rank: 0 open, 1 node, 2 covered); the scan goes
// on after that rank. This is the sequential algorithm itself; the CTA's
// threads share the forward scan (1024 ranks at a time) and the covering of
// each ball. nodes[] receives the nodes in order, *n_nodes their number.
// Runs only when some rank's forward R-slab exceeds the window of
// greedy_window_kernel (*span > window); returns at once otherwise.
__global__ void __launch_bounds__(1024) greedy_kernel(GridView g, const int* __restrict__ slot_rank,
                                                      const int* __restrict__ order, const double* __restrict__ V,
                                                      int P, double R2, unsigned char* rstate, int* __restrict__ nodes,
                                                      int* __restrict__ n_nodes, const int* __restrict__ span,
                                                      int window) {
    if (*span <= window) return;   // greedy_window_kernel has run
    __shared__ int s_next;
    __shared__ int s_beg[27], s_off[28];
    const int lane = threadIdx.x & 31;
    int pos = 0, nn = 0;
    while (pos < P) {
        // ---- the next open rank at or after pos (states are kept by rank)
        if (threadIdx.x == 0) s_next = P;
        __syncthreads();
        const int r = pos + (int)threadIdx.x;
        if (r < P && ((volatile unsigned char*)rstate)[r] == 0) atomicMin(&s_next, r);
        __syncthreads();
        const int f = s_next;
        if (f == P) {
            pos += 1024;
            continue;
        }
        // ---- rank f becomes node nn and covers its ball: warp 0 finds the
        // 27 cells' runs and their offsets (a shuffle scan)
        const int v = order[f];
        const double x = V[3 * (int64_t)v], y = V[3 * (int64_t)v + 1], z = V[3 * (int64_t)v + 2];
        if (threadIdx.x < 32) {
            int s0 = 0, s1 = 0;
            if (lane < 27) {
                long long c[3];
                g.cell(x, y, z, c);
                const long long cx = c[0] - 1 + lane / 9, cy = c[1] - 1 + (lane / 3) % 3, cz = c[2] - 1 + lane % 3;
                if (cx >= 0 && cy >= 0 && cz >= 0 && cx < g.dims[0] && cy < g.dims[1] && cz < g.dims[2])
                    g.range((unsigned long long)((cx * g.dims[1] + cy) * g.dims[2] + cz), &s0, &s1);
            }
            int incl = s1 - s0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane < 27) {
                s_beg[lane] = s0;
                s_off[lane + 1] = incl;
            }
            if (lane == 0) {
                s_off[0] = 0;
                rstate[f] = 1;
                nodes[nn] = v;
            }
        }
        __syncthreads();
        const int total = s_off[27];
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int k = 0;
            while (s_off[k + 1] <= t) ++k;
            const int sidx = s_beg[k] + (t - s_off[k]);
            if (sqd(x, y, z, g.xyz[3 * sidx], g.xyz[3 * sidx + 1], g.xyz[3 * sidx + 2]) < R2) {
                const int ru = slot_rank[sidx];
                if (((volatile unsigned char*)rstate)[ru] == 0) rstate[ru] = 2;
            }
        }
        ++nn;
        pos = f + 1;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_nodes = nn;
}

// Greedy sampling in a window of the visiting order (the source points are
// floats, so their float copies are exact). Per rank r: rend[r] = the first
// rank whose projection on the visiting axis exceeds r's by more than R
// (with a margin far above the projections' rounding), so every point
// strictly within R of rank r's point that comes after it in the order has
// a rank in (r, rend[r]). The CTA holds the ranks [lo, hi) (at most
// kGreedyWin, slot r mod kGreedyWin) with their coordinates (float and
// double), rend and state (0 open, 2 covered) in shared memory. Per node f:
// every warp finds the next open rank itself (4 ranks per lane, a ballot;
// the same rank in every warp); the window moves to [f, f + kGreedyWin) if
// it does not reach rend[f]; every thread tests the open ranks of
// (f, rend[f]) in float: a float squared distance is within a relative
// 4e-7 of the exact one, so below R^2 (1 - 1e-5) the point is covered,
// above R^2 (1 + 1e-5) it is not, and the thin shell between is decided by
// the double distance, as everywhere else; one CTA barrier per node. Used
// when every rend[r] - r fits the window (*span); greedy_kernel runs
// otherwise.
constexpr int kGreedyWin = 4096;

// projection of a point on the visiting axis, as keys_kernel forms it
__device__ __forceinline__ double axis_proj(double x, double y, double z, const double* sc) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x, sc[9]), __dmul_rn(y, sc[10])), __dmul_rn(z, sc[11]));
}

// per rank: double and float coordinates, projection
__global__ void greedy_coords_kernel(const int* __restrict__ order, const double* __restrict__ V, int P,
                                     const double* __restrict__ sc, double* __restrict__ Vr,
                                     float4* __restrict__ Vf, double* __restrict__ proj) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
        const int v = order[r];
        const double x = V[3 * (int64_t)v], y = V[3 * (int64_t)v + 1], z = V[3 * (int64_t)v + 2];
        Vr[3 * (int64_t)r] = x;
        Vr[3 * (int64_t)r + 1] = y;
        Vr[3 * (int64_t)r + 2] = z;
        Vf[r] = make_float4((float)x, (float)y, (float)z, 0.f);
        proj[r] = axis_proj(x, y, z, sc);
    }
}

// rend[r] by binary search of the (ascending) projections; the largest
// rend[r] - r into *span. Margin: |a.(p - q)| <= |a| |p - q|, and each
// computed projection is within 3.1 * 2^-53 * (|x| + |y| + |z|) of the
// exact one (the axis entries are at most 1); the bound adds R |a| 1e-9
// and 1e-9 (|x| + |y| + |z| + 3R), far above both.
__global__ void greedy_rend_kernel(const double* __restrict__ Vr, const double* __restrict__ proj, int P,
                                   const double* __restrict__ sc, double R, int* __restrict__ rend,
                                   int* __restrict__ span) {
    const double na = sqrt(sc[9] * sc[9] + sc[10] * sc[10] + sc[11] * sc[11]);
    int worst = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
        const double S = fabs(Vr[3 * (int64_t)r]) + fabs(Vr[3 * (int64_t)r + 1]) + fabs(Vr[3 * (int64_t)r + 2]);
        const double bound = proj[r] + R * na * (1.0 + 1e-9) + 1e-9 * (S + 3.0 * R);
        int lo = r + 1, hi = P;   // first rank in [r + 1, P] with proj > bound
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (proj[m] > bound) hi = m; else lo = m + 1;
        }
        rend[r] = lo;
        worst = max(worst, lo - r);
    }
    atomicMax(span, worst);
}

__global__ void __launch_bounds__(1024) greedy_window_kernel(const double* __restrict__ Vr,
                                                             const float4* __restrict__ Vf,
                                                             const int* __restrict__ rend,
                                                             const int* __restrict__ span, int P, double R2,
                                                             int* __restrict__ node_rank, int* __restrict__ n_nodes) {
    if (*span > kGreedyWin) return;   // greedy_kernel runs instead
    constexpr int W = kGreedyWin, M = kGreedyWin - 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* wf = reinterpret_cast<float4*>(smem);            // [W]
    double* wx = reinterpret_cast<double*>(wf + W);          // [3][W]
    int* wr = reinterpret_cast<int*>(wx + 3 * W);            // [W]
    unsigned char* ws = reinterpret_cast<unsigned char*>(wr + W);   // [W]
    const int lane = threadIdx.x & 31;
    // below thr_in a float squared distance is inside R for certain (its
    // relative error is below 4e-7; with R2 >= 1e-30 no subnormal term
    // matters); from thr_in to thr the double distance decides; at or above
    // thr the point is outside (R2 < 1e30: no float overflow near R)
    const bool all = !(R2 < 1e30);
    const float thr = all ? 0.f : (float)(R2 * (1.0 + 1e-5) + 1e-36);
    const float thr_in = (!all && R2 >= 1e-30) ? (float)(R2 * (1.0 - 1e-5)) : -1.f;
    int lo = 0, hi = 0;
    // the window becomes [nlo, min(P, nlo + W)): ranks from max(hi, nlo)
    // are loaded into slots of ranks below nlo (decided; the barrier first
    // lets every warp finish reading them)
    auto refill = [&](int nlo) {
        __syncthreads();
        const int nhi = min(P, nlo + W);
        for (int r = max(hi, nlo) + (int)threadIdx.x; r < nhi; r += blockDim.x) {
            const int q = r & M;
            wf[q] = Vf[r];
            wx[q] = Vr[3 * (int64_t)r];
            wx[W + q] = Vr[3 * (int64_t)r + 1];
            wx[2 * W + q] = Vr[3 * (int64_t)r + 2];
            wr[q] = rend[r];
            ws[q] = 0;
        }
        lo = nlo;
        hi = nhi;
        __syncthreads();
    };
    refill(0);
    int pos = 0, nn = 0;
    for (;;) {
        // every warp finds the next open rank f in [pos, hi) itself (4 ranks
        // per lane, a ballot): the states were written before the last
        // barrier and are not written again before the next, so every warp
        // finds the same f (-1: none)
        int f = -1;
        for (int base = pos & ~3; base < hi; base += 128) {
            const int r0 = base + 4 * lane;
            unsigned m = 0;   // bit k: rank r0 + k is open, in [pos, hi)
            if (r0 < hi) {
                const unsigned wv = *reinterpret_cast<const unsigned*>(ws + (r0 & M));
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (((wv >> (8 * k)) & 0xffu) == 0 && r0 + k >= pos && r0 + k < hi) m |= 1u << k;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, m != 0);
            if (bal) {
                const int src = __ffs(bal) - 1;
                const unsigned mm = __shfl_sync(0xffffffffu, m, src);
                f = base + 4 * src + __ffs(mm) - 1;
                break;
            }
        }
        if (f < 0) {   // every rank of [pos, hi) is decided
            if (hi >= P) break;
            const int h = hi;
            refill(h);
            pos = h;
            continue;
        }
        if (threadIdx.x == 0) node_rank[nn] = f;
        const int re = wr[f & M];
        if (re > hi) refill(f);   // re - f <= span <= W
        const int sf = f & M;
        const float4 pf = wf[sf];
        const double x = wx[sf], y = wx[W + sf], z = wx[2 * W + sf];
        // rank f itself is never read again (scans start after it)
        for (int r = f + 1 + (int)threadIdx.x; r < re; r += blockDim.x) {
            const int q = r & M;
            if (ws[q] != 0) continue;
            const float d2f = sqdf(pf, wf[q]);
            if (d2f < thr_in || ((all || d2f < thr) && sqd(x, y, z, wx[q], wx[W + q], wx[2 * W + q]) < R2)) ws[q] = 2;
        }
        ++nn;
        pos = f + 1;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_nodes = nn;
}

__global__ void rank_to_point_kernel(const int* __restrict__ n_nodes, const int* __restrict__ order,
                                     int* __restrict__ nodes) {
    const int N = *n_nodes;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) nodes[j] = order[nodes[j]];
}

// rank of each point in the visiting order, then of each grid slot's point
__global__ void rank_of_kernel(int P, const int* __restrict__ order, int* __restrict__ rank_of) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) rank_of[order[r]] = r;
}
__global__ void slot_rank_kernel(int P, const int* __restrict__ gitem, const int* __restrict__ rank_of,
                                 int* __restrict__ slot_rank) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P; s += gridDim.x * blockDim.x) slot_rank[s] = rank_of[gitem[s]];
}

// node positions and node-grid keys
__global__ void nodes_kernel(int N, const int* __restrict__ nodes, const double* __restrict__ V,
                             const double* __restrict__ sc, double h, long long d1, long long d2,
                             double* __restrict__ pn, unsigned long long* __restrict__ nkey, int* __restrict__ nval) {
    const double lo[3] = {sc[3], sc[4], sc[5]};
    const long long dims[3] = {(long long)sc[12], d1, d2};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const int i = nodes[j];
        long long c[3];
        for (int d = 0; d < 3; ++d) {
            const double x = V[3 * (int64_t)i + d];
            pn[3 * j + d] = x;
            long long v = (long long)floor((x - lo[d]) / h);
            c[d] = v < 0 ? 0 : (v > dims[d] - 1 ? dims[d] - 1 : v);
        }
        nkey[j] = (unsigned long long)((c[0] * d1 + c[1]) * d2 + c[2]);
        nval[j] = j;
    }
}

__global__ void node_grid_xyz_kernel(int N, const int* __restrict__ nsorted, const double* __restrict__ pn,
                                     double* __restrict__ nxyz) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) nxyz[3 * s + d] = pn[3 * nsorted[s] + d];
}

// influence sets: the K nearest nodes within R by (d^2, node id), weights of
// Eq. (weight_data) (1 - d^2/R^2)^3 normalised over the set, and the number
// of node pairs of each set (edges)
__global__ void __launch_bounds__(kT) influence_kernel(GridView g, const int* __restrict__ nsorted,
                                                       const int* __restrict__ pitem,
                                                       const double* __restrict__ pxyz, int64_t P, double R2, int K,
                                                       int* __restrict__ nidx, double* __restrict__ w,
                                                       int* __restrict__ npairs) {
    // points in the point grid's cell order (slot sl holds point pitem[sl],
    // coordinates pxyz): the lanes of a warp read the same node cells
    for (int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sl < P; sl += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = pitem[sl];
        const double x = pxyz[3 * sl], y = pxyz[3 * sl + 1], z = pxyz[3 * sl + 2];
        double bd[NRR_MAX_INFL];
        int bj[NRR_MAX_INFL];
        int n = 0;
        long long c[3];
        g.cell(x, y, z, c);
        for (long long cx = c[0] - 1; cx <= c[0] + 1; ++cx)
            for (long long cy = c[1] - 1; cy <= c[1] + 1; ++cy)
                for (long long cz = c[2] - 1; cz <= c[2] + 1; ++cz) {
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= g.dims[0] || cy >= g.dims[1] || cz >= g.dims[2]) continue;
                    int s0, s1;
                    g.range((unsigned long long)((cx * g.dims[1] + cy) * g.dims[2] + cz), &s0, &s1);
                    for (int s = s0; s < s1; ++s) {
                        const double d2 = sqd(x, y, z, g.xyz[3 * s], g.xyz[3 * s + 1], g.xyz[3 * s + 2]);
                        if (!(d2 < R2)) continue;
                        const int j = nsorted[s];
                        // sorted insertion by (d^2, node id), keeping the K smallest
                        if (n == K && !(d2 < bd[K - 1] || (d2 == bd[K - 1] && j < bj[K - 1]))) continue;
                        int pos = n < K ? n : K - 1;
                        while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bj[pos - 1] > j))) {
                            bd[pos] = bd[pos - 1];
                            bj[pos] = bj[pos - 1];
                            --pos;
                        }
                        bd[pos] = d2;
                        bj[pos] = j;
                        if (n < K) ++n;
                    }
                }
        double raw[NRR_MAX_INFL];
        double sum = 0.0;
        for (int s = 0; s < n; ++s) {
            const double a = 1.0 - bd[s] / R2;
            raw[s] = a * a * a;
        }
        for (int s = 0; s < n; ++s) sum += raw[s];
        for (int s = 0; s < K; ++s) {
            nidx[i * K + s] = s < n ? bj[s] : -1;
            w[i * K + s] = s < n ? raw[s] / sum : 0.0;
        }
        npairs[i] = n * (n - 1) / 2;
    }
}

__global__ void pair_keys_kernel(int64_t P, int K, const int* __restrict__ nidx, const int* __restrict__ off,
                                 unsigned long long* __restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        int o = off[i];
        for (int a = 0; a < K; ++a) {
            const int u = nidx[i * K + a];
            if (u < 0) break;
            for (int b = a + 1; b < K; ++b) {
                const int v = nidx[i * K + b];
                if (v < 0) break;
                const unsigned long long lo = (unsigned long long)min(u, v), hi = (unsigned long long)max(u, v);
                keys[o++] = (lo << 32) | hi;
            }
        }
    }
}

__global__ void unique_flags_kernel(int64_t n, const unsigned long long* __restrict__ keys, int* __restrict__ flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        flag[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1 : 0;
}

// unique edges (j < k) and both directed pairs of each
__global__ void edges_kernel(int64_t n, const unsigned long long* __restrict__ keys, const int* __restrict__ flag,
                             const int* __restrict__ pos, int* __restrict__ edges,
                             unsigned long long* __restrict__ dkeys) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        const int e = pos[k];
        const unsigned long long a = keys[k] >> 32, b = keys[k] & 0xffffffffull;
        edges[2 * e] = (int)a;
        edges[2 * e + 1] = (int)b;
        dkeys[2 * e] = (a << 32) | b;
        dkeys[2 * e + 1] = (b << 32) | a;
    }
}

// 1 / |p_i - p_j| of every directed pair and its per-CTA partial sums
__global__ void __launch_bounds__(kT) inv_len_kernel(int E2, const unsigned long long* __restrict__ dkeys,
                                                     const double* __restrict__ pn, double* __restrict__ inv,
                                                     double* __restrict__ part) {
    __shared__ double sh[kT / 32];
    const int per = (E2 + gridDim.x - 1) / gridDim.x;
    const int e0 = blockIdx.x * per, e1 = min(E2, e0 + per);
    double s = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += kT) {
        const int a = (int)(dkeys[e] >> 32), b = (int)(dkeys[e] & 0xffffffffull);
        const double v = 1.0 / sqrt(sqd(pn[3 * a], pn[3 * a + 1], pn[3 * a + 2], pn[3 * b], pn[3 * b + 1], pn[3 * b + 2]));
        inv[e] = v;
        s += v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void r_kernel(int E2, int nb, const double* __restrict__ part, double n_edges, double* __restrict__ r,
                         int* __restrict__ dpair, const unsigned long long* __restrict__ dkeys,
                         const double* __restrict__ inv) {
    __shared__ double s_sum;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        s_sum = t;
    }
    __syncthreads();
    const double sum = s_sum;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E2; e += gridDim.x * blockDim.x) {
        r[e] = 2.0 * n_edges * inv[e] / sum;
        dpair[2 * e] = (int)(dkeys[e] >> 32);
        dpair[2 * e + 1] = (int)(dkeys[e] & 0xffffffffull);
    }
}

// device buffers of one build, freed on every exit path
struct Scratch {
    std::vector<void*> p;
    ~Scratch() {
        for (void* q : p) cudaFree(q);
    }
    template <typename X>
    cudaError_t get(X** out, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(X));
        if (e == cudaSuccess) p.push_back(q);
        *out = (X*)q;
        return e;
    }
};

template <typename K, typename V>
cudaError_t sort_pairs(Scratch& s, const K* kin, K* kout, const V* vin, V* vout, int n, int end_bit, cudaStream_t st) {
    size_t tb = 0;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, vout, n, 0, end_bit, st);
    if (e != cudaSuccess) return e;
    void* tmp = nullptr;
    if ((e = s.get((unsigned char**)&tmp, tb)) != cudaSuccess) return e;
    return cub::DeviceRadixSort::SortPairs(tmp, tb, kin, kout, vin, vout, n, 0, end_bit, st);
}

template <typename K>
cudaError_t sort_keys(Scratch& s, const K* kin, K* kout, int n, cudaStream_t st) {
    size_t tb = 0;
    cudaError_t e = cub::DeviceRadixSort::SortKeys(nullptr, tb, kin, kout, n, 0, 64, st);
    if (e != cudaSuccess) return e;
    void* tmp = nullptr;
    if ((e = s.get((unsigned char**)&tmp, tb)) != cudaSuccess) return e;
    return cub::DeviceRadixSort::SortKeys(tmp, tb, kin, kout, n, 0, 64, st);
}

cudaError_t exclusive_sum(Scratch& s, const int* in, int* out, int n, cudaStream_t st) {
    size_t tb = 0;
    cudaError_t e = cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, st);
    if (e != cudaSuccess) return e;
    void* tmp = nullptr;
    if ((e = s.get((unsigned char**)&tmp, tb)) != cudaSuccess) return e;
    return cub::DeviceScan::ExclusiveSum(tmp, tb, in, out, n, st);
}


}  // namespace

// ---------------------------------------------------------------------------
// Hilbert orders of the source and target points (setup of the target leaves
// and of the source's internal order): one thread per point forms the code
// (nrr_curve_coord, nrr_hilbert3: the host's functions), then a stable radix
// sort of (code, index) pairs, whose ties keep the lower index as the host's
// sort of distinct (code, index) pairs does.
// ---------------------------------------------------------------------------
__global__ void curve_codes_kernel(const float* __restrict__ pts, int64_t n, double lo0, double lo1, double lo2,
                                   double e0, double e1, double e2, unsigned long long* __restrict__ code,
                                   int* __restrict__ idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cx = nrr_curve_coord(pts[3 * i], lo0, e0), cy = nrr_curve_coord(pts[3 * i + 1], lo1, e1),
                       cz = nrr_curve_coord(pts[3 * i + 2], lo2, e2);
        code[i] = nrr_hilbert3(cx, cy, cz);
        idx[i] = (int)i;
    }
}

// Algorithm 1 on the GPU (see the file comment). src: [P][3] float32, host or
// device. Fills g as nrr_build_graph does. Returns cudaSuccess or the first
// CUDA error; *rounds receives the number of greedy rounds.
cudaError_t nrr_build_graph_gpu(const float* src, int64_t P, double R, int K, HostGraph& g, cudaStream_t st,
                                int* rounds, double* lbar) {
#define GK(call)                                \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)
    Scratch s;
    const int n = (int)P;
    const double R2 = R * R;
    // NRR_SETUP_TIMES: the phases on stderr (each timed to the end of its
    // GPU work)
    const bool times = std::getenv("NRR_SETUP_TIMES") != nullptr;
    auto t_last = std::chrono::steady_clock::now();
    auto lap = [&](const char* what) {
        if (!times) return;
        cudaStreamSynchronize(st);
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "  graph on the GPU: %-28s %8.2f ms\n", what,
                     std::chrono::duration<double, std::milli>(now - t_last).count());
        t_last = now;
    };
    g.radius = R;
    g.K = K;
    float* fsrc = nullptr;
    double *V = nullptr, *part = nullptr, *sc = nullptr;
    GK(s.get(&fsrc, (size_t)P * 3));
    GK(cudaMemcpyAsync(fsrc, src, sizeof(float) * 3 * (size_t)P, cudaMemcpyDefault, st));
    GK(s.get(&V, (size_t)P * 3));
    GK(s.get(&part, (size_t)kRed * 12));
    GK(s.get(&sc, 16));
    to_double_kernel<<<blocks_for(3 * P), kT, 0, st>>>(fsrc, V, 3 * P);
    // ---- 1. PCA (mean and bounding box, then the covariance and its axis)
    moments_kernel<<<kRed, kT, 0, st>>>(V, P, 0, sc, part);
    finish_moments_kernel<<<1, 1, 0, st>>>(part, kRed, P, 0, sc);
    moments_kernel<<<kRed, kT, 0, st>>>(V, P, 1, sc, part);
    finish_moments_kernel<<<1, 1, 0, st>>>(part, kRed, P, 1, sc);
    GK(cudaGetLastError());
    double hsc[16];
    GK(cudaMemcpyAsync(hsc, sc, sizeof(double) * 12, cudaMemcpyDeviceToHost, st));
    GK(cudaStreamSynchronize(st));
    // grid of cell size R over the bounding box (the host code's grid)
    const double h = R > 0 ? R : 1.0;
    long long dims[3];
    for (int d = 0; d < 3; ++d) dims[d] = std::max<long long>(1, (long long)std::floor((hsc[6 + d] - hsc[3 + d]) / h) + 1);
    hsc[12] = (double)dims[0];
    GK(cudaMemcpyAsync(sc + 12, hsc + 12, sizeof(double), cudaMemcpyHostToDevice, st));
    lap("PCA");
    // ---- 2. the visiting order and the grid
    unsigned long long *pkey, *pkey_s, *ckey, *ckey_s;
    int *idx, *order, *gitem;
    double* gxyz;
    GK(s.get(&pkey, P)); GK(s.get(&pkey_s, P)); GK(s.get(&ckey, P)); GK(s.get(&ckey_s, P));
    GK(s.get(&idx, P)); GK(s.get(&order, P)); GK(s.get(&gitem, P));
    GK(s.get(&gxyz, (size_t)P * 3));
    keys_kernel<<<blocks_for(P), kT, 0, st>>>(V, P, sc, h, dims[1], dims[2], pkey, ckey, idx);
    GK(cudaGetLastError());
    GK(sort_pairs(s, pkey, pkey_s, idx, order, n, 64, st));
    GK(sort_pairs(s, ckey, ckey_s, idx, gitem, n, 64, st));
    float4* gf;
    GK(s.get(&gf, P));
    grid_data_kernel<<<blocks_for(P), kT, 0, st>>>(P, gitem, V, gxyz, gf);
    GK(cudaGetLastError());
    lap("visiting order and grid");
    // ---- 3. the greedy sampling (one CTA, node by node)
    const double cells_d = (double)dims[0] * (double)dims[1] * (double)dims[2];
    const bool dense = cells_d <= 4.0 * (double)P + 1048576.0;
    const long long cells = (long long)cells_d;
    int* cstart = nullptr;
    if (dense) {
        GK(s.get(&cstart, (size_t)cells + 1));
        cell_start_kernel<<<blocks_for(cells + 1), kT, 0, st>>>(ckey_s, n, cells, cstart);
    }
    unsigned char* state;
    int *nodes, *nnode;
    GK(s.get(&state, P));
    GK(s.get(&nodes, P));
    GK(s.get(&nnode, 1));
    GK(cudaMemsetAsync(state, 0, (size_t)P, st));
    GridView gv{ckey_s, gxyz, n, {hsc[3], hsc[4], hsc[5]}, h, {dims[0], dims[1], dims[2]}, cstart};
    // l-bar on the same grid (cell R) when asked for; read back with the
    // node count below
    double* d_lbar = nullptr;
    int* d_bad = nullptr;
    const int kk = (int)std::min<int64_t>(6, P - 1);
    // on a second stream: the greedy sampling below runs in one CTA and
    // leaves the other SMs to it
    struct SideStream {
        cudaStream_t s = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        ~SideStream() {
            if (s) cudaStreamDestroy(s);
            if (fork) cudaEventDestroy(fork);
            if (join) cudaEventDestroy(join);
        }
    } side;
    if (lbar) {
        *lbar = std::nan("");
        if (kk >= 1) {
            double *pp, *lpart;
            GK(s.get(&pp, P)); GK(s.get(&lpart, kRed)); GK(s.get(&d_lbar, 1)); GK(s.get(&d_bad, 1));
            GK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
            GK(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
            GK(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
            GK(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming));
            GK(cudaEventRecord(side.fork, st));
            GK(cudaStreamWaitEvent(side.s, side.fork, 0));
            int* d_badlist;
            GK(s.get(&d_badlist, kBadCap));
            switch (kk) {
                case 1: launch_spacing<1>(gv, gf, gitem, V, fsrc, n, pp, d_bad, d_badlist, side.s); break;
                case 2: launch_spacing<2>(gv, gf, gitem, V, fsrc, n, pp, d_bad, d_badlist, side.s); break;
                case 3: launch_spacing<3>(gv, gf, gitem, V, fsrc, n, pp, d_bad, d_badlist, side.s); break;
                case 4: launch_spacing<4>(gv, gf, gitem, V, fsrc, n, pp, d_bad, d_badlist, side.s); break;
                case 5: launch_spacing<5>(gv, gf, gitem, V, fsrc, n, pp, d_bad, d_badlist, side.s); break;
                default: launch_spacing<6>(gv, gf, gitem, V, fsrc, n, pp, d_bad, d_badlist, side.s); break;
            }
            sum_kernel<<<kRed, kT, 0, side.s>>>(pp, P, lpart);
            finish_sum_kernel<<<1, 1, 0, side.s>>>(lpart, kRed, 1.0 / ((double)P * kk), d_lbar);
            GK(cudaGetLastError());
            GK(cudaEventRecord(side.join, side.s));
        }
    }
    int *rank_of, *slot_rank;
    GK(s.get(&rank_of, P)); GK(s.get(&slot_rank, P));
    rank_of_kernel<<<blocks_for(P), kT, 0, st>>>(n, order, rank_of);
    slot_rank_kernel<<<blocks_for(P), kT, 0, st>>>(n, gitem, rank_of, slot_rank);
    // the window kernel when every rank's forward R-slab fits its window
    // (decided on the device), else the global-state kernel
    const size_t win_smem = (size_t)kGreedyWin * (16 + 24 + 4 + 1);
    {
        double *Vr, *proj;
        float4* Vf;
        int *rend, *span;
        GK(s.get(&Vr, (size_t)P * 3)); GK(s.get(&proj, P)); GK(s.get(&Vf, P));
        GK(s.get(&rend, P)); GK(s.get(&span, 1));
        GK(cudaMemsetAsync(span, 0, sizeof(int), st));
        GK(cudaMemsetAsync(nnode, 0, sizeof(int), st));
        GK(cudaFuncSetAttribute(greedy_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem));
        greedy_coords_kernel<<<blocks_for(P), kT, 0, st>>>(order, V, n, sc, Vr, Vf, proj);
        greedy_rend_kernel<<<blocks_for(P), kT, 0, st>>>(Vr, proj, n, sc, R, rend, span);
        greedy_window_kernel<<<1, 1024, win_smem, st>>>(Vr, Vf, rend, span, n, R2, nodes, nnode);
        rank_to_point_kernel<<<blocks_for(P), kT, 0, st>>>(nnode, order, nodes);
        greedy_kernel<<<1, 1024, 0, st>>>(gv, slot_rank, order, V, n, R2, state, nodes, nnode, span, kGreedyWin);
    }
    GK(cudaGetLastError());
    lap("greedy sampling (+ l-bar)");
    int N = 0;
    GK(cudaMemcpyAsync(&N, nnode, sizeof(int), cudaMemcpyDeviceToHost, st));
    double lb = std::nan("");
    int bad = 0;
    if (d_lbar) {
        GK(cudaStreamWaitEvent(st, side.join, 0));
        GK(cudaMemcpyAsync(&lb, d_lbar, sizeof(double), cudaMemcpyDeviceToHost, st));
        GK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    GK(cudaStreamSynchronize(st));
    if (rounds) *rounds = N;
    if (d_lbar && bad <= kBadCap) *lbar = lb;
    if (times && d_lbar) std::fprintf(stderr, "  graph on the GPU: l-bar points searched beyond R: %d\n", bad);
    int last[2];
    // ---- node positions and the node grid
    int *nval, *nsorted;
    double *pn, *nxyz;
    unsigned long long *nkey, *nkey_s;
    GK(s.get(&nval, N)); GK(s.get(&nsorted, N));
    GK(s.get(&pn, (size_t)N * 3)); GK(s.get(&nxyz, (size_t)N * 3));
    GK(s.get(&nkey, N)); GK(s.get(&nkey_s, N));
    nodes_kernel<<<blocks_for(N), kT, 0, st>>>(N, nodes, V, sc, h, dims[1], dims[2], pn, nkey, nval);
    GK(cudaGetLastError());
    GK(sort_pairs(s, nkey, nkey_s, nval, nsorted, N, 64, st));
    node_grid_xyz_kernel<<<blocks_for(N), kT, 0, st>>>(N, nsorted, pn, nxyz);
    lap("node grid");
    // ---- 4. influence sets, weights, edges, r_ij
    int *nidx, *npairs, *poff;
    double* w;
    GK(s.get(&nidx, (size_t)P * K)); GK(s.get(&w, (size_t)P * K));
    GK(s.get(&npairs, P)); GK(s.get(&poff, P));
    int* ncstart = nullptr;
    if (dense) {
        GK(s.get(&ncstart, (size_t)cells + 1));
        cell_start_kernel<<<blocks_for(cells + 1), kT, 0, st>>>(nkey_s, N, cells, ncstart);
    }
    GridView nv{nkey_s, nxyz, N, {hsc[3], hsc[4], hsc[5]}, h, {dims[0], dims[1], dims[2]}, ncstart};
    influence_kernel<<<blocks_for(P), kT, 0, st>>>(nv, nsorted, gitem, gxyz, P, R2, K, nidx, w, npairs);
    GK(cudaGetLastError());
    GK(exclusive_sum(s, npairs, poff, n, st));
    GK(cudaMemcpyAsync(&last[0], poff + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GK(cudaMemcpyAsync(&last[1], npairs + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GK(cudaStreamSynchronize(st));
    const int n_pk = last[0] + last[1];
    unsigned long long *pk, *pk_s;
    int *uflag, *upos;
    GK(s.get(&pk, n_pk)); GK(s.get(&pk_s, n_pk)); GK(s.get(&uflag, n_pk)); GK(s.get(&upos, n_pk));
    pair_keys_kernel<<<blocks_for(P), kT, 0, st>>>(P, K, nidx, poff, pk);
    GK(cudaGetLastError());
    int n_edges = 0;
    if (n_pk > 0) {
        GK(sort_keys(s, pk, pk_s, n_pk, st));
        unique_flags_kernel<<<blocks_for(n_pk), kT, 0, st>>>(n_pk, pk_s, uflag);
        GK(exclusive_sum(s, uflag, upos, n_pk, st));
        GK(cudaMemcpyAsync(&last[0], upos + n_pk - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GK(cudaMemcpyAsync(&last[1], uflag + n_pk - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GK(cudaStreamSynchronize(st));
        n_edges = last[0] + last[1];
    }
    const int E2 = 2 * n_edges;
    int *edges, *dpair;
    unsigned long long *dk, *dk_s;
    double *inv, *rr, *rpart;
    GK(s.get(&edges, 2 * (size_t)n_edges)); GK(s.get(&dpair, 2 * (size_t)E2));
    GK(s.get(&dk, E2)); GK(s.get(&dk_s, E2)); GK(s.get(&inv, E2)); GK(s.get(&rr, E2)); GK(s.get(&rpart, kRed));
    if (n_edges > 0) {
        edges_kernel<<<blocks_for(n_pk), kT, 0, st>>>(n_pk, pk_s, uflag, upos, edges, dk);
        GK(cudaGetLastError());
        GK(sort_keys(s, dk, dk_s, E2, st));
        inv_len_kernel<<<kRed, kT, 0, st>>>(E2, dk_s, pn, inv, rpart);
        r_kernel<<<blocks_for(E2), kT, 0, st>>>(E2, kRed, rpart, (double)n_edges, rr, dpair, dk_s, inv);
        GK(cudaGetLastError());
    }
    lap("influence, edges, r_ij");
    // ---- back to the host graph
    g.nodes.resize((size_t)N);
    g.nidx.resize((size_t)P * K);
    g.w.resize((size_t)P * K);
    g.edges.resize(2 * (size_t)n_edges);
    g.dpair.resize(2 * (size_t)E2);
    g.r.resize((size_t)E2);
    GK(cudaMemcpyAsync(g.nodes.data(), nodes, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, st));
    GK(cudaMemcpyAsync(g.nidx.data(), nidx, sizeof(int) * (size_t)P * K, cudaMemcpyDeviceToHost, st));
    GK(cudaMemcpyAsync(g.w.data(), w, sizeof(double) * (size_t)P * K, cudaMemcpyDeviceToHost, st));
    if (n_edges > 0) {
        GK(cudaMemcpyAsync(g.edges.data(), edges, sizeof(int) * 2 * (size_t)n_edges, cudaMemcpyDeviceToHost, st));
        GK(cudaMemcpyAsync(g.dpair.data(), dpair, sizeof(int) * 2 * (size_t)E2, cudaMemcpyDeviceToHost, st));
        GK(cudaMemcpyAsync(g.r.data(), rr, sizeof(double) * (size_t)E2, cudaMemcpyDeviceToHost, st));
    }
    GK(cudaStreamSynchronize(st));
    lap("copies to the host");
    return cudaSuccess;
#undef GK
}

cudaError_t nrr_curve_orders_gpu(const float* src, int64_t P, const float* tgt, int64_t T, const double lo[3],
                                 const double hi[3], cudaStream_t st, std::vector<int>& src_order,
                                 std::vector<uint64_t>& src_codes, std::vector<int>& tgt_order,
                                 std::vector<uint64_t>& tgt_codes) {
#define CK_(call)                               \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)
    Scratch s;
    const double e[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    const float* in[2] = {src, tgt};
    const int64_t n[2] = {P, T};
    std::vector<int>* ord[2] = {&src_order, &tgt_order};
    std::vector<uint64_t>* cod[2] = {&src_codes, &tgt_codes};
    for (int k = 0; k < 2; ++k) {
        const int64_t m = n[k];
        float* d_pts;
        unsigned long long *key, *key_s;
        int *idx, *idx_s;
        CK_(s.get(&d_pts, (size_t)m * 3)); CK_(s.get(&key, m)); CK_(s.get(&key_s, m));
        CK_(s.get(&idx, m)); CK_(s.get(&idx_s, m));
        CK_(cudaMemcpyAsync(d_pts, in[k], sizeof(float) * 3 * (size_t)m, cudaMemcpyDefault, st));
        curve_codes_kernel<<<blocks_for(m), kT, 0, st>>>(d_pts, m, lo[0], lo[1], lo[2], e[0], e[1], e[2], key, idx);
        CK_(cudaGetLastError());
        CK_(sort_pairs(s, key, key_s, idx, idx_s, (int)m, 63, st));
        ord[k]->resize((size_t)m);
        cod[k]->resize((size_t)m);
        CK_(cudaMemcpyAsync(ord[k]->data(), idx_s, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, st));
        CK_(cudaMemcpyAsync(cod[k]->data(), key_s, sizeof(uint64_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
    }
    CK_(cudaStreamSynchronize(st));
    return cudaSuccess;
#undef CK_
}
