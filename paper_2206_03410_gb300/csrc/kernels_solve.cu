// Solve of the surrogate normal equations K X = B (Eq. surr_solution) by
// block-Jacobi preconditioned conjugate gradients, warm-started at X^(k), in
// one persistent kernel that leaves G(X^(k)) in d.G (the Anderson mix that
// follows is in kernels_aa.cu).
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
#include <cooperative_groups.h>

#include <type_traits>

#include "nrr_device.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 128;
constexpr int kMaxRed = 12;  // values per reduction (at most)
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
    int skip_arrival;   // failure-detection test: this CTA does not arrive once

    // Returns false if the wait timed out or another CTA reported a failure.
    __device__ bool sync() {
        __syncthreads();
        if (threadIdx.x == 0) {
            int fail = 0;
            __threadfence();
            const bool skipped = skip_arrival != 0;
            const unsigned arrived = skipped ? 0u : atomicAdd(&st->bar_count, 1u);
            skip_arrival = 0;
            if (!skipped && arrived == nblocks - 1) {
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
    template <int K, typename A>
    __device__ bool run(Barrier& bar, const A (&v)[K], double* s_tmp, double (&out)[K]) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            A x = v[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) s_tmp[w * kMaxRed + j] = (double)x;
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

// 4x4 SPD inverse by Cholesky in type F. Returns false if not positive definite.
template <typename F>
__device__ bool spd_inverse4(const F A[16], F Inv[16]) {
    F L[16] = {0};
    for (int j = 0; j < 4; ++j) {
        F s = A[4 * j + j];
        for (int k = 0; k < j; ++k) s -= L[4 * j + k] * L[4 * j + k];
        if (!(s > F(0))) return false;
        L[4 * j + j] = sqrt(s);
        for (int i = j + 1; i < 4; ++i) {
            F t = A[4 * i + j];
            for (int k = 0; k < j; ++k) t -= L[4 * i + k] * L[4 * j + k];
            L[4 * i + j] = t / L[4 * j + j];
        }
    }
    // columns of inv(L), then Inv = inv(L)^T inv(L)
    F Li[16] = {0};
    for (int c = 0; c < 4; ++c) {
        for (int i = 0; i < 4; ++i) {
            F t = (i == c) ? F(1) : F(0);
            for (int k = 0; k < i; ++k) t -= L[4 * i + k] * Li[4 * k + c];
            Li[4 * i + c] = t / L[4 * i + i];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            F s = 0;
            for (int k = 0; k < 4; ++k) s += Li[4 * k + i] * Li[4 * k + j];
            Inv[4 * i + j] = s;
        }
    return true;
}

// four consecutive values from shared memory with vector loads
__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double (&o)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// a[c] for a runtime c in 0..2 without indexing (keeps a[] in registers)
template <typename T>
__device__ __forceinline__ T pick3(const T* a, int c) {
    return c == 0 ? a[0] : (c == 1 ? a[1] : a[2]);
}

// Row a of block blk of the K rows a cluster CTA keeps in shared memory.
// Layout, vector-major: block blk's 16-byte vectors v = 0 .. 16*sizeof(T)/16-1
// (row a = vectors a*sizeof(T)/4 ..) sit at vector index v * cap + blk, so the
// lanes of a warp that read the same row of consecutive blocks read
// consecutive 16-byte words (no bank conflicts between them).
__device__ __forceinline__ void krow(const float* K, int cap, int blk, int a, float (&o)[4]) {
    const float4 v = reinterpret_cast<const float4*>(K)[(size_t)a * cap + blk];
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void krow(const double* K, int cap, int blk, int a, double (&o)[4]) {
    const double2* K2 = reinterpret_cast<const double2*>(K);
    const double2 x = K2[(size_t)(2 * a) * cap + blk];
    const double2 y = K2[(size_t)(2 * a + 1) * cap + blk];
    o[0] = x.x; o[1] = x.y; o[2] = y.x; o[3] = y.y;
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
    __shared__ double s_scal[12];
    NrrState* st = d.st;
    if (st->done || st->skip) return;
    const int N = d.N;
    const int G = gridDim.x;
    const int per = (N + G - 1) / G;
    const int n0 = min(N, (int)blockIdx.x * per), n1 = min(N, n0 + per);
    const int npairs = (n1 - n0) * 3;
    // d.fault_barrier (a host-side test knob): CTA 0 skips its first arrival,
    // so every CTA's bounded wait runs out and records NRR_E_TIMEOUT
    Barrier bar{st, *(volatile unsigned*)&st->bar_gen, (unsigned)G, &s_flag,
                (d.fault_barrier && blockIdx.x == 0 && G > 1) ? 1 : 0};
    Red red{d.partials, 0};
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

    // initial residual with the warm start x = X^(k) (+ the previous MM
    // step once the stage has solved: K x = K X^(k) + K dx)
    const T* wdx = (d.warm_dx != nullptr && st->n_solves_stage > 0) ? d.warm_dx : nullptr;
    double acc[9];
    double sums[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) acc[j] = 0.0;
    for (int idx = threadIdx.x; idx < npairs; idx += kThreads) {
        const int n = n0 + idx / 3, c = idx % 3;
        T y[4];
        spmv_pair<T, false>(d, d.X, n, c, y);
        if (wdx) {
            T y2[4];
            spmv_pair<T, false>(d, wdx, n, c, y2);
            for (int a = 0; a < 4; ++a) y[a] += y2[a];
        }
        T rr[4];
        for (int a = 0; a < 4; ++a) {
            const T b = d.Bv[12 * n + 3 * a + c];
            rr[a] = b - y[a];
            d.r[12 * n + 3 * a + c] = rr[a];
            d.G[12 * n + 3 * a + c] = d.X[12 * n + 3 * a + c] + (wdx ? wdx[12 * n + 3 * a + c] : T(0));
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
    if (!red.run<9, double>(bar, acc, s_tmp, sums)) return;
    // CG scalars: thread 0 computes them (double), shared memory broadcasts
    double rz[3] = {sums[0], sums[1], sums[2]};
    double bb[3] = {sums[6], sums[7], sums[8]};
    if (threadIdx.x == 0) {
        double rel0 = 0.0;
        for (int c = 0; c < 3; ++c) rel0 = fmax(rel0, sqrt(sums[3 + c] / fmax(bb[c], 1e-300)));
        s_scal[4] = rel0;
    }
    __syncthreads();
    double rel = s_scal[4];
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
        if (!red.run<3, double>(bar, a3, s_tmp, s3)) return;
        if (threadIdx.x < 3) s_scal[threadIdx.x] = s3[threadIdx.x] != 0.0 ? rz[threadIdx.x] / s3[threadIdx.x] : 0.0;
        __syncthreads();
        const double al[3] = {s_scal[0], s_scal[1], s_scal[2]};
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
        if (!red.run<6, double>(bar, a6, s_tmp, s6)) return;
        ++it;
        if (threadIdx.x < 3) s_scal[8 + threadIdx.x] = rz[threadIdx.x] != 0.0 ? s6[threadIdx.x] / rz[threadIdx.x] : 0.0;
        if (threadIdx.x == 0) {
            double rel0 = 0.0;
            for (int c = 0; c < 3; ++c) rel0 = fmax(rel0, sqrt(s6[3 + c] / fmax(bb[c], 1e-300)));
            s_scal[4] = rel0;
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c) { beta_c[c] = s_scal[8 + c]; rz[c] = s6[c]; }
        rel = s_scal[4];
        __syncthreads();
    }

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->pcg_iters = it;
        st->pcg_res = rel;
    }
}


// ---------------------------------------------------------------------------
// Cluster variant: one thread-block cluster of C CTAs (C <= 16) solves the
// system. Each CTA keeps the K rows of its nodes, their block-Jacobi
// inverses and a window of the preconditioned residual (its own rows and
// copies of the neighbouring CTAs' rows its K rows reference, pushed by bulk
// asynchronous copies) in shared memory; the single reduction of each
// iteration uses the hardware cluster barrier, so an iteration touches no
// global memory. Used when the node count and the K rows fit (chosen at
// creation).
// ---------------------------------------------------------------------------
constexpr int kClusterThreads = 768;
constexpr int kClusterWarps = kClusterThreads / 32;

// Cluster-wide sums of K3 values per node and column: value j of column c
// is total 3 j + c. The thread of node ln and column c (four threads per
// node, the fourth without values) adds its values in three steps, each a
// fixed-shape tree, so every thread of every CTA gets bitwise the same sums
// on every run:
//  1. within the warp over its 8 nodes (shuffles across lanes 4k + c): lane
//     c < 3 then holds the warp's sums for column c and stores them;
//  2. over the warps of the CTA, one warp per total (K warps), which pushes
//     the CTA's sum into a slot of every CTA's shared memory before the
//     cluster barrier (push-based: after it each CTA reads local memory);
//  3. over the CTAs, again one warp per total, then a CTA barrier, after
//     which every thread reads the totals.
// One warp per total keeps the shuffle count of a reduction at about
// (3 K3 x warps + 10 K): the shuffle unit is shared by the CTA's 24 warps.
constexpr int kClusterMaxCtas = kNrrClusterMaxCtas;
// the block-Jacobi inverses are symmetric: their upper triangles (10 values)
// at a stride of 12 elements of T per node, which puts the float rows of 8
// consecutive nodes in distinct banks
constexpr int kMStride = 12;
__host__ __device__ constexpr int sym4u(int a, int t) { return a == 0 ? t : a == 1 ? 3 + t : a == 2 ? 5 + t : 9; }
// index of entry (a, t) of a symmetric 4x4 matrix in its packed upper triangle
__host__ __device__ constexpr int sym4(int a, int t) {
    return a > t ? sym4u(t, a) : sym4u(a, t);
}

// mbarrier and bulk-copy primitives (PTX) for the halo exchange
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ unsigned cluster_addr(const void* p, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
// bulk copy of `bytes` (a multiple of 16, 16-byte aligned ends) from this
// CTA's shared memory to another CTA's, completing on that CTA's mbarrier
__device__ __forceinline__ void bulk_push(unsigned dst, unsigned src, unsigned bytes, unsigned mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "r"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
// the halo copies of a CTA, precomputed: {destination, source, bytes,
// destination mbarrier} towards CTA r-1, then the same towards CTA r+1
// (bytes 0: no copy). The generic-proxy writes of the rows are made visible
// to the bulk copies first.
__device__ __forceinline__ void issue_halo(const unsigned* sp) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (sp[2]) bulk_push(sp[0], sp[1], sp[2], sp[3]);
    if (sp[6]) bulk_push(sp[4], sp[5], sp[6], sp[7]);
}

template <typename R>
struct ClusterSum {
    R* s_red;   // [2][kClusterMaxCtas][kMaxRed], written by every CTA
    R* s_tmp;   // [kClusterWarps][kMaxRed]: per-warp sums
    R* s_tot;   // [kMaxRed]: cluster totals
    int buf;
    int active_warps;   // warps whose threads may hold non-zero values
    const int* s_bad;   // set: this CTA failed; total 0 becomes NaN
    template <int K3>
    __device__ __forceinline__ void run(bool has, int c, const R (&v)[K3], R (&out)[3 * K3]) {
        constexpr int K = 3 * K3;
        static_assert(K <= kMaxRed && K <= kClusterWarps, "reduction size");
        cg::cluster_group cl = cg::this_cluster();
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (w < active_warps) {
            R x[K3];
#pragma unroll
            for (int j = 0; j < K3; ++j) x[j] = has ? v[j] : R(0);
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
#pragma unroll
                for (int j = 0; j < K3; ++j) x[j] += __shfl_xor_sync(0xffffffffu, x[j], o);
            }
            if (lane < 3) {
#pragma unroll
                for (int j = 0; j < K3; ++j) s_tmp[w * kMaxRed + 3 * j + lane] = x[j];
            }
        }
        __syncthreads();
        const int nr = (int)cl.num_blocks();
        if (w < K) {
            R y = lane < active_warps ? s_tmp[lane * kMaxRed + w] : R(0);
            if (w == 0 && s_bad != nullptr && *(volatile const int*)s_bad) y = (R)__int_as_float(0x7fc00000);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane < nr)
                cl.map_shared_rank(s_red, lane)[(buf * kClusterMaxCtas + (int)cl.block_rank()) * kMaxRed + w] = y;
        }
        cl.sync();   // release/acquire: every CTA's slot is written
        if (w < K) {
            R z = lane < nr ? s_red[(buf * kClusterMaxCtas + lane) * kMaxRed + w] : R(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
            if (lane == 0) s_tot[w] = z;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K; ++j) out[j] = s_tot[j];
        buf ^= 1;
    }
};

// Waits (every thread) for phase `parity` of the halo mbarrier, whose
// arrival thread 0 arms with the bytes the CTA receives. Bounded: if the
// rows have not all arrived after about two seconds, the thread records
// NRR_E_TIMEOUT in the state and marks the CTA failed (*bad); the next
// cluster reduction then carries NaN, so every CTA leaves the solve at the
// same point (the failed CTA arms and waits on the mbarrier no more: the
// solve ends at that reduction, before the next wait). Returns whether the
// rows arrived.
__device__ __forceinline__ bool halo_wait(unsigned long long* bar, unsigned parity, unsigned bytes, int* bad,
                                          NrrState* st) {
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, bytes);
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kSpinLimit) {
            atomicExch(&st->status, (int)NRR_E_TIMEOUT);
            *(volatile int*)bad = 1;
            return false;
        }
    }
    return true;
}

// One connected component of the node graph (warp-wide, all 32 lanes): if
// no node of it has alignment weight (anode == 0 for all), shift its nodes'
// translations in G so that their sum is that of X^(k), and count it.
template <typename T>
__device__ __forceinline__ void free_component(const DevProblem<T>& d, int comp, int lane) {
    const int c0 = d.comp_ptr[comp], c1 = d.comp_ptr[comp + 1];
    // weighted as soon as one node is (almost always in the first chunk)
    for (int k0 = c0; k0 < c1; k0 += 32) {
        const int k = k0 + lane;
        if (__any_sync(0xffffffffu, k < c1 && d.anode[d.comp_nodes[k]] != T(0))) return;
    }
    double sh[3] = {0.0, 0.0, 0.0};
    for (int k = c0 + lane; k < c1; k += 32) {
        const int j = d.comp_nodes[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) sh[a] += (double)d.G[12 * j + 9 + a] - (double)d.X[12 * j + 9 + a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sh[a] += __shfl_xor_sync(0xffffffffu, sh[a], o);
        sh[a] /= (double)(c1 - c0);
    }
    for (int k = c0 + lane; k < c1; k += 32) {
        const int j = d.comp_nodes[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) d.G[12 * j + 9 + a] = (T)((double)d.G[12 * j + 9 + a] - sh[a]);
    }
    if (lane == 0) atomicAdd(&d.st->n_singular, 1);
}

template <typename T>
__global__ void __launch_bounds__(kClusterThreads, 1)
    solve_cluster_kernel(DevProblem<T> d, int cap, NrrHaloWin win) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ T t_red[2 * kClusterMaxCtas * kMaxRed];
    __shared__ T t_tmp[kClusterWarps * kMaxRed];
    __shared__ T t_tot[kMaxRed];
    __shared__ __align__(8) unsigned long long s_bar;   // halo arrivals
    __shared__ int s_halo_bad;
    __shared__ unsigned s_push[8];
    NrrState* st = d.st;
    if (st->done || st->skip) return;   // the same decision in every CTA
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, bd = blockDim.x;
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        s_halo_bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // no CTA touches another's shared memory before every CTA of the cluster
    // runs: arrive now, wait after the local setup
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    long long* ts = (d.solve_stats != nullptr && blockIdx.x == 0 && threadIdx.x == 0) ? d.solve_stats : nullptr;
    int tsn = 0;
    auto stamp = [&]() { if (ts && tsn < 64) ts[tsn++] = clock64(); };
    stamp();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int N = d.N;
    const int per = (N + C - 1) / C;
    const int n0 = min(N, rank * per), n1 = min(N, n0 + per);
    const int cnt = n1 - n0;
    const int b0 = d.bsr_ptr[n0];
    const int nbl = d.bsr_ptr[n1] - b0;
    const int hmax = win.hmax;
    // this CTA's window, and the rows it pushes to CTA r-1 and CTA r+1
    int hlo = 0, hhi = 0, h_dn = 0, h_up = 0;
#pragma unroll
    for (int k = 0; k < kClusterMaxCtas; ++k) {
        if (k == rank) { hlo = win.lo[k]; hhi = win.hi[k]; }
        if (k == rank - 1) h_dn = win.hi[k];
        if (k == rank + 1) h_up = win.lo[k];
    }
    // shared layout (identical offsets in every CTA): K rows; the window of
    // u = M^-1 r (hmax halo rows, the CTA's own rows, hmax halo rows); preconditioner
    // blocks; per K block the window row of its column, or the owner rank
    // and local node of a column outside the window (bit 15 set)
    T* Kloc = reinterpret_cast<T*>(smem);
    T* zwin = Kloc + (size_t)cap * 16;
    T* zloc = zwin + (size_t)12 * hmax;
    T* Mloc = zwin + (size_t)12 * (2 * hmax + per);
    unsigned short* colloc = reinterpret_cast<unsigned short*>(Mloc + (size_t)per * kMStride);
    {
        // the K rows of this CTA's nodes, as 16-byte vectors, vector-major
        using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int kVpb = (int)sizeof(T);   // 16-byte vectors per 4x4 block
        const int nv = nbl * kVpb;
        const V4* src = reinterpret_cast<const V4*>(d.Kv + (size_t)b0 * 16);
        V4* dst = reinterpret_cast<V4*>(Kloc);
#pragma unroll 4
        for (int k = tid; k < nv; k += bd) dst[(size_t)(k % kVpb) * cap + k / kVpb] = __ldg(src + k);
    }
    for (int k = tid; k < nbl; k += bd) {
        const int col = d.bsr_col[b0 + k];
        unsigned short code;
        if (col >= n0 - hlo && col < n1 + hhi) {
            code = (unsigned short)(hmax + col - n0);
        } else {
            const int owner = col / per;
            code = (unsigned short)(0x8000u | ((unsigned)owner << 8) | (unsigned)(col - owner * per));
        }
        colloc[k] = code;
    }
    __syncthreads();
    for (int n = n0 + tid; n < n1; n += bd) {
        int bdg = d.bsr_ptr[n] - b0;
        while ((int)d.bsr_col[b0 + bdg] != n) ++bdg;
        // the preconditioner only steers CG: its inverse is formed in T
        T A[16], I[16];
        for (int a = 0; a < 4; ++a) {
            T k4[4];
            krow(Kloc, cap, bdg, a, k4);
            for (int t = 0; t < 4; ++t) A[4 * a + t] = k4[t];
        }
        if (!spd_inverse4(A, I)) {
            for (int t = 0; t < 16; ++t) I[t] = 0;
            for (int t = 0; t < 4; ++t) I[5 * t] = A[5 * t] > T(0) ? T(1) / A[5 * t] : T(1);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int t = a; t < 4; ++t) Mloc[kMStride * (n - n0) + sym4(a, t)] = I[4 * a + t];
    }
    __syncthreads();

    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    stamp();
    // halo exchange: once the CTA's new rows of u are written (after a CTA
    // barrier, lane 0 of the last warp) push the first hi[r-1] rows to CTA
    // r-1 and the last lo[r+1] rows to CTA r+1, with the copy descriptors
    // precomputed here; before the halo columns of each SpMV wait for the
    // rows this CTA receives (phase k of its mbarrier carries the halo of the
    // k-th u)
    const unsigned row_bytes = 12u * (unsigned)sizeof(T);
    const unsigned in_bytes = (unsigned)(hlo + hhi) * row_bytes;
    const int cnt_prev = rank > 0 ? min(N, rank * per) - min(N, (rank - 1) * per) : 0;
    unsigned long long* bar = &s_bar;
    if (tid == 0) {
        s_push[2] = s_push[6] = 0;
        if (h_dn > 0) {
            s_push[0] = cluster_addr(zwin + (size_t)12 * (hmax + cnt_prev), rank - 1);
            s_push[1] = smem_u32(zloc);
            s_push[2] = (unsigned)h_dn * row_bytes;
            s_push[3] = cluster_addr(bar, rank - 1);
        }
        if (h_up > 0) {
            s_push[4] = cluster_addr(zwin + (size_t)12 * (hmax - h_up), rank + 1);
            s_push[5] = smem_u32(zloc + (size_t)12 * (cnt - h_up));
            s_push[6] = (unsigned)h_up * row_bytes;
            s_push[7] = cluster_addr(bar, rank + 1);
        }
    }
    unsigned hphase = 0;
    // warps that hold work: four threads per node in the SpMV and the updates
    const int active_warps = min((int)(bd >> 5), (cnt * 4 + 31) / 32);
    ClusterSum<T> red{t_red, t_tmp, t_tot, 0, max(active_warps, 1), &s_halo_bad};
    const T tol = d.pcg_tol;
    // four threads per node: in the SpMV each takes every fourth block of
    // the node's row for all three columns; in the CG updates thread s < 3
    // owns column c = s of the node
    const int s4 = tid & 3;
    const bool node_ok = (tid >> 2) < cnt;
    const bool has = node_ok && s4 < 3;
    const int ln = node_ok ? tid >> 2 : 0;
    const int n = n0 + ln, c = s4 < 3 ? s4 : 0;
    const int rb0 = node_ok ? d.bsr_ptr[n] - b0 : 0, rb1 = node_ok ? d.bsr_ptr[n + 1] - b0 : 0;
    const T* Mi = Mloc + kMStride * ln;
    // window rows of this CTA's own nodes
    const unsigned own_lo = (unsigned)hmax, own_hi = (unsigned)(hmax + cnt);

    // Preconditioned CG in the form of Chronopoulos and Gear (J. Comput.
    // Appl. Math. 25, 1989), which has the iterates of PCG in exact
    // arithmetic: with u = M^-1 r and w = K u,
    //   gamma = r.u, delta = w.u, beta = gamma / gamma_old,
    //   alpha = gamma / (delta - beta gamma / alpha_old),
    //   p = u + beta p, s = w + beta s (= K p), x += alpha p, r -= alpha s.
    // One cluster-wide reduction per iteration (gamma, delta, r.r of the
    // three columns, after the SpMV). u reaches the neighbours by the halo
    // copies, pushed as soon as it is written; the SpMV takes the columns of
    // the CTA's own nodes first and waits for the halo before the others.
    // Without full windows (some column read from its owner CTA) a cluster
    // barrier publishes u before the SpMV.
    T x[4] = {0, 0, 0, 0}, r[4] = {0, 0, 0, 0}, p[4] = {0, 0, 0, 0}, sv[4] = {0, 0, 0, 0};
    T u[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
    const bool full = win.full != 0;
    // failure-detection test knob (host side): CTA 1 does not push the halo
    // of the first u, so its neighbours' bounded waits run out
    const bool skip_push = d.fault_halo != 0 && rank == 1;

    // u = M^-1 r for the node's column, into the CTA's window rows; then the
    // halo push and the SpMV w = K u (this thread's share of the row's
    // blocks, all three columns, 16-byte loads of K and u rows; the node's
    // four partial results added by shuffles)
#define NRR_CG_PRECONDITION()                                                                               \
    if (has) {                                                                                              \
        _Pragma("unroll") for (int a = 0; a < 4; ++a) {                                                     \
            u[a] = Mi[sym4(a, 0)] * r[0] + Mi[sym4(a, 1)] * r[1] + Mi[sym4(a, 2)] * r[2] + Mi[sym4(a, 3)] * r[3]; \
            zloc[12 * ln + 3 * a + c] = u[a];                                                               \
        }                                                                                                   \
    }
    // the row's blocks are sorted by column: those of the CTA's own nodes
    // form one range [ob0, ob1) of it
    int ob0 = rb0, ob1 = rb0;
    {
        int b = rb0;
        while (b < rb1 && !(colloc[b] >= own_lo && colloc[b] < own_hi)) ++b;
        ob0 = b;
        while (b < rb1 && colloc[b] >= own_lo && colloc[b] < own_hi) ++b;
        ob1 = b;
    }
    // this thread's blocks (every fourth from rb0 + s4) in [from, to)
    auto first_at = [&](int from) {
        const int b = rb0 + s4;
        return b >= from ? b : b + ((from - b + 3) >> 2) * 4;
    };
    auto spmv_range = [&](int from, int to, T (&wv)[12]) {
        for (int b = first_at(from); b < to; b += 4) {
            const unsigned cw = colloc[b];
            const T* zp = (cw & 0x8000u) ? cl.map_shared_rank(zloc, (int)((cw >> 8) & 15u)) + 12 * (cw & 0xffu)
                                         : zwin + 12 * cw;
            T zr[12];
#pragma unroll
            for (int k = 0; k < 12; k += 4) {
                T t4[4];
                load4(zp + k, t4);
                zr[k] = t4[0]; zr[k + 1] = t4[1]; zr[k + 2] = t4[2]; zr[k + 3] = t4[3];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T k4[4];
                krow(Kloc, cap, b, a, k4);
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    wv[3 * a + cc] += k4[0] * zr[cc] + k4[1] * zr[3 + cc] + k4[2] * zr[6 + cc] + k4[3] * zr[9 + cc];
            }
        }
    };
#define NRR_CG_SPMV()                                                                  \
    {                                                                                  \
        __syncthreads(); /* every thread's u rows are written */                     \
        if (tid == bd - 32 && !(skip_push && hphase == 0)) issue_halo(s_push);         \
        if (!full) cl.sync(); /* u rows read from their owners */                      \
        T wv[12];                                                                      \
        _Pragma("unroll") for (int k = 0; k < 12; ++k) wv[k] = 0;                    \
        spmv_range(ob0, ob1, wv);                                                      \
        halo_wait(bar, hphase & 1u, in_bytes, &s_halo_bad, st);                        \
        ++hphase;                                                                      \
        spmv_range(rb0, ob0, wv);                                                      \
        spmv_range(ob1, rb1, wv);                                                      \
        _Pragma("unroll") for (int k = 0; k < 12; ++k) {                               \
            wv[k] += __shfl_xor_sync(0xffffffffu, wv[k], 1);                           \
            wv[k] += __shfl_xor_sync(0xffffffffu, wv[k], 2);                           \
        }                                                                              \
        _Pragma("unroll") for (int a = 0; a < 4; ++a) w[a] = wv[3 * a + c];            \
    }

    // start: x = X^(k) (+ the previous MM step), r = B - K x, u = M^-1 r,
    // w = K u
    const T* wdx = (d.warm_dx != nullptr && d.st->n_solves_stage > 0) ? d.warm_dx : nullptr;
    T bb = 0;
    if (has) {
        T y[4] = {0, 0, 0, 0};
        for (int b = rb0; b < rb1; ++b) {
            const int k = d.bsr_col[b0 + b];
            T v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) v[t] = d.X[12 * k + 3 * t + c] + (wdx ? wdx[12 * k + 3 * t + c] : T(0));
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T k4[4];
                krow(Kloc, cap, b, a, k4);
                y[a] += k4[0] * v[0] + k4[1] * v[1] + k4[2] * v[2] + k4[3] * v[3];
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const T bv = d.Bv[12 * n + 3 * a + c];
            x[a] = d.X[12 * n + 3 * a + c] + (wdx ? wdx[12 * n + 3 * a + c] : T(0));
            r[a] = bv - y[a];
            bb += bv * bv;
        }
    }
    NRR_CG_PRECONDITION()
    stamp();
    NRR_CG_SPMV()
    // per column: r.u, w.u, r.r, B.B
    T acc4[4] = {0, 0, 0, 0}, s12[12];
    if (has) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            acc4[0] += r[a] * u[a];
            acc4[1] += w[a] * u[a];
            acc4[2] += r[a] * r[a];
        }
        acc4[3] = bb;
    }
    stamp();
    red.template run<4>(has, c, acc4, s12);
    stamp();
    const T bbc[3] = {s12[9] > T(0) ? s12[9] : T(1e-30), s12[10] > T(0) ? s12[10] : T(1e-30),
                      s12[11] > T(0) ? s12[11] : T(1e-30)};
    const T tol2 = tol * tol;
    // converged when every column has |r|^2 <= tol^2 |B|^2
    // a failed CTA (NaN in the sum of column 0) ends the solve everywhere
    const bool failed0 = s12[0] != s12[0];
    bool done = failed0 || (s12[6] <= tol2 * bbc[0] && s12[7] <= tol2 * bbc[1] && s12[8] <= tol2 * bbc[2]);
    T relmax2 = fmax(fmax(s12[6] / bbc[0], s12[7] / bbc[1]), s12[8] / bbc[2]);
    // this thread's column: gamma, alpha, beta
    T gam = pick3(s12, c);
    T dl0 = pick3(s12 + 3, c);
    T alph = dl0 != T(0) ? gam / dl0 : T(0), beta = 0;
    int it = 0;
    while (!done && it < d.pcg_max) {
        if (has) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                p[a] = u[a] + beta * p[a];
                sv[a] = w[a] + beta * sv[a];
                x[a] += alph * p[a];
                r[a] -= alph * sv[a];
            }
        }
        NRR_CG_PRECONDITION()
        if (it < 8) stamp();
        NRR_CG_SPMV()
        T a3[3] = {0, 0, 0}, s9[9];
        if (has) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                a3[0] += r[a] * u[a];
                a3[1] += w[a] * u[a];
                a3[2] += r[a] * r[a];
            }
        }
        if (it < 8) stamp();
        red.template run<3>(has, c, a3, s9);   // also: every CTA finished its SpMV
        if (it < 8) stamp();
        ++it;
        if (s9[0] != s9[0]) break;   // a CTA failed (or the recurrence broke down)
        done = s9[6] <= tol2 * bbc[0] && s9[7] <= tol2 * bbc[1] && s9[8] <= tol2 * bbc[2];
        relmax2 = fmax(fmax(s9[6] / bbc[0], s9[7] / bbc[1]), s9[8] / bbc[2]);
        const T gn = pick3(s9, c), dn = pick3(s9 + 3, c);
        const T be = gam != T(0) ? gn / gam : T(0);
        const T den = dn - (alph != T(0) ? be * gn / alph : T(0));
        beta = be;
        alph = den > T(0) ? gn / den : T(0);
        gam = gn;
    }
#undef NRR_CG_SPMV
#undef NRR_CG_PRECONDITION
    if (s_halo_bad) {
        // rows pushed to this CTA may still be in flight: let them land (a
        // bounded pause) before the cluster's CTAs leave
        const long long t0 = clock64();
        while (clock64() - t0 < 200000LL) {
        }
    }
    if (has) {
#pragma unroll
        for (int a = 0; a < 4; ++a) d.G[12 * n + 3 * a + c] = x[a];
    }
    if (rank == 0 && tid == 0) {
        st->pcg_iters = it;
        st->pcg_res = sqrt((double)relmax2);
    }
    stamp();
    if (ts) ts[63] = tsn;
    // no CTA may leave while another can still read its shared memory; the
    // barrier also publishes every CTA's G to the others
    cl.sync();
    // singular K (the free-translation fix of free_translation_kernel,
    // here for the passes' solves): one warp of the cluster per component
    if (d.fix_free && st->status == 0) {
        const int nwc = bd >> 5;
        for (int comp = rank * nwc + (tid >> 5); comp < d.n_comp; comp += C * nwc) free_component(d, comp, tid & 31);
    }
}

// ---------------------------------------------------------------------------
// Singular K (the paper is silent on it): a connected component of the node
// graph on which no point has alignment weight (every node's alignment part
// of its (t, t) entry of K, sum_i w^a_i w_ij^2, is exactly 0: the Welsch
// weights of all the points it influences underflowed) leaves the
// surrogate independent of the component's common translation, since
// D_ij does not change when t_i and t_j move together. K is then singular
// along that translation and the PCG solve leaves it (nearly) where the
// warm start X^(k) had it. This kernel fixes it exactly: G keeps the
// component's summed translation of X^(k),
//     t_j(G) -= (1/|C|) sum_{k in C} (t_k(G) - t_k(X^(k)))   for j in C,
// the minimiser of the surrogate whose update has no part along the null
// space. One warp per component; fixed-order sums; counts the components.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) free_translation_kernel(DevProblem<T> d) {
    NrrState* st = d.st;
    if (st->done || st->skip || st->status != 0) return;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int comp = gwarp; comp < d.n_comp; comp += nwarps) free_component(d, comp, lane);
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_free_translation(const DevProblem<T>& d, cudaStream_t s) {
    if (d.n_comp < 1) return cudaSuccess;
    const int grid = (d.n_comp + 7) / 8;
    free_translation_kernel<T><<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t nrr_launch_free_translation<float>(const DevProblem<float>&, cudaStream_t);
template cudaError_t nrr_launch_free_translation<double>(const DevProblem<double>&, cudaStream_t);

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

template <typename T>
size_t nrr_solve_cluster_smem(int cap, int per, int hmax) {
    return (size_t)cap * 16 * sizeof(T) + (size_t)(per + 2 * hmax) * 12 * sizeof(T) +
           (size_t)per * kMStride * sizeof(T) + (size_t)cap * sizeof(unsigned short) + 16;
}

// Prepares the cluster kernel for C CTAs with the given shared memory;
// returns the number of clusters that can be co-resident (0: not usable).
template <typename T>
size_t nrr_solve_cluster_static_smem() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, solve_cluster_kernel<T>) != cudaSuccess) {
        cudaGetLastError();
        return (size_t)1 << 30;
    }
    return fa.sharedSizeBytes;
}

// The dynamic shared-memory limit of the kernel is set to the largest value
// the device allows (a permission, identical for every context), so contexts
// with different needs can coexist; the amount used is given per launch.
template <typename T>
int nrr_solve_cluster_setup(int C, size_t smem, size_t optin) {
    const size_t max_dyn = optin - nrr_solve_cluster_static_smem<T>();
    cudaError_t e = cudaFuncSetAttribute(solve_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) { cudaGetLastError(); return 0; }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    e = cudaOccupancyMaxActiveClusters(&nc, solve_cluster_kernel<T>, &cfg);
    if (e != cudaSuccess) { cudaGetLastError(); return 0; }
    return nc;
}

template <typename T>
cudaError_t nrr_launch_solve_cluster(const DevProblem<T>& d, int C, int cap, const NrrHaloWin& win, size_t smem,
                                     cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, solve_cluster_kernel<T>, d, cap, win);
}

int nrr_solve_cluster_threads() { return kClusterThreads; }

template size_t nrr_solve_cluster_smem<float>(int, int, int);
template size_t nrr_solve_cluster_smem<double>(int, int, int);
template int nrr_solve_cluster_setup<float>(int, size_t, size_t);
template int nrr_solve_cluster_setup<double>(int, size_t, size_t);
template size_t nrr_solve_cluster_static_smem<float>();
template size_t nrr_solve_cluster_static_smem<double>();
template cudaError_t nrr_launch_solve_cluster<float>(const DevProblem<float>&, int, int, const NrrHaloWin&, size_t,
                                                     cudaStream_t);
template cudaError_t nrr_launch_solve_cluster<double>(const DevProblem<double>&, int, int, const NrrHaloWin&, size_t,
                                                      cudaStream_t);
