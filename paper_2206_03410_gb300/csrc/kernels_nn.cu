// Deformation (Eq. deformed_position) fused with the exact closest-point
// search rho(i) = argmin_u |u - v_hat_i| of Sec. 3.2 (Algorithm 2, first step
// of each pass), plus the stopping test of Algorithm 2.
//
// Design: one warp serves 32 Morton-consecutive source points (one per
// lane). The target is Morton-sorted into 32-point leaves with AABBs, and
// leaves into 32-leaf super tiles. Each lane starts from the distance to its
// previous correspondence (an actual target point, so a valid upper bound),
// the warp tests super-tile and leaf boxes against its query box and the
// warp's largest bound, and every surviving leaf is staged in shared memory
// and scanned by the lanes whose own box bound does not exclude it. Bounds
// are evaluated in float with directed rounding (round-down for lower
// bounds, round-up for the current best), so pruning never drops a point
// that could win or tie; the distance itself is evaluated in T. Ties go to
// the lowest caller index. Work per query is a few hundred distance
// evaluations instead of T; the kernel is bound by issue slots.
#include "nrr_device.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ float lo_f(double x) { return __double2float_rd(x); }
__device__ __forceinline__ float hi_f(double x) { return __double2float_ru(x); }
__device__ __forceinline__ float lo_f(float x) { return x; }
__device__ __forceinline__ float hi_f(float x) { return x; }

// Lower bound (rounded down) of the squared distance between box [alo, ahi]
// and box b = {lo x,y,z, hi x,y,z}.
__device__ __forceinline__ float box_gap2(float alox, float aloy, float aloz, float ahix,
                                          float ahiy, float ahiz, const float* b) {
    float gx = fmaxf(fmaxf(__fsub_rd(b[0], ahix), __fsub_rd(alox, b[3])), 0.f);
    float gy = fmaxf(fmaxf(__fsub_rd(b[1], ahiy), __fsub_rd(aloy, b[4])), 0.f);
    float gz = fmaxf(fmaxf(__fsub_rd(b[2], ahiz), __fsub_rd(aloz, b[5])), 0.f);
    return __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
}

// Upper bound in float of a squared distance in T, with a 2e-6 relative
// margin that covers the rounding of the float distance evaluation.
__device__ __forceinline__ float ub_f(float b) { return __fmul_ru(b, 1.000002f); }
__device__ __forceinline__ float ub_f(double b) { return __fmul_ru(__double2float_ru(b), 1.000002f); }

__device__ __forceinline__ float warp_max(float x) {
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float warp_min(float x) {
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

template <typename T>
__device__ __forceinline__ T sqdist(T ax, T ay, T az, T bx, T by, T bz) {
    T dx = ax - bx, dy = ay - by, dz = az - bz;
    return dx * dx + dy * dy + dz * dz;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) nn_kernel(DevProblem<T> d) {
    __shared__ TPoint<T> tile[kWarps][32];
    __shared__ double s_disp[kWarps];
    __shared__ int s_last;
    NrrState* st = d.st;
    if (MODE == NRR_MODE_PASS && st->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = d.P;
    const int i = (blockIdx.x * kWarps + warp) * 32 + lane;
    const bool valid = i < P;

    // ---- query point: v_hat_i (Eq. deformed_position) or v_i -------------
    T qx = 0, qy = 0, qz = 0;
    if (valid) {
        T vx = d.v[i], vy = d.v[P + i], vz = d.v[2 * P + i];
        if (MODE == NRR_MODE_RAW) {
            qx = vx; qy = vy; qz = vz;
        } else {
            const T* X = (MODE == NRR_MODE_EVAL) ? d.Xeval : d.X;
            for (int s = d.infl_ptr[i], e = d.infl_ptr[i + 1]; s < e; ++s) {
                const int j = d.infl_node[s];
                const T w = d.infl_w[s];
                const T* Xj = X + 12 * j;
                const T px = d.p[3 * j], py = d.p[3 * j + 1], pz = d.p[3 * j + 2];
                const T dx = vx - px, dy = vy - py, dz = vz - pz;
                // rows 0..2 of the block hold A_j^T, row 3 holds t_j
                const T ox = Xj[0] * dx + Xj[3] * dy + Xj[6] * dz + px + Xj[9];
                const T oy = Xj[1] * dx + Xj[4] * dy + Xj[7] * dz + py + Xj[10];
                const T oz = Xj[2] * dx + Xj[5] * dy + Xj[8] * dz + pz + Xj[11];
                qx += w * ox; qy += w * oy; qz += w * oz;
            }
        }
    }
    // ---- initial candidate: the previous correspondence --------------------
    T bx = 0, by = 0, bz = 0, best = 0;
    int bidx = 0x7fffffff;
    if (valid) {
        bx = d.u[i]; by = d.u[P + i]; bz = d.u[2 * P + i];
        bidx = d.rho[i];
        best = sqdist(qx, qy, qz, bx, by, bz);
    }
    // lane query box (float, rounded outwards) and the warp's query box
    const float lx = valid ? lo_f(qx) : INFINITY, ly = valid ? lo_f(qy) : INFINITY,
                lz = valid ? lo_f(qz) : INFINITY;
    const float hx = valid ? hi_f(qx) : -INFINITY, hy = valid ? hi_f(qy) : -INFINITY,
                hz = valid ? hi_f(qz) : -INFINITY;
    const float wlx = warp_min(lx), wly = warp_min(ly), wlz = warp_min(lz);
    const float whx = warp_max(hx), why = warp_max(hy), whz = warp_max(hz);
    const bool any_valid = __ballot_sync(0xffffffffu, valid) != 0;
    float UB = warp_max(valid ? ub_f(best) : 0.f);

    if (any_valid) {
        for (int s0 = 0; s0 < d.n_supers; s0 += 32) {
            const int s = s0 + lane;
            bool sc = s < d.n_supers &&
                      box_gap2(wlx, wly, wlz, whx, why, whz, d.super_box + 6 * s) <= UB;
            unsigned smask = __ballot_sync(0xffffffffu, sc);
            while (smask) {
                const int sb = __ffs(smask) - 1;
                smask &= smask - 1;
                const int base = (s0 + sb) * 32;
                // lane l holds the box of leaf base + l
                float bl[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
                bool lc = false;
                if (base + lane < d.n_leaves) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) bl[k] = d.leaf_box[6 * (base + lane) + k];
                    lc = box_gap2(wlx, wly, wlz, whx, why, whz, bl) <= UB;
                }
                unsigned lmask = __ballot_sync(0xffffffffu, lc);
                int lb = lmask ? __ffs(lmask) - 1 : -1;
                TPoint<T> cur;
                if (lb >= 0) cur = d.tpts[(size_t)(base + lb) * 32 + lane];
                while (lb >= 0) {
                    lmask &= lmask - 1;
                    const int nb = lmask ? __ffs(lmask) - 1 : -1;
                    TPoint<T> nxt;
                    if (nb >= 0) nxt = d.tpts[(size_t)(base + nb) * 32 + lane];   // prefetch
                    float b6[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) b6[k] = __shfl_sync(0xffffffffu, bl[k], lb);
                    const bool need = valid && box_gap2(lx, ly, lz, hx, hy, hz, b6) <= ub_f(best);
                    if (__ballot_sync(0xffffffffu, need)) {
                        tile[warp][lane] = cur;
                        __syncwarp();
                        if (need) {
#pragma unroll 8
                            for (int j = 0; j < 32; ++j) {
                                const TPoint<T> c = tile[warp][j];
                                const T dd = sqdist(qx, qy, qz, c.x, c.y, c.z);
                                if (dd < best || (dd == best && c.idx < bidx)) {
                                    best = dd; bidx = c.idx;
                                    bx = c.x; by = c.y; bz = c.z;
                                }
                            }
                        }
                        __syncwarp();
                    }
                    cur = nxt;
                    lb = nb;
                }
                UB = warp_max(valid ? ub_f(best) : 0.f);
            }
        }
    }

    // ---- outputs ------------------------------------------------------------
    const int wb = (MODE == NRR_MODE_RAW) ? 0 : (st->vk ^ 1);
    double dv2 = 0.0;
    if (valid) {
        d.rho[i] = bidx;
        d.d2[i] = best;
        d.u[i] = bx; d.u[P + i] = by; d.u[2 * P + i] = bz;
        if (MODE != NRR_MODE_RAW) {
            T* vh = d.vhat + (size_t)wb * 3 * P;
            vh[i] = qx; vh[P + i] = qy; vh[2 * P + i] = qz;
            if (MODE == NRR_MODE_PASS && st->pending_stop && st->have_vk) {
                const T* vk = d.vhat + (size_t)(wb ^ 1) * 3 * P;
                const double ex = (double)qx - (double)vk[i];
                const double ey = (double)qy - (double)vk[P + i];
                const double ez = (double)qz - (double)vk[2 * P + i];
                dv2 = ex * ex + ey * ey + ez * ez;
            }
        }
    }
    if constexpr (MODE == NRR_MODE_PASS) {
    // ---- stopping test of Algorithm 2 (max displacement) --------------------
    for (int o = 16; o > 0; o >>= 1) dv2 = fmax(dv2, __shfl_xor_sync(0xffffffffu, dv2, o));
    if (lane == 0) s_disp[warp] = dv2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = s_disp[0];
        for (int w = 1; w < kWarps; ++w) m = fmax(m, s_disp[w]);
        // non-negative doubles order like their bit patterns
        atomicMax(&st->disp_bits, (unsigned long long)__double_as_longlong(m));
        __threadfence();
        const unsigned t = atomicAdd(&st->cnt_nn, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    st->cnt_nn = 0;
    st->vlast = wb;
    if (st->pending_stop) {
        const double disp = sqrt(__longlong_as_double((long long)atomicAdd(&st->disp_bits, 0ull)));
        st->max_disp = disp;
        st->pending_stop = 0;
        if (disp < st->eps || st->n_solves_stage >= st->max_iters_stage) nrr_end_stage(st);
    }
    st->disp_bits = 0ull;
    }
}

}  // namespace

template <typename T>
cudaError_t nrr_launch_nn(const DevProblem<T>& d, int mode, int grid, cudaStream_t s) {
    (void)grid;
    const int g = (d.P + kThreads - 1) / kThreads;
    if (g == 0) return cudaSuccess;
    switch (mode) {
        case NRR_MODE_PASS: nn_kernel<T, NRR_MODE_PASS><<<g, kThreads, 0, s>>>(d); break;
        case NRR_MODE_EVAL: nn_kernel<T, NRR_MODE_EVAL><<<g, kThreads, 0, s>>>(d); break;
        default: nn_kernel<T, NRR_MODE_RAW><<<g, kThreads, 0, s>>>(d); break;
    }
    return cudaGetLastError();
}

template cudaError_t nrr_launch_nn<float>(const DevProblem<float>&, int, int, cudaStream_t);
template cudaError_t nrr_launch_nn<double>(const DevProblem<double>&, int, int, cudaStream_t);
