// Deformation (Eq. deformed_position) fused with the exact closest-point
// search rho(i) = argmin_u |u - v_hat_i| of Sec. 3.2 (Algorithm 2, first step
// of each pass), plus the stopping test of Algorithm 2.
//
// Design: one warp serves consecutive source points along a Hilbert
// curve. The target is sorted along the same curve into 32-point leaves with
// AABBs, and leaves into 32-leaf super tiles. Each lane starts from the distance to its
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
// leaves staged per batch (independent asynchronous copies); 32 KiB of
// shared memory per CTA for float points, 32 KiB for double points
template <typename T>
struct Batch { static constexpr int value = sizeof(T) == 4 ? 8 : 4; };

// 16-byte global->shared asynchronous copy (cp.async, cached in L2 only:
// a staged point is read once, from shared memory, and L1 is kept for the
// tile and leaf boxes) and the wait for all of a thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void stage_point(TPoint<float>* dst, const TPoint<float>* src) {
    cp_async16(dst, src);
}
__device__ __forceinline__ void stage_point(TPoint<double>* dst, const TPoint<double>* src) {
    cp_async16(dst, src);
    cp_async16(reinterpret_cast<char*>(dst) + 16, reinterpret_cast<const char*>(src) + 16);
}

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

template <typename T>
__device__ __forceinline__ T sqdist(T ax, T ay, T az, T bx, T by, T bz) {
    T dx = ax - bx, dy = ay - by, dz = az - bz;
    return dx * dx + dy * dy + dz * dz;
}

// Group arg-min over the LPQ lanes that share a query: smallest distance,
// ties to the lowest caller index.
template <typename T, int LPQ>
__device__ __forceinline__ void group_argmin(T& best, int& bidx, T& bx, T& by, T& bz) {
#pragma unroll
    for (int o = LPQ / 2; o > 0; o >>= 1) {
        const T od = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        const T ox = __shfl_xor_sync(0xffffffffu, bx, o);
        const T oy = __shfl_xor_sync(0xffffffffu, by, o);
        const T oz = __shfl_xor_sync(0xffffffffu, bz, o);
        if (od < best || (od == best && oi < bidx)) { best = od; bidx = oi; bx = ox; by = oy; bz = oz; }
    }
}

// Float path: a candidate is the 64-bit key (bits of d^2 << 32 | caller
// index); for d^2 >= 0 the bits of a float order like its value, so the
// smallest key is the smallest distance with ties to the lowest index. The
// winner's coordinates are fetched once at the end from its slot in the
// target array (slot -1: the initial candidate, whose coordinates are known).
__device__ __forceinline__ unsigned long long cand_key(float dd, int idx) {
    return ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned)idx;
}

template <int LPQ>
__device__ __forceinline__ void group_argmin_key(unsigned long long& key, int& pos) {
#pragma unroll
    for (int o = LPQ / 2; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int op = __shfl_xor_sync(0xffffffffu, pos, o);
        if (ok < key) { key = ok; pos = op; }
    }
}

template <typename T, int LPQ>
__device__ __forceinline__ T group_min(T v) {
#pragma unroll
    for (int o = LPQ / 2; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        v = ov < v ? ov : v;
    }
    return v;
}

// LPQ lanes serve one query: a warp serves 32 / LPQ curve-consecutive source
// points, and each lane scans 32 / LPQ of the 32 points of every leaf that
// its query needs. Splitting a query over several lanes shortens the serial
// work of the slowest warps (queries far from the target, e.g. over holes),
// and fewer queries per warp keep the warp's candidate set tight.
template <typename T, int MODE, int LPQ>
__global__ void __launch_bounds__(kThreads) nn_kernel(DevProblem<T> d) {
    constexpr int QPW = 32 / LPQ;   // queries per warp
    constexpr int PPL = 32 / LPQ;   // points of a leaf per lane
    constexpr int kBatch = Batch<T>::value;
    __shared__ TPoint<T> tile[kWarps][kBatch][32];
    __shared__ float s_gb[kWarps][4][8];
    __shared__ double s_disp[kWarps];
    __shared__ int s_last;
    NrrState* st = d.st;
    if (MODE == NRR_MODE_PASS && st->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane % LPQ;
    const int P = d.P;
    const int i = (blockIdx.x * kWarps + warp) * QPW + lane / LPQ;
    const bool valid = i < P;
    const long long t_start = clock64();
    unsigned n_super = 0, n_staged = 0, n_scanned = 0;

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
    // float path: packed key and slot of the best candidate
    unsigned long long bkey = sizeof(T) == 4 && valid ? cand_key((float)best, bidx) : 0ull;
    int bpos = -1;
    T gbest = best;   // best over the lanes of the query (pruning bound)
    // lane query box (float, rounded outwards) and the warp's query box
    const float lx = valid ? lo_f(qx) : INFINITY, ly = valid ? lo_f(qy) : INFINITY,
                lz = valid ? lo_f(qz) : INFINITY;
    const float hx = valid ? hi_f(qx) : -INFINITY, hy = valid ? hi_f(qy) : -INFINITY,
                hz = valid ? hi_f(qz) : -INFINITY;
    // boxes of the four 8-lane groups of the warp and their largest bounds,
    // kept in shared memory: a super tile or leaf is a candidate if it comes
    // within the bound of any group's box
    {
        float g[6] = {lx, ly, lz, hx, hy, hz};
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) g[k] = fminf(g[k], __shfl_xor_sync(0xffffffffu, g[k], o));
#pragma unroll
            for (int k = 3; k < 6; ++k) g[k] = fmaxf(g[k], __shfl_xor_sync(0xffffffffu, g[k], o));
        }
        if ((lane & 7) == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) s_gb[warp][lane >> 3][k] = g[k];
        }
    }
    const bool any_valid = __ballot_sync(0xffffffffu, valid) != 0;
    auto refresh_bounds = [&]() {
        float u = valid ? ub_f(gbest) : 0.f;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) u = fmaxf(u, __shfl_xor_sync(0xffffffffu, u, o));
        if ((lane & 7) == 0) s_gb[warp][lane >> 3][6] = u;
        __syncwarp();
    };
    auto candidate = [&](const float* box) {
        bool c = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float* gk = s_gb[warp][k];
            c = c || box_gap2(gk[0], gk[1], gk[2], gk[3], gk[4], gk[5], box) <= gk[6];
        }
        return c;
    };
    refresh_bounds();

    if (any_valid) {
        for (int s0 = 0; s0 < d.n_supers; s0 += 32) {
            const int s = s0 + lane;
            bool sc = s < d.n_supers && candidate(d.super_box + 6 * s);
            unsigned smask = __ballot_sync(0xffffffffu, sc);
            while (smask) {
                const int sb = __ffs(smask) - 1;
                smask &= smask - 1;
                const int base = (s0 + sb) * 32;
                ++n_super;
                // lane l holds the box of leaf base + l
                float bl[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
                bool lc = false;
                if (base + lane < d.n_leaves) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) bl[k] = d.leaf_box[6 * (base + lane) + k];
                    lc = candidate(bl);
                }
                unsigned lmask = __ballot_sync(0xffffffffu, lc);
                while (lmask) {
                    // up to kBatch leaves that some query of the warp needs
                    int ids[kBatch];
                    int cnt = 0;
                    while (lmask && cnt < kBatch) {
                        const int lb = __ffs(lmask) - 1;
                        lmask &= lmask - 1;
                        float b6[6];
#pragma unroll
                        for (int k = 0; k < 6; ++k) b6[k] = __shfl_sync(0xffffffffu, bl[k], lb);
                        const bool need = valid && box_gap2(lx, ly, lz, hx, hy, hz, b6) <= ub_f(gbest);
                        if (__ballot_sync(0xffffffffu, need)) ids[cnt++] = lb;
                    }
                    // stage them with independent asynchronous copies
                    n_staged += cnt;
#pragma unroll
                    for (int k = 0; k < kBatch; ++k)
                        if (k < cnt) stage_point(&tile[warp][k][lane], d.tpts + (size_t)(base + ids[k]) * 32 + lane);
                    cp_async_wait_all();
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < kBatch; ++k) {
                        if (k >= cnt) break;
                        float b6[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) b6[q] = __shfl_sync(0xffffffffu, bl[q], ids[k]);
                        const bool need = valid && box_gap2(lx, ly, lz, hx, hy, hz, b6) <= ub_f(gbest);
                        if (__ballot_sync(0xffffffffu, need)) {
                            ++n_scanned;
                            if (need) {
#pragma unroll
                                for (int j = 0; j < PPL; ++j) {
                                    const TPoint<T> c = tile[warp][k][sub + j * LPQ];
                                    const T dd = sqdist(qx, qy, qz, c.x, c.y, c.z);
                                    if constexpr (sizeof(T) == 4) {
                                        const unsigned long long key = cand_key((float)dd, c.idx);
                                        if (key < bkey) {
                                            bkey = key;
                                            bpos = (base + ids[k]) * 32 + sub + j * LPQ;
                                        }
                                    } else {
                                        if (dd < best || (dd == best && c.idx < bidx)) {
                                            best = dd; bidx = c.idx;
                                            bx = c.x; by = c.y; bz = c.z;
                                        }
                                    }
                                }
                            }
                            if constexpr (sizeof(T) == 4) best = (T)__uint_as_float((unsigned)(bkey >> 32));
                            gbest = group_min<T, LPQ>(best);
                        }
                    }
                    __syncwarp();
                }
                refresh_bounds();
            }
        }
    }
    if constexpr (sizeof(T) == 4) {
        group_argmin_key<LPQ>(bkey, bpos);
        best = (T)__uint_as_float((unsigned)(bkey >> 32));
        bidx = (int)(unsigned)(bkey & 0xffffffffull);
        if (valid && bpos >= 0) {
            const TPoint<T> c = d.tpts[bpos];
            bx = c.x; by = c.y; bz = c.z;
        }
    } else {
        group_argmin<T, LPQ>(best, bidx, bx, by, bz);
    }
    if (d.nn_stats != nullptr && lane == 0) {
        unsigned long long* o = d.nn_stats + 4 * (size_t)(blockIdx.x * kWarps + warp);
        o[0] = (unsigned long long)(clock64() - t_start);
        o[1] = n_super; o[2] = n_staged; o[3] = n_scanned;
    }

    // ---- outputs ------------------------------------------------------------
    const int wb = (MODE == NRR_MODE_RAW) ? 0 : (st->vk ^ 1);
    double dv2 = 0.0;
    if (valid && sub == 0) {
        d.rho[i] = bidx;
        d.d2[i] = best;
        d.u[i] = bx; d.u[P + i] = by; d.u[2 * P + i] = bz;
        if (MODE != NRR_MODE_RAW) {
            T* vh = d.vhat + (size_t)wb * 3 * P;
            vh[i] = qx; vh[P + i] = qy; vh[2 * P + i] = qz;
            if (MODE == NRR_MODE_PASS && st->pending_stop && st->have_vk) {
                const T* vk = d.vhat + (size_t)(wb ^ 1) * 3 * P;
                const double dx = (double)qx - (double)vk[i];
                const double dy = (double)qy - (double)vk[P + i];
                const double dz = (double)qz - (double)vk[2 * P + i];
                dv2 = dx * dx + dy * dy + dz * dz;
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
        // with an energy test the stage ends on it (or I_max) only
        if ((st->rel_tol <= 0 && disp < st->eps) || st->n_solves_stage >= st->max_iters_stage) nrr_end_stage(st);
    }
    st->disp_bits = 0ull;
    }
}

}  // namespace

template <typename T, int LPQ>
cudaError_t launch_nn_lpq(const DevProblem<T>& d, int mode, cudaStream_t s) {
    const int per_cta = kWarps * (32 / LPQ);
    const int g = (d.P + per_cta - 1) / per_cta;
    if (g == 0) return cudaSuccess;
    switch (mode) {
        case NRR_MODE_PASS: nn_kernel<T, NRR_MODE_PASS, LPQ><<<g, kThreads, 0, s>>>(d); break;
        case NRR_MODE_EVAL: nn_kernel<T, NRR_MODE_EVAL, LPQ><<<g, kThreads, 0, s>>>(d); break;
        default: nn_kernel<T, NRR_MODE_RAW, LPQ><<<g, kThreads, 0, s>>>(d); break;
    }
    return cudaGetLastError();
}

// lanes per query: the launch tuning parameter of the search (1, 2, 4 or 8)
template <typename T>
cudaError_t nrr_launch_nn(const DevProblem<T>& d, int mode, int lanes_per_query, cudaStream_t s) {
    switch (lanes_per_query) {
        case 1: return launch_nn_lpq<T, 1>(d, mode, s);
        case 2: return launch_nn_lpq<T, 2>(d, mode, s);
        case 4: return launch_nn_lpq<T, 4>(d, mode, s);
        default: return launch_nn_lpq<T, 8>(d, mode, s);
    }
}

template cudaError_t nrr_launch_nn<float>(const DevProblem<float>&, int, int, cudaStream_t);
template cudaError_t nrr_launch_nn<double>(const DevProblem<double>&, int, int, cudaStream_t);
