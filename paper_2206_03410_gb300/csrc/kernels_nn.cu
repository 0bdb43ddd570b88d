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

// The query of source point i: v_hat_i of Eq. (deformed_position) at the
// pass's iterate (or at Xeval), or v_i itself (MODE_RAW). One definition
// for both closest-point kernels, so that they see the same query bits.
template <typename T, int MODE>
__device__ __forceinline__ void query_point(const DevProblem<T>& d, int i, T& qx, T& qy, T& qz) {
    const int P = d.P;
    const T vx = d.v[i], vy = d.v[P + i], vz = d.v[2 * P + i];
    if (MODE == NRR_MODE_RAW) {
        qx = vx; qy = vy; qz = vz;
        return;
    }
    qx = 0; qy = 0; qz = 0;
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

// Outputs of a closest-point search (rho, d^2, the closest coordinates u and
// v_hat in the non-kept buffer) for the thread that owns query i (``write``),
// and in a pass the stopping test of Algorithm 2: the largest displacement
// of v_hat from the kept iterate's, reduced over the grid (the CTA's kWarps
// warps, then a 64-bit atomic max of the bits of non-negative doubles); the
// last CTA to finish ends the stage when the displacement is below eps or
// the stage has run I_max solves. Shared by both closest-point kernels (256
// threads per CTA).
template <typename T, int MODE>
__device__ __forceinline__ void search_outputs(const DevProblem<T>& d, int i, bool write, int bidx, T best, T bx,
                                               T by, T bz, T qx, T qy, T qz, double* s_disp, int* s_last) {
    NrrState* st = d.st;
    const int P = d.P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wb = (MODE == NRR_MODE_RAW) ? 0 : (st->vk ^ 1);
    double dv2 = 0.0;
    if (write) {
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
            *s_last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (!*s_last || threadIdx.x != 0) return;
        __threadfence();
        st->cnt_nn = 0;
        st->vlast = wb;
        if (st->pending_stop) {
            const double disp = sqrt(__longlong_as_double((long long)atomicAdd(&st->disp_bits, 0ull)));
            st->max_disp = disp;
            st->pending_stop = 0;
            // with an energy test the stage ends on it (or I_max) only
            if ((st->rel_tol <= 0 && disp < st->eps) || st->n_solves_stage >= st->max_iters_stage)
                nrr_end_stage(st);
        }
        st->disp_bits = 0ull;
    }
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
    if (valid) query_point<T, MODE>(d, i, qx, qy, qz);
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

    // mega tiles (32 super tiles each) first, then the super tiles of each
    // candidate mega tile: super tiles are visited in the same order as by
    // a flat scan, the tests of those whose mega tile is out of reach are
    // skipped (a mega tile's box holds its super tiles' boxes, and bounds
    // only shrink)
    for (int m0 = 0; any_valid && m0 < d.n_megas; m0 += 32) {
        const int m = m0 + lane;
        unsigned mmask = __ballot_sync(0xffffffffu, m < d.n_megas && candidate(d.mega_box + 6 * m));
        while (mmask) {
            const int s0 = (m0 + __ffs(mmask) - 1) * 32;
            mmask &= mmask - 1;
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

    // ---- outputs and the stopping test ----------------------------------------
    search_outputs<T, MODE>(d, i, valid && sub == 0, bidx, best, bx, by, bz, qx, qy, qz, s_disp, &s_last);
}

// ---------------------------------------------------------------------------
// Tensor-core candidate search (float path). The same outputs as nn_kernel,
// bit for bit: the closest point rho(i) (ties to the lowest caller index),
// its float squared distance and coordinates, v_hat and the stopping test.
//
// A CTA serves 128 curve-consecutive source points (the M = 128 rows of a
// tcgen05.mma). Its candidate target points are the union of the leaves
// that any of its sixteen 8-query boxes may need under the queries' current
// bounds (the distance to the previous correspondence), in chunks of four
// leaves (N = 128 columns). For every chunk two MMAs (kind::tf32, K = 8
// each, FP32 accumulator in tensor memory) form all 128 x 128 approximate
// squared distances at once, as one dot product of K = 16:
//   query row     [-2 x_hi, -2 x_hi, -2 x_lo, 1, 1, |x|^2_hi, |x|^2_lo, 0...]
//   candidate row [ y_hi,    y_lo,    y_hi, |y|^2_hi, |y|^2_lo, 1, 1, 0...]
// with x, y the float coordinates minus the CTA's centre and every value
// split into two TF32 parts (hi + lo), so that the product carries about 22
// significant bits: |x - y|^2 = |x|^2 + |y|^2 - 2 x.y up to
// delta = 2^-17 (|x| + R)^2, R the largest |y| among the candidates (the
// split and the FP32 accumulation err by less than a quarter of that).
// The epilogue reads each accumulator from tensor memory (tcgen05.ld) and
// keeps, per query and half of the columns, the eight smallest approximate
// distances; the halves are merged to eight, whose exact float distances
// and (d^2, caller index) keys (those of nn_kernel) are formed. With D the
// best of them, no candidate that was not kept can win when the eighth
// approximate distance exceeds D (1 + 2e-6) + delta (2e-6 covers the float
// rounding of the exact distances); a query for which this fails is
// searched exactly, alone, with nn_kernel's pruning. So the result is the
// exact search's; the tensor cores only choose where to look.
//
// Pipeline: two accumulators (256 tensor-memory columns) and two candidate
// tiles in shared memory; the MMA of chunk c runs while the epilogue reads
// chunk c - 1, and the target points of chunk c + 1 are loaded meanwhile.
// All waits on the MMA's completion are bounded: after about two seconds
// the kernel records NRR_E_TIMEOUT and finishes every query by the exact
// scan (freeing its tensor memory).
// ---------------------------------------------------------------------------
namespace tcs {
constexpr int kQ = 128;                 // queries per CTA: the MMA's M
constexpr int kN = 128;                 // candidates per chunk: the MMA's N
constexpr int kLeaves = kN / NRR_LEAF;  // leaves per chunk
constexpr int kCta = 256;               // warps w and w + 4 read the same tensor-memory lanes
constexpr int kGroups = 16;             // query boxes of 8 queries for the candidate test
constexpr int kListCap = 512;           // candidate leaves collected before they are processed
constexpr int kTop = 8;                 // best approximate candidates kept per query and half
constexpr unsigned kTmemCols = 2 * kN;  // two accumulators
constexpr float kDelta = 1.0f / 131072.0f;   // 2^-17
constexpr int kRowBytes = 64;           // 16 TF32 values per operand row
constexpr int kTileBytes = 128 * kRowBytes;
// byte offset of core matrix kc (4 TF32 values along K) of row r of a
// 128 x 16 TF32 operand tile in the tensor cores' K-major layout without
// swizzle: 8-row x 16-byte core matrices, those along K 128 bytes apart,
// row groups 512 bytes apart
__host__ __device__ constexpr int tile_off(int r, int kc) { return (r >> 3) * 512 + kc * 128 + (r & 7) * 16; }
// instruction descriptor of kind::tf32: D f32 (bits 4-5 = 1), A and B tf32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kN >> 3) << 17) |
                            ((unsigned)(kQ >> 4) << 24);
constexpr long long kSpin = 4000000000LL;   // clock64 cycles of a bounded wait

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of the K-slice starting at `start`:
// leading (K) byte offset 128, stride (8-row group) byte offset 512, the
// fixed version bits 46-48 = 1, no swizzle
__device__ __forceinline__ unsigned long long tile_desc(const void* start) {
    unsigned long long dsc = (unsigned long long)((smem_addr(start) & 0x3FFFFu) >> 4);
    dsc |= (unsigned long long)(128u >> 4) << 16;
    dsc |= (unsigned long long)(512u >> 4) << 32;
    dsc |= 1ull << 46;
    return dsc;
}

// round to TF32 (nearest, ties away), returned as a float
__device__ __forceinline__ float tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_done(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of an MMA completion barrier; false if it
// timed out (the caller records the failure).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity) {
    if (mbar_done(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_done(b, parity))
        if (clock64() - t0 > kSpin) return false;
    return true;
}

// 8 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(unsigned addr, float (&v)[8]) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// sorted insertion into a query's kTop best (approximate distance, slot)
__device__ __forceinline__ void top_insert(float (&tv)[kTop], int (&ts)[kTop], float v, int slot) {
    if (!(v < tv[kTop - 1])) return;
    tv[kTop - 1] = v;
    ts[kTop - 1] = slot;
#pragma unroll
    for (int k = kTop - 1; k > 0; --k) {
        if (tv[k] < tv[k - 1]) {
            const float fv = tv[k]; tv[k] = tv[k - 1]; tv[k - 1] = fv;
            const int fs = ts[k]; ts[k] = ts[k - 1]; ts[k - 1] = fs;
        }
    }
}

// one operand row (16 TF32 values) as four 16-byte core-matrix rows
struct Row16 {
    float v[16];
};
}  // namespace tcs

template <int MODE>
__global__ void __launch_bounds__(tcs::kCta, 2) nn_tc_kernel(DevProblem<float> d) {
    using namespace tcs;
    __shared__ __align__(1024) unsigned char sA[kTileBytes];
    __shared__ __align__(1024) unsigned char sB[2][kTileBytes];
    __shared__ int s_list[kListCap];
    __shared__ int s_slot[3][kN];          // target slot of each candidate column (-1: none), by chunk % 3
    __shared__ float s_gb[kGroups][8];     // query boxes and their bounds
    __shared__ float s_tv[kQ][kTop];       // second half's best, for the merge
    __shared__ int s_ts[kQ][kTop];
    __shared__ float s_ext[kQ / 32][6];
    __shared__ float s_ctr[3];
    __shared__ int s_cnt[kCta / 32];
    __shared__ unsigned s_Ru;              // bits of the largest candidate |y| (non-negative float)
    __shared__ unsigned s_tslot;
    __shared__ int s_fail;
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ double s_disp[kCta / 32];
    __shared__ int s_last;
    NrrState* st = d.st;
    if (MODE == NRR_MODE_PASS && st->done) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (kQ - 1);
    const bool owner = tid < kQ;           // owns query `row`; the other half helps the epilogue
    const int half = tid >> 7;
    const int P = d.P;
    const int i = blockIdx.x * kQ + row;
    const bool valid = owner && i < P;
    const bool row_valid = i < P;          // the row holds a query (either half)
    const long long t_start = clock64();

    // ---- queries and their initial candidate (the previous correspondence)
    float qx = 0.f, qy = 0.f, qz = 0.f, bx = 0.f, by = 0.f, bz = 0.f, best = 0.f;
    unsigned long long bkey = 0ull;
    int bpos = -1;
    if (valid) {
        query_point<float, MODE>(d, i, qx, qy, qz);
        bx = d.u[i]; by = d.u[P + i]; bz = d.u[2 * P + i];
        best = sqdist(qx, qy, qz, bx, by, bz);
        bkey = cand_key(best, d.rho[i]);
    }
    // ---- the CTA's centre (midpoint of its queries' box) and query boxes
    if (owner) {
        float e[6] = {valid ? qx : INFINITY, valid ? qy : INFINITY, valid ? qz : INFINITY,
                      valid ? qx : -INFINITY, valid ? qy : -INFINITY, valid ? qz : -INFINITY};
        float ub = valid ? ub_f(best) : 0.f;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) e[k] = fminf(e[k], __shfl_xor_sync(0xffffffffu, e[k], o));
#pragma unroll
            for (int k = 3; k < 6; ++k) e[k] = fmaxf(e[k], __shfl_xor_sync(0xffffffffu, e[k], o));
            ub = fmaxf(ub, __shfl_xor_sync(0xffffffffu, ub, o));
        }
        if ((lane & 7) == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) s_gb[row >> 3][k] = e[k];
            s_gb[row >> 3][6] = ub;
        }
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) e[k] = fminf(e[k], __shfl_xor_sync(0xffffffffu, e[k], o));
#pragma unroll
            for (int k = 3; k < 6; ++k) e[k] = fmaxf(e[k], __shfl_xor_sync(0xffffffffu, e[k], o));
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) s_ext[warp][k] = e[k];
        }
    }
    if (tid == 0) {
        s_Ru = 0u;
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid < 3) {
        float lo = s_ext[0][tid], hi = s_ext[0][3 + tid];
        for (int w = 1; w < kQ / 32; ++w) { lo = fminf(lo, s_ext[w][tid]); hi = fmaxf(hi, s_ext[w][3 + tid]); }
        s_ctr[tid] = 0.5f * (lo + hi);
    }
    __syncthreads();
    const unsigned taddr = s_tslot;
    const float cx = s_ctr[0], cy = s_ctr[1], cz = s_ctr[2];
    // ---- query rows of the A operand (zeros for rows without a query)
    float xn = 0.f;   // |x| of this query, for its error bound
    if (owner) {
        Row16 a;
#pragma unroll
        for (int k = 0; k < 16; ++k) a.v[k] = 0.f;
        if (valid) {
            const float x[3] = {qx - cx, qy - cy, qz - cz};
            const float nq = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            const float nh = tf32(nq);
            xn = sqrtf(nq);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float h = tf32(x[k]);
                a.v[k] = -2.f * h;
                a.v[3 + k] = -2.f * h;
                a.v[6 + k] = -2.f * tf32(x[k] - h);
            }
            a.v[9] = 1.f; a.v[10] = 1.f; a.v[11] = nh; a.v[12] = tf32(nq - nh);
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
            *reinterpret_cast<float4*>(sA + tile_off(row, kc)) =
                make_float4(a.v[4 * kc], a.v[4 * kc + 1], a.v[4 * kc + 2], a.v[4 * kc + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();

    float tv[kTop];
    int ts[kTop];
#pragma unroll
    for (int k = 0; k < kTop; ++k) { tv[k] = INFINITY; ts[k] = -1; }
    unsigned phase[2] = {0u, 0u};
    int chunk = 0;          // chunks issued so far
    int n_cand = 0;         // candidate leaves (statistics)
    bool failed = false;

    // chunks of the collected leaves. Iteration c builds the candidate rows
    // of chunk c, issues its two MMAs, loads the points of chunk c + 1 and
    // runs the epilogue of chunk c - 1 behind the MMAs: every thread reads
    // 64 accumulator columns of its query's row, 8 at a time, and keeps the
    // eight smallest. (The column slots of a chunk sit in s_slot[ch % 3]:
    // the chunk after next writes its own while a slow thread may still read
    // these.) One call site per step keeps the kernel's code small.
    auto process = [&](int nlist) {
        const int nch = (nlist + kLeaves - 1) / kLeaves;
        TPoint<float> pt{};
        int slot = -1;
        const int r = tid >> 1, hv = tid & 1;
#pragma unroll 1
        for (int c = 0; c <= nch; ++c) {
            if (c < nch) {
                // the target point of this thread's candidate row (two
                // threads per row, one per half of its 16 values)
                if (c == 0) {
                    const int li = r >> 5;
                    slot = -1;
                    if (li < nlist) {
                        const int sl = s_list[li] * NRR_LEAF + (r & 31);
                        pt = d.tpts[sl];
                        if (pt.idx != 0x7fffffff) slot = sl;   // not a padding point
                    }
                }
                const int b = chunk & 1;
                float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (slot >= 0) {
                    const float y[3] = {pt.x - cx, pt.y - cy, pt.z - cz};
                    const float ny = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
                    float h[3], l[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) { h[k] = tf32(y[k]); l[k] = tf32(y[k] - h[k]); }
                    if (hv == 0) {
                        // values 0..7: y_hi, y_lo, y_hi(0..1)
                        w[0] = h[0]; w[1] = h[1]; w[2] = h[2]; w[3] = l[0];
                        w[4] = l[1]; w[5] = l[2]; w[6] = h[0]; w[7] = h[1];
                        atomicMax(&s_Ru, __float_as_uint(sqrtf(ny)));
                    } else {
                        // values 8..15: y_hi(2), |y|^2 hi, lo, 1, 1, 0, 0, 0
                        const float nh = tf32(ny);
                        w[0] = h[2]; w[1] = nh; w[2] = tf32(ny - nh); w[3] = 1.f; w[4] = 1.f;
                    }
                }
                *reinterpret_cast<float4*>(sB[b] + tile_off(r, 2 * hv)) = make_float4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<float4*>(sB[b] + tile_off(r, 2 * hv + 1)) = make_float4(w[4], w[5], w[6], w[7]);
                if (hv == 0) s_slot[chunk % 3][r] = slot;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (tid == 0 && !s_fail) {
                    const unsigned dcol = taddr + (unsigned)(b * kN);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        // K values 8 ks .. 8 ks + 7: core matrices 2 ks and 2 ks + 1
                        const unsigned long long da = tile_desc(sA + ks * 256);
                        const unsigned long long db = tile_desc(sB[b] + ks * 256);
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                            "l"(da), "l"(db), "r"(kIdesc), "r"((unsigned)ks)
                            : "memory");
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_addr(&s_mbar[b]))
                        : "memory");
                }
                // the next chunk's point, loaded behind the MMAs
                const int li = (c + 1) * kLeaves + (r >> 5);
                slot = -1;
                if (c + 1 < nch && li < nlist) {
                    const int sl = s_list[li] * NRR_LEAF + (r & 31);
                    pt = d.tpts[sl];
                    if (pt.idx != 0x7fffffff) slot = sl;
                }
                ++chunk;
            }
            if (c == 0) continue;
            // ---- epilogue of chunk ch = chunk - 1 - (c < nch)
            const int ch = c < nch ? chunk - 2 : chunk - 1;
            const int b = ch & 1;
            if (!failed) {
                // warp-uniform outcome: tcgen05.ld needs the whole warp
                const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&s_mbar[b], phase[b]));
                if (!ok) {
                    failed = true;
                    s_fail = 1;
                    atomicExch(&st->status, (int)NRR_E_TIMEOUT);
                }
            }
            phase[b] ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!failed) {
                const unsigned base = taddr + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(b * kN + half * 64);
                const int* slots = s_slot[ch % 3] + half * 64;
#pragma unroll 1
                for (int part = 0; part < 8; ++part) {
                    float v[8];
                    tmem_ld8(base + (unsigned)(part * 8), v);
                    if (row_valid) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int sl = slots[part * 8 + j];
                            if (v[j] < tv[kTop - 1] && sl >= 0) top_insert(tv, ts, v[j], sl);
                        }
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    };

    // ---- candidate leaves: eight super tiles per round, one per warp; a
    // super tile (then a leaf) is a candidate if it comes within the bound
    // of any query box; leaves are listed in super-tile, then leaf order
    auto box_ok = [&](const float* box) {
        bool c = false;
#pragma unroll
        for (int g = 0; g < kGroups; ++g)
            c = c || box_gap2(s_gb[g][0], s_gb[g][1], s_gb[g][2], s_gb[g][3], s_gb[g][4], s_gb[g][5], box) <= s_gb[g][6];
        return c;
    };
    int nlist = 0;
    for (int s0 = 0; s0 < d.n_supers; s0 += kCta / 32) {
        const int S = s0 + warp;
        bool gs = false;
        if (S < d.n_supers && lane < kGroups) {
            const float* sbx = d.super_box + 6 * S;
            gs = box_gap2(s_gb[lane][0], s_gb[lane][1], s_gb[lane][2], s_gb[lane][3], s_gb[lane][4], s_gb[lane][5],
                          sbx) <= s_gb[lane][6];
        }
        unsigned lmask = 0u;
        if (__any_sync(0xffffffffu, gs)) {
            const int L = S * 32 + lane;
            const bool lc = L < d.n_leaves && box_ok(d.leaf_box + 6 * L);
            lmask = __ballot_sync(0xffffffffu, lc);
        }
        if (lane == 0) s_cnt[warp] = __popc(lmask);
        __syncthreads();
        int off = nlist, total = 0;
#pragma unroll
        for (int w = 0; w < kCta / 32; ++w) {
            const int cw = s_cnt[w];
            if (w < warp) off += cw;
            total += cw;
        }
        if (lmask & (1u << lane)) s_list[off + __popc(lmask & ((1u << lane) - 1u))] = S * 32 + lane;
        __syncthreads();
        nlist += total;
        n_cand += total;
        if (nlist > kListCap - 32 * (kCta / 32) || s0 + kCta / 32 >= d.n_supers) {
            process(nlist);
            nlist = 0;
        }
    }

    // ---- merge the halves' best eight, exact re-rank, completeness test
    if (!owner) {
#pragma unroll
        for (int k = 0; k < kTop; ++k) { s_tv[row][k] = tv[k]; s_ts[row][k] = ts[k]; }
    }
    __syncthreads();
    bool fallback = false;
    if (valid) {
#pragma unroll
        for (int k = 0; k < kTop; ++k) top_insert(tv, ts, s_tv[row][k], s_ts[row][k]);
        float D = INFINITY;   // best exact float distance among the kept candidates
        if (!failed) {
#pragma unroll
            for (int k = 0; k < kTop; ++k) {
                if (ts[k] >= 0) {
                    const TPoint<float> c = d.tpts[ts[k]];
                    const float dd = sqdist(qx, qy, qz, c.x, c.y, c.z);
                    D = fminf(D, dd);
                    const unsigned long long key = cand_key(dd, c.idx);
                    if (key < bkey) { bkey = key; bpos = ts[k]; }
                }
            }
        }
        const float Ru = __uint_as_float(s_Ru);
        const float r = __fadd_ru(xn, Ru);
        const float delta = __fmul_ru(kDelta, __fmul_ru(r, r));
        fallback = failed || !(tv[kTop - 1] > __fadd_ru(__fmul_ru(D, 1.000002f), delta));
        if (fallback) {
            // exact search of this query alone, pruned by its own box
            float ub = ub_f(__uint_as_float((unsigned)(bkey >> 32)));
            for (int S = 0; S < d.n_supers; ++S) {
                if (box_gap2(qx, qy, qz, qx, qy, qz, d.super_box + 6 * S) > ub) continue;
                for (int L = S * 32; L < min(d.n_leaves, S * 32 + 32); ++L) {
                    if (box_gap2(qx, qy, qz, qx, qy, qz, d.leaf_box + 6 * L) > ub) continue;
#pragma unroll 8
                    for (int j = 0; j < NRR_LEAF; ++j) {
                        const TPoint<float> c = d.tpts[L * NRR_LEAF + j];
                        const unsigned long long key = cand_key(sqdist(qx, qy, qz, c.x, c.y, c.z), c.idx);
                        if (key < bkey) { bkey = key; bpos = L * NRR_LEAF + j; }
                    }
                    ub = ub_f(__uint_as_float((unsigned)(bkey >> 32)));
                }
            }
        }
    }
    // ---- tensor memory back, statistics, outputs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        if (s_fail) {
            // let an MMA still in flight finish (bounded) before freeing
            const long long t0 = clock64();
            while (clock64() - t0 < 200000LL) {
            }
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
    }
    if (d.nn_stats != nullptr) {
        const int nfb = __syncthreads_count(fallback);
        if (tid == 0) {
            unsigned long long* o = d.nn_stats + 4 * (size_t)blockIdx.x;
            o[0] = (unsigned long long)(clock64() - t_start);
            o[1] = (unsigned long long)n_cand;
            o[2] = (unsigned long long)chunk;
            o[3] = (unsigned long long)nfb;
        }
    }
    const float bst = __uint_as_float((unsigned)(bkey >> 32));
    const int bidx = (int)(unsigned)(bkey & 0xffffffffull);
    if (valid && bpos >= 0) {
        const TPoint<float> c = d.tpts[bpos];
        bx = c.x; by = c.y; bz = c.z;
    }
    search_outputs<float, MODE>(d, i, valid, bidx, bst, bx, by, bz, qx, qy, qz, s_disp, &s_last);
}

// The alignment state at Xeval with the closest points held (the surrogate
// of the preliminary version's solver): v_hat_i of Eq. (deformed_position)
// into the non-kept buffer and d_i^2 = |v_hat_i - u_i|^2 to the held
// closest point u_i; rho and u unchanged.
template <typename T>
__global__ void __launch_bounds__(kThreads) fixed_corr_kernel(DevProblem<T> d) {
    NrrState* st = d.st;
    const int P = d.P;
    const int wb = st->vk ^ 1;
    T* vh = d.vhat + (size_t)wb * 3 * P;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        T qx, qy, qz;
        query_point<T, NRR_MODE_EVAL>(d, i, qx, qy, qz);
        vh[i] = qx; vh[P + i] = qy; vh[2 * P + i] = qz;
        d.d2[i] = sqdist(qx, qy, qz, d.u[i], d.u[P + i], d.u[2 * P + i]);
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

// The tensor-core candidate search (float path, pass or evaluation mode).
cudaError_t nrr_launch_nn_tc(const DevProblem<float>& d, int mode, cudaStream_t s) {
    const int g = (d.P + tcs::kQ - 1) / tcs::kQ;
    if (g == 0) return cudaSuccess;
    if (mode == NRR_MODE_PASS) nn_tc_kernel<NRR_MODE_PASS><<<g, tcs::kCta, 0, s>>>(d);
    else if (mode == NRR_MODE_EVAL) nn_tc_kernel<NRR_MODE_EVAL><<<g, tcs::kCta, 0, s>>>(d);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t nrr_launch_fixed_corr(const DevProblem<T>& d, cudaStream_t s) {
    const int g = (d.P + kThreads - 1) / kThreads;
    if (g == 0) return cudaSuccess;
    fixed_corr_kernel<T><<<g, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}
template cudaError_t nrr_launch_fixed_corr<float>(const DevProblem<float>&, cudaStream_t);
template cudaError_t nrr_launch_fixed_corr<double>(const DevProblem<double>&, cudaStream_t);

template cudaError_t nrr_launch_nn<float>(const DevProblem<float>&, int, int, cudaStream_t);
template cudaError_t nrr_launch_nn<double>(const DevProblem<double>&, int, int, cudaStream_t);
