// Device data layout and kernel entry points of one registration problem.
//
// HBM layout (T = float for the mixed path, double for the FP64 path):
//   source, internal Hilbert-curve order:  v [3][P] SoA; influence lists in CSR
//     (infl_ptr [P+1], infl_node/infl_w [nnz]); per pass v_hat [2][3][P],
//     closest target coordinates u [3][P], caller index rho [P], d2 [P],
//     alignment weights wa [P].
//   target, internal Hilbert-curve order:  tpts [n_leaves*32] {x,y,z,caller idx},
//     padded with +inf points; AABBs of 32-point leaves (float [6]) and of
//     32-leaf super tiles (float [6]).
//   graph: nodes p [N][3]; directed pairs (e_i, e_j, e_r) sorted by (i, j)
//     with CSR adj_ptr [N+1] over e_i and e_rev [E2] (reverse pair);
//     reg weights wr [E2]; rotations Rm [N][9].
//   system: block-sparse K in BSR with 4x4 blocks on the node-graph pattern
//     (bsr_ptr [N+1], bsr_col [nblk], bsr_edge [nblk] = directed pair (row,
//     col) or -1 on the diagonal), Kv [nblk][16], B [N][12]; per block the
//     list of (point, slot_row, slot_col) contributions (ent_ptr, ent) and
//     their skinning weights (ent_q, one value per entry).
//   iterates: X, G, Gprev, Fprev [N][12]; Anderson rings dF, dG [m][N*12];
//     PCG vectors r, z, p, q [N*12], block-Jacobi inverse Minv [N][16].
#pragma once

#include <cuda_runtime.h>

#include "nrr_internal.h"

// Halo windows of the cluster solve (at most 16 CTAs): CTA r keeps, beside
// its own z rows, copies of the z rows of the last lo[r] nodes of CTA r-1
// and of the first hi[r] nodes of CTA r+1 (the nodes its K rows reference
// there, at most hmax on each side), which those CTAs push to it with bulk
// asynchronous copies each CG iteration. Columns outside the window are read
// from the owner's shared memory.
constexpr int kNrrClusterMaxCtas = 16;
struct NrrHaloWin {
    int hmax;
    int full;   // 1: every column of every CTA lies in its window
    short lo[kNrrClusterMaxCtas];
    short hi[kNrrClusterMaxCtas];
};

template <typename T>
struct __align__(16) TPoint {
    T x, y, z;
    int idx;
};

template <typename T>
struct DevProblem {
    int P, N, E2, n_leaves, n_supers, n_megas, nblk;
    int aa_m;
    int robust;         // nrr_robust: Welsch's function or an l2 variant
    int pcg_max;
    T pcg_tol;
    // source
    const T* v;
    const int* infl_ptr;
    const int* infl_node;
    const T* infl_w;
    const T* p;
    // target
    const TPoint<T>* tpts;
    const float* leaf_box;
    const float* super_box;
    const float* mega_box;   // boxes of 32 consecutive super tiles
    // iterates
    T* X;
    T* Xeval;
    T* G;
    T* Gprev;
    T* Fprev;
    // PCG warm start of a pass's solve: X^(k) + warm_dx once the stage has
    // solved before (the previous MM step F^(k-1) = G^(k-1) - X^(k-1));
    // NULL: X^(k) alone (solves outside a pass)
    const T* warm_dx;
    // 1: the cluster solve applies the singular-K fix itself (a pass's
    // solve); 0: solves outside a pass
    int fix_free;
    T* dF;
    T* dG;
    // per point
    T* vhat;        // [2][3][P]
    T* u;           // [3][P]
    int* rho;       // [P] caller target index
    T* d2;          // [P]
    T* wa;          // [P]
    T* pts;         // [P][8] per pass: v_i, w^a_i, Q_i = u_rho(i) - pbar_i, 0
                    // (energy_kernel; the assembly gathers one row per entry)
    // graph edges
    const int* e_i;
    const int* e_j;
    const T* e_r;
    const int* adj_ptr;
    const int* e_rev;
    T* wr;
    T* Rm;
    // assembly
    const int* bsr_ptr;
    const int* bsr_col;
    const int* bsr_edge;
    const int* ent_ptr;
    const int* ent;         // packed (point << 6 | slot_row << 3 | slot_col)
    const T* ent_q;         // [n_ent] weight of the entry: w_in on a diagonal block (n, n),
                            // w_in w_ik (rounded once, from double) on a block (n, k)
    const int* blk_row;     // [nblk] row node of each block
    const int* diag_blk;    // [N] block (n, n) of each node
    const int* offd_blk;    // [nblk - N] the off-diagonal blocks, in BSR order
    // assembly work descriptors (static), one load each: per node n
    // {diagonal block, entry begin, entry end, first edge of n}; per
    // off-diagonal block (BSR order) {block, entry begin, entry end, directed
    // pair (n, k)} and {n, k, reverse pair, 0}
    const int4* asm_diag;
    const int4* asm_off;
    const int4* asm_off2;
    const T* pbar;          // [3][P] sum_j w_ij p_j (constant part of Q_i)
    T* Kv;
    T* Bv;
    T* anode;               // [N] alignment part of each node's (t, t) entry of K
    // connected components of the node graph: nodes of component c are
    // comp_nodes[comp_ptr[c] .. comp_ptr[c+1])
    int n_comp;
    const int* comp_ptr;
    const int* comp_nodes;
    // PCG
    T* r;
    T* z;
    T* pv;
    T* q;
    T* Minv;
    // reductions
    double* partials;   // [max_ctas * NRR_PARTIAL_STRIDE]
    double* xpartials;  // [n_xpart][4] E_reg at nu_r and nu_r / 2, E_rot, the nu_r read (xterm_kernel's CTAs)
    int n_xpart;        // CTAs of xterm_kernel
    NrrState* st;
    // optional per-warp counters of the closest-point search (NULL: off):
    // [warps][4] = {cycles, super tiles visited, leaves staged, leaves scanned}
    unsigned long long* nn_stats;
    // optional phase timestamps of the cluster solve (CTA 0, thread 0; NULL: off)
    long long* solve_stats;
    // failure-detection test knob (NRR_FAULT_BARRIER, read on the host at
    // creation): the grid-wide solve's CTA 0 skips its first barrier arrival
    int fault_barrier;
    int fault_halo;      // test knob: CTA 1 of the cluster solve skips its first halo push
};

#define NRR_PARTIAL_STRIDE 32

enum NrrMode { NRR_MODE_PASS = 0, NRR_MODE_EVAL = 1, NRR_MODE_RAW = 2 };

// Launch helpers (defined in the kernel translation units).
template <typename T>
cudaError_t nrr_launch_nn(const DevProblem<T>& d, int mode, int lanes_per_query, cudaStream_t s);
// v_hat at Xeval and d^2 to the held closest points u (rho, u unchanged).
template <typename T>
cudaError_t nrr_launch_fixed_corr(const DevProblem<T>& d, cudaStream_t s);
// Vector kernels of the L-BFGS comparison solver (kernels_lbfgs.cu), on n =
// 12 N values: the two-loop direction d = -H g from a ring of mk pairs
// (S, Y [m][n], newest at slot (head - 1) mod m) with scal[0] = g.d and
// scal[1] = |g|; Xout = Xk + t d; the new pair s = Xt - Xk, y = gn - g
// into slot `slot` with scal[2..5] = y.s, |y|, |s|, |gn|, then Xk = Xt and
// g = gn; and the largest |a_i - b_i| of two v_hat buffers into scal[6].
template <typename T>
cudaError_t nrr_launch_lbfgs_dir(int n, const double* g, const double* S, const double* Y, int mk, int head, int m,
                                 double* dvec, double* scal, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_lbfgs_axpy(int n, const T* Xk, double t, const double* dvec, T* Xout, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_lbfgs_pair(int n, T* Xk, const T* Xt, double* g, const double* gn, double* S, double* Y,
                                  int slot, double* scal, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_max_disp(int P, const T* a, const T* b, double* scal, cudaStream_t s);

// Tensor-core candidate search with an exact float re-rank (float path,
// NRR_MODE_PASS or NRR_MODE_EVAL): the outputs of nrr_launch_nn, bit for bit.
cudaError_t nrr_launch_nn_tc(const DevProblem<float>& d, int mode, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_energy(const DevProblem<T>& d, int mode, int grid, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_assemble(const DevProblem<T>& d, int grid, cudaStream_t s);
// Regularisation and rotation terms (X only; d.n_xpart CTAs).
template <typename T>
cudaError_t nrr_launch_xterm(const DevProblem<T>& d, int mode, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_solve(const DevProblem<T>& d, int grid, cudaStream_t s, bool cooperative);
template <typename T>
cudaError_t nrr_launch_aa(const DevProblem<T>& d, int grid, cudaStream_t s);
// Components of the node graph without alignment weight (K singular along
// their common translation): G keeps the component's summed translation of
// X (one warp per component; kernels_solve.cu).
template <typename T>
cudaError_t nrr_launch_free_translation(const DevProblem<T>& d, cudaStream_t s);
// kernels one pass launches: closest points, X-only terms, energy, assembly,
// solve, free translations (a kernel of its own after the grid-wide solve
// only), Anderson differences/Gram solve, Anderson mix
constexpr int kNrrLaunchesPerPass = 8;
__host__ __device__ constexpr int nrr_launches_per_pass(bool cluster_solve) {
    return cluster_solve ? kNrrLaunchesPerPass - 1 : kNrrLaunchesPerPass;
}
template <typename T>
cudaError_t nrr_launch_gradient(const DevProblem<T>& d, double* grad_X, double* grad_v, const int* order,
                                int grid, cudaStream_t s);
// Unrolled backward (kernels_unroll.cu): per-point and per-node adjoint
// contributions of one MM step given lambda = K^-1 g_bar and X' = X^(k+1);
// adds dL/dv to gv (caller order) and writes the new g_bar to gd and gt.
template <typename T>
cudaError_t nrr_launch_adjoint(const DevProblem<T>& d, const T* lam, const T* Xn, const int* order, T* ebuf,
                               double* gv, double* gd, T* gt, cudaStream_t s);
template <typename T>
cudaError_t nrr_launch_to_t(const double* in, T* out, int n, cudaStream_t s);

// 1/x for x > 0: a float reciprocal refined by two Newton steps in double
// (relative error about 2^-52; a double division costs several times more
// on this GPU's FP64 units), or the division when x lies outside the float
// range.
__device__ __forceinline__ double nrr_recip(double x) {
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
    double r = (double)__frcp_rn((float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// The m x m Anderson system for a compile-time m (every array in
// registers: one thread runs it, and local-memory round trips would
// dominate): the Gram matrix of the ring with the new slot's row tot[0..M)
// (gram_old: the kept entries, by ring slot), a ridge of 1e-10 times the
// mean diagonal entry, right-hand side tot[kM..kM+M), solved by an LDL^T
// factorisation in FP64 (one reciprocal per column on the serial path, no
// square roots; L_ij d_j kept in the upper part as scratch). Returns false
// if a pivot is not positive (the Gram matrix plus ridge is not numerically
// positive definite).
template <int M>
__device__ __forceinline__ bool nrr_aa_solve(const double* gram_old, const double (&tot)[2 * NRR_AA_MMAX], int slot,
                                             double (&th)[NRR_AA_MMAX]) {
    constexpr int kM = NRR_AA_MMAX;
    double Gm[M][M], rhs[M], dinv[M];
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
#pragma unroll
        for (int b = 0; b < M; ++b) Gm[a][b] = a == slot ? tot[b] : (b == slot ? tot[a] : gram_old[a * kM + b]);
        rhs[a] = tot[kM + a];
        tr += Gm[a][a];
    }
    const double lam = 1e-10 * tr / M;
#pragma unroll
    for (int a = 0; a < M; ++a) Gm[a][a] += lam;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double dj = Gm[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) dj -= Gm[j][k] * Gm[k][j];
        if (!(dj > 0)) return false;
        dinv[j] = nrr_recip(dj);
#pragma unroll
        for (int i = j + 1; i < M; ++i) {
            double t = Gm[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= Gm[i][k] * Gm[k][j];
            Gm[j][i] = t;
            Gm[i][j] = t * dinv[j];
        }
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        double t = rhs[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= Gm[i][k] * th[k];
        th[i] = t;
    }
#pragma unroll
    for (int i = 0; i < M; ++i) th[i] *= dinv[i];
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
        double t = th[i];
#pragma unroll
        for (int k = i + 1; k < M; ++k) t -= Gm[k][i] * th[k];
        th[i] = t;
    }
    return true;
}

// The Anderson step after its sums (one thread): the system of
// nrr_aa_solve for the ring's mk entries, theta set to 0 if the solve
// fails or |theta| > 1e4. th receives theta (kM entries). With `write` the
// state is updated: the kept Gram row, theta, the ring counters and the
// solve counters. Returns the number of coefficients used (mk, or 0).
__device__ inline int nrr_aa_finish(NrrState* st, const double* gram_old, const double (&tot)[2 * NRR_AA_MMAX],
                                    int mk, int slot, bool insert, int aa_m, double (&th)[NRR_AA_MMAX], bool write) {
    constexpr int kM = NRR_AA_MMAX;
    static_assert(kM == 8, "one case per ring size");
    bool ok = false;
    switch (mk) {
        case 1: ok = nrr_aa_solve<1>(gram_old, tot, slot, th); break;
        case 2: ok = nrr_aa_solve<2>(gram_old, tot, slot, th); break;
        case 3: ok = nrr_aa_solve<3>(gram_old, tot, slot, th); break;
        case 4: ok = nrr_aa_solve<4>(gram_old, tot, slot, th); break;
        case 5: ok = nrr_aa_solve<5>(gram_old, tot, slot, th); break;
        case 6: ok = nrr_aa_solve<6>(gram_old, tot, slot, th); break;
        case 7: ok = nrr_aa_solve<7>(gram_old, tot, slot, th); break;
        case 8: ok = nrr_aa_solve<8>(gram_old, tot, slot, th); break;
        default: break;
    }
    if (ok) {
        double nrm = 0.0;
#pragma unroll
        for (int i = 0; i < kM; ++i)
            if (i < mk) nrm += th[i] * th[i];
        ok = isfinite(nrm) && nrm <= 1e8;   // |theta| <= 1e4
    }
#pragma unroll
    for (int i = 0; i < kM; ++i) th[i] = (ok && i < mk) ? th[i] : 0.0;
    if (write) {
        // the new Gram row is kept for the next passes
#pragma unroll
        for (int b = 0; b < kM; ++b)
            if (b < mk) {
                st->gram[slot * kM + b] = tot[b];
                st->gram[b * kM + slot] = tot[b];
            }
#pragma unroll
        for (int i = 0; i < kM; ++i) st->theta[i] = th[i];
        st->aa_mk = ok ? mk : 0;
        st->aa_count = mk;
        st->aa_head = insert ? (slot + 1) % aa_m : slot;
        st->n_solves_stage += 1;
        st->n_solves += 1;
        st->pending_stop = 1;
        st->solved = 1;
    }
    return ok ? mk : 0;
}

// Stage transition of Algorithm 2 (halve nu_a and nu_r, recompute alpha and
// beta with Eq. WeightSettings, restart the stage). Single device thread.
__device__ __forceinline__ void nrr_stage_weights(NrrState* st) {
    const bool w = st->robust == NRR_WELSCH;
    st->alpha = st->alpha_fixed >= 0 ? st->alpha_fixed
                                     : st->k_alpha * st->n_src / st->n_edges *
                                           (w ? (st->nu_r * st->nu_r) / (st->nu_a * st->nu_a) : 1.0);
    st->beta = st->beta_fixed >= 0 ? st->beta_fixed
                                   : st->k_beta * st->n_src / st->n_nodes /
                                         (w ? 2.0 * st->nu_a * st->nu_a : 1.0);
}

__device__ __forceinline__ void nrr_end_stage(NrrState* st) {
    if (st->nu_a == st->nu_a_min) {
        st->done = 1;
        return;
    }
    st->nu_a = fmax(st->nu_a * 0.5, st->nu_a_min);
    st->nu_r = st->nu_r * 0.5;
    st->stage += 1;
    nrr_stage_weights(st);
    st->E_prev = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    st->n_solves_stage = 0;
    st->aa_count = 0;
    st->aa_head = 0;
    st->just_reverted = 0;
    st->pending_stop = 0;
}
