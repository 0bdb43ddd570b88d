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
