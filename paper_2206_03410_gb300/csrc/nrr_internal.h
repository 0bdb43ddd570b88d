// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <functional>
#include <string>
#include <vector>

#include "nrr.h"

#define NRR_AA_MMAX 8       // largest Anderson depth m
#define NRR_LEAF 32         // target points per leaf tile (one per lane)
#define NRR_MAX_INFL 8      // largest |I(v_i)|

// ---------------------------------------------------------------------------
// Device-resident control block of one context. Written by the kernels of a
// pass; the host reads it after a pass. Doubles first for alignment.
// ---------------------------------------------------------------------------
struct NrrState {
    double nu_a, nu_r, nu_a_min, alpha, beta;   // current stage
    double k_alpha, k_beta, alpha_fixed, beta_fixed;
    double n_src, n_edges, n_nodes;             // |V|, |E_G|, |V_G|
    double eps, rel_tol;
    double E, E_align, E_reg, E_rot;            // of the last evaluated iterate
    double E_prev;                              // last kept energy in stage
    double max_disp;                            // of the last stop test
    double pcg_res;                             // max relative residual
    double gram[NRR_AA_MMAX * NRR_AA_MMAX];     // dF_a . dF_b by ring slot
    double E_eval[4];                           // nrr_energy result
    double theta[NRR_AA_MMAX];                  // last Anderson coefficients
    unsigned long long disp_bits;               // running max of |dv|^2 bits
    int stage;
    int n_solves_stage, n_solves, n_passes, n_rejected;
    int max_iters_stage;
    int just_reverted;
    int pending_stop;       // 1: the previous pass solved; test at next pass
    int skip;               // 1: this pass stops after the energy
    int kept, solved;       // flags of the last pass
    int done;               // Algorithm 2 returned
    int status;             // nrr_status from device-side checks
    int aa_m, aa_count, aa_head, aa_mk;
    int robust;             // nrr_robust (alpha, beta rule of the stages)
    int pcg_iters;
    int n_singular;         // free components of the last solve (translation kept)
    int vk;                 // which v_hat buffer holds the kept iterate
    int vlast;              // which v_hat buffer was written last
    int have_vk;            // v_hat of a kept iterate exists
    unsigned int cnt_nn, cnt_energy;   // last-block-done counters
    unsigned int bar_count, bar_gen;   // grid barrier of the solve kernel
};

// Host-side graph (Algorithm 1), all in caller point indices.
struct HostGraph {
    double radius = 0, lbar = 0;
    int K = 8;                        // max influence
    std::vector<int> nodes;           // source index of node j
    std::vector<int> nidx;            // [P*K], -1 padded, nearest first
    std::vector<double> w;            // [P*K]
    std::vector<int> edges;           // [n_edges*2], j<k sorted
    std::vector<int> dpair;           // [2*n_edges*2] directed (i,j) sorted
    std::vector<double> r;            // [2*n_edges]
};

// graph_build.cpp
// Runs f(begin, end) over [0, n) in contiguous chunks on the host's cores
// (setup work; f writes only the outputs of its own range).
void nrr_parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f);
// The number of chunks nrr_parallel_for would use for n items, and f(chunk,
// begin, end) over [0, n) split into nchunks contiguous chunks, each on its
// own host thread (chunk boundaries depend on n and nchunks only).
int nrr_setup_chunks(int64_t n);
void nrr_parallel_chunks(int64_t n, int nchunks, const std::function<void(int64_t, int64_t, int64_t)>& f);
double nrr_mean_spacing(const double* V, int64_t P, int k);
void nrr_build_graph(const double* V, int64_t P, double R, int K, HostGraph& g);
// Pieces of Algorithm 1 shared by the point-cloud and mesh constructions:
// the visiting order (ascending projection on the PCA axis of the largest
// covariance eigenvalue, ties to the lower index), and the influence sets
// (the K nearest nodes of each point, ties to the lower node id), weights of
// Eq. (weight_data), edges and r_ij from the (point, node, D^2) influences
// of the greedy pass, appended in node order; g.nodes must hold the nodes.
struct NrrInfl {
    int pt;
    int node;
    double d2;
};
std::vector<int> nrr_pca_order(const double* V, int64_t P);
void nrr_finish_graph(const double* V, int64_t P, double R, int K, const std::vector<NrrInfl>& trip,
                      HostGraph& g);
// geodesic.cpp: Algorithm 1 on a triangle-mesh source (faces F [nF][3]
// vertex indices): the ball B(v) by breadth-first search along mesh edges,
// exact geodesic distances on its sub-mesh, influence where D < R. Returns
// false with a message for a non-manifold edge (three or more faces), a bad
// index or a degenerate face.
bool nrr_build_graph_mesh(const double* V, int64_t P, const int* F, int64_t nF, double R, int K, HostGraph& g,
                          std::string& err);
// l-bar of a mesh: the mean length of its (undirected) edges.
double nrr_mesh_mean_edge(const double* V, const int* F, int64_t nF);
// Algorithm 1 with radius R (> 0), or with 5 l-bar (radius <= 0), and l-bar
// (the mean 6-NN spacing) into g.lbar if need_lbar or radius <= 0 (else
// NaN); with a given radius the two run concurrently. Returns false (and
// builds nothing) if the radius would be 5 l-bar = 0.
bool nrr_graph_and_spacing(const double* V, int64_t P, double radius, int K, bool need_lbar, HostGraph& g);

#ifdef __CUDACC__
#define NRR_HD __host__ __device__
#else
#define NRR_HD
#endif
// Hilbert index of a 3-D point with 21 bits per axis, after J. Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707 (2004): the axes are
// converted in place to the "transposed" Hilbert index, whose bits are then
// interleaved most significant first. (Host and device: one definition.)
NRR_HD inline uint64_t nrr_hilbert3(uint32_t x, uint32_t y, uint32_t z) {
    const int bits = 21;
    uint32_t X[3] = {x, y, z};
    const uint32_t M = 1u << (bits - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t Pm = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= Pm;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & Pm;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t h = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
    return h;
}
// the 21-bit grid coordinate of p on an axis of the bounding box [lo, lo + ext]
// (IEEE double subtraction, division and product: the same on host and device)
NRR_HD inline uint32_t nrr_curve_coord(float p, double lo, double ext) {
    double f = ext > 0 ? ((double)p - lo) / ext : 0.0;
    f = fmin(fmax(f, 0.0), 1.0);
    return (uint32_t)llround(f * 2097151.0);
}
// graph_gpu.cu: the Hilbert orders of the source and the target (host
// arrays [n][3]) over the box [lo, hi], on the GPU: per point its code
// (nrr_curve_coord per axis, nrr_hilbert3), then a stable radix sort of
// (code, index); the orders and the sorted codes come back to the host.
cudaError_t nrr_curve_orders_gpu(const float* src, int64_t P, const float* tgt, int64_t T, const double lo[3],
                                 const double hi[3], cudaStream_t st, std::vector<int>& src_order,
                                 std::vector<uint64_t>& src_codes, std::vector<int>& tgt_order,
                                 std::vector<uint64_t>& tgt_codes);

// graph_gpu.cu: Algorithm 1 on the GPU (the same graph as nrr_build_graph);
// src [P][3] float32 host or device; *rounds = greedy rounds run; with lbar
// non-NULL also l-bar (the mean 6-NN spacing, nrr_mean_spacing's per-point
// values, summed in another order) on the graph's grid, or NaN when a
// point's 6 nearest others are not all within R (then the host computes it).
cudaError_t nrr_build_graph_gpu(const float* src, int64_t P, double R, int K, HostGraph& g, cudaStream_t st,
                                int* rounds, double* lbar = nullptr);

// Records msg as the global last error (nrr_last_error(NULL)); returns code.
nrr_status nrr_set_global_error(nrr_status code, const char* msg);

// Error helpers
struct NrrError {
    nrr_status code;
    std::string msg;
};
