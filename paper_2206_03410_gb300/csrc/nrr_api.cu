// C ABI of the registration library (include/nrr.h): context creation,
// per-pass launch sequence captured in a CUDA graph, and accessors.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nrr_device.cuh"

int nrr_solve_threads();
template <typename T>
int nrr_solve_max_blocks_per_sm();
int nrr_solve_cluster_threads();
template <typename T>
size_t nrr_solve_cluster_smem(int cap, int per, int hmax);
template <typename T>
int nrr_solve_cluster_setup(int C, size_t smem, size_t optin);
template <typename T>
size_t nrr_solve_cluster_static_smem();
template <typename T>
cudaError_t nrr_launch_solve_cluster(const DevProblem<T>& d, int C, int cap, const NrrHaloWin& win, size_t smem,
                                     cudaStream_t s);

namespace {

thread_local std::string g_last_error;

template <typename T>
struct Buffers {
    DevProblem<T> d{};
};

}  // namespace

nrr_status nrr_set_global_error(nrr_status code, const char* msg) {
    g_last_error = msg;
    return code;
}

struct nrr_ctx {
    nrr_params prm{};
    bool fp64 = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t aux = nullptr;                 // parallel branch of a pass
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    int64_t P = 0, T = 0;
    int N = 0, E2 = 0, nblk = 0, n_leaves = 0, n_supers = 0;
    HostGraph hg;
    std::vector<int> src_order;   // internal -> caller
    std::vector<int> src_rank;    // caller -> internal
    std::vector<int> bsr_ptr, bsr_col;
    std::vector<void*> allocs;
    NrrState* d_state = nullptr;
    NrrState* h_state = nullptr;
    DevProblem<float> df{};
    DevProblem<double> dd{};
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    cudaGraphExec_t loop_exec = nullptr;   // passes repeated on the device (nrr_solve)
    NrrState** d_states1 = nullptr;        // {d_state}, for the loop's control kernel
    int* d_ctrl = nullptr;                 // loop control: [0] passes run, [1] cap
    int* h_ctrl = nullptr;                 // pinned staging of the cap
    nrr_step_info* d_hist = nullptr;       // records of the last device-side loop's passes
    int hist_n = 0;                        // records of the last nrr_solve
    bool coop = true;
    int grid_energy = 0, grid_asm = 0, grid_solve = 0, grid_aa = 0, num_sms = 0;
    int nn_lpq = 8;                    // closest points: lanes per query (1, 2, 4, 8)
    bool nn_tc = false;                // closest points: tensor-core candidates (float path)
    int* d_order = nullptr;            // internal -> caller source index (gradients)
    double* d_grad = nullptr;          // gradient staging [N*12 + P*3]
    void* d_tune = nullptr;            // autotuner scratch: warm start and output of a solve, [2][N][12] in T
    // unrolled MM steps (nrr_unroll / nrr_backward mode 1)
    int unroll_K = -1;                 // steps of the last nrr_unroll (-1: none)
    double unroll_prm[4] = {0, 0, 0, 0};   // nu_a, nu_r, alpha, beta of that run
    void* d_ck = nullptr;              // checkpoints X^(0..K) [K+1][N][12] in T
    int ck_cap = 0;                    // checkpoints the buffer holds
    void* d_adj = nullptr;             // zero, lambda, g_bar [N][12] and e [3][P] in T
    double* d_adjd = nullptr;          // g_bar [N][12] and dL/dv [P][3] in double
    size_t nn_stats_n = 0;             // per-warp search counters (debug, opt-in)
    int cl_C = 0, cl_cap = 0;          // cluster solve: CTAs per cluster, K blocks per CTA
    int bal_nodes = 0;                 // batch policy -2: most nodes per CTA (0: unset)
    size_t cl_smem = 0;
    NrrHaloWin cl_win{};               // cluster solve: halo windows
    double diag = 0.0;
    double nu_a0 = 0.0, nu_r0 = 0.0;   // first-stage parameters
    uint64_t problem_hash = 0;         // inputs, graph and parameters (checkpoints)
    // the preliminary version's solver (nrr_solve_lbfgs): history pairs
    // S, Y [m][12N], gradients g, g_new and the direction [12N] (double),
    // scalars [8], the inner iterate X_k [12N] and v_hat at the outer
    // iterate [3P] (context precision)
    double* lb_buf = nullptr;
    void* lb_t = nullptr;
    int lb_m = 0;
    bool failed = false;
    std::string err;
};

namespace {

// NVTX range around a host call (visible in Nsight Systems / Compute
// timelines; a no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Wall-clock phases of nrr_create, printed to stderr when the environment
// variable NRR_SETUP_TIMES is set (profiling of the host setup).
struct SetupTimer {
    bool on = std::getenv("NRR_SETUP_TIMES") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void lap(const char* what) {
        nvtxMarkA(what);
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "nrr_create %-22s %8.2f ms\n", what,
                     std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

nrr_status fail(nrr_ctx* c, nrr_status code, const std::string& msg) {
    if (c) c->err = msg;
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, e_ == cudaErrorMemoryAllocation ? NRR_E_OOM : NRR_E_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

template <typename P>
cudaError_t dalloc(nrr_ctx* c, P** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(P));
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = (P*)q;
    return cudaMemsetAsync(q, 0, count * sizeof(P), c->stream);
}

template <typename P>
cudaError_t upload(nrr_ctx* c, P** p, const std::vector<P>& h) {
    cudaError_t e = dalloc(c, p, h.size());
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(P), cudaMemcpyHostToDevice, c->stream);
}

bool finite3(const std::vector<float>& v) {
    for (float x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// Copies n floats from a host or device pointer to a host vector.
cudaError_t fetch_floats(const float* src, size_t n, std::vector<float>& out, cudaStream_t s) {
    out.resize(n);
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(out.data(), src, n * sizeof(float), cudaMemcpyDefault, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// Eq. (WeightSettings); for the l2 variants without the factors that scale
// Welsch's curvature at zero.
void host_stage_weights(NrrState& st) {
    const bool w = st.robust == NRR_WELSCH;
    st.alpha = st.alpha_fixed >= 0 ? st.alpha_fixed
                                   : st.k_alpha * st.n_src / st.n_edges *
                                         (w ? (st.nu_r * st.nu_r) / (st.nu_a * st.nu_a) : 1.0);
    st.beta = st.beta_fixed >= 0 ? st.beta_fixed
                                 : st.k_beta * st.n_src / st.n_nodes / (w ? 2.0 * st.nu_a * st.nu_a : 1.0);
}

void host_restart_stage(NrrState& st) {
    st.E_prev = std::numeric_limits<double>::infinity();
    st.n_solves_stage = 0;
    st.aa_count = 0;
    st.aa_head = 0;
    st.just_reverted = 0;
    st.pending_stop = 0;
    st.have_vk = 0;
    st.skip = 0;
    st.done = 0;
}

template <typename T>
DevProblem<T>& prob(nrr_ctx* c);
template <>
DevProblem<float>& prob<float>(nrr_ctx* c) { return c->df; }
template <>
DevProblem<double>& prob<double>(nrr_ctx* c) { return c->dd; }

nrr_status pull_state(nrr_ctx* c) {
    CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(NrrState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}

nrr_status push_state(nrr_ctx* c) {
    CK(cudaMemcpyAsync(c->d_state, c->h_state, sizeof(NrrState), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}

template <typename T>
cudaError_t launch_solve_on(nrr_ctx* c, const DevProblem<T>& d) {
    if (c->cl_C > 0) return nrr_launch_solve_cluster<T>(d, c->cl_C, c->cl_cap, c->cl_win, c->cl_smem, c->stream);
    return nrr_launch_solve<T>(d, c->grid_solve, c->stream, c->coop);
}

template <typename T>
cudaError_t launch_solve(nrr_ctx* c) { return launch_solve_on<T>(c, prob<T>(c)); }

// The closest-point search of the context's launch shape: the exact pruned
// search, or (float path, pass and evaluation modes) the tensor-core
// candidate search with its exact re-rank; both give the same outputs.
template <typename T>
cudaError_t launch_search(nrr_ctx* c, const DevProblem<T>& d, int mode) {
    return nrr_launch_nn<T>(d, mode, c->nn_lpq, c->stream);
}
template <>
cudaError_t launch_search<float>(nrr_ctx* c, const DevProblem<float>& d, int mode) {
    if (c->nn_tc && mode != NRR_MODE_RAW) return nrr_launch_nn_tc(d, mode, c->stream);
    return nrr_launch_nn<float>(d, mode, c->nn_lpq, c->stream);
}

// The solve step of a pass: PCG, then the free-translation fix of singular
// components (a kernel of its own after the grid-wide solve; the cluster
// solve applies it in its last phase).
template <typename T>
cudaError_t launch_solve_step(nrr_ctx* c) {
    cudaError_t e = launch_solve<T>(c);
    if (e != cudaSuccess) return e;
    if (c->cl_C > 0) return cudaSuccess;
    return nrr_launch_free_translation<T>(prob<T>(c), c->stream);
}

// Whether the cluster solve with C CTAs can run: every CTA's K rows fit in
// shared memory and one such cluster can be resident. Fills the launch
// parameters (K blocks per CTA, halo windows, dynamic shared memory). The
// halo window of CTA r reaches from its lowest to its highest column
// (clamped to the neighbouring CTAs' nodes and to what shared memory holds
// beside the K rows); columns outside it are read from the owner CTA.
template <typename T>
bool cluster_fits(nrr_ctx* c, int C, int* cap_out, NrrHaloWin* win_out, size_t* smem_out) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int N = c->N;
    if (C < 1 || C > 16) return false;
    const int per = (N + C - 1) / C;
    if (per * 4 > nrr_solve_cluster_threads() || per >= 4096) return false;
    int cap = 0;
    for (int r = 0; r < C; ++r) {
        const int n0 = std::min(N, r * per), n1 = std::min(N, n0 + per);
        cap = std::max(cap, c->bsr_ptr[(size_t)n1] - c->bsr_ptr[(size_t)n0]);
    }
    const size_t base = nrr_solve_cluster_smem<T>(cap, per, 0);
    const size_t stat = nrr_solve_cluster_static_smem<T>();
    if (base + stat > (size_t)optin) return false;
    NrrHaloWin win{};
    int want = 0;
    for (int r = 0; r < C; ++r) {
        const int n0 = std::min(N, r * per), n1 = std::min(N, n0 + per);
        int lo = 0, hi = 0;
        if (n1 > n0) {
            const int* col = c->bsr_col.data();
            const int cmin = *std::min_element(col + c->bsr_ptr[(size_t)n0], col + c->bsr_ptr[(size_t)n1]);
            const int cmax = *std::max_element(col + c->bsr_ptr[(size_t)n0], col + c->bsr_ptr[(size_t)n1]);
            const int prev = n0 - std::min(N, std::max(0, r - 1) * per);   // nodes of CTA r-1
            const int next = std::min(N, n1 + per) - n1;                   // nodes of CTA r+1
            lo = std::min(std::max(0, n0 - cmin), prev);
            hi = std::min(std::max(0, cmax + 1 - n1), next);
        }
        win.lo[r] = (short)lo;
        win.hi[r] = (short)hi;
        want = std::max(want, std::max(lo, hi));
    }
    const size_t row2 = 2 * 12 * sizeof(T);   // one halo row on each side
    const int room = (int)std::min<size_t>(((size_t)optin - base - stat) / row2, 4096);
    win.hmax = std::min(want, room);
    // full: no CTA reads a column outside its window (the windows reach
    // every referenced column and no column lies beyond a neighbour)
    win.full = want <= room ? 1 : 0;
    for (int r = 0; r < C && win.full; ++r) {
        const int n0 = std::min(N, r * per), n1 = std::min(N, n0 + per);
        for (int b = c->bsr_ptr[(size_t)n0]; b < c->bsr_ptr[(size_t)n1]; ++b) {
            const int col = c->bsr_col[(size_t)b];
            if (col < n0 - win.lo[r] || col >= n1 + win.hi[r]) { win.full = 0; break; }
        }
    }
    for (int r = 0; r < C; ++r) {
        win.lo[r] = (short)std::min<int>(win.lo[r], win.hmax);
        win.hi[r] = (short)std::min<int>(win.hi[r], win.hmax);
    }
    if (std::getenv("NRR_NO_HALO")) {
        win = NrrHaloWin{};
    }
    const size_t smem = nrr_solve_cluster_smem<T>(cap, per, win.hmax);
    if (nrr_solve_cluster_setup<T>(C, smem, (size_t)optin) < 1) return false;
    *cap_out = cap;
    *win_out = win;
    *smem_out = smem;
    return true;
}

// Sets the solve to the cluster of C CTAs (C >= 1, must fit) or to the
// grid-wide solve (C = 0).
template <typename T>
bool set_solver(nrr_ctx* c, int C) {
    if (C == 0) {
        c->cl_C = 0;
        return true;
    }
    int cap = 0;
    size_t smem = 0;
    NrrHaloWin win{};
    if (!cluster_fits<T>(c, C, &cap, &win, &smem)) return false;
    c->cl_C = C;
    c->cl_cap = cap;
    c->cl_win = win;
    c->cl_smem = smem;
    return true;
}

// Chooses the cluster solve when one cluster of up to 16 CTAs can hold the
// K rows of its nodes in shared memory; otherwise the grid-wide solve.
template <typename T>
void choose_solver(nrr_ctx* c) {
    c->cl_C = 0;
    if (std::getenv("NRR_NO_CLUSTER")) return;
    // a cluster whose CTAs hold their K rows: by default the largest (more
    // SMs for one pair), with solve_ctas = -1 the smallest (cheaper barriers,
    // SMs left free for the other pairs of a batch)
    int forced = c->prm.solve_ctas > 0 ? c->prm.solve_ctas : 0;
    if (const char* e = std::getenv("NRR_CLUSTER_CTAS")) forced = std::atoi(e);
    const bool smallest = c->prm.solve_ctas < 0;
    const int order_small[5] = {1, 2, 4, 8, 16}, order_large[5] = {16, 8, 4, 2, 1};
    // balanced (batches): the smallest cluster whose CTAs hold at most
    // bal_nodes nodes each, so that the pairs' clusters share the SMs in
    // proportion to their systems
    if (c->prm.solve_ctas == -2 && c->bal_nodes > 0 && forced == 0) {
        for (int C : order_small)
            if ((c->N + C - 1) / C <= c->bal_nodes && set_solver<T>(c, C)) return;
        for (int C : order_large)
            if (set_solver<T>(c, C)) return;
        return;
    }
    for (int C : (smallest ? order_small : order_large)) {
        if (forced > 0 && C != forced) continue;
        if (set_solver<T>(c, C)) return;
    }
}

// One pass. The regularisation and rotation terms depend on X only: they run
// on the auxiliary stream (a parallel branch of the captured graph) beside
// the closest-point search, and the energy kernel waits for both.
template <typename T>
cudaError_t launch_pass(nrr_ctx* c) {
    DevProblem<T>& d = prob<T>(c);
    cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
    if (e == cudaSuccess) e = nrr_launch_xterm<T>(d, NRR_MODE_PASS, c->aux);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->aux);
    if (e != cudaSuccess) return e;
    e = launch_search<T>(c, d, NRR_MODE_PASS);
    if (e != cudaSuccess) return e;
    e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    if (e != cudaSuccess) return e;
    e = nrr_launch_energy<T>(d, NRR_MODE_PASS, c->grid_energy, c->stream);
    if (e != cudaSuccess) return e;
    e = nrr_launch_assemble<T>(d, c->grid_asm, c->stream);
    if (e != cudaSuccess) return e;
    e = launch_solve_step<T>(c);
    if (e != cudaSuccess) return e;
    return nrr_launch_aa<T>(d, c->grid_aa, c->stream);
}

cudaError_t launch_pass_any(nrr_ctx* c) { return c->fp64 ? launch_pass<double>(c) : launch_pass<float>(c); }

// Passes of one nrr_solve whose summaries the device-side loop records.
constexpr int kBatchCreateThreads = 8;   // host threads of nrr_batch_create
constexpr int kHistCap = 8192;

// The summary of a context state after a pass (host and device).
__host__ __device__ void fill_info(const NrrState& s, nrr_step_info* info) {
    if (!info) return;
    info->E = s.E; info->E_align = s.E_align; info->E_reg = s.E_reg; info->E_rot = s.E_rot;
    info->nu_a = s.nu_a; info->nu_r = s.nu_r; info->alpha = s.alpha; info->beta = s.beta;
    info->max_disp = s.max_disp;
    info->pcg_rel_residual = s.pcg_res;
    info->kept = s.kept; info->solved = s.solved; info->stage = s.stage; info->done = s.done;
    info->pcg_iters = s.pcg_iters; info->aa_mk = s.aa_mk;
    info->n_passes = s.n_passes; info->n_solves = s.n_solves; info->n_rejected = s.n_rejected;
    info->status = s.status;
    info->n_singular = s.n_singular;
    info->warning = s.n_singular > 0 ? NRR_E_SINGULAR : NRR_OK;
}

// Control of a device-side pass loop (one CTA): copies every context's
// done flag, status and counters to `flags` (when given), records the state
// of a single context after each pass in `hist` (when given, up to hist_cap
// passes), counts the contexts still running, and lets the loop's body run
// again while one is running, none has failed, fewer than ctrl[1] passes ran
// in this launch and more than half of the `members` contexts whose passes
// the body holds are still running (below that the host recaptures a
// smaller body).
__global__ void loop_control(NrrState* const* st, int n, int members, int* flags, int* ctrl,
                             nrr_step_info* hist, int hist_cap, cudaGraphConditionalHandle h) {
    __shared__ int s_run, s_err;
    if (threadIdx.x == 0) { s_run = 0; s_err = 0; }
    __syncthreads();
    int run = 0, err = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const NrrState* s = st[i];
        if (flags) {
            flags[4 * i + 0] = s->done;
            flags[4 * i + 1] = s->status;
            flags[4 * i + 2] = s->n_passes;
            flags[4 * i + 3] = s->n_solves;
        }
        err |= s->status != 0;
        run += s->status == 0 && !s->done;
    }
    if (run) atomicAdd(&s_run, run);
    if (err) atomicOr(&s_err, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int k = ctrl[0] + 1;
        ctrl[0] = k;
        // a single context's pass record (the loop's history)
        if (hist && k <= hist_cap) fill_info(*st[0], hist + (k - 1));
        const bool more = s_run > 0 && !s_err && k < ctrl[1] && 2 * s_run > members;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// Builds `*out`: one conditional WHILE node whose body is what `body`
// enqueues on `stream` (captured into the body graph) followed by
// loop_control. The handle starts at 1 on every launch, so a launch runs the
// body at least once.
template <typename F>
cudaError_t build_loop_graph(cudaStream_t stream, F&& body, NrrState* const* st, int n, int members,
                             int* flags, int* ctrl, nrr_step_info* hist, int hist_cap, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h{};
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams prm{};
    cudaGraph_t bodyg = nullptr;
    if (e == cudaSuccess) {
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = h;
        prm.conditional.type = cudaGraphCondTypeWhile;
        prm.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm);
        if (e == cudaSuccess) bodyg = prm.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(stream, bodyg, nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t be = body();
        if (be == cudaSuccess) {
            loop_control<<<1, 256, 0, stream>>>(st, n, members, flags, ctrl, hist, hist_cap, h);
            be = cudaGetLastError();
        }
        cudaGraph_t captured = nullptr;
        cudaError_t ee = cudaStreamEndCapture(stream, &captured);
        e = be != cudaSuccess ? be : ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
    }
    return e;
}

nrr_status capture_graph(nrr_ctx* c) {
    c->use_graph = false;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->loop_exec) {
        cudaGraphExecDestroy(c->loop_exec);
        c->loop_exec = nullptr;
    }
    if (std::getenv("NRR_NO_GRAPH")) return NRR_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return NRR_OK;
    }
    cudaError_t le = launch_pass_any(c);
    cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess || g == nullptr) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return NRR_OK;   // direct launches instead
    }
    cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        c->gexec = nullptr;
        return NRR_OK;
    }
    c->use_graph = true;
    // the same pass as the body of a device-side loop (nrr_solve); without
    // it nrr_solve launches the pass graph from the host
    if (c->d_states1 && !std::getenv("NRR_HOST_LOOP"))
        build_loop_graph(c->stream, [c]() { return launch_pass_any(c); }, c->d_states1, 1, 1, nullptr,
                         c->d_ctrl, c->d_hist, kHistCap, &c->loop_exec);
    return NRR_OK;
}

nrr_status run_pass(nrr_ctx* c) {
    if (c->use_graph) CK(cudaGraphLaunch(c->gexec, c->stream));
    else CK(launch_pass_any(c));
    return NRR_OK;
}



// ---------------------------------------------------------------------------
// Creation
// ---------------------------------------------------------------------------
// 64-bit hash of the bytes of a problem (source, target, graph, parameters),
// stored in checkpoints so that a state saved from another problem of the
// same sizes is refused. Word-wise multiply-xorshift mixing; not
// cryptographic.
struct ProblemHash {
    uint64_t h = 0x9e3779b97f4a7c15ull;
    void word(uint64_t w) {
        h ^= w + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h *= 0xff51afd7ed558ccdull;
        h ^= h >> 33;
    }
    // arrays of 1 MiB and more: fixed 256 KiB blocks hashed on the host's
    // cores, their hashes then taken in order (independent of the threads)
    void bytes(const void* p, size_t n) {
        constexpr size_t kBlock = (size_t)1 << 18;
        if (n >= ((size_t)1 << 20)) {
            const unsigned char* b = static_cast<const unsigned char*>(p);
            const int64_t nb = (int64_t)((n + kBlock - 1) / kBlock);
            std::vector<uint64_t> sub((size_t)nb);
            nrr_parallel_chunks(nb, (int)std::min<int64_t>(nb, 16), [&](int64_t, int64_t k0, int64_t k1) {
                for (int64_t k = k0; k < k1; ++k) {
                    ProblemHash ph;
                    ph.bytes_serial(b + (size_t)k * kBlock, std::min(kBlock, n - (size_t)k * kBlock));
                    sub[(size_t)k] = ph.h;
                }
            });
            for (uint64_t w : sub) word(w);
            word((uint64_t)n);
            return;
        }
        bytes_serial(p, n);
    }
    void bytes_serial(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        size_t k = 0;
        for (; k + 8 <= n; k += 8) {
            uint64_t w;
            std::memcpy(&w, b + k, 8);
            word(w);
        }
        uint64_t t = 0;
        for (size_t j = 0; k + j < n; ++j) t |= (uint64_t)b[k + j] << (8 * j);
        word(t ^ ((uint64_t)n << 56));
    }
    template <typename V>
    void vec(const std::vector<V>& v) { bytes(v.data(), v.size() * sizeof(V)); }
};

uint64_t problem_hash(const std::vector<float>& src, const std::vector<float>& tgt, const HostGraph& g,
                      const nrr_params& prm) {
    ProblemHash ph;
    ph.vec(src);
    ph.vec(tgt);
    ph.vec(g.nodes);
    ph.vec(g.nidx);
    ph.vec(g.w);
    ph.vec(g.edges);
    ph.vec(g.r);
    const double dp[] = {prm.graph_radius, prm.nu_a, prm.nu_r, prm.nu_a_min, prm.k_alpha, prm.k_beta, prm.alpha,
                         prm.beta, prm.eps, prm.rel_energy_tol, prm.pcg_tol};
    const int ip[] = {prm.max_influence, prm.anneal, prm.aa_m, prm.max_iters_per_stage, prm.precision,
                      prm.pcg_max_iters, prm.robust, prm.nu_schedule};
    ph.bytes(dp, sizeof dp);
    ph.bytes(ip, sizeof ip);
    return ph.h;
}

// Algorithm 1 on the GPU (graph_gpu.cu) with l-bar on a host thread beside
// it when the parameters need it (or first, when the radius defaults to
// 5 l-bar). src: the float source points (host or device).
nrr_status graph_on_device(const float* src, const std::vector<double>& V, int64_t P, double radius, int K,
                           bool need_lbar, cudaStream_t st, HostGraph& g) {
    double lbar = std::nan("");
    double R = radius;
    const bool lbar_first = R <= 0;
    if (lbar_first) {
        lbar = nrr_mean_spacing(V.data(), P, 6);
        R = 5.0 * lbar;
        if (!(R > 0)) return nrr_set_global_error(NRR_E_INVALID, "graph radius 5 l-bar is not positive");
    }
    // with a given radius, l-bar comes from the GPU beside the graph (on the
    // graph's grid, points whose 6 nearest others are not all within R by
    // brute force); the host computes it only if there are too many of them
    int rounds = 0;
    double lb_gpu = std::nan("");
    const cudaError_t e = nrr_build_graph_gpu(src, P, R, K, g, st, &rounds, (!lbar_first && need_lbar) ? &lb_gpu : nullptr);
    if (e != cudaSuccess)
        return nrr_set_global_error(e == cudaErrorMemoryAllocation ? NRR_E_OOM : NRR_E_CUDA,
                                    (std::string("deformation graph on the GPU: ") + cudaGetErrorString(e)).c_str());
    if (!lbar_first && need_lbar) lbar = std::isnan(lb_gpu) ? nrr_mean_spacing(V.data(), P, 6) : lb_gpu;
    g.lbar = lbar;
    return NRR_OK;
}

// Algorithm 1 on a triangle-mesh source (faces already on the host): l-bar
// is the mean mesh edge length, the radius 5 l-bar unless given.
nrr_status graph_from_mesh(const std::vector<double>& V, int64_t P, const std::vector<int>& F, double radius,
                           int K, HostGraph& g, const char* who) {
    const int64_t nF = (int64_t)(F.size() / 3);
    for (int x : F)
        if (x < 0 || x >= P) return nrr_set_global_error(NRR_E_INVALID, (std::string(who) + ": face index out of range").c_str());
    const double lbar = nrr_mesh_mean_edge(V.data(), F.data(), nF);
    const double R = radius > 0 ? radius : 5.0 * lbar;
    if (!(R > 0) || !std::isfinite(R))
        return nrr_set_global_error(NRR_E_INVALID, (std::string(who) + ": radius 5 l-bar is not positive").c_str());
    std::string err;
    if (!nrr_build_graph_mesh(V.data(), P, F.data(), nF, R, K, g, err))
        return nrr_set_global_error(NRR_E_INVALID, (std::string(who) + ": " + err).c_str());
    g.lbar = lbar;
    return NRR_OK;
}

// Hilbert orders of source and target over their common bounding box (on
// the GPU: nrr_curve_orders_gpu).
struct CurveOrders {
    double diag = 0.0;
    std::vector<int> src_order, tgt_order;
    std::vector<uint64_t> src_codes, tgt_codes;
    cudaError_t compute(const std::vector<float>& src, int64_t P, const std::vector<float>& tgt, int64_t Tn,
                        cudaStream_t st) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = 0; i < P; ++i)
            for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], (double)src[3 * i + a]); hi[a] = std::max(hi[a], (double)src[3 * i + a]); }
        for (int64_t i = 0; i < Tn; ++i)
            for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], (double)tgt[3 * i + a]); hi[a] = std::max(hi[a], (double)tgt[3 * i + a]); }
        const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        diag = std::sqrt(dx * dx + dy * dy + dz * dz);
        return nrr_curve_orders_gpu(src.data(), P, tgt.data(), Tn, lo, hi, st, src_order, src_codes, tgt_order,
                                    tgt_codes);
    }
};

template <typename T>
nrr_status build_device(nrr_ctx* c, const std::vector<float>& src, const std::vector<float>& tgt, CurveOrders& co,
                        SetupTimer& tm) {
    DevProblem<T>& d = prob<T>(c);
    const int64_t P = c->P, Tn = c->T;
    const HostGraph& g = c->hg;
    const int K = g.K, N = c->N;
    c->diag = co.diag;
    c->src_order.swap(co.src_order);
    std::vector<uint64_t>& src_codes = co.src_codes;
    std::vector<uint64_t>& tgt_codes = co.tgt_codes;
    std::vector<int>& tgt_order = co.tgt_order;
    c->src_rank.assign((size_t)P, 0);
    nrr_parallel_for(P, [&](int64_t i0, int64_t i1) {
        for (int64_t ii = i0; ii < i1; ++ii) c->src_rank[(size_t)c->src_order[(size_t)ii]] = (int)ii;
    });

    // the target's leaves, tiles and the initial correspondence guess depend
    // on the curve orders only: built on another thread beside the
    // graph-dependent structures below
    struct Leaves {
        int nl = 0, ns = 0, nm = 0;
        std::vector<TPoint<T>> tp;
        std::vector<float> lbox, sbox, mbox;
        std::vector<T> u0;
        std::vector<int> rho0;
    } lv;
    struct Joiner {
        std::thread t;
        ~Joiner() { if (t.joinable()) t.join(); }
    } leaves_thread{std::thread([&]() {
        // target leaves (32 curve-consecutive points) and super tiles
        const int nl = (int)((Tn + NRR_LEAF - 1) / NRR_LEAF);
        const int ns = (nl + 31) / 32;
        lv.nl = nl;
        lv.ns = ns;
        std::vector<TPoint<T>>& tp = lv.tp;
        tp.resize((size_t)nl * NRR_LEAF);
        std::vector<float>& lbox = lv.lbox;
        std::vector<float>& sbox = lv.sbox;
        lbox.resize((size_t)nl * 6);
        sbox.resize((size_t)ns * 6);
        nrr_parallel_for((int64_t)tp.size(), [&](int64_t k0, int64_t k1) {
            for (int64_t k = k0; k < k1; ++k) {
                if (k < Tn) {
                    const int t = tgt_order[(size_t)k];
                    tp[(size_t)k].x = (T)tgt[3 * (size_t)t];
                    tp[(size_t)k].y = (T)tgt[3 * (size_t)t + 1];
                    tp[(size_t)k].z = (T)tgt[3 * (size_t)t + 2];
                    tp[(size_t)k].idx = t;
                } else {
                    tp[(size_t)k].x = tp[(size_t)k].y = tp[(size_t)k].z = std::numeric_limits<T>::infinity();
                    tp[(size_t)k].idx = 0x7fffffff;
                }
            }
        });
        nrr_parallel_for(nl, [&](int64_t L0, int64_t L1) {
            for (int64_t L = L0; L < L1; ++L) {
                float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
                for (int64_t k = L * NRR_LEAF; k < std::min<int64_t>(Tn, (L + 1) * NRR_LEAF); ++k) {
                    const int t = tgt_order[(size_t)k];
                    for (int a = 0; a < 3; ++a) {
                        b[a] = std::min(b[a], tgt[3 * (size_t)t + a]);
                        b[3 + a] = std::max(b[3 + a], tgt[3 * (size_t)t + a]);
                    }
                }
                std::memcpy(&lbox[(size_t)L * 6], b, sizeof(b));
            }
        });
        for (int S = 0; S < ns; ++S) {
            float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
            for (int L = S * 32; L < std::min(nl, (S + 1) * 32); ++L)
                for (int a = 0; a < 3; ++a) {
                    b[a] = std::min(b[a], lbox[(size_t)L * 6 + a]);
                    b[3 + a] = std::max(b[3 + a], lbox[(size_t)L * 6 + 3 + a]);
                }
            std::memcpy(&sbox[(size_t)S * 6], b, sizeof(b));
        }
        const int nm = (ns + 31) / 32;
        lv.nm = nm;
        std::vector<float>& mbox = lv.mbox;
        mbox.resize((size_t)nm * 6);
        for (int M = 0; M < nm; ++M) {
            float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
            for (int S = M * 32; S < std::min(ns, (M + 1) * 32); ++S)
                for (int a = 0; a < 3; ++a) {
                    b[a] = std::min(b[a], sbox[(size_t)S * 6 + a]);
                    b[3 + a] = std::max(b[3 + a], sbox[(size_t)S * 6 + 3 + a]);
                }
            std::memcpy(&mbox[(size_t)M * 6], b, sizeof(b));
        }
        // initial correspondence guess: the target point next along the curve
        std::vector<T>& u0 = lv.u0;
        std::vector<int>& rho0 = lv.rho0;
        u0.resize((size_t)(3 * P));
        rho0.resize((size_t)P);
        nrr_parallel_for(P, [&](int64_t i0, int64_t i1) {
            for (int64_t ii = i0; ii < i1; ++ii) {
                size_t pos = (size_t)(std::lower_bound(tgt_codes.begin(), tgt_codes.end(), src_codes[(size_t)ii]) -
                                      tgt_codes.begin());
                if (pos >= (size_t)Tn) pos = (size_t)Tn - 1;
                for (int a = 0; a < 3; ++a)
                    u0[(size_t)(a * P + ii)] = a == 0 ? tp[pos].x : (a == 1 ? tp[pos].y : tp[pos].z);
                rho0[(size_t)ii] = tp[pos].idx;
            }
        });
    })};

    // source SoA and influence CSR in internal order (per point the count,
    // then the rows, on the host's cores)
    std::vector<T> v((size_t)(3 * P));
    std::vector<int> infl_ptr((size_t)P + 1, 0), infl_node;
    std::vector<T> infl_w;
    nrr_parallel_for(P, [&](int64_t i0, int64_t i1) {
        for (int64_t ii = i0; ii < i1; ++ii) {
            const int i = c->src_order[(size_t)ii];
            for (int a = 0; a < 3; ++a) v[(size_t)(a * P + ii)] = (T)src[3 * (size_t)i + a];
            int k = 0;
            while (k < K && g.nidx[(size_t)i * K + k] >= 0) ++k;
            infl_ptr[(size_t)ii + 1] = k;
        }
    });
    for (int64_t ii = 0; ii < P; ++ii) infl_ptr[(size_t)ii + 1] += infl_ptr[(size_t)ii];
    infl_node.resize((size_t)infl_ptr[(size_t)P]);
    infl_w.resize((size_t)infl_ptr[(size_t)P]);
    nrr_parallel_for(P, [&](int64_t i0, int64_t i1) {
        for (int64_t ii = i0; ii < i1; ++ii) {
            const int i = c->src_order[(size_t)ii];
            for (int k = 0, o = infl_ptr[(size_t)ii]; o < infl_ptr[(size_t)ii + 1]; ++k, ++o) {
                infl_node[(size_t)o] = g.nidx[(size_t)i * K + k];
                infl_w[(size_t)o] = (T)g.w[(size_t)i * K + k];
            }
        }
    });
    tm.lap("  source SoA + influence CSR");
    std::vector<T> p((size_t)N * 3);
    for (int j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) p[(size_t)3 * j + a] = (T)src[3 * (size_t)g.nodes[(size_t)j] + a];
    // directed pairs (sorted by (i, j)), adjacency and reverse index
    const int E2 = c->E2;
    std::vector<int> e_i((size_t)E2), e_j((size_t)E2), adj_ptr((size_t)N + 1, 0), e_rev((size_t)E2);
    std::vector<T> e_r((size_t)E2);
    for (int e = 0; e < E2; ++e) {
        e_i[(size_t)e] = g.dpair[2 * (size_t)e];
        e_j[(size_t)e] = g.dpair[2 * (size_t)e + 1];
        e_r[(size_t)e] = (T)g.r[(size_t)e];
        adj_ptr[(size_t)e_i[(size_t)e] + 1]++;
    }
    for (int n = 0; n < N; ++n) adj_ptr[(size_t)n + 1] += adj_ptr[(size_t)n];
    for (int e = 0; e < E2; ++e) {
        const int a = e_i[(size_t)e], b = e_j[(size_t)e];
        auto first = e_j.begin() + adj_ptr[(size_t)b], last = e_j.begin() + adj_ptr[(size_t)b + 1];
        auto it = std::lower_bound(first, last, a);
        e_rev[(size_t)e] = (int)(it - e_j.begin());
    }
    // BSR pattern: the diagonal plus the neighbours of each node
    std::vector<int>& bp = c->bsr_ptr;
    std::vector<int>& bc = c->bsr_col;
    std::vector<int> be;
    bp.assign((size_t)N + 1, 0);
    bc.clear();
    for (int n = 0; n < N; ++n) {
        bool put_diag = false;
        for (int e = adj_ptr[(size_t)n]; e < adj_ptr[(size_t)n + 1]; ++e) {
            if (!put_diag && e_j[(size_t)e] > n) { bc.push_back(n); be.push_back(-1); put_diag = true; }
            bc.push_back(e_j[(size_t)e]);
            be.push_back(e);
        }
        if (!put_diag) { bc.push_back(n); be.push_back(-1); }
        bp[(size_t)n + 1] = (int)bc.size();
    }
    c->nblk = (int)bc.size();
    auto block_of = [&](int a, int b) {
        auto first = bc.begin() + bp[(size_t)a], last = bc.begin() + bp[(size_t)a + 1];
        return (int)(std::lower_bound(first, last, b) - bc.begin());
    };
    tm.lap("  edges + BSR pattern");
    // per-block contribution lists (point, slot_row, slot_col), by point:
    // the block of every (point, slot, slot) in parallel, then a counting
    // sort by block that keeps point order
    std::vector<int64_t> pent((size_t)P + 1, 0);
    for (int64_t ii = 0; ii < P; ++ii) {
        const int64_t k = infl_ptr[(size_t)ii + 1] - infl_ptr[(size_t)ii];
        pent[(size_t)ii + 1] = pent[(size_t)ii] + k * k;
    }
    std::vector<int> eblk((size_t)pent[(size_t)P]);
    nrr_parallel_for(P, [&](int64_t i0, int64_t i1) {
        for (int64_t ii = i0; ii < i1; ++ii) {
            int64_t o = pent[(size_t)ii];
            for (int sa = infl_ptr[(size_t)ii]; sa < infl_ptr[(size_t)ii + 1]; ++sa)
                for (int sb = infl_ptr[(size_t)ii]; sb < infl_ptr[(size_t)ii + 1]; ++sb)
                    eblk[(size_t)o++] = block_of(infl_node[(size_t)sa], infl_node[(size_t)sb]);
        }
    });
    tm.lap("  entry blocks");
    // stable counting sort by block: per chunk of points a histogram, then
    // each chunk's start in every block (chunks in point order), then the
    // chunks fill their entries in parallel
    const int nblk = c->nblk;
    const int nch = (int)std::max<int64_t>(
        1, std::min<int64_t>(nrr_setup_chunks(P), ((int64_t)1 << 24) / std::max(1, nblk)));
    std::vector<int> hist((size_t)nch * nblk, 0);
    nrr_parallel_chunks(P, nch, [&](int64_t t, int64_t i0, int64_t i1) {
        int* h = hist.data() + (size_t)t * nblk;
        for (int64_t o = pent[(size_t)i0]; o < pent[(size_t)i1]; ++o) h[eblk[(size_t)o]]++;
    });
    std::vector<int> ent_cnt((size_t)nblk + 1, 0), run((size_t)nblk, 0);
    nrr_parallel_for(nblk, [&](int64_t b0, int64_t b1) {
        for (int t = 0; t < nch; ++t)
            for (int64_t b = b0; b < b1; ++b) run[(size_t)b] += hist[(size_t)t * nblk + b];
    });
    for (int b = 0; b < nblk; ++b) ent_cnt[(size_t)b + 1] = ent_cnt[(size_t)b] + run[(size_t)b];
    nrr_parallel_for(nblk, [&](int64_t b0, int64_t b1) {
        for (int64_t b = b0; b < b1; ++b) run[(size_t)b] = ent_cnt[(size_t)b];
        for (int t = 0; t < nch; ++t)
            for (int64_t b = b0; b < b1; ++b) {
                const int k = hist[(size_t)t * nblk + b];
                hist[(size_t)t * nblk + b] = run[(size_t)b];
                run[(size_t)b] += k;
            }
    });
    std::vector<int> ent((size_t)ent_cnt[(size_t)nblk]);
    nrr_parallel_chunks(P, nch, [&](int64_t t, int64_t i0, int64_t i1) {
        int* fillp = hist.data() + (size_t)t * nblk;
        for (int64_t ii = i0; ii < i1; ++ii) {
            const int b0 = infl_ptr[(size_t)ii];
            int64_t o = pent[(size_t)ii];
            for (int sa = b0; sa < infl_ptr[(size_t)ii + 1]; ++sa)
                for (int sb = b0; sb < infl_ptr[(size_t)ii + 1]; ++sb) {
                    const int blk = eblk[(size_t)o++];
                    ent[(size_t)fillp[blk]++] = (int)((ii << 6) | ((sa - b0) << 3) | (sb - b0));
                }
        }
    });
    tm.lap("BSR + contribution lists");
    // connected components of the node graph (union-find over the edges),
    // nodes listed by component in increasing order
    std::vector<int> comp_ptr, comp_nodes;
    {
        std::vector<int> parent((size_t)N);
        for (int j = 0; j < N; ++j) parent[(size_t)j] = j;
        auto root = [&](int x) {
            while (parent[(size_t)x] != x) {
                parent[(size_t)x] = parent[(size_t)parent[(size_t)x]];
                x = parent[(size_t)x];
            }
            return x;
        };
        for (size_t e = 0; e + 1 < g.edges.size(); e += 2) {
            const int a = root(g.edges[e]), b = root(g.edges[e + 1]);
            if (a != b) parent[(size_t)std::max(a, b)] = std::min(a, b);
        }
        std::vector<int> label((size_t)N, -1), count;
        for (int j = 0; j < N; ++j) {
            const int r = root(j);
            if (label[(size_t)r] < 0) { label[(size_t)r] = (int)count.size(); count.push_back(0); }
            label[(size_t)j] = label[(size_t)r];
            count[(size_t)label[(size_t)j]]++;
        }
        comp_ptr.assign(count.size() + 1, 0);
        for (size_t k = 0; k < count.size(); ++k) comp_ptr[k + 1] = comp_ptr[k] + count[k];
        comp_nodes.assign((size_t)N, 0);
        std::vector<int> fill(comp_ptr.begin(), comp_ptr.end() - 1);
        for (int j = 0; j < N; ++j) comp_nodes[(size_t)fill[(size_t)label[(size_t)j]]++] = j;
    }
    tm.lap("  components");
    // one weight per entry: w_in on a diagonal block (the entry's two slots
    // are the same node), w_in w_ik (product in double, rounded once) off it
    std::vector<T> ent_q(ent.size());
    nrr_parallel_for((int64_t)ent.size(), [&](int64_t e0, int64_t e1) {
        for (int64_t e = e0; e < e1; ++e) {
            const int ii = ent[(size_t)e] >> 6, sa = (ent[(size_t)e] >> 3) & 7, sb = ent[(size_t)e] & 7;
            const double wa_ = (double)infl_w[(size_t)infl_ptr[(size_t)ii] + sa];
            const double wb_ = (double)infl_w[(size_t)infl_ptr[(size_t)ii] + sb];
            ent_q[(size_t)e] = (T)(sa == sb ? wa_ : wa_ * wb_);
        }
    });
    std::vector<int> blk_row((size_t)c->nblk);
    for (int n = 0; n < N; ++n)
        for (int b = bp[(size_t)n]; b < bp[(size_t)n + 1]; ++b) blk_row[(size_t)b] = n;
    std::vector<T> pbar((size_t)(3 * P), (T)0);
    nrr_parallel_for(P, [&](int64_t i0, int64_t i1) {
        for (int64_t ii = i0; ii < i1; ++ii) {
            double acc[3] = {0, 0, 0};
            for (int s = infl_ptr[(size_t)ii]; s < infl_ptr[(size_t)ii + 1]; ++s) {
                const int j = infl_node[(size_t)s];
                for (int a = 0; a < 3; ++a)
                    acc[a] += (double)infl_w[(size_t)s] * (double)src[3 * (size_t)g.nodes[(size_t)j] + a];
            }
            for (int a = 0; a < 3; ++a) pbar[(size_t)(a * P + ii)] = (T)acc[a];
        }
    });
    tm.lap("  entry weights, pbar");
    leaves_thread.t.join();
    const int nl = lv.nl, ns = lv.ns, nm = lv.nm;
    c->n_leaves = nl;
    c->n_supers = ns;
    std::vector<TPoint<T>>& tp = lv.tp;
    std::vector<float>& lbox = lv.lbox;
    std::vector<float>& sbox = lv.sbox;
    std::vector<float>& mbox = lv.mbox;
    std::vector<T>& u0 = lv.u0;
    std::vector<int>& rho0 = lv.rho0;
    // identity transforms
    std::vector<T> X0((size_t)N * 12, (T)0);
    for (int j = 0; j < N; ++j) { X0[(size_t)12 * j + 0] = 1; X0[(size_t)12 * j + 4] = 1; X0[(size_t)12 * j + 8] = 1; }

    tm.lap("leaves + initial bound");
    d.P = (int)P; d.N = N; d.E2 = E2; d.n_leaves = nl; d.n_supers = ns; d.n_megas = nm; d.nblk = c->nblk;
    d.aa_m = c->prm.aa_m;
    d.robust = c->prm.robust;
    d.pcg_max = c->prm.pcg_max_iters;
    d.pcg_tol = (T)c->prm.pcg_tol;
    T *pv_, *pw_, *pp_, *er_;
    int *ip_, *in_, *ei_, *ej_, *ap_, *rv_, *bp_, *bc_, *be_, *ep_, *en_, *rho_;
    TPoint<T>* tp_;
    float *lb_, *sb_, *mb_;
    CK(upload(c, &pv_, v)); d.v = pv_;
    CK(upload(c, &ip_, infl_ptr)); d.infl_ptr = ip_;
    CK(upload(c, &in_, infl_node)); d.infl_node = in_;
    CK(upload(c, &pw_, infl_w)); d.infl_w = pw_;
    CK(upload(c, &pp_, p)); d.p = pp_;
    CK(upload(c, &tp_, tp)); d.tpts = tp_;
    CK(upload(c, &lb_, lbox)); d.leaf_box = lb_;
    CK(upload(c, &sb_, sbox)); d.super_box = sb_;
    CK(upload(c, &mb_, mbox)); d.mega_box = mb_;
    CK(upload(c, &ei_, e_i)); d.e_i = ei_;
    CK(upload(c, &ej_, e_j)); d.e_j = ej_;
    CK(upload(c, &er_, e_r)); d.e_r = er_;
    CK(upload(c, &ap_, adj_ptr)); d.adj_ptr = ap_;
    CK(upload(c, &rv_, e_rev)); d.e_rev = rv_;
    CK(upload(c, &bp_, bp)); d.bsr_ptr = bp_;
    CK(upload(c, &bc_, bc)); d.bsr_col = bc_;
    CK(upload(c, &be_, be)); d.bsr_edge = be_;
    CK(upload(c, &ep_, ent_cnt)); d.ent_ptr = ep_;
    CK(upload(c, &en_, ent)); d.ent = en_;
    {
        T *ew_, *pb_;
        int* br_;
        CK(upload(c, &ew_, ent_q)); d.ent_q = ew_;
        CK(upload(c, &pb_, pbar)); d.pbar = pb_;
        CK(upload(c, &br_, blk_row)); d.blk_row = br_;
        std::vector<int> diag_blk((size_t)N), offd_blk;
        for (int n = 0; n < N; ++n)
            for (int b = bp[(size_t)n]; b < bp[(size_t)n + 1]; ++b) {
                if (bc[(size_t)b] == n) diag_blk[(size_t)n] = b;
                else offd_blk.push_back(b);
            }
        int *db_, *ob_;
        CK(upload(c, &db_, diag_blk)); d.diag_blk = db_;
        CK(upload(c, &ob_, offd_blk)); d.offd_blk = ob_;
        std::vector<int4> adiag((size_t)N), aoff(offd_blk.size()), aoff2(offd_blk.size());
        for (int n = 0; n < N; ++n) {
            const int b = diag_blk[(size_t)n];
            adiag[(size_t)n] = make_int4(b, ent_cnt[(size_t)b], ent_cnt[(size_t)b + 1], adj_ptr[(size_t)n]);
        }
        for (size_t q = 0; q < offd_blk.size(); ++q) {
            const int b = offd_blk[q];
            const int e = be[(size_t)b];
            aoff[q] = make_int4(b, ent_cnt[(size_t)b], ent_cnt[(size_t)b + 1], e);
            aoff2[q] = make_int4(blk_row[(size_t)b], bc[(size_t)b], e_rev[(size_t)e], 0);
        }
        int4 *ad_, *ao_, *ao2_;
        CK(upload(c, &ad_, adiag)); d.asm_diag = ad_;
        CK(upload(c, &ao_, aoff)); d.asm_off = ao_;
        CK(upload(c, &ao2_, aoff2)); d.asm_off2 = ao2_;
    }
    CK(upload(c, &d.X, X0));
    CK(dalloc(c, &d.Xeval, (size_t)N * 12));
    CK(dalloc(c, &d.G, (size_t)N * 12));
    CK(upload(c, &d.Gprev, X0));
    CK(dalloc(c, &d.Fprev, (size_t)N * 12));
    d.warm_dx = d.Fprev;
    d.fix_free = 1;
    const int mm = std::max(1, c->prm.aa_m);
    CK(dalloc(c, &d.dF, (size_t)mm * N * 12));
    CK(dalloc(c, &d.dG, (size_t)mm * N * 12));
    CK(dalloc(c, &d.vhat, (size_t)6 * P));
    CK(upload(c, &d.u, u0));
    CK(upload(c, &rho_, rho0)); d.rho = rho_;
    CK(dalloc(c, &d.d2, (size_t)P));
    CK(dalloc(c, &d.wa, (size_t)P));
    CK(dalloc(c, &d.pts, (size_t)P * 8));
    CK(dalloc(c, &d.wr, (size_t)E2));
    CK(dalloc(c, &d.Rm, (size_t)N * 9));
    CK(dalloc(c, &d.Kv, (size_t)c->nblk * 16));
    CK(dalloc(c, &d.anode, (size_t)N));
    {
        int *cp_, *cn_;
        CK(upload(c, &cp_, comp_ptr)); d.comp_ptr = cp_;
        CK(upload(c, &cn_, comp_nodes)); d.comp_nodes = cn_;
        d.n_comp = (int)comp_ptr.size() - 1;
    }
    CK(dalloc(c, &d.Bv, (size_t)N * 12));
    CK(dalloc(c, &d.r, (size_t)N * 12));
    CK(dalloc(c, &d.z, (size_t)N * 12));
    CK(dalloc(c, &d.pv, (size_t)N * 12));
    CK(dalloc(c, &d.q, (size_t)N * 12));
    CK(dalloc(c, &d.Minv, (size_t)N * 16));
    const int max_ctas = std::max({c->grid_energy, c->grid_solve, 1});
    CK(dalloc(c, &d.partials, (size_t)2 * max_ctas * NRR_PARTIAL_STRIDE));
    // few CTAs: the kernel runs beside the closest-point search and should
    // take few of its SM slots
    d.n_xpart = std::max(1, std::min(std::max(1, c->num_sms / 4), (c->E2 + c->N + 255) / 256));
    CK(dalloc(c, &d.xpartials, (size_t)4 * d.n_xpart));
    d.st = c->d_state;
    d.nn_stats = nullptr;
    d.solve_stats = nullptr;
    d.fault_barrier = std::getenv("NRR_FAULT_BARRIER") ? 1 : 0;
    d.fault_halo = std::getenv("NRR_FAULT_HALO") ? 1 : 0;
    if (std::getenv("NRR_SOLVE_STATS")) {
        long long* ss = nullptr;
        CK(dalloc(c, &ss, 64));
        d.solve_stats = ss;
    }
    tm.lap("uploads");
    if (std::getenv("NRR_NN_STATS")) {
        // the most warps a search launches: 8 lanes per query, 4 queries
        // per warp, whole CTAs of 8 warps
        const size_t warps = ((size_t)P + 31) / 32 * 8;
        unsigned long long* ns = nullptr;
        CK(dalloc(c, &ns, warps * 4));
        d.nn_stats = ns;
        c->nn_stats_n = warps;
    }
    return NRR_OK;
}

template <typename T>
nrr_status median_distance(nrr_ctx* c, double* out) {
    DevProblem<T>& d = prob<T>(c);
    CK(nrr_launch_nn<T>(d, NRR_MODE_RAW, c->nn_lpq, c->stream));
    std::vector<T> d2((size_t)c->P);
    CK(cudaMemcpyAsync(d2.data(), d.d2, sizeof(T) * (size_t)c->P, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<double> dist((size_t)c->P);
    for (size_t i = 0; i < dist.size(); ++i) dist[i] = std::sqrt((double)d2[i]);
    // the middle element(s) by selection, not a full sort
    const size_t n = dist.size();
    std::nth_element(dist.begin(), dist.begin() + n / 2, dist.end());
    const double hi = dist[n / 2];
    if (n % 2) {
        *out = hi;
    } else {
        const double lo = *std::max_element(dist.begin(), dist.begin() + n / 2);
        *out = (lo + hi) / 2.0;
    }
    return NRR_OK;
}

template <typename T>
nrr_status read_X(nrr_ctx* c, const T* src, double* X) {
    std::vector<T> h((size_t)c->N * 12);
    CK(cudaMemcpyAsync(h.data(), src, sizeof(T) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<double> o(h.begin(), h.end());
    CK(cudaMemcpy(X, o.data(), sizeof(double) * o.size(), cudaMemcpyDefault));
    return NRR_OK;
}

template <typename T>
nrr_status write_X(nrr_ctx* c, T* dst, const double* X) {
    std::vector<double> h((size_t)c->N * 12);
    CK(cudaMemcpy(h.data(), X, sizeof(double) * h.size(), cudaMemcpyDefault));
    for (double x : h)
        if (!std::isfinite(x)) return fail(c, NRR_E_INVALID, "X has non-finite entries");
    std::vector<T> t(h.begin(), h.end());
    CK(cudaMemcpyAsync(dst, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}


// ---------------------------------------------------------------------------
// Unrolled MM steps: K plain MM steps (no Anderson mix, no safeguard) at the
// current stage's nu_a, nu_r, alpha, beta, with X^(0..K) kept as checkpoints;
// the backward recomputes closest points, weights and K at each checkpoint
// and solves the adjoint system with the same PCG.
// ---------------------------------------------------------------------------

// Runs the off-trajectory work of nrr_unroll / nrr_backward with the pass
// flags cleared, then puts the solver state back (the evaluations wrote
// v_hat into the non-kept buffer, as nrr_energy does).
struct StateGuard {
    nrr_ctx* c;
    NrrState saved{};
    bool is_open = false;
    nrr_status open() {
        nrr_status st = pull_state(c);
        if (st != NRR_OK) return st;
        saved = *c->h_state;
        is_open = true;
        c->h_state->done = 0;
        c->h_state->skip = 0;
        return push_state(c);
    }
    nrr_status close() {
        is_open = false;
        *c->h_state = saved;
        c->h_state->vlast = saved.vk ^ 1;
        return push_state(c);
    }
    // an early return (an error) still puts the state back
    ~StateGuard() {
        if (is_open) close();
    }
};

template <typename T>
nrr_status unroll_buffers(nrr_ctx* c, int K) {
    const size_t n12 = (size_t)c->N * 12, P = (size_t)c->P;
    if (c->ck_cap < K + 1) {
        if (c->d_ck) { CK(cudaFree(c->d_ck)); c->d_ck = nullptr; c->ck_cap = 0; }
        const int cap = std::max(K + 1, 11);
        CK(cudaMalloc(&c->d_ck, sizeof(T) * n12 * (size_t)cap));
        c->ck_cap = cap;
    }
    if (!c->d_adj) {
        CK(cudaMalloc(&c->d_adj, sizeof(T) * (3 * n12 + 3 * P)));
        CK(cudaMemsetAsync(c->d_adj, 0, sizeof(T) * n12, c->stream));   // the zero warm start
    }
    if (!c->d_adjd) CK(cudaMalloc(&c->d_adjd, sizeof(double) * (n12 + 3 * P)));
    if (!c->d_order) {
        CK(cudaMalloc(&c->d_order, sizeof(int) * P));
        CK(cudaMemcpyAsync(c->d_order, c->src_order.data(), sizeof(int) * P, cudaMemcpyHostToDevice, c->stream));
    }
    return NRR_OK;
}

// Closest points, Welsch weights, rotations and K, B at the checkpoint Xk.
template <typename T>
nrr_status unroll_system_at(nrr_ctx* c, const T* Xk) {
    DevProblem<T>& d = prob<T>(c);
    CK(cudaMemcpyAsync(d.Xeval, Xk, sizeof(T) * 12 * (size_t)c->N, cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_search<T>(c, d, NRR_MODE_EVAL));
    CK(nrr_launch_xterm<T>(d, NRR_MODE_EVAL, c->stream));
    CK(nrr_launch_energy<T>(d, NRR_MODE_EVAL, c->grid_energy, c->stream));
    CK(nrr_launch_assemble<T>(d, c->grid_asm, c->stream));
    return NRR_OK;
}

template <typename T>
nrr_status unroll_t(nrr_ctx* c, int K, const double* X0, double* XK) {
    nrr_status st = unroll_buffers<T>(c, K);
    if (st != NRR_OK) return st;
    const size_t n12 = (size_t)c->N * 12;
    T* ck = (T*)c->d_ck;
    st = write_X<T>(c, ck, X0);
    if (st != NRR_OK) return st;
    StateGuard guard{c};
    st = guard.open();
    if (st != NRR_OK) return st;
    c->unroll_prm[0] = c->h_state->nu_a;
    c->unroll_prm[1] = c->h_state->nu_r;
    c->unroll_prm[2] = c->h_state->alpha;
    c->unroll_prm[3] = c->h_state->beta;
    for (int k = 0; k < K; ++k) {
        st = unroll_system_at<T>(c, ck + (size_t)k * n12);
        if (st != NRR_OK) return st;
        DevProblem<T> ds = prob<T>(c);
        ds.X = ck + (size_t)k * n12;          // warm start X^(k)
        ds.warm_dx = nullptr;
        ds.fix_free = 0;
        ds.G = ck + (size_t)(k + 1) * n12;    // X^(k+1) = K^-1 B
        CK(launch_solve_on<T>(c, ds));
    }
    st = pull_state(c);
    if (st != NRR_OK) return st;
    const int dev_status = c->h_state->status;
    st = guard.close();
    if (st != NRR_OK) return st;
    if (dev_status != 0) return fail(c, (nrr_status)dev_status, "nrr_unroll: device-side check failed");
    c->unroll_K = K;
    if (XK) return read_X<T>(c, ck + (size_t)K * n12, XK);
    return NRR_OK;
}

template <typename T>
nrr_status unroll_backward_t(nrr_ctx* c, const double* C, double* grad_X, double* grad_src) {
    const int K = c->unroll_K;
    const size_t n12 = (size_t)c->N * 12, P = (size_t)c->P;
    T* ck = (T*)c->d_ck;
    T* zero = (T*)c->d_adj;
    T* lam = zero + n12;
    T* gt = lam + n12;
    T* ebuf = gt + n12;
    double* gd = c->d_adjd;
    double* gv = gd + n12;
    DevProblem<T>& d = prob<T>(c);
    StateGuard guard{c};
    nrr_status st = guard.open();
    if (st != NRR_OK) return st;
    const NrrState& h = *c->h_state;
    if (h.nu_a != c->unroll_prm[0] || h.nu_r != c->unroll_prm[1] || h.alpha != c->unroll_prm[2] ||
        h.beta != c->unroll_prm[3]) {
        guard.close();
        return fail(c, NRR_E_STATE, "nrr_backward mode 1: the stage changed since nrr_unroll");
    }
    CK(cudaMemsetAsync(gv, 0, sizeof(double) * 3 * P, c->stream));
    if (C == nullptr) {
        // L = E(X^(K)): closest points held at X^(K)
        CK(cudaMemcpyAsync(d.Xeval, ck + (size_t)K * n12, sizeof(T) * n12, cudaMemcpyDeviceToDevice, c->stream));
        CK(launch_search<T>(c, d, NRR_MODE_EVAL));
        CK(nrr_launch_xterm<T>(d, NRR_MODE_EVAL, c->stream));
        CK(nrr_launch_energy<T>(d, NRR_MODE_EVAL, c->grid_energy, c->stream));
        const int grid = std::max(1, (c->N + 31) / 32);
        CK(nrr_launch_gradient<T>(d, gd, gv, c->d_order, grid, c->stream));
    } else {
        std::vector<double> hC(n12);
        CK(cudaMemcpy(hC.data(), C, sizeof(double) * n12, cudaMemcpyDefault));
        for (double x : hC)
            if (!std::isfinite(x)) { guard.close(); return fail(c, NRR_E_INVALID, "cotangent has non-finite entries"); }
        CK(cudaMemcpyAsync(gd, hC.data(), sizeof(double) * n12, cudaMemcpyHostToDevice, c->stream));
    }
    CK(nrr_launch_to_t<T>(gd, gt, (int)n12, c->stream));
    for (int k = K - 1; k >= 0; --k) {
        st = unroll_system_at<T>(c, ck + (size_t)k * n12);
        if (st != NRR_OK) return st;
        DevProblem<T> ds = d;
        ds.X = zero;     // warm start 0
        ds.warm_dx = nullptr;
        ds.fix_free = 0;
        ds.Bv = gt;      // K lambda = g_bar
        ds.G = lam;
        CK(launch_solve_on<T>(c, ds));
        CK(nrr_launch_adjoint<T>(d, lam, ck + (size_t)(k + 1) * n12, c->d_order, ebuf, gv, gd, gt, c->stream));
    }
    if (grad_X) CK(cudaMemcpyAsync(grad_X, gd, sizeof(double) * n12, cudaMemcpyDefault, c->stream));
    if (grad_src) CK(cudaMemcpyAsync(grad_src, gv, sizeof(double) * 3 * P, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    st = pull_state(c);
    if (st != NRR_OK) return st;
    const int dev_status = c->h_state->status;
    st = guard.close();
    if (st != NRR_OK) return st;
    if (dev_status != 0) return fail(c, (nrr_status)dev_status, "nrr_backward: device-side check failed");
    return NRR_OK;
}


// ---------------------------------------------------------------------------
// Autotuner: the launch shapes of the two kernels whose best shape depends on
// the problem - lanes per closest-point query and the CTAs of the cluster
// solve (or the grid-wide solve) - are timed on the context's own data and
// the fastest is kept. Results can be cached in a text table keyed by the
// precision and the half-octave buckets of P, T and N.
// ---------------------------------------------------------------------------
struct TuneKey {
    int fp64, bP, bT, bN;
};

int half_octave(int64_t x) { return (int)std::floor(2.0 * std::log2((double)std::max<int64_t>(x, 1))); }

TuneKey tune_key(const nrr_ctx* c) { return {c->fp64 ? 1 : 0, half_octave(c->P), half_octave(c->T), half_octave(c->N)}; }

// Last line of the table that matches key:
// "nrr-tune <fp64> <bP> <bT> <bN> <lpq> <ctas> [<tensor cores>]".
bool table_lookup(const char* path, const TuneKey& k, int* lpq, int* ctas, int* tc = nullptr) {
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        int a[7] = {0, 0, 0, 0, 0, 0, 0};
        const int n = std::sscanf(line, "nrr-tune %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6]);
        if (n >= 6 && a[0] == k.fp64 && a[1] == k.bP && a[2] == k.bT && a[3] == k.bN) {
            *lpq = a[4];
            *ctas = a[5];
            if (tc) *tc = n == 7 ? a[6] : 0;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void table_append(const char* path, const TuneKey& k, int lpq, int ctas, int tc = 0) {
    FILE* f = path ? std::fopen(path, "a") : nullptr;
    if (!f) return;
    std::fprintf(f, "nrr-tune %d %d %d %d %d %d %d\n", k.fp64, k.bP, k.bT, k.bN, lpq, ctas, tc);
    std::fclose(f);
}

// Mean device milliseconds of reps launches of f() on the context's stream,
// after one untimed launch.
template <typename F>
nrr_status time_launches(nrr_ctx* c, int reps, F&& f, double* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    cudaError_t e = f();
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = f();
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(e);
    *ms = (double)t / reps;
    return NRR_OK;
}

bool valid_lpq(int v) { return v == 1 || v == 2 || v == 4 || v == 8; }

// Applies a launch configuration (validated) and recaptures the pass graph.
template <typename T>
nrr_status apply_config(nrr_ctx* c, int lpq, int ctas, int tc) {
    if (!valid_lpq(lpq)) return fail(c, NRR_E_INVALID, "lanes per query must be 1, 2, 4 or 8");
    if (tc != 0 && tc != 1) return fail(c, NRR_E_INVALID, "nn_tensor_cores must be 0 or 1");
    if (tc && c->fp64) return fail(c, NRR_E_INVALID, "the tensor-core search serves the mixed-precision path only");
    if (ctas < 0 || ctas > 16 || !set_solver<T>(c, ctas))
        return fail(c, NRR_E_INVALID, "the cluster solve with " + std::to_string(ctas) + " CTAs does not fit");
    c->nn_lpq = lpq;
    c->nn_tc = tc != 0;
    return capture_graph(c);
}

template <typename T>
nrr_status tune_t(nrr_ctx* c, int reps, int* best_lpq, int* best_ctas, int* best_tc, double* nn_ms,
                  double* solve_ms) {
    DevProblem<T>& d = prob<T>(c);
    const size_t n12 = (size_t)c->N * 12;
    if (!c->d_tune) CK(cudaMalloc(&c->d_tune, 2 * sizeof(T) * n12));
    T* x0 = (T*)c->d_tune;
    // a surrogate system to time the solve on: the first pass from the
    // start; the solve is then timed from that pass's own warm start X^(0)
    // (the pass's mix already holds its solution)
    nrr_status st = nrr_reset(c);
    if (st != NRR_OK) return st;
    CK(cudaMemcpyAsync(x0, d.X, sizeof(T) * n12, cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_pass_any(c));
    CK(cudaMemcpyAsync(d.Xeval, d.X, sizeof(T) * n12, cudaMemcpyDeviceToDevice, c->stream));
    // closest points at the current iterate, per lanes-per-query
    *nn_ms = INFINITY;
    for (int lpq : {1, 2, 4, 8}) {
        double ms = 0;
        st = time_launches(c, reps, [&]() { return nrr_launch_nn<T>(d, NRR_MODE_EVAL, lpq, c->stream); }, &ms);
        if (st != NRR_OK) return st;
        if (ms < *nn_ms) { *nn_ms = ms; *best_lpq = lpq; }
    }
    if (!std::isfinite(*nn_ms)) *best_lpq = c->nn_lpq;
    *best_tc = 0;
    if (!c->fp64) {
        // the tensor-core candidate search (same results as the exact one)
        double ms = 0;
        st = time_launches(c, reps, [&]() { return nrr_launch_nn_tc(c->df, NRR_MODE_EVAL, c->stream); }, &ms);
        if (st != NRR_OK) return st;
        if (ms < *nn_ms) { *nn_ms = ms; *best_tc = 1; }
    }
    // the solve of that system, per cluster size (0: grid-wide); the
    // solution goes to scratch, the pass state is not touched
    DevProblem<T> ds = d;
    ds.X = x0;
    ds.warm_dx = nullptr;
    ds.fix_free = 0;
    ds.G = x0 + n12;
    *solve_ms = INFINITY;
    const int keep_C = c->cl_C;
    for (int C : {16, 8, 4, 2, 1, 0}) {
        if (!set_solver<T>(c, C)) continue;
        if (C == 0 && !c->coop) continue;
        double ms = 0;
        st = time_launches(c, reps, [&]() { return launch_solve_on<T>(c, ds); }, &ms);
        if (st != NRR_OK) {
            // a shape the device cannot launch (resources): not a candidate
            cudaGetLastError();
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return st;
            continue;
        }
        if (ms < *solve_ms) { *solve_ms = ms; *best_ctas = C; }
    }
    if (!std::isfinite(*solve_ms)) *best_ctas = keep_C;
    st = pull_state(c);
    if (st != NRR_OK) return st;
    if (c->h_state->status != 0) return fail(c, (nrr_status)c->h_state->status, "nrr_tune: device-side check failed");
    // the evaluations wrote v_hat into the non-kept buffer
    c->h_state->vlast = c->h_state->vk ^ 1;
    st = push_state(c);
    if (st != NRR_OK) return st;
    st = apply_config<T>(c, *best_lpq, *best_ctas, *best_tc);
    if (st != NRR_OK) return st;
    return nrr_reset(c);
}


// ---------------------------------------------------------------------------
// The preliminary version's solver (Sec. 3.3.4, the Remark on the
// preliminary version; Sec. 4.3), as a comparison solver on the same energy:
// each outer iteration holds the closest points at X^k, which makes E a
// non-quadratic surrogate (it keeps Welsch's functions and the rotation
// term), and minimises it by an inner L-BFGS with a backtracking line search
// (sufficient decrease c1) that ends at |g| <= g_tol |g_0| or after
// max_inner steps. The nu annealing, alpha, beta and the stopping tests are
// those of Algorithm 2. Every evaluation (closest points, energy terms,
// gradient, direction, trial point) runs in the library's kernels; the host
// takes the accept/reject decisions from the energies it reads back.
// ---------------------------------------------------------------------------
void host_end_stage(NrrState& s) {
    if (s.nu_a == s.nu_a_min) {
        s.done = 1;
        return;
    }
    s.nu_a = std::max(s.nu_a * 0.5, s.nu_a_min);
    s.nu_r = s.nu_r * 0.5;
    s.stage += 1;
    host_stage_weights(s);
    s.E_prev = std::numeric_limits<double>::infinity();
    s.n_solves_stage = 0;
}

template <typename T>
nrr_status lbfgs_t(nrr_ctx* c, const nrr_lbfgs_params& lb, int max_outer) {
    DevProblem<T>& d = prob<T>(c);
    const int n = c->N * 12;
    const size_t P = (size_t)c->P;
    const int m = lb.m;
    if (c->lb_m < m || !c->lb_buf) {
        if (c->lb_buf) { CK(cudaFree(c->lb_buf)); c->lb_buf = nullptr; }
        CK(cudaMalloc(&c->lb_buf, sizeof(double) * ((size_t)2 * m * n + 3 * (size_t)n + 8)));
        c->lb_m = m;
    }
    if (!c->lb_t) CK(cudaMalloc(&c->lb_t, sizeof(T) * ((size_t)n + 3 * P)));
    if (!c->d_order) {
        CK(cudaMalloc(&c->d_order, sizeof(int) * P));
        CK(cudaMemcpyAsync(c->d_order, c->src_order.data(), sizeof(int) * P, cudaMemcpyHostToDevice, c->stream));
    }
    double* S = c->lb_buf;
    double* Y = S + (size_t)m * n;
    double* g = Y + (size_t)m * n;
    double* gn = g + n;
    double* dv = gn + n;
    double* scal = dv + n;
    T* Xk = (T*)c->lb_t;
    T* vk = Xk + n;
    double hs[8];
    const int grid_g = std::max(1, (c->N + 31) / 32);
    nrr_status st = pull_state(c);
    if (st != NRR_OK) return st;
    NrrState& h = *c->h_state;
    const size_t vbytes = sizeof(T) * 3 * P;
    auto vhat_eval = [&]() { return d.vhat + (size_t)(h.vk ^ 1) * 3 * P; };
    // energy at Xeval, with the closest points searched (true) or held
    auto energy_at_eval = [&](bool search, double* E) -> nrr_status {
        if (search) CK(launch_search<T>(c, d, NRR_MODE_EVAL));
        else CK(nrr_launch_fixed_corr<T>(d, c->stream));
        CK(nrr_launch_xterm<T>(d, NRR_MODE_EVAL, c->stream));
        CK(nrr_launch_energy<T>(d, NRR_MODE_EVAL, c->grid_energy, c->stream));
        CK(cudaMemcpyAsync(c->h_state->E_eval, &c->d_state->E_eval, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *E = c->h_state->E_eval[0];
        return NRR_OK;
    };
    auto read_scal = [&]() -> nrr_status {
        CK(cudaMemcpyAsync(hs, scal, sizeof hs, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return NRR_OK;
    };
    for (int outer = 0; outer < max_outer && !h.done; ++outer) {
        // the device state (stage parameters read by the kernels) follows
        // the host's decisions of the previous iteration
        if (outer > 0) {
            if ((st = push_state(c)) != NRR_OK) return st;
        }
        if ((st = pull_state(c)) != NRR_OK) return st;
        if (h.status != 0) break;
        // ---- closest points and the energy at X^k (stopping tests as Algorithm 2)
        CK(cudaMemcpyAsync(d.Xeval, d.X, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream));
        double E = 0.0;
        if ((st = energy_at_eval(true, &E)) != NRR_OK) return st;
        h.E = E;
        h.E_align = h.E_eval[1]; h.E_reg = h.E_eval[2]; h.E_rot = h.E_eval[3];
        h.n_passes += 1;
        h.kept = 1;
        h.solved = 0;
        if (h.rel_tol > 0 && std::isfinite(h.E_prev) && std::fabs(h.E_prev - E) < h.rel_tol * std::fabs(h.E_prev)) {
            host_end_stage(h);
            continue;
        }
        h.E_prev = E;
        CK(cudaMemcpyAsync(vk, vhat_eval(), vbytes, cudaMemcpyDeviceToDevice, c->stream));
        // ---- inner L-BFGS on the surrogate (closest points held)
        CK(cudaMemcpyAsync(Xk, d.X, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream));
        CK(nrr_launch_gradient<T>(d, g, nullptr, c->d_order, grid_g, c->stream));
        double f = E, g0 = 0.0;
        int mk = 0, head = 0;
        for (int it = 0; it < lb.max_inner; ++it) {
            CK(nrr_launch_lbfgs_dir<T>(n, g, S, Y, mk, head, m, dv, scal, c->stream));
            if ((st = read_scal()) != NRR_OK) return st;
            if (it == 0) g0 = hs[1];
            if (!(hs[1] > lb.g_tol * g0)) break;
            const double gd = hs[0];
            double t = 1.0, Et = 0.0;
            bool accepted = false;
            for (int k = 0; k <= lb.max_halvings; ++k) {
                CK(nrr_launch_lbfgs_axpy<T>(n, Xk, t, dv, d.Xeval, c->stream));
                if ((st = energy_at_eval(false, &Et)) != NRR_OK) return st;
                if (Et <= f + lb.c1 * t * gd) { accepted = true; break; }
                t *= 0.5;
            }
            if (!accepted) break;
            CK(nrr_launch_gradient<T>(d, gn, nullptr, c->d_order, grid_g, c->stream));
            CK(nrr_launch_lbfgs_pair<T>(n, Xk, d.Xeval, g, gn, S, Y, head, scal, c->stream));
            if ((st = read_scal()) != NRR_OK) return st;
            if (hs[2] > 1e-12 * hs[3] * hs[4]) {
                head = (head + 1) % m;
                mk = std::min(mk + 1, m);
            }
            f = Et;
        }
        // ---- the new outer iterate and its displacement
        CK(cudaMemcpyAsync(d.X, Xk, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(d.Xeval, Xk, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream));
        CK(nrr_launch_fixed_corr<T>(d, c->stream));
        CK(nrr_launch_max_disp<T>((int)P, vhat_eval(), vk, scal, c->stream));
        if ((st = read_scal()) != NRR_OK) return st;
        h.max_disp = std::sqrt(hs[6]);
        h.solved = 1;
        h.n_solves += 1;
        h.n_solves_stage += 1;
        if ((h.rel_tol <= 0 && h.max_disp < h.eps) || h.n_solves_stage >= h.max_iters_stage) host_end_stage(h);
    }
    // later passes of Algorithm 2 start a fresh Anderson history; the
    // evaluation buffer holds v_hat at the last iterate
    h.aa_count = 0;
    h.aa_head = 0;
    h.just_reverted = 0;
    h.pending_stop = 0;
    h.skip = 0;
    h.vlast = h.vk ^ 1;
    return push_state(c);
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the solver state that a pass reads and that later
// passes do not rebuild - the device control block, the iterate X, the MM
// results G, G_prev, F_prev, the Anderson rings dF, dG and both deformed-
// source buffers (the stop test compares with the kept one). Layout: a
// header {magic, version, precision, P, N, m, problem hash}, then NrrState, then the
// arrays in that order, in the context's precision.
// ---------------------------------------------------------------------------
struct CkptHeader {
    uint64_t magic;      // "nrr-ckpt"
    uint32_t version, fp64;
    int64_t P, N, m;
    uint64_t problem;    // hash of the inputs, the graph and the parameters
};
constexpr uint32_t kCkptVersion = 2u;
constexpr uint64_t kCkptMagic = 0x74706b632d72726eull;

size_t ckpt_bytes(const nrr_ctx* c) {
    const size_t esz = c->fp64 ? sizeof(double) : sizeof(float);
    const size_t m = (size_t)std::max(1, c->prm.aa_m);
    const size_t n12 = (size_t)c->N * 12;
    return sizeof(CkptHeader) + sizeof(NrrState) + esz * (4 * n12 + 2 * m * n12 + 6 * (size_t)c->P);
}

template <typename T>
nrr_status ckpt_copy(nrr_ctx* c, unsigned char* host, bool save) {
    DevProblem<T>& d = prob<T>(c);
    const size_t m = (size_t)std::max(1, c->prm.aa_m);
    const size_t n12 = (size_t)c->N * 12;
    T* arrays[6] = {d.X, d.G, d.Gprev, d.Fprev, d.dF, d.dG};
    const size_t counts[6] = {n12, n12, n12, n12, m * n12, m * n12};
    unsigned char* p = host;
    for (int k = 0; k < 6; ++k) {
        const size_t nb = sizeof(T) * counts[k];
        if (save) CK(cudaMemcpyAsync(p, arrays[k], nb, cudaMemcpyDeviceToHost, c->stream));
        else CK(cudaMemcpyAsync(arrays[k], p, nb, cudaMemcpyHostToDevice, c->stream));
        p += nb;
    }
    const size_t nv = sizeof(T) * 6 * (size_t)c->P;
    if (save) CK(cudaMemcpyAsync(p, d.vhat, nv, cudaMemcpyDeviceToHost, c->stream));
    else CK(cudaMemcpyAsync(d.vhat, p, nv, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void nrr_params_default(nrr_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->graph_radius = 0.0;
    p->max_influence = 8;
    p->nu_a = 0.0;
    p->nu_r = 0.0;
    p->nu_a_min = 0.0;
    p->anneal = 1;
    p->k_alpha = 100.0;
    p->k_beta = 1.0;
    p->alpha = -1.0;
    p->beta = -1.0;
    p->aa_m = 5;
    p->max_iters_per_stage = 100;
    p->max_total_passes = 100000;
    p->eps = 0.0;
    p->rel_energy_tol = 0.0;
    p->precision = NRR_MIXED;
    p->pcg_tol = 0.0;
    p->pcg_max_iters = 500;
    p->solve_ctas = 0;
    p->robust = NRR_WELSCH;
    p->nu_schedule = NRR_NU_ANNEAL;
    p->graph_on_gpu = 0;
}

const char* nrr_last_error(const nrr_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

void nrr_destroy(nrr_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
    if (c->d_states1) cudaFree(c->d_states1);
    if (c->d_hist) cudaFree(c->d_hist);
    if (c->d_ctrl) cudaFree(c->d_ctrl);
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    for (void* p : c->allocs) cudaFree(p);
    if (c->d_order) cudaFree(c->d_order);
    if (c->d_grad) cudaFree(c->d_grad);
    if (c->d_tune) cudaFree(c->d_tune);
    if (c->d_ck) cudaFree(c->d_ck);
    if (c->d_adj) cudaFree(c->d_adj);
    if (c->d_adjd) cudaFree(c->d_adjd);
    if (c->lb_buf) cudaFree(c->lb_buf);
    if (c->lb_t) cudaFree(c->lb_t);
    if (c->d_state) cudaFree(c->d_state);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

nrr_status nrr_create(nrr_ctx** out, const float* src_xyz, const float* src_nrm, int64_t P,
                      const float* tgt_xyz, const float* tgt_nrm, int64_t T,
                      const nrr_params* params, void* cuda_stream) {
    NvtxRange nvtx_range("nrr_create");
    nrr_ctx* c = nullptr;
    if (!out) return fail(nullptr, NRR_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!src_xyz || !tgt_xyz) return fail(nullptr, NRR_E_INVALID, "point arrays must not be NULL");
    if (P < 1 || T < 1) return fail(nullptr, NRR_E_INVALID, "P and T must be >= 1");
    if (P >= (1LL << 25) || T >= (1LL << 30)) return fail(nullptr, NRR_E_INVALID, "P must be < 2^25 and T < 2^30");
    nrr_params prm;
    if (params) prm = *params; else nrr_params_default(&prm);
    if (prm.max_influence < 1 || prm.max_influence > NRR_MAX_INFL)
        return fail(nullptr, NRR_E_INVALID, "max_influence must be in 1..8");
    if (prm.aa_m < 0 || prm.aa_m > NRR_AA_MMAX) return fail(nullptr, NRR_E_INVALID, "aa_m must be in 0..8");
    if (prm.precision != NRR_FP64 && prm.precision != NRR_MIXED)
        return fail(nullptr, NRR_E_INVALID, "precision must be NRR_FP64 or NRR_MIXED");
    if (prm.max_iters_per_stage < 1 || prm.pcg_max_iters < 1 || prm.max_total_passes < 1)
        return fail(nullptr, NRR_E_INVALID, "iteration caps must be >= 1");
    if (prm.src_faces && (prm.n_src_faces < 1 || prm.n_src_faces > (1LL << 28)))
        return fail(nullptr, NRR_E_INVALID, "n_src_faces must be in 1..2^28 when src_faces is given");
    if (prm.src_faces && prm.graph_on_gpu)
        return fail(nullptr, NRR_E_INVALID, "graph_on_gpu is not available for a mesh source (src_faces)");
    if (prm.solve_ctas < -1 || prm.solve_ctas > 16)
        return fail(nullptr, NRR_E_INVALID, "solve_ctas must be in -1..16");
    if (prm.robust < NRR_WELSCH || prm.robust > NRR_L2_TRUNCATED)
        return fail(nullptr, NRR_E_INVALID, "robust must be NRR_WELSCH, NRR_L2 or NRR_L2_TRUNCATED");
    if (prm.graph_on_gpu != 0 && prm.graph_on_gpu != 1)
        return fail(nullptr, NRR_E_INVALID, "graph_on_gpu must be 0 or 1");
    if (prm.nu_schedule < NRR_NU_ANNEAL || prm.nu_schedule > NRR_NU_FIXED_MED)
        return fail(nullptr, NRR_E_INVALID, "nu_schedule must be one of nrr_nu_schedule");
    if (!(std::isfinite(prm.graph_radius) && std::isfinite(prm.nu_a) && std::isfinite(prm.nu_r) &&
          std::isfinite(prm.nu_a_min) && std::isfinite(prm.eps) && std::isfinite(prm.k_alpha) &&
          std::isfinite(prm.k_beta) && std::isfinite(prm.alpha) && std::isfinite(prm.beta)))
        return fail(nullptr, NRR_E_INVALID, "parameters must be finite");
    if (prm.pcg_tol <= 0) prm.pcg_tol = prm.precision == NRR_FP64 ? 1e-12 : 1e-6;

    c = new (std::nothrow) nrr_ctx();
    if (!c) return fail(nullptr, NRR_E_OOM, "host allocation failed");
    std::unique_ptr<nrr_ctx, void (*)(nrr_ctx*)> guard(c, nrr_destroy);
    c->prm = prm;
    c->fp64 = prm.precision == NRR_FP64;
    c->P = P;
    c->T = T;
    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    SetupTimer tm;
    std::vector<float> src, tgt, tmp;
    CK(fetch_floats(src_xyz, (size_t)P * 3, src, c->stream));
    CK(fetch_floats(tgt_xyz, (size_t)T * 3, tgt, c->stream));
    if (!finite3(src) || !finite3(tgt)) return fail(nullptr, NRR_E_INVALID, "non-finite point coordinates");
    if (src_nrm) {
        CK(fetch_floats(src_nrm, (size_t)P * 3, tmp, c->stream));
        if (!finite3(tmp)) return fail(nullptr, NRR_E_INVALID, "non-finite source normals");
    }
    if (tgt_nrm) {
        CK(fetch_floats(tgt_nrm, (size_t)T * 3, tmp, c->stream));
        if (!finite3(tmp)) return fail(nullptr, NRR_E_INVALID, "non-finite target normals");
    }
    tm.lap("inputs");
    CurveOrders co;
    CK(co.compute(src, P, tgt, T, c->stream));
    tm.lap("curve orders");
    // l-bar, radius and the deformation graph (Algorithm 1)
    std::vector<double> V(src.begin(), src.end());
    const bool need_lbar = prm.graph_radius <= 0 || prm.nu_r <= 0 || prm.nu_a_min <= 0;
    if (prm.src_faces) {
        std::vector<int> F((size_t)prm.n_src_faces * 3);
        CK(cudaMemcpyAsync(F.data(), prm.src_faces, sizeof(int) * F.size(), cudaMemcpyDefault, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const nrr_status gs = graph_from_mesh(V, P, F, prm.graph_radius, prm.max_influence, c->hg, "nrr_create");
        if (gs != NRR_OK) return gs;
    } else if (prm.graph_on_gpu) {
        const nrr_status gs = graph_on_device(src.data(), V, P, prm.graph_radius, prm.max_influence, need_lbar,
                                              c->stream, c->hg);
        if (gs != NRR_OK) return gs;
    } else if (!nrr_graph_and_spacing(V.data(), P, prm.graph_radius, prm.max_influence, need_lbar, c->hg)) {
        return fail(nullptr, NRR_E_INVALID, "graph radius must be positive");
    }
    tm.lap("l-bar + graph (Algorithm 1)");
    c->N = (int)c->hg.nodes.size();
    c->E2 = (int)c->hg.r.size();
    c->problem_hash = problem_hash(src, tgt, c->hg, prm);
    // launch geometry
    if (const char* e = std::getenv("NRR_NN_LPQ")) {
        const int v = std::atoi(e);
        if (v == 1 || v == 2 || v == 4 || v == 8) c->nn_lpq = v;
    }
    c->grid_energy = 2 * c->num_sms;
    // assembly: one warp per diagonal block, one per four off-diagonal blocks
    c->grid_asm = std::max(1, std::min(16 * c->num_sms, (c->N + (c->E2 + 3) / 4 + 7) / 8));
    // Anderson kernels: one element of X per thread up to grid_energy CTAs
    // (the partials buffer is sized for grid_energy)
    c->grid_aa = std::max(1, std::min(c->grid_energy, (c->N * 12 + 255) / 256));
    {
        const int per_cta = nrr_solve_threads() / 3;   // (node, column) pairs per thread
        int want = std::max(1, (c->N + per_cta - 1) / per_cta);
        const int occ = c->fp64 ? nrr_solve_max_blocks_per_sm<double>() : nrr_solve_max_blocks_per_sm<float>();
        c->grid_solve = std::max(1, std::min(want, c->num_sms * std::max(1, occ)));
        c->grid_solve = std::min(c->grid_solve, c->num_sms);
    }
    // device state
    CK(cudaMalloc(&c->d_state, sizeof(NrrState)));
    CK(cudaMallocHost(&c->h_state, sizeof(NrrState)));
    std::memset(c->h_state, 0, sizeof(NrrState));
    CK(cudaMalloc(&c->d_hist, sizeof(nrr_step_info) * kHistCap));
    CK(cudaMalloc(&c->d_states1, sizeof(NrrState*)));
    CK(cudaMemcpy(c->d_states1, &c->d_state, sizeof(NrrState*), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_ctrl, 2 * sizeof(int)));
    CK(cudaMallocHost(&c->h_ctrl, 2 * sizeof(int)));
    tm.lap("hash + state buffers");
    nrr_status st = c->fp64 ? build_device<double>(c, src, tgt, co, tm) : build_device<float>(c, src, tgt, co, tm);
    if (st != NRR_OK) return st;
    if (c->fp64) choose_solver<double>(c); else choose_solver<float>(c);
    tm.lap("solver choice");
    NrrState& s = *c->h_state;
    s.k_alpha = prm.k_alpha; s.k_beta = prm.k_beta;
    s.alpha_fixed = prm.alpha; s.beta_fixed = prm.beta;
    s.n_src = (double)P; s.n_edges = std::max(1.0, (double)c->hg.edges.size() / 2.0); s.n_nodes = std::max(1, c->N);
    s.eps = prm.eps > 0 ? prm.eps : 1e-5 * c->diag;
    s.rel_tol = prm.rel_energy_tol;
    s.max_iters_stage = prm.max_iters_per_stage;
    s.aa_m = prm.aa_m;
    s.robust = prm.robust;
    s.nu_a = 1.0; s.nu_r = 1.0;
    CK(cudaMemcpyAsync(c->d_state, c->h_state, sizeof(NrrState), cudaMemcpyHostToDevice, c->stream));
    double nu_a0 = prm.nu_a;
    if (nu_a0 <= 0) {
        st = c->fp64 ? median_distance<double>(c, &nu_a0) : median_distance<float>(c, &nu_a0);
        if (st != NRR_OK) return st;
    }
    tm.lap("median distance");
    double nu_min = prm.nu_a_min > 0 ? prm.nu_a_min : c->hg.lbar / std::sqrt(3.0);
    if (!prm.anneal) nu_min = nu_a0;
    s.nu_a_min = nu_min;
    s.nu_a = std::max(nu_a0, nu_min);
    s.nu_r = prm.nu_r > 0 ? prm.nu_r : 3.0 * c->hg.lbar;
    if (!(s.nu_a > 0) || !(s.nu_r > 0)) return fail(nullptr, NRR_E_INVALID, "nu_a and nu_r must be positive");
    if (prm.nu_schedule != NRR_NU_ANNEAL) {
        // the stages the annealing would run: nu_a halves (clamped at
        // nu_a_min), nu_r halves, until nu_a == nu_a_min
        double na = s.nu_a, nr = s.nu_r;
        while (na != s.nu_a_min) {
            na = std::max(na * 0.5, s.nu_a_min);
            nr = nr * 0.5;
        }
        if (prm.nu_schedule == NRR_NU_FIXED_MIN) { s.nu_a = na; s.nu_r = nr; }
        else if (prm.nu_schedule == NRR_NU_FIXED_MED) { s.nu_a = (s.nu_a + na) / 2.0; s.nu_r = (s.nu_r + nr) / 2.0; }
        s.nu_a_min = s.nu_a;
    }
    if (prm.robust == NRR_L2) s.nu_a_min = s.nu_a;   // no nu in the energy: one stage
    host_stage_weights(s);
    host_restart_stage(s);
    c->nu_a0 = s.nu_a;
    c->nu_r0 = s.nu_r;
    st = push_state(c);
    if (st != NRR_OK) return st;
    st = capture_graph(c);
    if (st != NRR_OK) return st;
    tm.lap("state + graph capture");
    guard.release();
    *out = c;
    return NRR_OK;
}

nrr_status nrr_step(nrr_ctx* c, nrr_step_info* info) {
    NvtxRange nvtx_range("nrr_step");
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    if (c->h_state->done) return fail(c, NRR_E_STATE, "the solve has already returned");
    nrr_status st = run_pass(c);
    if (st != NRR_OK) { c->failed = true; return st; }
    st = pull_state(c);
    if (st != NRR_OK) { c->failed = true; return st; }
    fill_info(*c->h_state, info);
    if (c->h_state->status != 0) {
        c->failed = true;
        return fail(c, (nrr_status)c->h_state->status, "device-side wait timed out");
    }
    return NRR_OK;
}

nrr_status nrr_solve(nrr_ctx* c, int max_passes, nrr_step_info* info) {
    NvtxRange nvtx_range("nrr_solve");
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    const int cap = max_passes > 0 ? max_passes : c->prm.max_total_passes;
    nrr_status st = pull_state(c);
    if (st != NRR_OK) return st;
    const int start = c->h_state->n_passes;
    if (c->use_graph && c->loop_exec && !c->h_state->done) {
        // every pass on the device: one launch, one read of the state
        c->h_ctrl[0] = 0;
        c->h_ctrl[1] = cap;
        CK(cudaMemcpyAsync(c->d_ctrl, c->h_ctrl, 2 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CK(cudaGraphLaunch(c->loop_exec, c->stream));
        CK(cudaMemcpyAsync(c->h_ctrl, c->d_ctrl, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        st = pull_state(c);
        c->hist_n = std::min(c->h_ctrl[0], kHistCap);
        if (st != NRR_OK) { c->failed = true; return st; }
        if (c->h_state->status != 0) {
            c->failed = true;
            fill_info(*c->h_state, info);
            return fail(c, (nrr_status)c->h_state->status, "device-side wait timed out");
        }
        fill_info(*c->h_state, info);
        return c->h_state->done ? NRR_OK : NRR_E_NOT_CONVERGED;
    }
    c->hist_n = 0;   // the host-launched loop records no history
    int launched = 0;
    const int batch = 4;
    while (!c->h_state->done && c->h_state->n_passes - start < cap) {
        const int left = cap - (c->h_state->n_passes - start);
        const int nb = std::min(batch, left);
        for (int k = 0; k < nb; ++k) {
            st = run_pass(c);
            if (st != NRR_OK) { c->failed = true; return st; }
        }
        launched += nb;
        st = pull_state(c);
        if (st != NRR_OK) { c->failed = true; return st; }
        if (c->h_state->status != 0) {
            c->failed = true;
            fill_info(*c->h_state, info);
            return fail(c, (nrr_status)c->h_state->status, "device-side wait timed out");
        }
    }
    fill_info(*c->h_state, info);
    return c->h_state->done ? NRR_OK : NRR_E_NOT_CONVERGED;
}

nrr_status nrr_enqueue_passes(nrr_ctx* c, int n) {
    if (!c || n < 0) return fail(c, NRR_E_INVALID, "bad argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    for (int k = 0; k < n; ++k) {
        nrr_status st = run_pass(c);
        if (st != NRR_OK) { c->failed = true; return st; }
    }
    return NRR_OK;
}

nrr_status nrr_time_kernels(nrr_ctx* c, int n, double out_ms[6]) {
    if (!c || n < 0 || !out_ms) return fail(c, NRR_E_INVALID, "bad argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    constexpr int kSteps = 6;
    cudaEvent_t ev[kSteps + 1];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    nrr_status result = NRR_OK;
    for (int k = 0; k < n && result == NRR_OK; ++k) {
        cudaError_t e = cudaEventRecord(ev[0], c->stream);
        for (int s = 0; s < kSteps && e == cudaSuccess; ++s) {
            if (c->fp64) {
                DevProblem<double>& d = c->dd;
                e = s == 0 ? launch_search<double>(c, d, NRR_MODE_PASS)
                  : s == 1 ? nrr_launch_xterm<double>(d, NRR_MODE_PASS, c->stream)
                  : s == 2 ? nrr_launch_energy<double>(d, NRR_MODE_PASS, c->grid_energy, c->stream)
                  : s == 3 ? nrr_launch_assemble<double>(d, c->grid_asm, c->stream)
                  : s == 4 ? launch_solve_step<double>(c)
                           : nrr_launch_aa<double>(d, c->grid_aa, c->stream);
            } else {
                DevProblem<float>& d = c->df;
                e = s == 0 ? launch_search<float>(c, d, NRR_MODE_PASS)
                  : s == 1 ? nrr_launch_xterm<float>(d, NRR_MODE_PASS, c->stream)
                  : s == 2 ? nrr_launch_energy<float>(d, NRR_MODE_PASS, c->grid_energy, c->stream)
                  : s == 3 ? nrr_launch_assemble<float>(d, c->grid_asm, c->stream)
                  : s == 4 ? launch_solve_step<float>(c)
                           : nrr_launch_aa<float>(d, c->grid_aa, c->stream);
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev[s + 1], c->stream);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[kSteps]);
        for (int s = 0; s < kSteps && e == cudaSuccess; ++s) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
            out_ms[s] += ms;
        }
        if (e != cudaSuccess) {
            c->failed = true;
            result = fail(c, NRR_E_CUDA, std::string("nrr_time_kernels: ") + cudaGetErrorString(e));
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return result;
}

nrr_status nrr_reset(nrr_ctx* c) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    std::vector<double> I((size_t)c->N * 12, 0.0);
    for (int j = 0; j < c->N; ++j) { I[(size_t)12 * j] = 1; I[(size_t)12 * j + 4] = 1; I[(size_t)12 * j + 8] = 1; }
    nrr_status st = c->fp64 ? write_X<double>(c, c->dd.X, I.data()) : write_X<float>(c, c->df.X, I.data());
    if (st != NRR_OK) return st;
    st = pull_state(c);
    if (st != NRR_OK) return st;
    NrrState& s = *c->h_state;
    s.nu_a = c->nu_a0;
    s.nu_r = c->nu_r0;
    s.stage = 0;
    s.n_passes = s.n_solves = s.n_rejected = 0;
    s.max_disp = 0;
    s.kept = s.solved = 0;
    host_stage_weights(s);
    host_restart_stage(s);
    return push_state(c);
}

nrr_status nrr_energy(nrr_ctx* c, const double* X, double out_terms[4]) {
    NvtxRange nvtx_range("nrr_energy");
    if (!c || !out_terms) return fail(c, NRR_E_INVALID, "NULL argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    nrr_status st;
    if (c->fp64) {
        if (X) { st = write_X<double>(c, c->dd.Xeval, X); if (st != NRR_OK) return st; }
        else CK(cudaMemcpyAsync(c->dd.Xeval, c->dd.X, sizeof(double) * 12 * (size_t)c->N, cudaMemcpyDeviceToDevice, c->stream));
        CK(launch_search<double>(c, c->dd, NRR_MODE_EVAL));
        CK(nrr_launch_xterm<double>(c->dd, NRR_MODE_EVAL, c->stream));
        CK(nrr_launch_energy<double>(c->dd, NRR_MODE_EVAL, c->grid_energy, c->stream));
    } else {
        if (X) { st = write_X<float>(c, c->df.Xeval, X); if (st != NRR_OK) return st; }
        else CK(cudaMemcpyAsync(c->df.Xeval, c->df.X, sizeof(float) * 12 * (size_t)c->N, cudaMemcpyDeviceToDevice, c->stream));
        CK(launch_search<float>(c, c->df, NRR_MODE_EVAL));
        CK(nrr_launch_xterm<float>(c->df, NRR_MODE_EVAL, c->stream));
        CK(nrr_launch_energy<float>(c->df, NRR_MODE_EVAL, c->grid_energy, c->stream));
    }
    st = pull_state(c);
    if (st != NRR_OK) return st;
    for (int k = 0; k < 4; ++k) out_terms[k] = c->h_state->E_eval[k];
    // the evaluation wrote v_hat, rho and d2 of X into the non-kept buffers
    c->h_state->vlast = c->h_state->vk ^ 1;
    return push_state(c);
}

nrr_status nrr_set_transforms(nrr_ctx* c, const double* X) {
    if (!c || !X) return fail(c, NRR_E_INVALID, "NULL argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    nrr_status st = c->fp64 ? write_X<double>(c, c->dd.X, X) : write_X<float>(c, c->df.X, X);
    if (st != NRR_OK) return st;
    st = pull_state(c);
    if (st != NRR_OK) return st;
    host_restart_stage(*c->h_state);
    return push_state(c);
}

nrr_status nrr_set_stage(nrr_ctx* c, double nu_a, double nu_r) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (!(nu_a > 0) || !(nu_r > 0) || !std::isfinite(nu_a) || !std::isfinite(nu_r))
        return fail(c, NRR_E_INVALID, "nu_a and nu_r must be positive and finite");
    nrr_status st = pull_state(c);
    if (st != NRR_OK) return st;
    NrrState& s = *c->h_state;
    s.nu_a = std::max(nu_a, s.nu_a_min);
    s.nu_r = nu_r;
    host_stage_weights(s);
    host_restart_stage(s);
    return push_state(c);
}

nrr_status nrr_get_transforms(nrr_ctx* c, double* X) {
    if (!c || !X) return fail(c, NRR_E_INVALID, "NULL argument");
    return c->fp64 ? read_X<double>(c, c->dd.X, X) : read_X<float>(c, c->df.X, X);
}

nrr_status nrr_get_mm_solution(nrr_ctx* c, double* G) {
    if (!c || !G) return fail(c, NRR_E_INVALID, "NULL argument");
    return c->fp64 ? read_X<double>(c, c->dd.Gprev, G) : read_X<float>(c, c->df.Gprev, G);
}

nrr_status nrr_get_search_stats(nrr_ctx* c, unsigned long long* out, int64_t max_warps, int64_t* n_warps) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    const unsigned long long* src = c->fp64 ? c->dd.nn_stats : c->df.nn_stats;
    const int per_warp = c->nn_tc ? 128 : 32 / c->nn_lpq;   // tensor-core search: per CTA of 128 queries
    const int64_t nw = (c->P + per_warp - 1) / per_warp;
    if (n_warps) *n_warps = src ? nw : 0;
    if (!src || !out) return NRR_OK;
    const int64_t n = std::min<int64_t>(std::min<int64_t>(nw, max_warps), (int64_t)c->nn_stats_n);
    CK(cudaMemcpyAsync(out, src, sizeof(unsigned long long) * 4 * (size_t)n, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}

nrr_status nrr_get_solve_stats(nrr_ctx* c, long long out[64]) {
    if (!c || !out) return fail(c, NRR_E_INVALID, "NULL argument");
    const long long* src = c->fp64 ? c->dd.solve_stats : c->df.solve_stats;
    if (!src) { std::memset(out, 0, 64 * sizeof(long long)); return NRR_OK; }
    CK(cudaMemcpyAsync(out, src, 64 * sizeof(long long), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}

nrr_status nrr_get_info(nrr_ctx* c, nrr_step_info* info) {
    if (!c || !info) return fail(c, NRR_E_INVALID, "NULL argument");
    nrr_status st = pull_state(c);
    if (st != NRR_OK) return st;
    fill_info(*c->h_state, info);
    return NRR_OK;
}

nrr_status nrr_get_history(nrr_ctx* c, nrr_step_info* out, int max_records, int* n_records) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (max_records < 0) return fail(c, NRR_E_INVALID, "max_records must be >= 0");
    const int n = out ? std::min(max_records, c->hist_n) : 0;
    if (n > 0) {
        CK(cudaMemcpyAsync(out, c->d_hist, sizeof(nrr_step_info) * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (n_records) *n_records = out ? n : c->hist_n;
    return NRR_OK;
}

nrr_status nrr_get_sizes(nrr_ctx* c, int64_t* P, int64_t* T, int64_t* N, int64_t* n_edges,
                         int32_t* max_influence) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (P) *P = c->P;
    if (T) *T = c->T;
    if (N) *N = c->N;
    if (n_edges) *n_edges = (int64_t)c->hg.edges.size() / 2;
    if (max_influence) *max_influence = c->hg.K;
    return NRR_OK;
}

struct nrr_graph {
    HostGraph g;
};

nrr_status nrr_graph_build(nrr_graph** out, const float* src_xyz, int64_t P, double radius, int max_influence) {
    if (!out || !src_xyz) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build: NULL argument");
    *out = nullptr;
    if (P < 1) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build: P < 1");
    if (!std::isfinite(radius)) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build: radius not finite");
    const int K = max_influence <= 0 ? 8 : max_influence;
    if (K > 8) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build: max_influence > 8");
    try {
        std::vector<double> V((size_t)P * 3);
        for (size_t k = 0; k < V.size(); ++k) {
            V[k] = (double)src_xyz[k];
            if (!std::isfinite(V[k])) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build: non-finite point");
        }
        std::unique_ptr<nrr_graph> g(new nrr_graph);
        if (!nrr_graph_and_spacing(V.data(), P, radius, K, true, g->g))
            return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build: radius 5 l-bar is not positive");
        *out = g.release();
        return NRR_OK;
    } catch (const std::bad_alloc&) {
        return nrr_set_global_error(NRR_E_OOM, "nrr_graph_build: out of host memory");
    }
}

nrr_status nrr_graph_build_mesh(nrr_graph** out, const float* src_xyz, int64_t P, const int32_t* faces,
                                int64_t n_faces, double radius, int max_influence) {
    if (!out || !src_xyz || !faces) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_mesh: NULL argument");
    *out = nullptr;
    if (P < 1 || P >= (1LL << 31)) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_mesh: P must be in 1..2^31-1");
    if (n_faces < 1 || n_faces > (1LL << 28))
        return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_mesh: n_faces must be in 1..2^28");
    if (!std::isfinite(radius)) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_mesh: radius not finite");
    const int K = max_influence <= 0 ? 8 : max_influence;
    if (K > 8) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_mesh: max_influence > 8");
    try {
        std::vector<double> V((size_t)P * 3);
        for (size_t k = 0; k < V.size(); ++k) {
            V[k] = (double)src_xyz[k];
            if (!std::isfinite(V[k])) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_mesh: non-finite point");
        }
        std::vector<int> F(faces, faces + 3 * n_faces);
        std::unique_ptr<nrr_graph> g(new nrr_graph);
        const nrr_status gs = graph_from_mesh(V, P, F, radius, K, g->g, "nrr_graph_build_mesh");
        if (gs != NRR_OK) return gs;
        *out = g.release();
        return NRR_OK;
    } catch (const std::bad_alloc&) {
        return nrr_set_global_error(NRR_E_OOM, "nrr_graph_build_mesh: out of host memory");
    }
}

nrr_status nrr_graph_build_gpu(nrr_graph** out, const float* src_xyz, int64_t P, double radius, int max_influence,
                               void* cuda_stream) {
    if (!out || !src_xyz) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_gpu: NULL argument");
    *out = nullptr;
    if (P < 1 || P >= (1LL << 25)) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_gpu: P must be in 1..2^25-1");
    if (!std::isfinite(radius)) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_gpu: radius not finite");
    const int K = max_influence <= 0 ? 8 : max_influence;
    if (K > 8) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_gpu: max_influence > 8");
    try {
        std::vector<float> src;
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (fetch_floats(src_xyz, (size_t)P * 3, src, st) != cudaSuccess)
            return nrr_set_global_error(NRR_E_CUDA, "nrr_graph_build_gpu: reading the points failed");
        if (!finite3(src)) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_build_gpu: non-finite point");
        std::vector<double> V(src.begin(), src.end());
        std::unique_ptr<nrr_graph> g(new nrr_graph);
        const nrr_status gs = graph_on_device(src.data(), V, P, radius, K, true, st, g->g);
        if (gs != NRR_OK) return gs;
        *out = g.release();
        return NRR_OK;
    } catch (const std::bad_alloc&) {
        return nrr_set_global_error(NRR_E_OOM, "nrr_graph_build_gpu: out of host memory");
    }
}

nrr_status nrr_graph_sizes(const nrr_graph* g, int64_t* N, int64_t* n_edges, int32_t* max_influence,
                           double* radius) {
    if (!g) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_sizes: graph is NULL");
    if (N) *N = (int64_t)g->g.nodes.size();
    if (n_edges) *n_edges = (int64_t)(g->g.edges.size() / 2);
    if (max_influence) *max_influence = g->g.K;
    if (radius) *radius = g->g.radius;
    return NRR_OK;
}

nrr_status nrr_graph_get(const nrr_graph* gh, int32_t* node_src, int32_t* nidx, double* w, int32_t* edges,
                         double* r, double* lbar) {
    if (!gh) return nrr_set_global_error(NRR_E_INVALID, "nrr_graph_get: graph is NULL");
    const HostGraph& g = gh->g;
    if (node_src) std::copy(g.nodes.begin(), g.nodes.end(), node_src);
    if (nidx) std::copy(g.nidx.begin(), g.nidx.end(), nidx);
    if (w) std::copy(g.w.begin(), g.w.end(), w);
    if (edges) std::copy(g.edges.begin(), g.edges.end(), edges);
    if (r) std::copy(g.r.begin(), g.r.end(), r);
    if (lbar) *lbar = g.lbar;
    return NRR_OK;
}

void nrr_graph_destroy(nrr_graph* g) { delete g; }

nrr_status nrr_get_graph(nrr_ctx* c, int32_t* node_src, int32_t* nidx, double* w, int32_t* edges,
                         double* r, double* lbar) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    const HostGraph& g = c->hg;
    if (node_src) std::copy(g.nodes.begin(), g.nodes.end(), node_src);
    if (nidx) std::copy(g.nidx.begin(), g.nidx.end(), nidx);
    if (w) std::copy(g.w.begin(), g.w.end(), w);
    if (edges) std::copy(g.edges.begin(), g.edges.end(), edges);
    if (r) std::copy(g.r.begin(), g.r.end(), r);
    if (lbar) *lbar = g.lbar;
    return NRR_OK;
}

}  // extern "C"

namespace {
template <typename T>
nrr_status get_points(nrr_ctx* c, const T* dev, int ncomp, double* out) {
    const size_t P = (size_t)c->P;
    std::vector<T> h(P * ncomp);
    CK(cudaMemcpyAsync(h.data(), dev, sizeof(T) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<double> o(P * ncomp);
    for (size_t ii = 0; ii < P; ++ii) {
        const size_t i = (size_t)c->src_order[ii];
        for (int a = 0; a < ncomp; ++a) o[i * ncomp + a] = (double)h[a * P + ii];
    }
    CK(cudaMemcpy(out, o.data(), sizeof(double) * o.size(), cudaMemcpyDefault));
    return NRR_OK;
}

template <typename T>
nrr_status get_system_t(nrr_ctx* c, double* Kd, double* B) {
    DevProblem<T>& d = prob<T>(c);
    const int N = c->N;
    std::vector<T> kv((size_t)c->nblk * 16), bv((size_t)N * 12);
    CK(cudaMemcpyAsync(kv.data(), d.Kv, sizeof(T) * kv.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(bv.data(), d.Bv, sizeof(T) * bv.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (Kd) {
        const size_t n4 = (size_t)4 * N;
        std::vector<double> K(n4 * n4, 0.0);
        for (int n = 0; n < N; ++n)
            for (int b = c->bsr_ptr[(size_t)n]; b < c->bsr_ptr[(size_t)n + 1]; ++b) {
                const int k = c->bsr_col[(size_t)b];
                for (int a = 0; a < 4; ++a)
                    for (int t = 0; t < 4; ++t)
                        K[(size_t)(4 * n + a) * n4 + 4 * k + t] = (double)kv[(size_t)16 * b + 4 * a + t];
            }
        CK(cudaMemcpy(Kd, K.data(), sizeof(double) * K.size(), cudaMemcpyDefault));
    }
    if (B) {
        std::vector<double> o(bv.begin(), bv.end());
        CK(cudaMemcpy(B, o.data(), sizeof(double) * o.size(), cudaMemcpyDefault));
    }
    return NRR_OK;
}
}  // namespace

extern "C" {

nrr_status nrr_get_deformed(nrr_ctx* c, double* v_hat) {
    if (!c || !v_hat) return fail(c, NRR_E_INVALID, "NULL argument");
    nrr_status st = pull_state(c);
    if (st != NRR_OK) return st;
    const int b = c->h_state->vlast;
    const size_t off = (size_t)b * 3 * (size_t)c->P;
    return c->fp64 ? get_points<double>(c, c->dd.vhat + off, 3, v_hat)
                   : get_points<float>(c, c->df.vhat + off, 3, v_hat);
}

nrr_status nrr_get_correspondence(nrr_ctx* c, int32_t* rho, double* d2) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    const size_t P = (size_t)c->P;
    if (rho) {
        std::vector<int> h(P), o(P);
        const int* src = c->fp64 ? c->dd.rho : c->df.rho;
        CK(cudaMemcpyAsync(h.data(), src, sizeof(int) * P, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t ii = 0; ii < P; ++ii) o[(size_t)c->src_order[ii]] = h[ii];
        CK(cudaMemcpy(rho, o.data(), sizeof(int) * P, cudaMemcpyDefault));
    }
    if (d2) {
        nrr_status st = c->fp64 ? get_points<double>(c, c->dd.d2, 1, d2) : get_points<float>(c, c->df.d2, 1, d2);
        if (st != NRR_OK) return st;
    }
    return NRR_OK;
}

nrr_status nrr_get_system(nrr_ctx* c, double* Kdense, double* B) {
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (Kdense && c->N > 4096) return fail(c, NRR_E_INVALID, "dense K only for N <= 4096");
    return c->fp64 ? get_system_t<double>(c, Kdense, B) : get_system_t<float>(c, Kdense, B);
}

nrr_status nrr_get_launch_config(nrr_ctx* c, nrr_launch_config* out) {
    if (!c || !out) return fail(c, NRR_E_INVALID, "NULL argument");
    out->nn_lanes_per_query = c->nn_lpq;
    out->nn_tensor_cores = c->nn_tc ? 1 : 0;
    out->solve_ctas = c->cl_C;
    out->nn_ms = 0.0;
    out->solve_ms = 0.0;
    out->pass_ms = 0.0;
    out->launches_per_pass = nrr_launches_per_pass(c->cl_C > 0);
    return NRR_OK;
}

nrr_status nrr_set_launch_config(nrr_ctx* c, const nrr_launch_config* cfg) {
    if (!c || !cfg) return fail(c, NRR_E_INVALID, "NULL argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    return c->fp64 ? apply_config<double>(c, cfg->nn_lanes_per_query, cfg->solve_ctas, cfg->nn_tensor_cores)
                   : apply_config<float>(c, cfg->nn_lanes_per_query, cfg->solve_ctas, cfg->nn_tensor_cores);
}

nrr_status nrr_tune(nrr_ctx* c, const char* table_path, int reps, nrr_launch_config* out) {
    NvtxRange nvtx_range("nrr_tune");
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    if (reps <= 0) reps = 5;
    if (reps > 1000) return fail(c, NRR_E_INVALID, "nrr_tune: reps must be at most 1000");
    const TuneKey key = tune_key(c);
    int lpq = 0, ctas = 0, tc = 0;
    double nn_ms = 0.0, solve_ms = 0.0;
    nrr_status st = NRR_E_INVALID;
    if (table_lookup(table_path, key, &lpq, &ctas, &tc)) {
        st = c->fp64 ? apply_config<double>(c, lpq, ctas, tc) : apply_config<float>(c, lpq, ctas, tc);
        if (st == NRR_OK) st = nrr_reset(c);
    }
    if (st != NRR_OK) {   // no usable entry: measure
        st = c->fp64 ? tune_t<double>(c, reps, &lpq, &ctas, &tc, &nn_ms, &solve_ms)
                     : tune_t<float>(c, reps, &lpq, &ctas, &tc, &nn_ms, &solve_ms);
        if (st != NRR_OK) return st;
        table_append(table_path, key, lpq, ctas, tc);
    }
    if (out) {
        out->nn_lanes_per_query = lpq;
        out->solve_ctas = ctas;
        out->nn_ms = nn_ms;
        out->solve_ms = solve_ms;
        out->pass_ms = 0.0;
        out->launches_per_pass = nrr_launches_per_pass(c->cl_C > 0);
        out->nn_tensor_cores = tc;
    }
    return NRR_OK;
}

nrr_status nrr_get_state_size(nrr_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(c, NRR_E_INVALID, "NULL argument");
    *bytes = ckpt_bytes(c);
    return NRR_OK;
}

nrr_status nrr_save_state(nrr_ctx* c, void* buf, size_t bytes) {
    NvtxRange nvtx_range("nrr_save_state");
    if (!c || !buf) return fail(c, NRR_E_INVALID, "NULL argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    if (bytes < ckpt_bytes(c)) return fail(c, NRR_E_INVALID, "nrr_save_state: buffer smaller than nrr_get_state_size");
    nrr_status st = pull_state(c);
    if (st != NRR_OK) return st;
    std::vector<unsigned char> h(ckpt_bytes(c));
    CkptHeader hd{kCkptMagic, kCkptVersion, c->fp64 ? 1u : 0u, c->P, (int64_t)c->N,
                  (int64_t)std::max(1, c->prm.aa_m), c->problem_hash};
    std::memcpy(h.data(), &hd, sizeof hd);
    std::memcpy(h.data() + sizeof hd, c->h_state, sizeof(NrrState));
    unsigned char* arrays = h.data() + sizeof hd + sizeof(NrrState);
    st = c->fp64 ? ckpt_copy<double>(c, arrays, true) : ckpt_copy<float>(c, arrays, true);
    if (st != NRR_OK) return st;
    CK(cudaMemcpy(buf, h.data(), h.size(), cudaMemcpyDefault));
    return NRR_OK;
}

nrr_status nrr_load_state(nrr_ctx* c, const void* buf, size_t bytes) {
    NvtxRange nvtx_range("nrr_load_state");
    if (!c || !buf) return fail(c, NRR_E_INVALID, "NULL argument");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    if (bytes < ckpt_bytes(c)) return fail(c, NRR_E_INVALID, "nrr_load_state: buffer smaller than nrr_get_state_size");
    std::vector<unsigned char> h(ckpt_bytes(c));
    CK(cudaMemcpy(h.data(), buf, h.size(), cudaMemcpyDefault));
    CkptHeader hd;
    std::memcpy(&hd, h.data(), sizeof hd);
    if (hd.magic != kCkptMagic || hd.version != kCkptVersion || hd.fp64 != (c->fp64 ? 1u : 0u) || hd.P != c->P ||
        hd.N != (int64_t)c->N || hd.m != (int64_t)std::max(1, c->prm.aa_m) || hd.problem != c->problem_hash)
        return fail(c, NRR_E_INVALID, "nrr_load_state: the state was saved from a different problem or precision");
    NrrState s;
    std::memcpy(&s, h.data() + sizeof hd, sizeof s);
    // counters of the last-block and barrier protocols start from zero
    s.cnt_nn = 0; s.cnt_energy = 0; s.bar_count = 0; s.disp_bits = 0ull;
    const unsigned char* arrays = h.data() + sizeof hd + sizeof(NrrState);
    nrr_status st = c->fp64 ? ckpt_copy<double>(c, const_cast<unsigned char*>(arrays), false)
                            : ckpt_copy<float>(c, const_cast<unsigned char*>(arrays), false);
    if (st != NRR_OK) return st;
    *c->h_state = s;
    return push_state(c);
}

nrr_status nrr_backward(nrr_ctx* c, int mode, const double* X, double* grad_X, double* grad_src) {
    NvtxRange nvtx_range("nrr_backward");
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (mode != 0 && mode != 1) return fail(c, NRR_E_INVALID, "nrr_backward: mode must be 0 or 1");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    if (mode == 1) {
        if (c->unroll_K < 0) return fail(c, NRR_E_STATE, "nrr_backward mode 1 needs a previous nrr_unroll");
        return c->fp64 ? unroll_backward_t<double>(c, X, grad_X, grad_src)
                       : unroll_backward_t<float>(c, X, grad_X, grad_src);
    }
    // evaluate closest points, weights and rotations at X (as nrr_energy)
    double terms[4];
    nrr_status st = nrr_energy(c, X, terms);
    if (st != NRR_OK) return st;
    if (!c->d_order) {
        CK(cudaMalloc(&c->d_order, sizeof(int) * (size_t)c->P));
        CK(cudaMemcpyAsync(c->d_order, c->src_order.data(), sizeof(int) * (size_t)c->P, cudaMemcpyHostToDevice,
                           c->stream));
    }
    if (!c->d_grad) {
        CK(cudaMalloc(&c->d_grad, sizeof(double) * ((size_t)c->N * 12 + (size_t)c->P * 3)));
    }
    double* gX = c->d_grad;
    double* gv = c->d_grad + (size_t)c->N * 12;
    const int grid = std::max(1, (c->N + 31) / 32);
    if (c->fp64) CK(nrr_launch_gradient<double>(c->dd, grad_X ? gX : nullptr, grad_src ? gv : nullptr, c->d_order, grid, c->stream));
    else CK(nrr_launch_gradient<float>(c->df, grad_X ? gX : nullptr, grad_src ? gv : nullptr, c->d_order, grid, c->stream));
    if (grad_X) CK(cudaMemcpyAsync(grad_X, gX, sizeof(double) * (size_t)c->N * 12, cudaMemcpyDefault, c->stream));
    if (grad_src) CK(cudaMemcpyAsync(grad_src, gv, sizeof(double) * (size_t)c->P * 3, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NRR_OK;
}

void nrr_lbfgs_params_default(nrr_lbfgs_params* p) {
    if (!p) return;
    p->m = 5;
    p->c1 = 1e-4;
    p->g_tol = 1e-3;
    p->max_inner = 20;
    p->max_halvings = 30;
}

nrr_status nrr_solve_lbfgs(nrr_ctx* c, const nrr_lbfgs_params* params, int max_outer, nrr_step_info* info) {
    NvtxRange nvtx_range("nrr_solve_lbfgs");
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    nrr_lbfgs_params lb;
    if (params) lb = *params; else nrr_lbfgs_params_default(&lb);
    if (lb.m < 1 || lb.m > NRR_AA_MMAX || lb.max_inner < 1 || lb.max_halvings < 0 || lb.max_halvings > 60 ||
        !(lb.c1 > 0 && lb.c1 < 1) || !(lb.g_tol >= 0 && lb.g_tol < 1))
        return fail(c, NRR_E_INVALID, "nrr_solve_lbfgs: m in 1..8, max_inner >= 1, max_halvings in 0..60, "
                                      "0 < c1 < 1, 0 <= g_tol < 1");
    const int cap = max_outer > 0 ? max_outer : c->prm.max_total_passes;
    nrr_status st = c->fp64 ? lbfgs_t<double>(c, lb, cap) : lbfgs_t<float>(c, lb, cap);
    if (st != NRR_OK) { c->failed = true; return st; }
    st = pull_state(c);
    if (st != NRR_OK) return st;
    fill_info(*c->h_state, info);
    if (c->h_state->status != 0) {
        c->failed = true;
        return fail(c, (nrr_status)c->h_state->status, "device-side check failed");
    }
    return c->h_state->done ? NRR_OK : NRR_E_NOT_CONVERGED;
}

nrr_status nrr_unroll(nrr_ctx* c, int K, const double* X0, double* XK) {
    NvtxRange nvtx_range("nrr_unroll");
    if (!c) return fail(nullptr, NRR_E_INVALID, "ctx is NULL");
    if (!X0) return fail(c, NRR_E_INVALID, "nrr_unroll: X0 is NULL");
    if (K < 0 || K > 1024) return fail(c, NRR_E_INVALID, "nrr_unroll: K must be in 0..1024");
    if (c->failed) return fail(c, NRR_E_STATE, "context failed earlier: " + c->err);
    c->unroll_K = -1;
    return c->fp64 ? unroll_t<double>(c, K, X0, XK) : unroll_t<float>(c, K, X0, XK);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent pairs: one context per pair; one CUDA graph runs one
// pass of every pair as parallel branches, then gathers every pair's flags
// so that a single small read tells the host which pairs have returned.
// ---------------------------------------------------------------------------
struct nrr_batch {
    std::vector<nrr_ctx*> ctx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraphExec_t gexec = nullptr;
    NrrState** d_states = nullptr;
    int* d_flags = nullptr;
    int* h_flags = nullptr;
    std::vector<int> captured;   // pairs whose pass the batch graph holds
    cudaGraphExec_t loop_exec = nullptr;   // the same passes repeated on the device
    int* d_ctrl = nullptr;                 // loop control: [0] passes run, [1] cap
    int* h_ctrl = nullptr;
    std::string err;
};

namespace {

__global__ void gather_flags(NrrState* const* st, int n, int* flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        flags[4 * i + 0] = st[i]->done;
        flags[4 * i + 1] = st[i]->status;
        flags[4 * i + 2] = st[i]->n_passes;
        flags[4 * i + 3] = st[i]->n_solves;
    }
}

nrr_status batch_fail(nrr_batch* b, nrr_status code, const std::string& msg) {
    if (b) b->err = msg;
    g_last_error = msg;
    return code;
}

nrr_status batch_capture(nrr_batch* b, const std::vector<int>& members);

#define BK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return batch_fail(b, e_ == cudaErrorMemoryAllocation ? NRR_E_OOM : NRR_E_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

}  // namespace


namespace {

// Captures the batch graph: fork the pass of every member pair onto its own
// stream, join, gather the flags of all pairs.
nrr_status batch_capture(nrr_batch* b, const std::vector<int>& members) {
    const int n = (int)b->ctx.size();
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->captured = members;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaEventRecord(b->events[(size_t)n], b->stream);
    for (int i : members) {
        if (ce != cudaSuccess) break;
        nrr_ctx* c = b->ctx[(size_t)i];
        ce = cudaStreamWaitEvent(c->stream, b->events[(size_t)n], 0);
        if (ce == cudaSuccess) ce = launch_pass_any(c);
        if (ce == cudaSuccess) ce = cudaEventRecord(b->events[(size_t)i], c->stream);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->stream, b->events[(size_t)i], 0);
    }
    if (ce == cudaSuccess) {
        gather_flags<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_states, n, b->d_flags);
        ce = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (ce != cudaSuccess || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return batch_fail(b, NRR_E_CUDA, std::string("batch graph capture failed: ") +
                                             cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    BK(ie);
    // the members' passes as the body of a device-side loop that runs
    // until every pair has returned, a pair failed, the cap is reached, or
    // half of the members have returned (then the host recaptures)
    if (b->loop_exec) {
        cudaGraphExecDestroy(b->loop_exec);
        b->loop_exec = nullptr;
    }
    if (!std::getenv("NRR_HOST_LOOP")) {
        auto body = [b, &members]() {
            const int n_all = (int)b->ctx.size();
            cudaError_t e = cudaEventRecord(b->events[(size_t)n_all], b->stream);
            for (int i : members) {
                if (e != cudaSuccess) break;
                nrr_ctx* c = b->ctx[(size_t)i];
                e = cudaStreamWaitEvent(c->stream, b->events[(size_t)n_all], 0);
                if (e == cudaSuccess) e = launch_pass_any(c);
                if (e == cudaSuccess) e = cudaEventRecord(b->events[(size_t)i], c->stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->events[(size_t)i], 0);
            }
            return e;
        };
        build_loop_graph(b->stream, body, b->d_states, n, (int)members.size(), b->d_flags, b->d_ctrl, nullptr, 0,
                         &b->loop_exec);
    }
    return NRR_OK;
}

std::vector<int> all_pairs(const nrr_batch* b) {
    std::vector<int> v(b->ctx.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = (int)i;
    return v;
}

// Applies one launch policy to every pair of a batch: lanes per query and
// each pair's smallest (policy -1) or largest (policy 0) fitting cluster.
nrr_status batch_apply(nrr_batch* b, int lpq, int policy) {
    // policy -2: all pairs' nodes spread over the SMs
    int64_t sum_n = 0;
    for (nrr_ctx* c : b->ctx) sum_n += c->N;
    const int sms = std::max(1, b->ctx.empty() ? 1 : b->ctx[0]->num_sms);
    const int bal = (int)std::max<int64_t>(64, (sum_n + sms - 1) / sms);
    for (nrr_ctx* c : b->ctx) {
        c->bal_nodes = bal;
        c->nn_lpq = lpq;
        c->prm.solve_ctas = policy;
        if (c->fp64) choose_solver<double>(c); else choose_solver<float>(c);
        nrr_status st = capture_graph(c);
        if (st != NRR_OK) return st;
    }
    return batch_capture(b, all_pairs(b));
}

}  // namespace

extern "C" {

nrr_status nrr_batch_tune(nrr_batch* b, const char* table_path, int reps, nrr_launch_config* out) {
    NvtxRange nvtx_range("nrr_batch_tune");
    if (!b) return batch_fail(nullptr, NRR_E_INVALID, "batch is NULL");
    if (reps <= 0) reps = 3;
    if (reps > 1000) return batch_fail(b, NRR_E_INVALID, "nrr_batch_tune: reps must be at most 1000");
    int64_t sumP = 0, sumN = 0;
    for (nrr_ctx* c : b->ctx) { sumP += c->P; sumN += c->N; }
    // key: precision, pair count, total points and nodes (half octaves)
    const TuneKey key = {b->ctx[0]->fp64 ? 3 : 2, half_octave((int64_t)b->ctx.size()), half_octave(sumP),
                         half_octave(sumN)};
    int lpq = 0, policy = 0;
    double best_ms = 0.0;
    nrr_status st = NRR_E_INVALID;
    if (table_lookup(table_path, key, &lpq, &policy) && valid_lpq(lpq) && (policy >= -2 && policy <= 0)) {
        st = batch_apply(b, lpq, policy);
    }
    if (st != NRR_OK) {
        best_ms = INFINITY;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        BK(cudaEventCreate(&e0));
        BK(cudaEventCreate(&e1));
        for (int cl : {4, 8, 2})
            for (int pol : {-1, 0, -2}) {
                st = batch_apply(b, cl, pol);
                if (st == NRR_OK) st = nrr_batch_reset(b);
                if (st != NRR_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
                cudaError_t e = cudaGraphLaunch(b->gexec, b->stream);   // untimed first pass
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->gexec, b->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    BK(e);
                }
                if (t / reps < best_ms) { best_ms = t / reps; lpq = cl; policy = pol; }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        st = batch_apply(b, lpq, policy);
        if (st != NRR_OK) return st;
        table_append(table_path, key, lpq, policy);
    }
    st = nrr_batch_reset(b);
    if (st != NRR_OK) return st;
    if (out) {
        out->nn_lanes_per_query = lpq;
        out->solve_ctas = policy;
        out->nn_ms = 0.0;
        out->solve_ms = 0.0;
        out->pass_ms = best_ms;
        out->launches_per_pass = 0;
        out->nn_tensor_cores = 0;
    }
    return NRR_OK;
}

void nrr_batch_destroy(nrr_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->loop_exec) cudaGraphExecDestroy(b->loop_exec);
    if (b->d_ctrl) cudaFree(b->d_ctrl);
    if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
    for (nrr_ctx* c : b->ctx) nrr_destroy(c);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    if (b->d_states) cudaFree(b->d_states);
    if (b->d_flags) cudaFree(b->d_flags);
    if (b->h_flags) cudaFreeHost(b->h_flags);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

nrr_status nrr_batch_create(nrr_batch** out, int n_pairs, const float* const* src_xyz, const int64_t* P,
                            const float* const* tgt_xyz, const int64_t* T, const nrr_params* params,
                            int params_per_pair, void* cuda_stream) {
    nrr_batch* b = nullptr;
    if (!out || n_pairs < 1 || !src_xyz || !P || !tgt_xyz || !T)
        return batch_fail(nullptr, NRR_E_INVALID, "nrr_batch_create: bad arguments");
    *out = nullptr;
    b = new (std::nothrow) nrr_batch();
    if (!b) return batch_fail(nullptr, NRR_E_OOM, "host allocation failed");
    std::unique_ptr<nrr_batch, void (*)(nrr_batch*)> guard(b, nrr_batch_destroy);
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        BK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    // the pairs' contexts are independent: created by a few host threads at
    // once (each on its own stream, on the caller's device), kept in pair
    // order; the first failing pair (lowest index) is reported
    {
        int device = 0;
        BK(cudaGetDevice(&device));
        std::vector<nrr_ctx*> made((size_t)n_pairs, nullptr);
        std::vector<nrr_status> stat((size_t)n_pairs, NRR_OK);
        std::vector<std::string> msg((size_t)n_pairs);
        std::atomic<int> next{0};
        auto work = [&]() {
            if (cudaSetDevice(device) != cudaSuccess) return;
            for (int i = next.fetch_add(1); i < n_pairs; i = next.fetch_add(1)) {
                const nrr_params* pp = params ? (params_per_pair ? &params[i] : params) : nullptr;
                nrr_params q;
                if (pp) q = *pp; else nrr_params_default(&q);
                if (q.solve_ctas == 0) q.solve_ctas = -1;   // smallest cluster inside a batch
                stat[(size_t)i] = nrr_create(&made[(size_t)i], src_xyz[i], nullptr, P[i], tgt_xyz[i], nullptr, T[i],
                                             &q, nullptr);
                if (stat[(size_t)i] != NRR_OK) msg[(size_t)i] = g_last_error;
            }
        };
        const int nth = std::max(1, std::min(n_pairs, kBatchCreateThreads));
        std::vector<std::thread> th;
        for (int k = 1; k < nth; ++k) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
        for (int i = 0; i < n_pairs; ++i) b->ctx.push_back(made[(size_t)i]);   // destroyed with the batch
        for (int i = 0; i < n_pairs; ++i)
            if (stat[(size_t)i] != NRR_OK || !made[(size_t)i])
                return batch_fail(b, stat[(size_t)i] != NRR_OK ? stat[(size_t)i] : NRR_E_CUDA,
                                  "pair " + std::to_string(i) + ": " + msg[(size_t)i]);
    }
    const int n = n_pairs;
    std::vector<NrrState*> sts((size_t)n);
    for (int i = 0; i < n; ++i) sts[(size_t)i] = b->ctx[(size_t)i]->d_state;
    BK(cudaMalloc(&b->d_states, sizeof(NrrState*) * (size_t)n));
    BK(cudaMemcpy(b->d_states, sts.data(), sizeof(NrrState*) * (size_t)n, cudaMemcpyHostToDevice));
    BK(cudaMalloc(&b->d_flags, sizeof(int) * 4 * (size_t)n));
    BK(cudaMallocHost(&b->h_flags, sizeof(int) * 4 * (size_t)n));
    BK(cudaMalloc(&b->d_ctrl, 2 * sizeof(int)));
    BK(cudaMallocHost(&b->h_ctrl, 2 * sizeof(int)));
    b->events.resize((size_t)n + 1);
    for (auto& e : b->events) BK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    nrr_status cst = batch_capture(b, all_pairs(b));
    if (cst != NRR_OK) return cst;
    guard.release();
    *out = b;
    return NRR_OK;
}

nrr_status nrr_batch_solve(nrr_batch* b, int max_passes, nrr_step_info* infos) {
    NvtxRange nvtx_range("nrr_batch_solve");
    if (!b) return batch_fail(nullptr, NRR_E_INVALID, "batch is NULL");
    const int n = (int)b->ctx.size();
    int cap = max_passes;
    if (cap <= 0) {
        cap = 0;
        for (nrr_ctx* c : b->ctx) cap = std::max(cap, c->prm.max_total_passes);
    }
    int launched = 0;
    bool all_done = false;
    // the graph holds every pair at the start; when half of its pairs have
    // returned it is recaptured with the pairs still running (passes of
    // returned pairs do nothing, but their launches still cost)
    if ((int)b->captured.size() != n) {
        nrr_status cst = batch_capture(b, all_pairs(b));
        if (cst != NRR_OK) return cst;
    }
    // NRR_BATCH_TIMES: each launch's captured pairs, passes and wall time
    // on stderr (profiling of the batch's phases)
    const bool times = std::getenv("NRR_BATCH_TIMES") != nullptr;
    while (!all_done && launched < cap) {
        const auto t_launch = std::chrono::steady_clock::now();
        const int launched_before = launched;
        if (b->loop_exec) {
            // passes repeat on the device until every pair has returned or
            // half of the captured pairs have (the cap and failures too)
            b->h_ctrl[0] = 0;
            b->h_ctrl[1] = cap - launched;
            BK(cudaMemcpyAsync(b->d_ctrl, b->h_ctrl, 2 * sizeof(int), cudaMemcpyHostToDevice, b->stream));
            BK(cudaGraphLaunch(b->loop_exec, b->stream));
            BK(cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        } else {
            const int nb = std::min(4, cap - launched);
            for (int k = 0; k < nb; ++k) BK(cudaGraphLaunch(b->gexec, b->stream));
            b->h_ctrl[0] = nb;
        }
        BK(cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int) * 4 * (size_t)n, cudaMemcpyDeviceToHost, b->stream));
        BK(cudaStreamSynchronize(b->stream));
        launched += b->h_ctrl[0];
        if (times)
            std::fprintf(stderr, "nrr_batch_solve: %3d pairs captured, %5d passes, %9.2f ms\n",
                         (int)b->captured.size(), launched - launched_before,
                         std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_launch).count());
        all_done = true;
        std::vector<int> running;
        for (int i = 0; i < n; ++i) {
            if (b->h_flags[4 * i + 1] != 0)
                return batch_fail(b, (nrr_status)b->h_flags[4 * i + 1],
                                  "pair " + std::to_string(i) + ": device-side wait timed out");
            if (b->h_flags[4 * i] == 0) running.push_back(i);
        }
        all_done = running.empty();
        if (!all_done && 2 * running.size() <= b->captured.size()) {
            nrr_status cst = batch_capture(b, running);
            if (cst != NRR_OK) return cst;
        }
    }
    if (infos)
        for (int i = 0; i < n; ++i) {
            nrr_status st = nrr_get_info(b->ctx[(size_t)i], &infos[i]);
            if (st != NRR_OK) return st;
        }
    return all_done ? NRR_OK : NRR_E_NOT_CONVERGED;
}

nrr_status nrr_batch_reset(nrr_batch* b) {
    if (!b) return batch_fail(nullptr, NRR_E_INVALID, "batch is NULL");
    for (nrr_ctx* c : b->ctx) {
        nrr_status st = nrr_reset(c);
        if (st != NRR_OK) return st;
    }
    return NRR_OK;
}

nrr_status nrr_batch_get_context(nrr_batch* b, int i, nrr_ctx** out) {
    if (!b || !out || i < 0 || i >= (int)b->ctx.size()) return batch_fail(b, NRR_E_INVALID, "bad pair index");
    *out = b->ctx[(size_t)i];
    return NRR_OK;
}

}  // extern "C"
