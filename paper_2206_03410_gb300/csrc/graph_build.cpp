// Host construction of the embedded deformation graph (Sec. 3.1, Algorithm 1)
// for point clouds, with Euclidean distances in place of geodesics, plus the
// mean point spacing l-bar and the space-filling-curve ordering used by the
// search structures.
//
// Built once per problem in nrr_create (setup, not part of the per-iteration
// path). Compiled with -ffp-contract=off so that every squared distance is
// evaluated as dx*dx + dy*dy + dz*dz with separate roundings on every host.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <cstring>
#include <functional>
#include <iterator>
#include <thread>

#include "nrr_internal.h"

namespace {

// Number of host threads for setup work on n items, at least `grain` items
// per thread.
int64_t setup_threads(int64_t n, int64_t grain = 4096) {
    const int64_t hw = (int64_t)std::max(1u, std::thread::hardware_concurrency());
    return std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(hw, 64), n / grain));
}

// A pool of host worker threads (one fewer than the cores), started on
// first use: a parallel call queues a job of nt tasks, the workers and the
// calling thread claim tasks from it, and the call returns once every task
// has run and no worker still holds the job. Calls may come from several
// threads at once and from inside tasks (the caller can always finish its
// own job alone), so setup work pays no thread creation per call.
class SetupPool {
    struct Job {
        const std::function<void(int64_t)>* f;
        int64_t n;
        std::atomic<int64_t> next{0};
        int users = 0;   // workers inside run() (under the mutex)
    };
    std::mutex m_;
    std::condition_variable work_, idle_;
    std::deque<Job*> q_;
    std::vector<std::thread> th_;
    bool stop_ = false;

    static void run(Job* j) {
        for (int64_t k = j->next.fetch_add(1); k < j->n; k = j->next.fetch_add(1)) (*j->f)(k);
    }
    void loop() {
        std::unique_lock<std::mutex> lk(m_);
        for (;;) {
            work_.wait(lk, [&] { return stop_ || !q_.empty(); });
            if (stop_) return;
            Job* j = q_.front();
            if (j->next.load() >= j->n) {   // exhausted: off the queue
                q_.pop_front();
                continue;
            }
            ++j->users;
            lk.unlock();
            run(j);
            lk.lock();
            if (--j->users == 0) idle_.notify_all();
        }
    }

public:
    explicit SetupPool(int workers) {
        for (int k = 0; k < workers; ++k) th_.emplace_back([this] { loop(); });
    }
    ~SetupPool() {
        {
            std::lock_guard<std::mutex> lk(m_);
            stop_ = true;
        }
        work_.notify_all();
        for (auto& t : th_) t.join();
    }
    void parallel(int64_t n, const std::function<void(int64_t)>& f) {
        Job j;
        j.f = &f;
        j.n = n;
        {
            std::lock_guard<std::mutex> lk(m_);
            q_.push_back(&j);
        }
        work_.notify_all();
        run(&j);
        std::unique_lock<std::mutex> lk(m_);
        for (auto it = q_.begin(); it != q_.end(); ++it)
            if (*it == &j) { q_.erase(it); break; }
        idle_.wait(lk, [&] { return j.users == 0; });
    }
    static SetupPool& get() {
        static SetupPool pool((int)std::max(1u, std::thread::hardware_concurrency()) - 1);
        return pool;
    }
};

// Runs f(chunk, begin, end) over [0, n) split into nt contiguous chunks on
// the host's cores (setup work; each chunk writes only its own outputs, so
// results do not depend on the number of threads).
template <class F>
void parallel_chunks_idx(int64_t n, int64_t nt, F&& f) {
    if (nt <= 1) { f((int64_t)0, (int64_t)0, n); return; }
    const int64_t per = (n + nt - 1) / nt;
    const std::function<void(int64_t)> task = [&](int64_t t) {
        const int64_t b = std::min(n, t * per), e = std::min(n, b + per);
        f(t, b, e);
    };
    SetupPool::get().parallel(nt, task);
}

template <class F>
void parallel_chunks(int64_t n, F&& f, int64_t grain = 4096) {
    parallel_chunks_idx(n, setup_threads(n, grain), [&f](int64_t, int64_t b, int64_t e) { f(b, e); });
}

// Sorts v (whose elements are all distinct) with chunks sorted in parallel
// and merged pairwise in parallel; the result is the unique sorted order.
template <class E>
void parallel_sort(std::vector<E>& v) {
    const int64_t n = (int64_t)v.size();
    int64_t nt = setup_threads(n);
    if (nt <= 1) { std::sort(v.begin(), v.end()); return; }
    const int64_t per = (n + nt - 1) / nt;
    std::vector<int64_t> bounds;
    for (int64_t t = 0; t <= nt; ++t) bounds.push_back(std::min(n, t * per));
    parallel_chunks_idx(n, nt, [&](int64_t t, int64_t, int64_t) {
        std::sort(v.begin() + bounds[(size_t)t], v.begin() + bounds[(size_t)t + 1]);
    });
    while (bounds.size() > 2) {
        std::vector<int64_t> next;
        std::vector<std::thread> th;
        for (size_t k = 0; k + 2 < bounds.size(); k += 2) {
            const int64_t a = bounds[k], m = bounds[k + 1], b = bounds[k + 2];
            th.emplace_back([&v, a, m, b]() { std::inplace_merge(v.begin() + a, v.begin() + m, v.begin() + b); });
            next.push_back(a);
        }
        if (bounds.size() % 2 == 0) next.push_back(bounds[bounds.size() - 2]);
        next.push_back(bounds.back());
        for (auto& x : th) x.join();
        bounds.swap(next);
    }
}

// Sorts pairs (u, v) with 0 <= u, v < n lexicographically and removes
// duplicates: two stable counting passes (by v, then by u).
void sort_unique_pairs(std::vector<std::pair<int, int>>& e, int n) {
    if (e.size() < 2) return;
    std::vector<std::pair<int, int>> tmp(e.size());
    std::vector<int> cnt((size_t)n + 1);
    auto pass = [&](std::vector<std::pair<int, int>>& from, std::vector<std::pair<int, int>>& to, bool by_u) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (const auto& x : from) cnt[(size_t)(by_u ? x.first : x.second) + 1]++;
        for (int k = 0; k < n; ++k) cnt[(size_t)k + 1] += cnt[(size_t)k];
        for (const auto& x : from) to[(size_t)cnt[(size_t)(by_u ? x.first : x.second)]++] = x;
    };
    pass(e, tmp, false);
    pass(tmp, e, true);
    e.erase(std::unique(e.begin(), e.end()), e.end());
}

// Uniform grid over a point set: the point indices sorted by (cell key,
// index) and, per occupied cell, its run of them. Cells are found through a
// dense table of the occupied cells' ranks when the grid has few cells for
// the points (the common case), else by binary search of the sorted keys.
struct Grid {
    double lo[3];
    double h;
    int64_t dims[3];
    std::vector<int> items;          // point indices by (cell key, index)
    std::vector<double> pxyz;        // their coordinates, in the same order [n][3]
    std::vector<int64_t> ukeys;      // occupied cells' keys, ascending
    std::vector<int> ustart;         // their runs in items (ukeys.size() + 1)
    std::vector<int> dense;          // key -> rank in ukeys, or -1 (if used)

    int64_t key(int64_t x, int64_t y, int64_t z) const {
        return (x * dims[1] + y) * dims[2] + z;
    }
    void cell_of(const double* p, int64_t c[3]) const {
        for (int d = 0; d < 3; ++d) {
            int64_t v = (int64_t)std::floor((p[d] - lo[d]) / h);
            c[d] = std::min<int64_t>(std::max<int64_t>(v, 0), dims[d] - 1);
        }
    }
    void build(const double* V, int64_t n, double cell) {
        double hi[3];
        for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], V[3 * i + d]);
                hi[d] = std::max(hi[d], V[3 * i + d]);
            }
        h = cell > 0 ? cell : 1.0;
        for (int d = 0; d < 3; ++d)
            dims[d] = std::max<int64_t>(1, (int64_t)std::floor((hi[d] - lo[d]) / h) + 1);
        std::vector<std::pair<int64_t, int>> kv((size_t)n);
        parallel_chunks(n, [&](int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                int64_t c[3];
                cell_of(V + 3 * i, c);
                kv[(size_t)i] = {key(c[0], c[1], c[2]), (int)i};
            }
        });
        parallel_sort(kv);   // (cell, index) pairs are distinct
        items.resize((size_t)n);
        ukeys.clear();
        ustart.clear();
        for (size_t i = 0; i < kv.size(); ++i) {
            items[i] = kv[i].second;
            if (i == 0 || kv[i].first != kv[i - 1].first) {
                ukeys.push_back(kv[i].first);
                ustart.push_back((int)i);
            }
        }
        ustart.push_back((int)n);
        pxyz.resize((size_t)n * 3);
        parallel_chunks(n, [&](int64_t s0, int64_t s1) {
            for (int64_t s = s0; s < s1; ++s)
                for (int d = 0; d < 3; ++d) pxyz[(size_t)(3 * s + d)] = V[3 * (int64_t)items[(size_t)s] + d];
        });
        // dims[d] <= extent / h + 1 each; the product can overflow only for
        // absurd extents, which take the sparse path
        const double total = (double)dims[0] * (double)dims[1] * (double)dims[2];
        dense.clear();
        if (total <= 4.0 * (double)n + 1048576.0) {
            dense.assign((size_t)total, -1);
            for (size_t u = 0; u < ukeys.size(); ++u) dense[(size_t)ukeys[u]] = (int)u;
        }
    }
    // rank of cell (x, y, z) among the occupied cells, or -1
    int find(int64_t x, int64_t y, int64_t z) const {
        if (x < 0 || y < 0 || z < 0 || x >= dims[0] || y >= dims[1] || z >= dims[2]) return -1;
        const int64_t k = key(x, y, z);
        if (!dense.empty()) return dense[(size_t)k];
        auto it = std::lower_bound(ukeys.begin(), ukeys.end(), k);
        return (it != ukeys.end() && *it == k) ? (int)(it - ukeys.begin()) : -1;
    }
    template <class F>
    void visit_cell(int64_t x, int64_t y, int64_t z, F&& f) const {
        const int u = find(x, y, z);
        if (u < 0) return;
        for (int s = ustart[(size_t)u], e = ustart[(size_t)u + 1]; s < e; ++s) f(items[(size_t)s]);
    }
    // f(point index, its coordinates) for the points of cell (x, y, z)
    template <class F>
    void visit_cell_xyz(int64_t x, int64_t y, int64_t z, F&& f) const {
        const int u = find(x, y, z);
        if (u < 0) return;
        for (int s = ustart[(size_t)u], e = ustart[(size_t)u + 1]; s < e; ++s)
            f(items[(size_t)s], pxyz.data() + 3 * (size_t)s);
    }
};

inline double sqd(const double* a, const double* b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (Golub & Van
// Loan, Sec. 8.5): returns eigenvalues in ev and eigenvectors as columns of Q.
void jacobi_eig3(const double Ain[9], double ev[3], double Q[9]) {
    double A[9];
    std::memcpy(A, Ain, sizeof(A));
    for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        if (off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double apq = A[3 * p + q];
                if (apq == 0.0) continue;
                double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                // A <- J^T A J with J the rotation in the (p,q) plane
                for (int k = 0; k < 3; ++k) {
                    double akp = A[3 * k + p], akq = A[3 * k + q];
                    A[3 * k + p] = c * akp - s * akq;
                    A[3 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[3 * p + k], aqk = A[3 * q + k];
                    A[3 * p + k] = c * apk - s * aqk;
                    A[3 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double qkp = Q[3 * k + p], qkq = Q[3 * k + q];
                    Q[3 * k + p] = c * qkp - s * qkq;
                    Q[3 * k + q] = s * qkp + c * qkq;
                }
            }
    }
    ev[0] = A[0]; ev[1] = A[4]; ev[2] = A[8];
}

}  // namespace

void nrr_parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f) { parallel_chunks(n, f); }
int nrr_setup_chunks(int64_t n) { return (int)setup_threads(n); }
void nrr_parallel_chunks(int64_t n, int nchunks, const std::function<void(int64_t, int64_t, int64_t)>& f) {
    parallel_chunks_idx(n, nchunks, f);
}

double nrr_mean_spacing(const double* V, int64_t P, int k) {
    if (P < 2) return 0.0;
    const int kk = (int)std::min<int64_t>(k, P - 1);
    // cells of about three point spacings (from the bbox and the count); the
    // points of each cell scan the candidates of its 27 neighbouring cells,
    // gathered once per cell, and fall back to a growing shell search when
    // their kk-th neighbour is not certified within that block
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < P; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], V[3 * i + d]);
            hi[d] = std::max(hi[d], V[3 * i + d]);
        }
    const double diag = std::sqrt(sqd(lo, hi));
    double cell = diag / std::sqrt((double)P) * 3.0;
    if (!(cell > 0)) cell = 1.0;
    Grid g;
    g.build(V, P, cell);
    // cells as runs of g.items (sorted by cell key)
    const std::vector<int>& run_start = g.ustart;
    const int64_t n_cells = (int64_t)run_start.size() - 1;
    // per point: the sum of its kk nearest distances, then a sum in point order
    std::vector<double> per_point((size_t)P, 0.0);
    // continues the search of point i over the shells of cells s >= 2 around
    // its cell (best: the kk nearest among shells 0 and 1, ascending)
    auto shell_search = [&](int64_t i, std::vector<double>& best) {
        const double* q = V + 3 * i;
        int64_t c[3];
        g.cell_of(q, c);
        for (int64_t s = 2;; ++s) {
            for (int64_t x = c[0] - s; x <= c[0] + s; ++x)
                for (int64_t y = c[1] - s; y <= c[1] + s; ++y)
                    for (int64_t z = c[2] - s; z <= c[2] + s; ++z) {
                        if (std::max({std::llabs(x - c[0]), std::llabs(y - c[1]), std::llabs(z - c[2])}) != s)
                            continue;
                        g.visit_cell(x, y, z, [&](int j) {
                            if (j == (int)i) return;
                            double d2 = sqd(q, V + 3 * (int64_t)j);
                            if (d2 < best[(size_t)kk - 1]) {
                                size_t pos = (size_t)kk - 1;
                                while (pos > 0 && best[pos - 1] > d2) { best[pos] = best[pos - 1]; --pos; }
                                best[pos] = d2;
                            }
                        });
                    }
            const double reach = (double)s * g.h;
            const bool out_of_grid = s > std::max({g.dims[0], g.dims[1], g.dims[2]});
            if (best[(size_t)kk - 1] <= reach * reach || out_of_grid) break;
        }
    };
    parallel_chunks(n_cells, [&](int64_t c0, int64_t c1) {
        std::vector<double> best;
        std::vector<int> cand;
        std::vector<double> cx, cy, cz, d2v;   // candidate coordinates (SoA), distances
        for (int64_t cidx = c0; cidx < c1; ++cidx) {
            const int64_t s0 = run_start[(size_t)cidx], s1 = run_start[(size_t)cidx + 1];
            int64_t c[3];
            g.cell_of(V + 3 * (int64_t)g.items[(size_t)s0], c);
            cand.clear(); cx.clear(); cy.clear(); cz.clear();
            for (int64_t x = c[0] - 1; x <= c[0] + 1; ++x)
                for (int64_t y = c[1] - 1; y <= c[1] + 1; ++y)
                    for (int64_t z = c[2] - 1; z <= c[2] + 1; ++z)
                        g.visit_cell_xyz(x, y, z, [&](int j, const double* p) {
                            cand.push_back(j);
                            cx.push_back(p[0]); cy.push_back(p[1]); cz.push_back(p[2]);
                        });
            const size_t nc = cand.size();
            d2v.resize(nc);
            for (int64_t sidx = s0; sidx < s1; ++sidx) {
                const int64_t i = g.items[(size_t)sidx];
                const double qx = V[3 * i], qy = V[3 * i + 1], qz = V[3 * i + 2];
                // the same arithmetic as sqd(q, p), for all candidates
                for (size_t t = 0; t < nc; ++t) {
                    const double dx = qx - cx[t], dy = qy - cy[t], dz = qz - cz[t];
                    d2v[t] = dx * dx + dy * dy + dz * dz;
                }
                best.assign((size_t)kk, INFINITY);
                double worst = INFINITY;
                for (size_t t = 0; t < nc; ++t) {
                    const double d2 = d2v[t];
                    if (d2 < worst && cand[t] != (int)i) {
                        size_t pos = (size_t)kk - 1;
                        while (pos > 0 && best[pos - 1] > d2) { best[pos] = best[pos - 1]; --pos; }
                        best[pos] = d2;
                        worst = best[(size_t)kk - 1];
                    }
                }
                // every point outside the 27 cells is at least one cell width away
                if (!(best[(size_t)kk - 1] <= g.h * g.h)) shell_search(i, best);
                double sp = 0.0;
                for (int t = 0; t < kk; ++t) sp += std::sqrt(best[(size_t)t]);
                per_point[(size_t)i] = sp;
            }
        }
    }, 64);
    double total = 0.0;
    for (int64_t i = 0; i < P; ++i) total += per_point[(size_t)i];
    return total / ((double)P * kk);
}

std::vector<int> nrr_pca_order(const double* V, int64_t P) {
    // PCA axis of the largest covariance eigenvalue
    double mu[3] = {0, 0, 0};
    for (int64_t i = 0; i < P; ++i)
        for (int d = 0; d < 3; ++d) mu[d] += V[3 * i + d];
    for (int d = 0; d < 3; ++d) mu[d] /= (double)P;
    double C[9] = {0};
    for (int64_t i = 0; i < P; ++i) {
        double c[3] = {V[3 * i] - mu[0], V[3 * i + 1] - mu[1], V[3 * i + 2] - mu[2]};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[3 * a + b] += c[a] * c[b];
    }
    for (int i = 0; i < 9; ++i) C[i] /= (double)P;
    double ev[3], Q[9];
    jacobi_eig3(C, ev, Q);
    int top = 0;
    for (int i = 1; i < 3; ++i) if (ev[i] > ev[top]) top = i;
    double ax[3] = {Q[0 * 3 + top], Q[1 * 3 + top], Q[2 * 3 + top]};
    int big = 0;
    for (int i = 1; i < 3; ++i) if (std::fabs(ax[i]) > std::fabs(ax[big])) big = i;
    if (ax[big] < 0) for (double& a : ax) a = -a;
    std::vector<double> proj((size_t)P);
    for (int64_t i = 0; i < P; ++i)
        proj[(size_t)i] = V[3 * i] * ax[0] + V[3 * i + 1] * ax[1] + V[3 * i + 2] * ax[2];
    // ascending projection, ties to the lower index: (projection, index)
    // pairs are distinct
    std::vector<std::pair<double, int>> pk((size_t)P);
    for (int64_t i = 0; i < P; ++i) pk[(size_t)i] = {proj[(size_t)i], (int)i};
    parallel_sort(pk);
    std::vector<int> order((size_t)P);
    for (int64_t i = 0; i < P; ++i) order[(size_t)i] = pk[(size_t)i].second;
    return order;
}

void nrr_build_graph(const double* V, int64_t P, double R, int K, HostGraph& g) {
    const double R2 = R * R;
    const std::vector<int> order = nrr_pca_order(V, P);
    // Greedy radius sampling: a point becomes a node if it has no influencing
    // node yet; the new node influences every point strictly within R.
    Grid grid;
    grid.build(V, P, R);
    // (point, node, squared distance) of every influence, appended in node
    // order; a point is covered once some node influences it
    std::vector<NrrInfl> trip;
    trip.reserve((size_t)P * 4);
    std::vector<unsigned char> covered((size_t)P, 0);
    g.nodes.clear();
    for (int i : order) {
        if (!g.nodes.empty() && covered[(size_t)i]) continue;
        int j = (int)g.nodes.size();
        g.nodes.push_back(i);
        const double* q = V + 3 * (int64_t)i;
        int64_t c[3];
        grid.cell_of(q, c);
        for (int64_t x = c[0] - 1; x <= c[0] + 1; ++x)
            for (int64_t y = c[1] - 1; y <= c[1] + 1; ++y)
                for (int64_t z = c[2] - 1; z <= c[2] + 1; ++z)
                    grid.visit_cell_xyz(x, y, z, [&](int pt, const double* pp) {
                        const double d2 = sqd(q, pp);
                        if (d2 < R2) {
                            trip.push_back({pt, j, d2});
                            covered[(size_t)pt] = 1;
                        }
                    });
    }
    nrr_finish_graph(V, P, R, K, trip, g);
}

void nrr_finish_graph(const double* V, int64_t P, double R, int K, const std::vector<NrrInfl>& trip,
                      HostGraph& g) {
    g.radius = R;
    g.K = K;
    const double R2 = R * R;
    // grouped by point (counting sort, node order kept within a point): per
    // chunk of the triples a histogram over the points, then every chunk
    // scatters its triples after those of the earlier chunks
    std::vector<int64_t> iptr((size_t)P + 1, 0);
    std::vector<std::pair<double, int>> iv(trip.size());
    {
        const int64_t nT = (int64_t)trip.size();
        const int64_t nc = setup_threads(nT, 16384);
        std::vector<std::vector<int>> cnt((size_t)nc);
        parallel_chunks_idx(nT, nc, [&](int64_t t, int64_t a, int64_t b) {
            std::vector<int>& h = cnt[(size_t)t];
            h.assign((size_t)P, 0);
            for (int64_t e = a; e < b; ++e) h[(size_t)trip[(size_t)e].pt]++;
        });
        // per point: its total, and each chunk's first slot relative to it
        parallel_chunks(P, [&](int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                int run = 0;
                for (int64_t t = 0; t < nc; ++t) {
                    const int c = cnt[(size_t)t][(size_t)i];
                    cnt[(size_t)t][(size_t)i] = run;
                    run += c;
                }
                iptr[(size_t)i + 1] = run;
            }
        });
        for (int64_t i = 0; i < P; ++i) iptr[(size_t)i + 1] += iptr[(size_t)i];
        parallel_chunks_idx(nT, nc, [&](int64_t t, int64_t a, int64_t b) {
            std::vector<int>& h = cnt[(size_t)t];
            for (int64_t e = a; e < b; ++e) {
                const NrrInfl& x = trip[(size_t)e];
                iv[(size_t)(iptr[(size_t)x.pt] + h[(size_t)x.pt]++)] = {x.d2, x.node};
            }
        });
    }
    // Influence sets: the K nearest nodes, weights of Eq. (weight_data);
    // point chunks in parallel, each with its own list of node pairs
    g.nidx.assign((size_t)P * K, -1);
    g.w.assign((size_t)P * K, 0.0);
    const int64_t nt = setup_threads(P);
    std::vector<std::vector<std::pair<int, int>>> chunk_edges((size_t)nt);
    parallel_chunks_idx(P, nt, [&](int64_t t, int64_t i0, int64_t i1) {
    std::vector<std::pair<int, int>>& edge_list = chunk_edges[(size_t)t];
    for (int64_t i = i0; i < i1; ++i) {
        std::pair<double, int>* L = iv.data() + iptr[(size_t)i];
        const size_t nl = (size_t)(iptr[(size_t)i + 1] - iptr[(size_t)i]);
        std::sort(L, L + nl);
        int n = (int)std::min<size_t>(nl, (size_t)K);
        double raw[NRR_MAX_INFL];
        double sum = 0.0;
        for (int s = 0; s < n; ++s) {
            double a = 1.0 - L[(size_t)s].first / R2;
            raw[s] = a * a * a;
        }
        for (int s = 0; s < n; ++s) sum += raw[s];
        for (int s = 0; s < n; ++s) {
            g.nidx[(size_t)i * K + s] = L[(size_t)s].second;
            g.w[(size_t)i * K + s] = raw[s] / sum;
        }
        for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b) {
                int u = L[(size_t)a].second, v = L[(size_t)b].second;
                edge_list.push_back({std::min(u, v), std::max(u, v)});
            }
    }
    sort_unique_pairs(edge_list, (int)g.nodes.size());
    });
    // the chunks' lists are sorted and unique: merge them pairwise
    while (chunk_edges.size() > 1) {
        std::vector<std::vector<std::pair<int, int>>> next;
        for (size_t k = 0; k + 1 < chunk_edges.size(); k += 2) {
            std::vector<std::pair<int, int>> m;
            m.reserve(chunk_edges[k].size() + chunk_edges[k + 1].size());
            std::set_union(chunk_edges[k].begin(), chunk_edges[k].end(), chunk_edges[k + 1].begin(),
                           chunk_edges[k + 1].end(), std::back_inserter(m));
            next.push_back(std::move(m));
        }
        if (chunk_edges.size() % 2) next.push_back(std::move(chunk_edges.back()));
        chunk_edges.swap(next);
    }
    std::vector<std::pair<int, int>> edge_list;
    if (!chunk_edges.empty()) edge_list.swap(chunk_edges[0]);
    g.edges.clear();
    for (auto& e : edge_list) { g.edges.push_back(e.first); g.edges.push_back(e.second); }
    std::vector<std::pair<int, int>> dp;
    for (auto& e : edge_list) { dp.push_back(e); dp.push_back({e.second, e.first}); }
    std::sort(dp.begin(), dp.end());
    g.dpair.clear();
    for (auto& e : dp) { g.dpair.push_back(e.first); g.dpair.push_back(e.second); }
    // r_ij of Sec. 3.2
    size_t E2 = dp.size();
    std::vector<double> inv(E2);
    double inv_sum = 0.0;
    for (size_t e = 0; e < E2; ++e) {
        const double* a = V + 3 * (int64_t)g.nodes[(size_t)dp[e].first];
        const double* b = V + 3 * (int64_t)g.nodes[(size_t)dp[e].second];
        inv[e] = 1.0 / std::sqrt(sqd(a, b));
        inv_sum += inv[e];
    }
    g.r.resize(E2);
    for (size_t e = 0; e < E2; ++e) g.r[e] = 2.0 * (double)edge_list.size() * inv[e] / inv_sum;
}

bool nrr_graph_and_spacing(const double* V, int64_t P, double radius, int K, bool need_lbar, HostGraph& g) {
    double lbar = std::nan("");
    if (radius > 0) {
        // the graph does not need l-bar: its search runs on other threads
        // while Algorithm 1's greedy pass (sequential) holds one
        std::thread t;
        if (need_lbar) t = std::thread([&]() { lbar = nrr_mean_spacing(V, P, 6); });
        struct Join {
            std::thread& t;
            ~Join() { if (t.joinable()) t.join(); }
        } join{t};
        nrr_build_graph(V, P, radius, K, g);
    } else {
        lbar = nrr_mean_spacing(V, P, 6);
        const double R = 5.0 * lbar;
        if (!(R > 0)) return false;   // e.g. all points identical
        nrr_build_graph(V, P, R, K, g);
    }
    g.lbar = lbar;
    return true;
}

