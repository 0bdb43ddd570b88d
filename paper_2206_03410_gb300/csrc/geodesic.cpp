// Algorithm 1 (Sec. 3.1) on a triangle-mesh source: the ball B(v) of a new
// node by breadth-first search along mesh edges, exact geodesic distances
// D(v, q) on the sub-mesh of the faces incident to B(v), and the influence
// sets of Eq. (InfluenceNodes) with the weights of Eq. (weight_data) from D.
//
// Exact geodesics by window propagation (continuous Dijkstra): a shortest
// path on a polyhedral surface is straight inside faces, stays straight
// across an edge once the two faces are unfolded into one plane, and bends
// only at vertices whose total face angle is at least 2 pi or that lie on
// the boundary. A window is a set of such straight paths: an interval
// [b0, b1] of an edge, the unfolded position S of the vertex they start
// from (the source or a vertex where paths bend, a pseudo-source) in the
// edge's frame, and sigma, the distance from the source to that vertex;
// a point X of the interval is reached at sigma + |S - X|. Windows are
// processed in increasing order of their smallest distance; a window
// crossing a face splits into the parts of the two far edges that its
// paths reach, the far vertex gets a distance when a path reaches it, and
// a vertex where paths may bend emits new windows (sigma = its distance)
// into every face around it whenever its distance improves. Windows are not
// merged; two tests drop windows that cannot carry a shortest path:
//  * their smallest distance is at least R (only D < R matters);
//  * an endpoint of their edge reaches the whole interval more cheaply
//    along the edge: d(B) + |B X| < sigma + |S X| holds for all X of the
//    interval if it holds at the interval's end farthest from B (the
//    difference of the two sides only grows towards B), and a shortest
//    path cannot pass through a point that another path reaches sooner.
// The paper uses the VTP algorithm for the same exact distances.
#include <algorithm>
#include <cmath>
#include <queue>
#include <string>
#include <vector>

#include "nrr_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

double dist3(const double* a, const double* b) {
    const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return std::sqrt(dx * dx + dy * dy + dz * dz);
}

// Faces, the face across each face edge, vertex -> faces, vertex
// neighbours, and the total face angle and boundary flag of each vertex.
struct MeshTopo {
    int64_t P = 0, nF = 0;
    const double* V = nullptr;
    const int* F = nullptr;
    std::vector<int> across;        // [nF][3]: face across edge k = (F[k], F[k+1 mod 3]), -1 on the boundary
    std::vector<int> vf_ptr, vf;    // faces around each vertex
    std::vector<int> nb_ptr, nb;    // mesh neighbours of each vertex
    std::vector<double> angle;      // total face angle at each vertex
    std::vector<char> boundary;     // vertex on the mesh boundary

    bool build(const double* V_, int64_t P_, const int* F_, int64_t nF_, std::string& err) {
        V = V_; P = P_; F = F_; nF = nF_;
        for (int64_t f = 0; f < nF; ++f) {
            const int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
            if (a < 0 || b < 0 || c < 0 || a >= P || b >= P || c >= P) {
                err = "face " + std::to_string(f) + " has a vertex index out of range";
                return false;
            }
            if (a == b || b == c || a == c) {
                err = "face " + std::to_string(f) + " repeats a vertex";
                return false;
            }
        }
        // edges (lo, hi, face * 3 + k), sorted: equal edges are adjacent
        struct HalfEdge { int lo, hi; int64_t fk; };
        std::vector<HalfEdge> he((size_t)(3 * nF));
        for (int64_t f = 0; f < nF; ++f)
            for (int k = 0; k < 3; ++k) {
                const int u = F[3 * f + k], v = F[3 * f + (k + 1) % 3];
                he[(size_t)(3 * f + k)] = {std::min(u, v), std::max(u, v), 3 * f + k};
            }
        std::sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
            return x.lo != y.lo ? x.lo < y.lo : x.hi != y.hi ? x.hi < y.hi : x.fk < y.fk;
        });
        across.assign((size_t)(3 * nF), -1);
        std::vector<std::vector<int>> nbv((size_t)P);
        for (size_t i = 0; i < he.size();) {
            size_t j = i;
            while (j < he.size() && he[j].lo == he[i].lo && he[j].hi == he[i].hi) ++j;
            if (j - i > 2) {
                err = "edge (" + std::to_string(he[i].lo) + ", " + std::to_string(he[i].hi) +
                      ") is shared by more than two faces";
                return false;
            }
            if (j - i == 2) {
                across[(size_t)he[i].fk] = (int)(he[i + 1].fk / 3);
                across[(size_t)he[i + 1].fk] = (int)(he[i].fk / 3);
            }
            nbv[(size_t)he[i].lo].push_back(he[i].hi);
            nbv[(size_t)he[i].hi].push_back(he[i].lo);
            i = j;
        }
        nb_ptr.assign((size_t)P + 1, 0);
        for (int64_t v = 0; v < P; ++v) nb_ptr[(size_t)v + 1] = nb_ptr[(size_t)v] + (int)nbv[(size_t)v].size();
        nb.resize((size_t)nb_ptr[(size_t)P]);
        for (int64_t v = 0; v < P; ++v)
            std::copy(nbv[(size_t)v].begin(), nbv[(size_t)v].end(), nb.begin() + nb_ptr[(size_t)v]);
        vf_ptr.assign((size_t)P + 1, 0);
        for (int64_t f = 0; f < nF; ++f)
            for (int k = 0; k < 3; ++k) vf_ptr[(size_t)F[3 * f + k] + 1]++;
        for (int64_t v = 0; v < P; ++v) vf_ptr[(size_t)v + 1] += vf_ptr[(size_t)v];
        vf.resize((size_t)vf_ptr[(size_t)P]);
        std::vector<int> fill(vf_ptr.begin(), vf_ptr.end() - 1);
        angle.assign((size_t)P, 0.0);
        boundary.assign((size_t)P, 0);
        for (int64_t f = 0; f < nF; ++f)
            for (int k = 0; k < 3; ++k) {
                const int v = F[3 * f + k], a = F[3 * f + (k + 1) % 3], b = F[3 * f + (k + 2) % 3];
                vf[(size_t)fill[(size_t)v]++] = (int)f;
                const double la = dist3(V + 3 * (int64_t)v, V + 3 * (int64_t)a);
                const double lb = dist3(V + 3 * (int64_t)v, V + 3 * (int64_t)b);
                const double lab = dist3(V + 3 * (int64_t)a, V + 3 * (int64_t)b);
                if (!(la > 0) || !(lb > 0) || !(lab > 0)) {
                    err = "face " + std::to_string(f) + " has an edge of zero length";
                    return false;
                }
                const double c = (la * la + lb * lb - lab * lab) / (2.0 * la * lb);
                angle[(size_t)v] += std::acos(std::max(-1.0, std::min(1.0, c)));
                if (across[(size_t)(3 * f + k)] < 0) {
                    boundary[(size_t)F[3 * f + k]] = 1;
                    boundary[(size_t)F[3 * f + (k + 1) % 3]] = 1;
                }
            }
        return true;
    }
    double len(int a, int b) const { return dist3(V + 3 * (int64_t)a, V + 3 * (int64_t)b); }
};

// A window on the edge a -> b (frame: a at the origin, b at (L, 0)); it
// entered that edge from face `from` (on the negative-y side) and enters the
// face across the edge next.
struct Window {
    double key;          // smallest distance of its points
    int from, a, b;
    double L, b0, b1;    // interval [b0, b1] of [0, L]
    double sx, sy;       // source in the frame (sy <= 0)
    double sigma;
};
struct WindowOrder {
    bool operator()(const Window& x, const Window& y) const { return x.key > y.key; }
};

// Geodesic distances from one vertex over a sub-mesh (faces stamped with
// the current node), reused across nodes: per-vertex and per-face stamps
// replace clearing.
class GeodesicSolver {
  public:
    explicit GeodesicSolver(const MeshTopo& m)
        : m_(m), face_stamp_((size_t)m.nF, -1), vert_stamp_((size_t)m.P, -1), d_((size_t)m.P, 0.0) {}

    // Marks the faces around the vertices of `ball` as the sub-mesh of this
    // run; the sub-mesh boundary is where a face edge has no sub-mesh face
    // across it.
    void set_submesh(const std::vector<int>& ball) {
        ++run_;
        for (int q : ball)
            for (int k = m_.vf_ptr[(size_t)q]; k < m_.vf_ptr[(size_t)q + 1]; ++k) face_stamp_[(size_t)m_.vf[(size_t)k]] = run_;
    }

    // D(s, q) for the vertices q reached below `limit` (others: +inf).
    bool solve(int s, double limit, std::string& err) {
        limit_ = limit;
        heap_ = {};
        set_dist(s, 0.0);
        emit_from(s);
        long long processed = 0;
        while (!heap_.empty()) {
            Window w = heap_.top();
            heap_.pop();
            if (++processed > kMaxWindows) {
                err = "geodesic window propagation exceeded its limit";
                return false;
            }
            if (dominated(w)) continue;
            propagate(w);
        }
        return true;
    }

    double dist(int v) const { return vert_stamp_[(size_t)v] == run_ ? d_[(size_t)v] : INFINITY; }

  private:
    static constexpr long long kMaxWindows = 20000000;

    bool in_sub(int f) const { return f >= 0 && face_stamp_[(size_t)f] == run_; }

    void set_dist(int v, double d) {
        vert_stamp_[(size_t)v] = run_;
        d_[(size_t)v] = d;
    }

    // A vertex where shortest paths may bend: total face angle at least
    // 2 pi (flat vertices included, for paths that pass exactly through
    // them), or on the boundary of the mesh or of the sub-mesh.
    bool bend_vertex(int v) const {
        if (m_.boundary[(size_t)v] || m_.angle[(size_t)v] >= 2.0 * kPi - 1e-9) return true;
        for (int k = m_.vf_ptr[(size_t)v]; k < m_.vf_ptr[(size_t)v + 1]; ++k)
            if (!in_sub(m_.vf[(size_t)k])) return true;
        return false;
    }

    // Offers distance d to vertex v; on improvement a bending vertex emits
    // windows.
    void offer(int v, double d) {
        if (d < dist(v)) {
            set_dist(v, d);
            if (bend_vertex(v) && d < limit_) emit_from(v);
        }
    }

    // Windows of the paths that start at vertex v (distance dist(v)): one on
    // the far edge of each sub-mesh face around v.
    void emit_from(int v) {
        const double sigma = dist(v);
        for (int k = m_.vf_ptr[(size_t)v]; k < m_.vf_ptr[(size_t)v + 1]; ++k) {
            const int f = m_.vf[(size_t)k];
            if (!in_sub(f)) continue;
            const int* F = m_.F + 3 * (int64_t)f;
            const int kv = F[0] == v ? 0 : F[1] == v ? 1 : 2;
            // the far edge runs F[kv+1] -> F[kv+2] in the face's order, so v
            // lies to its left; the window's frame needs the face on the
            // negative side: orient it F[kv+2] -> F[kv+1]
            const int a = F[(kv + 2) % 3], b = F[(kv + 1) % 3];
            const double L = m_.len(a, b), la = m_.len(a, v), lb = m_.len(b, v);
            const double x = (L * L + la * la - lb * lb) / (2.0 * L);
            const double y = -std::sqrt(std::max(la * la - x * x, 0.0));
            push(Window{0.0, f, a, b, L, 0.0, L, x, y, sigma});
        }
    }

    static double seg_dist(double sx, double sy, double b0, double b1) {
        const double x = std::min(std::max(sx, b0), b1);
        return std::hypot(sx - x, sy);
    }

    bool dominated(const Window& w) const {
        if (w.key >= limit_) return true;
        const double da = dist(w.a), db = dist(w.b);
        if (db + (w.L - w.b0) < w.sigma + std::hypot(w.sx - w.b0, w.sy)) return true;
        if (da + w.b1 < w.sigma + std::hypot(w.sx - w.b1, w.sy)) return true;
        return false;
    }

    void push(Window w) {
        if (!(w.b1 >= w.b0)) return;
        // endpoints reached by the window
        const double tol = 1e-12 * w.L;
        if (w.b0 <= tol) offer(w.a, w.sigma + std::hypot(w.sx, w.sy));
        if (w.b1 >= w.L - tol) offer(w.b, w.sigma + std::hypot(w.sx - w.L, w.sy));
        w.key = w.sigma + seg_dist(w.sx, w.sy, w.b0, w.b1);
        if (dominated(w)) return;
        heap_.push(w);
    }

    // Crosses the face beyond the window's edge.
    void propagate(const Window& w) {
        // the face across a -> b other than w.from
        int g = -1;
        {
            const int* F = m_.F + 3 * (int64_t)w.from;
            for (int k = 0; k < 3; ++k) {
                const int u = F[k], v = F[(k + 1) % 3];
                if ((u == w.a && v == w.b) || (u == w.b && v == w.a)) g = m_.across[(size_t)(3 * (int64_t)w.from + k)];
            }
        }
        if (!in_sub(g)) return;
        const int* G = m_.F + 3 * (int64_t)g;
        const int c = G[0] != w.a && G[0] != w.b ? G[0] : G[1] != w.a && G[1] != w.b ? G[1] : G[2];
        const double lac = m_.len(w.a, c), lbc = m_.len(w.b, c);
        const double cx = (w.L * w.L + lac * lac - lbc * lbc) / (2.0 * w.L);
        const double cy = std::sqrt(std::max(lac * lac - cx * cx, 0.0));
        // cone from S through (b0, 0) (left ray d0) and (b1, 0) (right ray d1)
        const double d0x = w.b0 - w.sx, d0y = -w.sy;
        const double d1x = w.b1 - w.sx, d1y = -w.sy;
        const double qx = cx - w.sx, qy = cy - w.sy;
        const double right = d1x * qy - d1y * qx;   // >= 0: C not right of the cone
        const double left = qx * d0y - qy * d0x;    // >= 0: C not left of the cone
        // intersection parameter t in [0, 1] along p -> q of the line
        // through S with direction (dx, dy)
        auto hit = [&](double px, double py, double ex, double ey, double dx, double dy) {
            const double den = ex * dy - ey * dx;
            if (den == 0.0) return 0.0;
            const double t = ((w.sx - px) * dy - (w.sy - py) * dx) / den;
            return std::min(1.0, std::max(0.0, t));
        };
        const double acx = cx, acy = cy;              // A -> C
        const double cbx = w.L - cx, cby = -cy;       // C -> B
        if (right >= 0.0 && left >= 0.0) {
            offer(c, w.sigma + std::hypot(qx, qy));
            child(w, g, w.a, c, 0.0, 0.0, acx, acy, hit(0.0, 0.0, acx, acy, d0x, d0y), 1.0);
            child(w, g, c, w.b, cx, cy, cbx, cby, 0.0, hit(cx, cy, cbx, cby, d1x, d1y));
        } else if (right < 0.0) {
            // the cone lies left of C: its paths leave through A -> C
            child(w, g, w.a, c, 0.0, 0.0, acx, acy, hit(0.0, 0.0, acx, acy, d0x, d0y),
                  hit(0.0, 0.0, acx, acy, d1x, d1y));
        } else {
            // right of C: through C -> B
            child(w, g, c, w.b, cx, cy, cbx, cby, hit(cx, cy, cbx, cby, d0x, d0y),
                  hit(cx, cy, cbx, cby, d1x, d1y));
        }
    }

    // The window on edge u -> v of face g (u at (px, py) in the parent frame,
    // direction (ex, ey) to v), interval t in [t0, t1] of its length.
    void child(const Window& w, int g, int u, int v, double px, double py, double ex, double ey, double t0,
               double t1) {
        const double L = std::hypot(ex, ey);
        const double ux = ex / L, uy = ey / L;
        // frame of u -> v: x along it, y to its left; face g lies on its right
        const double rx = w.sx - px, ry = w.sy - py;
        const double sx = rx * ux + ry * uy;
        const double sy = -rx * uy + ry * ux;
        push(Window{0.0, g, u, v, L, std::min(t0, t1) * L, std::max(t0, t1) * L, sx, sy, w.sigma});
    }

    const MeshTopo& m_;
    std::vector<int> face_stamp_, vert_stamp_;
    std::vector<double> d_;
    int run_ = 0;
    double limit_ = INFINITY;
    std::priority_queue<Window, std::vector<Window>, WindowOrder> heap_;
};

}  // namespace

double nrr_mesh_mean_edge(const double* V, const int* F, int64_t nF) {
    std::vector<std::pair<int, int>> e;
    e.reserve((size_t)(3 * nF));
    for (int64_t f = 0; f < nF; ++f)
        for (int k = 0; k < 3; ++k) {
            const int u = F[3 * f + k], v = F[3 * f + (k + 1) % 3];
            e.push_back({std::min(u, v), std::max(u, v)});
        }
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    if (e.empty()) return 0.0;
    double s = 0.0;
    for (const auto& x : e) s += dist3(V + 3 * (int64_t)x.first, V + 3 * (int64_t)x.second);
    return s / (double)e.size();
}

bool nrr_build_graph_mesh(const double* V, int64_t P, const int* F, int64_t nF, double R, int K, HostGraph& g,
                          std::string& err) {
    MeshTopo m;
    if (!m.build(V, P, F, nF, err)) return false;
    const double R2 = R * R;
    const std::vector<int> order = nrr_pca_order(V, P);
    GeodesicSolver geo(m);
    std::vector<NrrInfl> trip;
    std::vector<unsigned char> covered((size_t)P, 0), in_ball((size_t)P, 0);
    std::vector<int> ball;
    g.nodes.clear();
    for (int i : order) {
        if (!g.nodes.empty() && covered[(size_t)i]) continue;
        const int j = (int)g.nodes.size();
        g.nodes.push_back(i);
        // B(v_i): breadth-first along mesh edges through |v_i - q| < R
        const double* vi = V + 3 * (int64_t)i;
        ball.assign(1, i);
        in_ball[(size_t)i] = 1;
        for (size_t k = 0; k < ball.size(); ++k) {
            const int a = ball[k];
            for (int e = m.nb_ptr[(size_t)a]; e < m.nb_ptr[(size_t)a + 1]; ++e) {
                const int b = m.nb[(size_t)e];
                if (in_ball[(size_t)b]) continue;
                const double* q = V + 3 * (int64_t)b;
                const double dx = q[0] - vi[0], dy = q[1] - vi[1], dz = q[2] - vi[2];
                if (dx * dx + dy * dy + dz * dz < R2) {
                    in_ball[(size_t)b] = 1;
                    ball.push_back(b);
                }
            }
        }
        geo.set_submesh(ball);
        if (!geo.solve(i, R, err)) return false;
        // ball order is the breadth-first order; influences within one node
        // in increasing vertex order (the grouping by point keeps node order)
        std::sort(ball.begin(), ball.end());
        for (int q : ball) {
            in_ball[(size_t)q] = 0;
            const double d = geo.dist(q);
            if (d < R) {
                trip.push_back({q, j, d * d});
                covered[(size_t)q] = 1;
            }
        }
    }
    nrr_finish_graph(V, P, R, K, trip, g);
    return true;
}
