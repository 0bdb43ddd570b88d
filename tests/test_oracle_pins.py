"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics: closed forms, invariants, special cases that reduce to library
routines, brute force on tiny inputs, and a hand-worked example.

Every check here is independent of the oracle's own formulas: a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.spatial

import synth
from oracle import anderson, graph as G, model as M, surrogate as S
from oracle.solver import Params, Registration

HERE = os.path.dirname(os.path.abspath(__file__))


def _rng(s=0):
    return np.random.default_rng(s)


def _near_identity_X(N, rng, scale=0.05):
    X = M.identity_X(N).reshape(N, 4, 3)
    X = X + scale * rng.standard_normal(X.shape)
    return X.reshape(N, 12)


@pytest.fixture(scope="module")
def small():
    pair = synth.tiny_pair(400, 450, seed=3, noise=0.002, outliers=0.05)
    g = G.build_graph(pair.src.astype(np.float64), 0.35)
    return pair, g


# ---------------------------------------------------------------- Welsch ---

def test_welsch_closed_forms():
    """Eq. (Welsch_func): psi(0)=0, psi(nu)=1-e^{-1/2}, bounded by 1, and the
    l0 limit as nu -> 0 (Sec. 3.2)."""
    nu = 0.7
    assert M.welsch(0.0, nu) == 0.0
    assert abs(M.welsch(nu * nu, nu) - (1 - math.exp(-0.5))) < 1e-15
    x = np.linspace(0, 50, 1001)
    v = M.welsch(x * x, nu)
    assert np.all(v <= 1.0) and np.all(v[x < 5] < 1.0) and np.all(np.diff(v) >= 0)
    assert abs(M.welsch(1.0, 1e-3) - 1.0) < 1e-15


def test_welsch_surrogate_majorizes_and_touches():
    """Eq. (WelschSurrogateFunc) bounds psi from above and touches it at
    x = y with equal slope (Sec. 3.3.1)."""
    nu = 0.3
    xs = np.linspace(0, 3, 301)
    for y in np.linspace(0, 3, 61):
        s = M.welsch_surrogate(xs, y, nu)
        f = M.welsch(xs * xs, nu)
        assert np.all(s >= f - 1e-15)
        assert abs(M.welsch_surrogate(y, y, nu) - M.welsch(y * y, nu)) < 1e-15
        h = 1e-6
        ds = (M.welsch_surrogate(y + h, y, nu) - M.welsch_surrogate(y - h, y, nu)) / (2 * h)
        df = (M.welsch((y + h) ** 2, nu) - M.welsch((y - h) ** 2, nu)) / (2 * h)
        assert abs(ds - df) < 1e-7


# ----------------------------------------------------------------- graph ---

def test_graph_hand_worked_line():
    """Algorithm 1 on 11 collinear points, worked by hand (golden file)."""
    with open(os.path.join(HERE, "golden", "line_graph.json")) as f:
        gold = json.load(f)
    x = np.array(gold["points_x"])
    V = np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1)
    g = G.build_graph(V, gold["radius"])
    assert g.nodes.tolist() == gold["nodes"]
    for i, inf in enumerate(gold["influence"]):
        got = [int(j) for j in g.nidx[i] if j >= 0]
        assert got == inf, (i, got, inf)
    assert g.edges.tolist() == gold["edges"]
    raw = np.array([(1 - 0.01 / 0.0625) ** 3, (1 - 0.04 / 0.0625) ** 3])
    assert np.allclose(g.w[1, :2], raw / raw.sum(), rtol=0, atol=1e-15)


def test_pca_axis_matches_svd():
    V = _rng(1).standard_normal((300, 3)) * np.array([3.0, 1.0, 0.5])
    a = G.pca_axis(V)
    _, _, vt = np.linalg.svd(V - V.mean(0))
    assert min(np.linalg.norm(a - vt[0]), np.linalg.norm(a + vt[0])) < 1e-10
    assert a[np.argmax(np.abs(a))] > 0


def test_graph_invariants_brute_force(small):
    """Nodes are R-separated; every point has a non-empty influence set equal
    to the brute-force set of nodes within R (cap 8 not binding here);
    weights sum to one (Eq. weight_data); edges join co-influencing nodes;
    mean r_ij over directed pairs is 1 and r_ij is proportional to 1/|p_i-p_j|."""
    pair, g = small
    V = pair.src.astype(np.float64)
    R = g.radius
    dn = scipy.spatial.distance.cdist(g.p, g.p)
    np.fill_diagonal(dn, np.inf)
    assert dn.min() >= R
    dv = scipy.spatial.distance.cdist(V, g.p)
    for i in range(V.shape[0]):
        brute = sorted(np.nonzero(dv[i] < R)[0].tolist(), key=lambda j: (dv[i, j], j))
        got = [int(j) for j in g.nidx[i] if j >= 0]
        assert got == brute[:8] and len(got) >= 1
    ws = g.w.sum(axis=1)
    assert np.allclose(ws, 1.0, atol=1e-14)
    expect = set()
    for i in range(V.shape[0]):
        ids = [int(j) for j in g.nidx[i] if j >= 0]
        for a in ids:
            for b in ids:
                if a < b:
                    expect.add((a, b))
    assert set(map(tuple, g.edges.tolist())) == expect
    assert abs(g.r.mean() - 1.0) < 1e-13
    d = np.linalg.norm(g.p[g.dpair[:, 0]] - g.p[g.dpair[:, 1]], axis=1)
    assert np.allclose(g.r * d, (g.r * d)[0], rtol=1e-12)


def test_mean_spacing_matches_kdtree():
    V = _rng(2).random((500, 3))
    tree = scipy.spatial.cKDTree(V)
    d, _ = tree.query(V, k=7)
    assert abs(G.mean_spacing(V) - d[:, 1:].mean()) < 1e-13


# ---------------------------------------------------------------- deform ---

def test_deform_identity_translation_affine(small):
    """Eq. (deformed_position) with the partition of unity: X = I gives v,
    equal translations give v + t, and node-consistent affine maps give the
    global map A v + t exactly."""
    pair, g = small
    V = pair.src.astype(np.float64)
    N = g.N
    assert np.allclose(M.deform(V, g.nidx, g.w, g.p, M.identity_X(N)), V, atol=1e-14)
    t = np.array([0.3, -0.2, 0.1])
    X = M.identity_X(N).reshape(N, 4, 3)
    X[:, 3, :] = t
    assert np.allclose(M.deform(V, g.nidx, g.w, g.p, X.reshape(N, 12)), V + t, atol=1e-14)
    A = np.array([[1.1, 0.2, -0.1], [0.05, 0.9, 0.3], [-0.2, 0.1, 1.2]])
    X = np.zeros((N, 4, 3))
    X[:, :3, :] = A.T
    X[:, 3, :] = t - g.p + g.p @ A.T          # t_j = t - p_j + A p_j
    out = M.deform(V, g.nidx, g.w, g.p, X.reshape(N, 12))
    assert np.allclose(out, V @ A.T + t, atol=1e-13)


# ------------------------------------------------------------ closest pt ---

def test_closest_points_match_kdtree_and_ties():
    rng = _rng(4)
    U = rng.random((700, 3))
    Q = rng.random((300, 3))
    rho, d2 = M.closest_points(Q, U)
    d, idx = scipy.spatial.cKDTree(U).query(Q)
    assert np.allclose(np.sqrt(d2), d, atol=1e-14)
    # where the kd-tree's pick differs it must be an exact tie
    assert np.all((rho == idx) | (np.abs(d2 - d * d) < 1e-15))
    # exact duplicates: lowest index wins
    U2 = np.concatenate([U, U])
    rho2, _ = M.closest_points(Q, U2)
    assert np.array_equal(rho2, rho)
    rho3, _ = M.closest_points(Q, np.concatenate([U[:5], U]))
    assert np.all(rho3 == np.where(rho < 5, rho, rho + 5))


# ---------------------------------------------------------------- energy ---

def test_energy_zero_for_identical_shapes():
    """Source = target and X = I: closest points are the points themselves,
    D_ij = 0 and A = I, so E = 0 (Eq. objective_func)."""
    pair = synth.tiny_pair(300, 300, seed=5)
    V = pair.src.astype(np.float64)
    reg = Registration(V, V, Params(radius=0.4, nu_a=0.1, nu_r=0.1, nu_a_min=0.1))
    E, t = reg.energy()
    assert E == 0.0 and t["E_align"] == 0.0 and t["E_reg"] == 0.0 and t["E_rot"] == 0.0


def test_rotation_projection_and_rot_energy():
    """proj_R gives an orthonormal matrix with det +1; for A = R0 S with S
    symmetric positive definite it returns R0 (polar decomposition); and
    |A - proj_R(A)|_F^2 = sum (sigma_i - 1)^2 with sigma from eig(A^T A)."""
    rng = _rng(6)
    for _ in range(50):
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        B = rng.standard_normal((3, 3))
        Sm = B @ B.T + 0.5 * np.eye(3)
        A = q @ Sm
        Rm = M.proj_rotation(A)
        assert np.allclose(Rm.T @ Rm, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(Rm) - 1) < 1e-13
        assert np.allclose(Rm, q, atol=1e-12)
        sig = np.sqrt(np.linalg.eigvalsh(A.T @ A))
        assert abs(np.sum((A - Rm) ** 2) - np.sum((sig - 1) ** 2)) < 1e-10
    # reflection: det < 0 flips the smallest singular direction
    A = np.diag([2.0, 1.0, -0.5])
    assert np.allclose(M.proj_rotation(A), np.diag([1.0, 1.0, 1.0]))


def test_reg_residual_zero_for_rigid_field(small):
    """D_ij vanishes when all nodes carry the same affine map (Eq. reg_diff)."""
    pair, g = small
    A = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    t = np.array([0.1, 0.2, 0.3])
    X = np.zeros((g.N, 4, 3))
    X[:, :3, :] = A.T
    X[:, 3, :] = t - g.p + g.p @ A.T
    D = M.reg_residuals(g.p, g.dpair, g.r, X.reshape(g.N, 12))
    assert np.abs(D).max() < 1e-13


# ------------------------------------------------------------- surrogate ---

def _state(pair, g, X, nu_a=0.05, nu_r=0.1):
    V = pair.src.astype(np.float64)
    U = pair.tgt.astype(np.float64)
    t = M.energy_terms(V, U, g, X, nu_a, nu_r)
    return V, U, t


def test_matrix_form_equals_sums(small):
    """|W_a(FX-Q)|^2, |W_r(HX-Y)|^2 and |JX-Z|^2 (Sec. 3.3.2) equal the
    term-by-term surrogates of Eqs. (AlignQuadSurrogate), (ERegSurrogate) and
    the rotation surrogate at an arbitrary X."""
    pair, g = small
    rng = _rng(7)
    Xk = _near_identity_X(g.N, rng)
    nu_a, nu_r = 0.05, 0.1
    V, U, t = _state(pair, g, Xk, nu_a, nu_r)
    _, _, parts = S.normal_equations(V, U, g, t, nu_a, nu_r, 1.0, 1.0)
    X = _near_identity_X(g.N, rng).reshape(4 * g.N, 3)
    vh = M.deform(V, g.nidx, g.w, g.p, X.reshape(g.N, 12))
    wa = np.exp(-t["d2"] / (2 * nu_a ** 2)) / (2 * nu_a ** 2)
    ref_a = np.sum(wa * np.sum((vh - U[t["rho"]]) ** 2, axis=1))
    got_a = np.sum(parts["wa"][:, None] * (parts["F"] @ X - parts["Q"]) ** 2)
    assert abs(got_a - ref_a) < 1e-10 * abs(ref_a)
    D = M.reg_residuals(g.p, g.dpair, g.r, X.reshape(g.N, 12))
    Dk = t["D"]
    wr = np.exp(-np.sum(Dk ** 2, 1) / (2 * nu_r ** 2)) / (2 * nu_r ** 2)
    ref_r = np.sum(wr * np.sum(D ** 2, axis=1))
    got_r = np.sum(parts["wr"][:, None] * (parts["H"] @ X - parts["Y"]) ** 2)
    assert abs(got_r - ref_r) < 1e-10 * abs(ref_r)
    A = M.A_of(X.reshape(g.N, 12))
    ref_o = np.sum((A - t["R"]) ** 2)
    got_o = np.sum((parts["J"] @ X - parts["Z"]) ** 2)
    assert abs(got_o - ref_o) < 1e-10 * abs(ref_o)


def test_normal_equations_minimise_surrogate(small):
    """The solution of K X = B zeroes the gradient of the term-by-term
    surrogate (central differences) and the surrogate with the dropped
    constants restored majorises E and touches it at X^k (Eq. MMConditions)."""
    pair, g = small
    rng = _rng(8)
    Xk = _near_identity_X(g.N, rng, 0.02)
    nu_a, nu_r, alpha, beta = 0.05, 0.1, 2.0, 0.5
    V, U, t = _state(pair, g, Xk, nu_a, nu_r)
    K, B, _ = S.normal_equations(V, U, g, t, nu_a, nu_r, alpha, beta)
    Kd = K.toarray()
    assert np.allclose(Kd, Kd.T, atol=1e-12)
    assert np.linalg.eigvalsh(Kd).min() > 0
    Xs = S.solve_normal_equations(K, B)
    # the dense Cholesky the oracle uses for small systems and the sparse LU
    # it uses for large ones agree, and both leave a residual at rounding
    Bm = np.asarray(B).reshape(-1, 3)
    Xlu = np.asarray(S.spla.spsolve(K.tocsc(), Bm)).reshape(Xs.shape)
    assert np.abs(Xlu - Xs).max() <= 1e-10 * np.abs(Xs).max()
    knorm = np.linalg.norm(Kd, 2)
    for Xsol in (Xs, Xlu):
        # backward error of a backward-stable direct solve
        res = Kd @ Xsol.reshape(-1, 3) - Bm
        assert np.linalg.norm(res) <= 1e-13 * knorm * np.linalg.norm(Xsol)
    f = lambda X: S.surrogate_value(V, U, g, t, X, nu_a, nu_r, alpha, beta)
    flat = Xs.ravel()
    h = 1e-5
    for idx in rng.choice(flat.size, 12, replace=False):
        e = np.zeros_like(flat)
        e[idx] = h
        gd = (f((flat + e).reshape(Xs.shape)) - f((flat - e).reshape(Xs.shape))) / (2 * h)
        assert abs(gd) < 1e-5 * (1 + abs(f(Xs))), (idx, gd)
    # majorisation and touching
    Ek = M.total_energy(t, alpha, beta)
    assert abs(f(Xk) - Ek) < 1e-10 * abs(Ek)
    for _ in range(10):
        X = Xk + 0.01 * rng.standard_normal(Xk.shape)
        tX = M.energy_terms(V, U, g, X, nu_a, nu_r)
        assert f(X) >= M.total_energy(tX, alpha, beta) - 1e-10


def test_known_affine_map_recovered_in_one_solve():
    """Target = global affine image of the source with known correspondences
    and beta = 0: one MM solve recovers the map on every node to 1e-10."""
    pair = synth.tiny_pair(500, 500, seed=9)
    V = pair.src.astype(np.float64)
    A = np.array([[1.05, 0.1, 0.0], [-0.08, 0.97, 0.05], [0.02, -0.03, 1.1]])
    t = np.array([0.02, -0.01, 0.03])
    U = V @ A.T + t
    g = G.build_graph(V, 0.35)
    X0 = M.identity_X(g.N)
    terms = M.energy_terms(V, U, g, X0, 0.2, 0.2, rho=np.arange(V.shape[0]))
    K, B, _ = S.normal_equations(V, U, g, terms, 0.2, 0.2, 1.0, 0.0)
    X = S.solve_normal_equations(K, B).reshape(g.N, 4, 3)
    assert np.allclose(X[:, :3, :], np.broadcast_to(A.T, (g.N, 3, 3)), atol=1e-10)
    assert np.allclose(X[:, 3, :], t - g.p + g.p @ A.T, atol=1e-10)


# ----------------------------------------------------------- algorithm 2 ---

@pytest.mark.parametrize("robust,aa_m", [("welsch", 5), ("l2", 5), ("l2r", 0), ("l2r", 5)])
def test_mm_monotone_and_aa_safeguard(robust, aa_m):
    """Kept energies never increase within a stage (Sec. 3.3, monotone MM
    plus the AA safeguard of Sec. 3.3.4), for Welsch's function and for the
    variants of Sec. 4.2 (plain MM on the truncated quadratic included)."""
    pair = synth.tiny_pair(600, 650, seed=10, noise=0.003, outliers=0.05)
    reg = Registration(pair.src, pair.tgt, Params(radius=0.35, aa_m=aa_m, robust=robust,
                                                  max_iters_per_stage=15))
    reg.solve(max_passes=60)
    by_stage = {}
    for r in reg.records:
        if r.kept:
            by_stage.setdefault(r.stage, []).append(r.E)
    assert by_stage
    for es in by_stage.values():
        assert all(b <= a * (1 + 1e-12) for a, b in zip(es, es[1:]))


def test_aa_m0_is_plain_mm():
    pair = synth.tiny_pair(300, 320, seed=11, noise=0.002)
    p = Params(radius=0.4, aa_m=0, max_iters_per_stage=6)
    a = Registration(pair.src, pair.tgt, p)
    a.solve(max_passes=6)
    b = Registration(pair.src, pair.tgt, p)
    for _ in range(6):
        if b.done:
            break
        t = b.terms()
        G_ = b.mm_map(t)
        b.step()
        assert np.array_equal(b.X, G_) or b.done
    assert np.array_equal(a.X, b.X)


def test_anderson_linear_contraction():
    """On an affine contraction G(x) = M x + b of dimension d, AA with
    m >= d reaches the fixed point after d + 1 mixes (the textbook
    equivalence with GMRES), up to the tiny ridge."""
    rng = _rng(12)
    d = 4
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    Mx = Q @ np.diag([0.9, 0.5, -0.3, 0.7]) @ Q.T
    b = rng.standard_normal(d)
    xstar = np.linalg.solve(np.eye(d) - Mx, b)
    aa = anderson.Anderson(m=d)
    x = np.zeros(d)
    for _ in range(d + 2):
        x = aa.mix(Mx @ x + b, x)
    assert np.linalg.norm(x - xstar) < 1e-6 * np.linalg.norm(xstar)
    plain = np.zeros(d)
    for _ in range(d + 2):
        plain = Mx @ plain + b
    assert np.linalg.norm(plain - xstar) > 1e-2


def test_energy_gradient_matches_central_differences(small):
    """The analytic gradient of E with the closest points held fixed equals
    FP64 central differences (h = 1e-6) of E at points where no closest point
    changes within +-h (checked), for X and for the source positions."""
    pair, g = small
    rng = _rng(13)
    X = _near_identity_X(g.N, rng, 0.02)
    V = pair.src.astype(np.float64)
    U = pair.tgt.astype(np.float64)
    nu_a, nu_r, alpha, beta = 0.05, 0.1, 3.0, 0.7
    t0 = M.energy_terms(V, U, g, X, nu_a, nu_r)
    gX, gv = M.energy_gradient(V, U, g, X, nu_a, nu_r, alpha, beta)

    def E(Xv, Vv):
        t = M.energy_terms(Vv, U, g, Xv, nu_a, nu_r)
        assert np.array_equal(t["rho"], t0["rho"])     # no flip within the step
        return M.total_energy(t, alpha, beta)

    h = 1e-6
    flat = X.ravel()
    for idx in rng.choice(flat.size, 10, replace=False):
        e = np.zeros_like(flat)
        e[idx] = h
        fd = (E((flat + e).reshape(X.shape), V) - E((flat - e).reshape(X.shape), V)) / (2 * h)
        assert abs(fd - gX.ravel()[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, gX.ravel()[idx])
    for i in rng.choice(V.shape[0], 6, replace=False):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[i, c] += h
            Vm[i, c] -= h
            # node positions p_j are held constant: only v_i moves
            fd = (E(X, Vp) - E(X, Vm)) / (2 * h)
            assert abs(fd - gv[i, c]) < 1e-6 * max(1.0, abs(fd)), (i, c, fd, gv[i, c])


# ------------------------------------------------- unrolled MM derivative ---

def test_proj_rotation_vjp_matches_central_differences():
    """The reverse-mode derivative of proj_R equals FP64 central differences
    of <Rbar, proj_R(A)>, for det A > 0 (polar factor) and det A < 0 (the
    reflected singular vector), on random matrices."""
    from oracle import unrolled as UR
    rng = _rng(31)
    for flip in (False, True):
        for _ in range(4):
            A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
            if flip:
                A[:, 0] = -A[:, 0]
            if (np.linalg.det(A) < 0) != flip:
                continue
            Rbar = rng.standard_normal((3, 3))
            Abar = UR.proj_rotation_vjp(A, Rbar)
            h = 1e-6
            for a in range(3):
                for b in range(3):
                    Ap, Am = A.copy(), A.copy()
                    Ap[a, b] += h
                    Am[a, b] -= h
                    fd = (np.sum(Rbar * M.proj_rotation(Ap)) - np.sum(Rbar * M.proj_rotation(Am))) / (2 * h)
                    assert abs(fd - Abar[a, b]) < 1e-7 * max(1.0, abs(fd)), (flip, a, b, fd, Abar[a, b])


@pytest.fixture(scope="module")
def unroll_case():
    pair = synth.tiny_pair(300, 330, seed=8, noise=0.002, outliers=0.03)
    g = G.build_graph(pair.src.astype(np.float64), 0.4)
    X0 = _near_identity_X(g.N, _rng(5), 0.01)
    return pair.src.astype(np.float64), pair.tgt.astype(np.float64), g, X0


@pytest.mark.parametrize("loss", ["energy", "cotangent"])
def test_unrolled_backward_matches_central_differences(unroll_case, loss):
    """dL/dX^(0) and dL/dV of K = 3 unrolled MM steps (fixed nu, no AA)
    equal FP64 central differences (h = 1e-6) of the oracle's forward map, at
    points where no closest point of any step changes within +-h (checked);
    node positions and skinning weights are held constant."""
    from oracle import unrolled as UR
    V, U, g, X0 = unroll_case
    nu_a, nu_r, alpha, beta, K = 0.04, 0.12, 2.0, 0.5, 3
    C = _rng(6).standard_normal((g.N, 12)) if loss == "cotangent" else None
    Xs = UR.unrolled_forward(V, U, g, X0, nu_a, nu_r, alpha, beta, K)
    gX, gV = UR.unrolled_backward(V, U, g, Xs, nu_a, nu_r, alpha, beta, cotangent=C)
    _, rho0 = UR.unrolled_loss(V, U, g, X0, nu_a, nu_r, alpha, beta, K, C)

    def L(Xv, Vv):
        val, rhos = UR.unrolled_loss(Vv, U, g, Xv, nu_a, nu_r, alpha, beta, K, C)
        for a, b in zip(rhos, rho0):
            assert np.array_equal(a, b)           # no flip within the step
        return val

    rng = _rng(7)
    h = 1e-6
    flat = X0.ravel()
    for idx in rng.choice(flat.size, 12, replace=False):
        e = np.zeros_like(flat)
        e[idx] = h
        fd = (L((flat + e).reshape(X0.shape), V) - L((flat - e).reshape(X0.shape), V)) / (2 * h)
        assert abs(fd - gX.ravel()[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, gX.ravel()[idx])
    for i in rng.choice(V.shape[0], 5, replace=False):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[i, c] += h
            Vm[i, c] -= h
            fd = (L(X0, Vp) - L(X0, Vm)) / (2 * h)
            assert abs(fd - gV[i, c]) < 1e-6 * max(1.0, abs(fd)), (i, c, fd, gV[i, c])


# ------------------------------------------------- robust-norm variants ---

def test_variant_functions_closed_forms():
    """Sec. 4.2 variants: the squared l2 norm (weights 1) and the truncation
    at 3 nu_a (weight 1 strictly below, 0 from 3 nu_a on), against values
    worked by hand; Welsch's function unchanged."""
    nu = 0.5
    d2 = np.array([0.0, 0.25, 2.25, 4.0])      # d = 0, 0.5, 1.5 (= 3 nu), 2
    assert np.allclose(M.align_psi(d2, nu, "l2"), [0.0, 0.25, 2.25, 4.0])
    assert np.allclose(M.align_weight(d2, nu, "l2"), [1, 1, 1, 1])
    assert np.allclose(M.align_psi(d2, nu, "l2r"), [0.0, 0.25, 2.25, 2.25])
    assert np.array_equal(M.align_weight(d2, nu, "l2r"), [1.0, 1.0, 0.0, 0.0])
    assert np.allclose(M.reg_psi(d2, nu, "l2r"), d2) and np.allclose(M.reg_weight(d2, nu, "l2"), 1)
    assert np.allclose(M.align_psi(d2, nu, "welsch"), 1 - np.exp(-d2 / 0.5))
    # the truncated weight is the derivative of the truncated quadratic a.e.
    h = 1e-7
    for x2 in (0.3, 1.0, 3.0):
        fd = (M.align_psi(x2 + h, nu, "l2r") - M.align_psi(x2 - h, nu, "l2r")) / (2 * h)
        assert abs(fd - M.align_weight(x2, nu, "l2r")) < 1e-6


@pytest.mark.parametrize("robust", ["l2", "l2r"])
def test_variant_energy_gradient_matches_central_differences(small, robust):
    pair, g = small
    rng = _rng(23)
    X = _near_identity_X(g.N, rng, 0.02)
    V = pair.src.astype(np.float64)
    U = pair.tgt.astype(np.float64)
    nu_a, nu_r, alpha, beta = 0.05, 0.1, 3.0, 0.7
    t0 = M.energy_terms(V, U, g, X, nu_a, nu_r, robust=robust)
    gX, gv = M.energy_gradient(V, U, g, X, nu_a, nu_r, alpha, beta, robust=robust)

    def E(Xv):
        t = M.energy_terms(V, U, g, Xv, nu_a, nu_r, robust=robust)
        assert np.array_equal(t["rho"], t0["rho"])
        # no distance crosses the truncation within the step
        assert np.array_equal(t["d2"] < 9 * nu_a ** 2, t0["d2"] < 9 * nu_a ** 2)
        return M.total_energy(t, alpha, beta)

    h = 1e-6
    flat = X.ravel()
    for idx in rng.choice(flat.size, 10, replace=False):
        e = np.zeros_like(flat)
        e[idx] = h
        fd = (E((flat + e).reshape(X.shape)) - E((flat - e).reshape(X.shape))) / (2 * h)
        assert abs(fd - gX.ravel()[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, gX.ravel()[idx])


def test_l2_step_minimises_the_l2_energy_for_fixed_correspondences(small):
    """For the squared l2 norm the surrogate is the energy itself once the
    closest points are fixed: the MM step's solution G is the minimiser of
    E_l2(.; rho) (convex quadratic), so E_l2 rises in every direction from G
    and its central-difference gradient at G vanishes."""
    pair, g = small
    V = pair.src.astype(np.float64)
    U = pair.tgt.astype(np.float64)
    X = _near_identity_X(g.N, _rng(24), 0.01)
    nu_a, nu_r, alpha, beta = 0.05, 0.1, 3.0, 0.7
    t = M.energy_terms(V, U, g, X, nu_a, nu_r, robust="l2")
    K, B, _ = S.normal_equations(V, U, g, t, nu_a, nu_r, alpha, beta, robust="l2")
    Gs = S.solve_normal_equations(K, B)
    rho = t["rho"]

    def E(Xv):
        tt = M.energy_terms(V, U, g, Xv, nu_a, nu_r, rho=rho, robust="l2")
        # E_rot of the surrogate: |A - R(A^k)|^2 with R held at X
        A = M.A_of(Xv)
        return tt["E_align"] + alpha * tt["E_reg"] + beta * float(np.sum((A - t["R"]) ** 2))

    e0 = E(Gs)
    rng = _rng(25)
    for _ in range(5):
        D = rng.standard_normal(Gs.shape)
        assert E(Gs + 1e-3 * D) > e0
        fd = (E(Gs + 1e-6 * D) - E(Gs - 1e-6 * D)) / 2e-6
        assert abs(fd) < 1e-6 * max(1.0, e0)


def test_nu_fixed_variants_follow_the_annealing_schedule():
    """Welsch-fmax / fmin / fmed (Sec. 4.2) run one stage at the first
    stage's nu, at the last stage's, and at their means, the stages being
    those the annealed run actually visits."""
    pair = synth.tiny_pair(300, 330, seed=9, noise=0.002, outliers=0.03)
    base = dict(radius=0.35, nu_a=0.2, nu_r=0.4, nu_a_min=0.03, aa_m=0, max_iters_per_stage=3)
    ann = Registration(pair.src, pair.tgt, Params(**base))
    ann.solve()
    stages = sorted({(r.stage, r.nu_a, r.nu_r) for r in ann.records})
    first, last = stages[0][1:], stages[-1][1:]
    assert len(stages) == 4 and last[0] == 0.03          # 0.2 -> 0.1 -> 0.05 -> 0.03
    for which, want in [("max", first), ("min", last),
                        ("med", ((first[0] + last[0]) / 2, (first[1] + last[1]) / 2))]:
        r = Registration(pair.src, pair.tgt, Params(nu_fixed=which, **base))
        assert (r.nu_a, r.nu_r) == want
        r.solve()
        assert {rec.stage for rec in r.records} == {0}


def _solves_per_stage(reg):
    """Solves of each stage: the passes that reached the solve carry the
    displacement of their new iterate."""
    out = {}
    for r in reg.records:
        if not math.isnan(r.max_disp):
            out[r.stage] = out.get(r.stage, 0) + 1
    return [out.get(k, 0) for k in range(max(out) + 1)]


def test_stop_rules_displacement_or_energy():
    """Algorithm 2 ends a stage when the deformed source moves less than eps
    (or after I_max solves); with an energy tolerance, the rule the
    depth-scale workload is run to, a stage ends when two consecutive kept
    energies differ by less than that tolerance (or at I_max) and the
    displacement test is off."""
    pair = synth.tiny_pair(300, 330, seed=9, noise=0.002, outliers=0.03)
    base = dict(radius=0.35, nu_a=0.2, nu_r=0.4, nu_a_min=0.03, aa_m=0, max_iters_per_stage=3)
    # eps above any displacement: every stage ends after its first solve
    r = Registration(pair.src, pair.tgt, Params(eps=1e9, **base))
    r.solve()
    assert r.done and _solves_per_stage(r) == [1, 1, 1, 1]
    # an energy tolerance that never holds: I_max solves per stage, eps unused
    r = Registration(pair.src, pair.tgt, Params(eps=1e9, rel_energy_tol=1e-300, **base))
    r.solve()
    assert r.done and _solves_per_stage(r) == [3, 3, 3, 3]
    # a tolerance that always holds: the second kept pass of a stage ends it
    # without a solve
    r = Registration(pair.src, pair.tgt, Params(eps=1e9, rel_energy_tol=1.0, **base))
    r.solve()
    assert r.done and _solves_per_stage(r) == [1, 1, 1, 1]
    assert [math.isnan(x.max_disp) for x in r.records] == [False, True] * 4


def test_small_rigid_motion_recovered_by_algorithm_2():
    """Target = a small rigid motion of the source (no noise, no outliers;
    the largest displacement a fifth of the smallest distance between two
    source points, so every point's closest target is its own image):
    Algorithm 2 with its own closest points (no correspondence hook),
    Anderson mixing and annealing, run with a tight stopping threshold,
    reaches the motion (E = 0 at the exact map): every deformed point lies
    on its image to 1e-10 of the bounding-box diagonal, and the limit is a
    fixed point of the MM map."""
    pair = synth.tiny_pair(400, 400, seed=12)
    V = pair.src.astype(np.float64)
    d2 = np.sum((V[:, None, :] - V[None, :, :]) ** 2, axis=2)
    np.fill_diagonal(d2, np.inf)
    dmin = float(np.sqrt(d2.min()))
    ang = 0.1 * dmin / np.linalg.norm(V - V.mean(axis=0), axis=1).max()
    c, s = np.cos(ang), np.sin(ang)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    center = V.mean(axis=0)
    t = np.array([0.6, -0.4, 0.2]) * 0.1 * dmin
    U = (V - center) @ Rz.T + center + t
    assert np.linalg.norm(U - V, axis=1).max() <= 0.2 * dmin
    assert np.array_equal(M.closest_points(V, U)[0], np.arange(len(V)))
    diag = np.linalg.norm(np.maximum(V.max(0), U.max(0)) - np.minimum(V.min(0), U.min(0)))
    reg = Registration(V, U, Params(radius=0.35, aa_m=5, eps=1e-12 * diag))
    reg.solve()
    assert reg.done
    vh = M.deform(V, reg.graph.nidx, reg.graph.w, reg.graph.p, reg.X)
    assert np.abs(vh - U).max() < 1e-10 * diag
    # the limit is a fixed point of the MM map G (Sec. 3.3.4): one more
    # surrogate minimisation from it stays there
    G_ = reg.mm_map(reg.terms())
    assert np.abs(G_ - reg.X).max() < 1e-9 * np.abs(reg.X).max()


def test_revert_target_is_the_last_mm_result():
    """After the safeguard rejects an Anderson iterate (Algorithm 2), the
    next iterate is G^(k-1), the minimiser of the surrogate built at the last
    kept iterate X^(k-1): every directional derivative of that surrogate
    (summed term by term: Eqs. AlignQuadSurrogate and ERegSurrogate and the
    rotation surrogate; a quadratic in X, so central differences are exact
    up to rounding) vanishes at the new iterate, and not at X^(k-1) nor at
    the rejected iterate. The re-evaluated iterate is then kept, and by MM
    descent (Sec. 3.3.1: E(G) <= surrogate(G) <= surrogate(X^(k-1)) =
    E(X^(k-1))) its energy is at most the last kept energy."""
    pair = synth.tiny_pair(1200, 1320, seed=31, noise=0.002, outliers=0.05)
    reg = Registration(pair.src, pair.tgt, Params(radius=0.25, aa_m=5))
    evaluated = []
    rej = None
    for k in range(12):
        evaluated.append(reg.X.copy())
        rec = reg.step()
        if not rec.kept:
            rej = k
            break
    assert rej is not None and rej >= 2
    prev = reg.records[rej - 1]
    assert prev.kept and prev.stage == reg.records[rej].stage == reg.stage
    X_k1, X_rej, X_rev = evaluated[rej - 1], evaluated[rej], reg.X.copy()
    terms_k1 = reg.terms(X_k1)
    a, b = reg.weights()

    def ddir(X, D, h=1e-3):
        f = lambda Y: S.surrogate_value(reg.V, reg.U, reg.graph, terms_k1, Y, reg.nu_a, reg.nu_r, a, b)
        return (f(X + h * D) - f(X - h * D)) / (2 * h)

    rng = _rng(5)
    for _ in range(4):
        D = rng.standard_normal(X_rev.shape)
        g_rev, g_k1, g_rej = ddir(X_rev, D), ddir(X_k1, D), ddir(X_rej, D)
        assert abs(g_rev) < 1e-6 * abs(g_k1), (g_rev, g_k1)
        assert abs(g_rev) < 1e-6 * abs(g_rej), (g_rev, g_rej)
    nxt = reg.step()
    assert nxt.kept
    assert nxt.E <= prev.E * (1 + 1e-12), (nxt.E, prev.E)


def test_singular_system_keeps_free_translation():
    """Singular K (the paper is silent): an island of source points far from
    every target point at a small nu_a gets Welsch weights that underflow to
    0, so the island's component of the deformation graph has no alignment
    weight and K is singular along the component's common translation (an
    exact null vector: the indicator of the component's t rows). The
    oracle's minimiser then keeps the island's summed translation of X^k:
    it equals the minimum-norm update X^k + K^+ (B - K X^k) from an SVD
    least-squares solve, and every directional derivative of the surrogate
    (summed term by term) vanishes at it. The same pair with the island on
    the target has no free component."""
    pair = synth.island_pair(1200, 1300, seed=5)
    kw = dict(radius=0.3, aa_m=5, nu_a=0.03, nu_r=0.2, nu_a_min=0.03)
    reg = Registration(pair.src, pair.tgt, Params(**kw))
    g = reg.graph
    island_nodes = np.nonzero(g.p[:, 0] > 2.0)[0]
    assert len(island_nodes) >= 2
    X = _near_identity_X(g.N, _rng(3), scale=0.01)
    t = reg.terms(X)
    a, b = reg.weights()
    K, B, parts = S.normal_equations(reg.V, reg.U, g, t, reg.nu_a, reg.nu_r, a, b)
    free = S.free_components(g, parts["wa"])
    assert len(free) == 1 and np.array_equal(np.sort(free[0]), island_nodes)
    n = K.shape[0]
    null = np.zeros(n)
    null[4 * island_nodes + 3] = 1.0
    Kd = K.toarray()
    assert np.abs(Kd @ null).max() < 1e-12 * np.abs(Kd).max()
    G = S.solve_normal_equations(K, B, X, free)
    Xp = X.reshape(-1, 4, 3).reshape(n, 3)
    upd, *_ = np.linalg.lstsq(Kd, np.asarray(B) - Kd @ Xp, rcond=1e-10)
    G_min = (Xp + upd).reshape(-1, 4, 3).reshape(-1, 12)
    assert np.abs(G - G_min).max() < 1e-10 * np.abs(G_min).max()
    tG = G.reshape(-1, 4, 3)[island_nodes, 3, :].sum(axis=0)
    tX = X.reshape(-1, 4, 3)[island_nodes, 3, :].sum(axis=0)
    assert np.abs(tG - tX).max() < 1e-12
    f = lambda Y: S.surrogate_value(reg.V, reg.U, g, t, Y, reg.nu_a, reg.nu_r, a, b)
    rng = _rng(9)
    for _ in range(3):
        D = rng.standard_normal(G.shape)
        gG = (f(G + 1e-3 * D) - f(G - 1e-3 * D)) / 2e-3
        gX = (f(X + 1e-3 * D) - f(X - 1e-3 * D)) / 2e-3
        assert abs(gG) < 1e-6 * abs(gX), (gG, gX)
    # a pass of Algorithm 2 records the free component
    rec = reg.step()
    assert rec.kept and rec.n_singular == 1
    # the island on the target: no free component, the plain solve
    near = synth.island_pair(1200, 1300, seed=5, offset=0.0)
    reg2 = Registration(near.src, near.tgt, Params(**kw))
    t2 = reg2.terms()
    _, _, parts2 = S.normal_equations(reg2.V, reg2.U, reg2.graph, t2, reg2.nu_a, reg2.nu_r, a, b)
    assert S.free_components(reg2.graph, parts2["wa"]) == []


def test_lbfgs_two_loop_satisfies_the_secant_equation():
    """The two-loop recursion applies the L-BFGS inverse-Hessian estimate H,
    which satisfies the secant equation of its newest pair, H y = s, and is
    symmetric positive definite (g.d < 0 for d = -H g)."""
    from oracle.lbfgs import two_loop
    rng = _rng(21)
    n = 12
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    S = [rng.standard_normal(n) for _ in range(5)]
    Y = [A @ s for s in S]
    d = two_loop(Y[-1], S, Y)
    assert np.abs(d + S[-1]).max() < 1e-12 * np.abs(S[-1]).max()
    for _ in range(3):
        g = rng.standard_normal(n)
        assert float(np.dot(g, two_loop(g, S, Y))) < 0
    # no pairs: a unit-length steepest-descent step
    g = rng.standard_normal(n)
    assert np.allclose(two_loop(g, [], []), -g / np.linalg.norm(g), rtol=1e-15, atol=0)


def test_lbfgs_reaches_the_quadratic_minimiser():
    """With the squared-l2 robust function and beta = 0 the surrogate of the
    preliminary version's solver (closest points held) is the quadratic
    |F X - Q|^2 + alpha |H X - Y|^2, whose minimiser solves the normal
    equations K X = B (Sec. 3.3.2, all weights 1): the inner L-BFGS, run to a
    tight gradient tolerance, reaches that direct solution."""
    from oracle.lbfgs import LbfgsParams, LbfgsRegistration
    pair = synth.tiny_pair(500, 550, seed=41, noise=0.002)
    reg = LbfgsRegistration(pair.src, pair.tgt, Params(radius=0.35, robust="l2", beta=0.0, alpha=0.5),
                            LbfgsParams(max_inner=3000, g_tol=1e-11))
    X0 = _near_identity_X(reg.graph.N, _rng(2), scale=0.02)
    t = reg.terms(X0)
    a, b = reg.weights()
    K, B, _ = S.normal_equations(reg.V, reg.U, reg.graph, t, reg.nu_a, reg.nu_r, a, b, robust="l2")
    X_direct = S.solve_normal_equations(K, B)
    X_lb = reg.minimise_surrogate(X0, t["rho"])
    assert np.abs(X_lb - X_direct).max() < 1e-7 * np.abs(X_direct).max()


def test_lbfgs_outer_energies_decrease():
    """Each outer iteration minimises a majoriser of E that touches it at X^k
    (closest points held) with sufficient-decrease steps only, so the
    energies of the outer iterates never increase within a stage."""
    from oracle.lbfgs import LbfgsRegistration
    pair = synth.tiny_pair(600, 660, seed=43, noise=0.002, outliers=0.05)
    reg = LbfgsRegistration(pair.src, pair.tgt, Params(radius=0.3, max_iters_per_stage=6))
    recs = [reg.step() for _ in range(6)]
    assert all(r.stage == 0 for r in recs)
    E = [r.E for r in recs]
    assert all(E[k + 1] <= E[k] * (1 + 1e-12) for k in range(len(E) - 1)), E
    assert all(steps >= 1 for steps, _ in reg.inner)
