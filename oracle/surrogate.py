"""Quadratic surrogate and its minimiser (Sec. 3.3.1 and 3.3.2) in FP64.

The matrices are built exactly as the paper writes them:

  E_align(X|X^k) = |W_a (F X - Q)|_F^2,   F_ij = w_ij [v_i^T - p_j^T, 1],
                   Q_i = u_rho(i)^k - sum_j w_ij p_j,
                   W_a = diag(sqrt(w^a_i)), w^a_i = exp(-d_i^2 / 2nu_a^2) / (2 nu_a^2)
  E_reg(X|X^k)   = |W_r (H X - Y)|_F^2,   H row (i,j): r_ij [(p_i - p_j)^T, 1] at
                   X_j and [0, 0, 0, -r_ij] at X_i;  Y row: r_ij (p_i - p_j)^T
  E_rot(X|X^k)   = |J X - Z|_F^2,         J = diag(1,1,1,0, ...),
                   Z block j = [proj_R(A_j^k)^T; 0]
  K = F^T W_a^2 F + alpha H^T W_r^2 H + beta J^T J,
  B = F^T W_a^2 Q + alpha H^T W_r^2 Y + beta J^T J Z,   K X = B  (Eq. surr_solution).

The rotation surrogate is read with its square (|A - proj_R(A^k)|_F^2), the
form the matrix expression |J X - Z|_F^2 states.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.csgraph  # noqa: F401  (sp.csgraph)
import scipy.sparse.linalg as spla


def build_F(V, graph) -> sp.csr_matrix:
    V = np.asarray(V, dtype=np.float64)
    P, K = graph.nidx.shape
    rows, cols, vals = [], [], []
    for s in range(K):
        j = graph.nidx[:, s]
        m = np.nonzero(j >= 0)[0]
        jj = j[m]
        wv = graph.w[m, s]
        d = V[m] - graph.p[jj]
        for c in range(3):
            rows.append(m)
            cols.append(4 * jj + c)
            vals.append(wv * d[:, c])
        rows.append(m)
        cols.append(4 * jj + 3)
        vals.append(wv)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                          np.concatenate(cols))), shape=(P, 4 * graph.N))


def build_Q(U_rho: np.ndarray, graph) -> np.ndarray:
    Q = np.asarray(U_rho, dtype=np.float64).copy()
    for s in range(graph.nidx.shape[1]):
        j = graph.nidx[:, s]
        m = j >= 0
        Q[m] -= graph.w[m, s][:, None] * graph.p[j[m]]
    return Q


def build_H(graph):
    """Returns (H [2|E|, 4N] sparse, Y [2|E|, 3])."""
    E2 = len(graph.dpair)
    if E2 == 0:
        return sp.csr_matrix((0, 4 * graph.N)), np.zeros((0, 3))
    i, j = graph.dpair[:, 0], graph.dpair[:, 1]
    d = graph.p[i] - graph.p[j]
    r = graph.r
    e = np.arange(E2)
    rows = [e, e, e, e, e]
    cols = [4 * j + 0, 4 * j + 1, 4 * j + 2, 4 * j + 3, 4 * i + 3]
    vals = [r * d[:, 0], r * d[:, 1], r * d[:, 2], r, -r]
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                      np.concatenate(cols))), shape=(E2, 4 * graph.N))
    Y = r[:, None] * d
    return H, Y


def build_J(N: int) -> sp.csr_matrix:
    diag = np.tile(np.array([1.0, 1.0, 1.0, 0.0]), N)
    return sp.diags(diag, format="csr")


def build_Z(Rm: np.ndarray) -> np.ndarray:
    N = Rm.shape[0]
    Z = np.zeros((N, 4, 3))
    Z[:, :3, :] = np.transpose(Rm, (0, 2, 1))
    return Z.reshape(4 * N, 3)


def normal_equations(V, U, graph, terms, nu_a, nu_r, alpha, beta, robust="welsch"):
    """K and B of Eq. (surr_solution) at the state whose energy terms are
    ``terms`` (closest points, D_ij and rotations evaluated at X^k); the
    weights are those of the robust function ``robust`` (model.ROBUST)."""
    from . import model
    U = np.asarray(U, dtype=np.float64)
    F = build_F(V, graph)
    Q = build_Q(U[terms["rho"]], graph)
    wa = model.align_weight(terms["d2"], nu_a, robust)
    H, Y = build_H(graph)
    wr = model.reg_weight(np.sum(terms["D"] ** 2, axis=1), nu_r, robust)
    J = build_J(graph.N)
    Z = build_Z(terms["R"])
    Wa2 = sp.diags(wa)
    Wr2 = sp.diags(wr)
    K = (F.T @ Wa2 @ F + alpha * (H.T @ Wr2 @ H) + beta * (J.T @ J)).tocsr()
    B = F.T @ (wa[:, None] * Q) + alpha * (H.T @ (wr[:, None] * Y)) + beta * (J.T @ (J @ Z))
    return K, np.asarray(B), dict(F=F, Q=Q, wa=wa, H=H, Y=Y, wr=wr, J=J, Z=Z)


def free_components(graph, wa) -> list[np.ndarray]:
    """Connected components of the deformation graph on which the alignment
    term has no weight: every node j of the component has
    a_j = sum_i w^a_i w_ij^2 = 0 exactly (the (t_j, t_j) entry of
    F^T W_a F), which happens when the Welsch weights of all points the
    component influences underflow to 0. The surrogate then does not depend
    on the component's common translation (H annihilates it: D_ij does not
    change when t_i and t_j move together), so K is singular. Returns the
    node index arrays of those components (empty if K is regular in this
    respect)."""
    N = graph.N
    a = np.zeros(N)
    for s in range(graph.nidx.shape[1]):
        j = graph.nidx[:, s]
        m = j >= 0
        np.add.at(a, j[m], np.asarray(wa, dtype=np.float64)[m] * graph.w[m, s] ** 2)
    if len(graph.edges):
        e = np.asarray(graph.edges)
        adj = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(N, N))
    else:
        adj = sp.coo_matrix((N, N))
    n_comp, label = sp.csgraph.connected_components(adj, directed=False)
    out = []
    for c in range(n_comp):
        nodes = np.nonzero(label == c)[0]
        if np.all(a[nodes] == 0.0):
            out.append(nodes)
    return out


def solve_normal_equations(K, B, X_prev=None, free=()) -> np.ndarray:
    """Direct solve of K X = B (dense Cholesky for small systems, sparse LU
    otherwise). Returns X in [N,12] layout.

    ``free`` lists components whose common translation K does not determine
    (free_components); for each, the solution keeps the component's summed
    translation of ``X_prev`` ([N,12], the iterate the surrogate was built
    at): the constraint sum_{j in C} t_j = sum_{j in C} t_j(X_prev) is
    added with a Lagrange multiplier, per column of X, and the augmented
    system [[K, N], [N^T, 0]] is solved directly."""
    n = K.shape[0]
    if len(free) == 0:
        if n <= 4000:
            c = scipy.linalg.cho_factor(K.toarray(), lower=True)
            X = scipy.linalg.cho_solve(c, B)
        else:
            X = spla.spsolve(K.tocsc(), B)
        return np.asarray(X).reshape(n // 4, 4, 3).reshape(n // 4, 12)
    nc = len(free)
    rows = np.concatenate([4 * np.asarray(C) + 3 for C in free])
    cols = np.concatenate([np.full(len(C), k) for k, C in enumerate(free)])
    Nm = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, nc))
    Xp = np.asarray(X_prev, dtype=np.float64).reshape(n // 4, 4, 3).reshape(n, 3)
    A = sp.bmat([[K, Nm], [Nm.T, None]], format="csc")
    rhs = np.concatenate([np.asarray(B), Nm.T @ Xp])
    if n <= 4000:
        sol = scipy.linalg.solve(A.toarray(), rhs)
    else:
        sol = spla.spsolve(A, rhs)
    X = np.asarray(sol)[:n]
    return X.reshape(n // 4, 4, 3).reshape(n // 4, 12)


def surrogate_value(V, U, graph, terms_k, X, nu_a, nu_r, alpha, beta):
    """The surrogate E(X | X^k) of Eq. (surrogate_func) summed term by term
    (Eqs. ERegSurrogate, AlignQuadSurrogate and the rotation surrogate),
    with the constants the paper drops restored so that it equals E at X^k."""
    from . import model
    U = np.asarray(U, dtype=np.float64)
    vh = model.deform(V, graph.nidx, graph.w, graph.p, X)
    u = U[terms_k["rho"]]
    dk = np.sqrt(terms_k["d2"])
    dx = np.sqrt(np.sum((vh - u) ** 2, axis=1))
    s_align = np.sum(model.welsch_surrogate(dx, dk, nu_a))
    D = model.reg_residuals(graph.p, graph.dpair, graph.r, X)
    Dk = terms_k["D"]
    s_reg = np.sum(model.welsch_surrogate(np.sqrt(np.sum(D * D, axis=1)),
                                          np.sqrt(np.sum(Dk * Dk, axis=1)), nu_r))
    A = model.A_of(X)
    s_rot = np.sum((A - terms_k["R"]) ** 2)
    return float(s_align + alpha * s_reg + beta * s_rot)
