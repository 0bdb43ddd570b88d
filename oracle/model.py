"""Deformation model and objective (Sec. 3, Sec. 3.2) in FP64.

Transform layout: X has shape [N,12]; X[j].reshape(4,3) is the 4x3 block of
X_j in the paper's stacked X in R^{4N x 3}: rows 0..2 hold A_j^T and row 3
holds t_j^T, so that [ (v - p_j)^T, 1 ] @ block = (A_j (v - p_j) + t_j)^T.
"""
from __future__ import annotations

import numpy as np


def blocks(X: np.ndarray) -> np.ndarray:
    return np.asarray(X, dtype=np.float64).reshape(-1, 4, 3)


def A_of(X: np.ndarray) -> np.ndarray:
    """A_j for every node, shape [N,3,3]."""
    return np.transpose(blocks(X)[:, :3, :], (0, 2, 1))


def t_of(X: np.ndarray) -> np.ndarray:
    return blocks(X)[:, 3, :]


def identity_X(N: int) -> np.ndarray:
    X = np.zeros((N, 4, 3))
    X[:, 0, 0] = X[:, 1, 1] = X[:, 2, 2] = 1.0
    return X.reshape(N, 12)


def deform(V: np.ndarray, nidx: np.ndarray, w: np.ndarray, p: np.ndarray,
           X: np.ndarray) -> np.ndarray:
    """Eq. (deformed_position): v_hat_i = sum_j w_ij (A_j (v_i - p_j) + p_j + t_j)."""
    V = np.asarray(V, dtype=np.float64)
    A = A_of(X)
    t = t_of(X)
    out = np.zeros_like(V)
    for s in range(nidx.shape[1]):
        j = nidx[:, s]
        m = j >= 0
        jj = j[m]
        d = V[m] - p[jj]
        term = np.einsum("nab,nb->na", A[jj], d) + p[jj] + t[jj]
        out[m] += w[m, s][:, None] * term
    return out


def closest_points(Q: np.ndarray, U: np.ndarray, chunk: int = 256):
    """rho(i) = argmin_u |u - q_i| over the target points (Sec. 3.2), by
    brute force; equal distances resolve to the lowest target index.
    Returns (rho [n] int64, d2 [n] float64)."""
    Q = np.asarray(Q, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    n = Q.shape[0]
    rho = np.empty(n, dtype=np.int64)
    d2 = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        q = Q[s:s + chunk]
        dx = q[:, None, 0] - U[None, :, 0]
        dy = q[:, None, 1] - U[None, :, 1]
        dz = q[:, None, 2] - U[None, :, 2]
        dd = dx * dx + dy * dy + dz * dz
        a = np.argmin(dd, axis=1)          # first (lowest) index on ties
        rho[s:s + chunk] = a
        d2[s:s + chunk] = dd[np.arange(q.shape[0]), a]
    return rho, d2


def welsch(x2: np.ndarray, nu: float) -> np.ndarray:
    """Eq. (Welsch_func) applied to a squared argument: psi_nu(x) with x^2 given."""
    return 1.0 - np.exp(-np.asarray(x2, dtype=np.float64) / (2.0 * nu * nu))


# Robust functions of the alignment and regularisation terms. The paper's
# method uses Welsch's function; Sec. 4.2 compares it with two variants that
# replace it by the squared l2 norm, with all alignment weights 1 ("l2") or
# with an alignment weight 0 once a distance reaches 3 nu_a ("l2r"). The
# l2r weights are the MM weights of the truncated quadratic min(d^2, 9 nu_a^2),
# which is the energy read here for that variant; the regularisation term of
# both variants is sum |D_ij|^2.
ROBUST = ("welsch", "l2", "l2r")


def align_psi(d2: np.ndarray, nu_a: float, robust: str = "welsch") -> np.ndarray:
    """Per-point alignment energy as a function of the squared distance."""
    d2 = np.asarray(d2, dtype=np.float64)
    if robust == "welsch":
        return welsch(d2, nu_a)
    if robust == "l2":
        return d2.copy()
    if robust == "l2r":
        return np.minimum(d2, 9.0 * nu_a * nu_a)
    raise ValueError(robust)


def align_weight(d2: np.ndarray, nu_a: float, robust: str = "welsch") -> np.ndarray:
    """Derivative of align_psi w.r.t. the squared distance: the weight of the
    quadratic surrogate (Eq. AlignQuadSurrogate for Welsch's function)."""
    d2 = np.asarray(d2, dtype=np.float64)
    if robust == "welsch":
        return np.exp(-d2 / (2.0 * nu_a * nu_a)) / (2.0 * nu_a * nu_a)
    if robust == "l2":
        return np.ones_like(d2)
    if robust == "l2r":
        return (d2 < 9.0 * nu_a * nu_a).astype(np.float64)
    raise ValueError(robust)


def reg_psi(Dn2: np.ndarray, nu_r: float, robust: str = "welsch") -> np.ndarray:
    Dn2 = np.asarray(Dn2, dtype=np.float64)
    return welsch(Dn2, nu_r) if robust == "welsch" else Dn2.copy()


def reg_weight(Dn2: np.ndarray, nu_r: float, robust: str = "welsch") -> np.ndarray:
    Dn2 = np.asarray(Dn2, dtype=np.float64)
    if robust == "welsch":
        return np.exp(-Dn2 / (2.0 * nu_r * nu_r)) / (2.0 * nu_r * nu_r)
    return np.ones_like(Dn2)


def welsch_surrogate(x: np.ndarray, y: np.ndarray, nu: float) -> np.ndarray:
    """Eq. (WelschSurrogateFunc): psi(y) + (1 - psi(y)) / (2 nu^2) (x^2 - y^2)."""
    py = welsch(np.asarray(y) ** 2, nu)
    return py + (1.0 - py) / (2.0 * nu * nu) * (np.asarray(x) ** 2 - np.asarray(y) ** 2)


def reg_residuals(p: np.ndarray, dpair: np.ndarray, r: np.ndarray,
                  X: np.ndarray) -> np.ndarray:
    """Eq. (reg_diff): D_ij = r_ij (A_j (p_i - p_j) + p_j + t_j - (p_i + t_i))
    for every directed pair (i, j); shape [2|E_G|, 3]."""
    if len(dpair) == 0:
        return np.zeros((0, 3))
    A = A_of(X)
    t = t_of(X)
    i, j = dpair[:, 0], dpair[:, 1]
    d = p[i] - p[j]
    val = np.einsum("nab,nb->na", A[j], d) + p[j] + t[j] - (p[i] + t[i])
    return r[:, None] * val


def proj_rotation(A: np.ndarray) -> np.ndarray:
    """proj_R(A) = argmin over rotations R of |R - A|_F (Sec. 3.2), from the
    SVD A = U S V^T: R = U diag(1, 1, det(U V^T)) V^T. Batched over [...,3,3]."""
    U, _, Vt = np.linalg.svd(A)
    det = np.linalg.det(U @ Vt)
    D = np.zeros(A.shape[:-2] + (3,))
    D[..., 0] = 1.0
    D[..., 1] = 1.0
    D[..., 2] = det
    return U @ (D[..., :, None] * Vt)


def energy_terms(V, U, graph, X, nu_a, nu_r, rho=None, robust="welsch"):
    """Eq. (objective_func) terms at X. Returns dict with E_align, E_reg,
    E_rot, the closest points (rho, d2), v_hat, D and the rotations R.
    ``rho`` replaces the closest-point search (used only by tests that
    supply known correspondences); ``robust`` selects the variant of Sec.
    4.2 (see ROBUST)."""
    vh = deform(V, graph.nidx, graph.w, graph.p, X)
    U64 = np.asarray(U, dtype=np.float64)
    if rho is None:
        rho, d2 = closest_points(vh, U64)
    else:
        diff = vh - U64[rho]
        d2 = diff[:, 0] ** 2 + diff[:, 1] ** 2 + diff[:, 2] ** 2
    e_align = float(np.sum(align_psi(d2, nu_a, robust)))
    D = reg_residuals(graph.p, graph.dpair, graph.r, X)
    Dn2 = np.sum(D * D, axis=1)
    e_reg = float(np.sum(reg_psi(Dn2, nu_r, robust)))
    A = A_of(X)
    Rm = proj_rotation(A) if len(A) else A
    e_rot = float(np.sum((A - Rm) ** 2))
    return dict(E_align=e_align, E_reg=e_reg, E_rot=e_rot, rho=rho, d2=d2,
                vhat=vh, D=D, R=Rm)


def total_energy(terms: dict, alpha: float, beta: float) -> float:
    return terms["E_align"] + alpha * terms["E_reg"] + beta * terms["E_rot"]


def energy_gradient(V, U, graph, X, nu_a, nu_r, alpha, beta, rho=None, robust="welsch"):
    """Gradient of E (Eq. objective_func) with the closest points held at
    their values at X (rho is piecewise constant in X), the node positions
    p_j and the weights w_ij held constant.

    d psi_nu(x) / d(x^2) = exp(-x^2 / 2nu^2) / (2nu^2) = w (the surrogate's
    weight), so with r_i = v_hat_i - u_rho(i):
      dE/dX_j  = sum_i 2 w^a_i w_ij [v_i - p_j; 1] r_i^T
               + alpha sum_(i,j) 2 w^r_ij (h_j D_ij^T at X_j, h_i D_ij^T at X_i)
               + beta 2 [(A_j - proj_R(A_j))^T; 0]
      dE/dv_i  = 2 w^a_i (sum_j w_ij A_j)^T r_i
    (the rotation term's derivative is 2 (A - proj_R(A)) because proj_R(A)
    minimises the distance to the rotation group).
    Returns (grad_X [N,12], grad_v [P,3])."""
    V = np.asarray(V, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    t = energy_terms(V, U, graph, X, nu_a, nu_r, rho=rho, robust=robust)
    r = t["vhat"] - U[t["rho"]]
    wa = align_weight(t["d2"], nu_a, robust)
    N = graph.N
    gX = np.zeros((N, 4, 3))
    gv = np.zeros_like(V)
    A = A_of(X)
    for s in range(graph.nidx.shape[1]):
        j = graph.nidx[:, s]
        m = np.nonzero(j >= 0)[0]
        jj = j[m]
        wij = graph.w[m, s]
        a = np.concatenate([V[m] - graph.p[jj], np.ones((len(m), 1))], axis=1)   # [n,4]
        contrib = 2.0 * (wa[m] * wij)[:, None, None] * a[:, :, None] * r[m][:, None, :]
        np.add.at(gX, jj, contrib)
        gv[m] += 2.0 * wa[m, None] * wij[:, None] * np.einsum("nab,na->nb", A[jj], r[m])
    if len(graph.dpair):
        D = t["D"]
        wr = reg_weight(np.sum(D * D, axis=1), nu_r, robust)
        i, j = graph.dpair[:, 0], graph.dpair[:, 1]
        rr = graph.r
        hj = np.concatenate([rr[:, None] * (graph.p[i] - graph.p[j]), rr[:, None]], axis=1)
        hi = np.zeros((len(i), 4))
        hi[:, 3] = -rr
        cj = 2.0 * alpha * wr[:, None, None] * hj[:, :, None] * D[:, None, :]
        ci = 2.0 * alpha * wr[:, None, None] * hi[:, :, None] * D[:, None, :]
        np.add.at(gX, j, cj)
        np.add.at(gX, i, ci)
    gX[:, :3, :] += 2.0 * beta * np.transpose(A - t["R"], (0, 2, 1))
    return gX.reshape(N, 12), gv
