"""Unrolled MM steps and their reverse-mode derivative, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): the library's
unrolled backward is checked against this module, and this module is pinned
by central finite differences of its own forward map.

The map. K plain MM steps (Sec. 3.3.1-3.3.2) at fixed nu_a, nu_r, alpha,
beta, with no Anderson mixing and no safeguard (the accept/reject branch is
not differentiable):
    X^(k+1) = Phi(X^(k), V) = K(X^(k), V)^-1 B(X^(k), V)      (Eq. surr_solution)
with K, B the normal equations of the quadratic surrogate built at X^(k).
The paper does not differentiate its solver; the readings used here are:
  * the closest points rho(i) are piecewise constant in X and V: no
    gradient flows through the argmin, only through v_hat_i and d_i;
  * the node positions p_j, skinning weights w_ij, r_ij and the graph are
    constants, even though the nodes are source points: the source gradient
    flows through v_i in F (hence K, B) and in v_hat_i only;
  * the solve is exact (implicit differentiation): with lambda = K^-1 g_bar,
    dL/dB = lambda and dL/dK = -lambda X'^T, X' = X^(k+1);
  * the loss is L(X^(K)) = <C, X^(K)> for a given cotangent C, or E(X^(K))
    (Eq. objective_func, closest points held at X^(K)).

The dependence of K and B on X^(k) is through the weights W_a (d_i), W_r
(D_ij) and the rotation targets Z (proj_R(A_j)); F and Q carry the
dependence on V (F's entries w_ij (v_i - p_j)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import model, surrogate


# ------------------------------------------------------------ proj_R vjp ---

def proj_rotation_vjp(A: np.ndarray, Rbar: np.ndarray) -> np.ndarray:
    """Vector-Jacobian product of proj_R (Sec. 3.2) at A: returns dL/dA given
    dL/dR, batched over [..., 3, 3].

    With A = U S V^T (SVD), d = (1, 1, det(U V^T)) and R = U diag(d) V^T,
    write A = R S' with S' = V diag(d s) V^T symmetric. Differentiating
    A = R S' with R^T dR = Omega skew gives
        Omega S' + S' Omega = R^T dA - dA^T R,
    which in the bases U, V reads, with dU~ = U^T dA V and
    Omega~ = V^T Omega V:
        Omega~_kl (d_k s_k + d_l s_l) = d_k dU~_kl - d_l dU~_lk,
    and dR = U diag(d) Omega~ V^T. The adjoint of this linear map is taken
    entry by entry."""
    A = np.asarray(A, dtype=np.float64)
    Rbar = np.asarray(Rbar, dtype=np.float64)
    U, s, Vt = np.linalg.svd(A)
    V = np.swapaxes(Vt, -1, -2)
    det = np.linalg.det(U @ Vt)
    d = np.ones(A.shape[:-2] + (3,))
    d[..., 2] = det
    # G^ = diag(d) U^T Rbar V : dL = sum_kl G^_kl Omega~_kl
    Gh = d[..., :, None] * (np.swapaxes(U, -1, -2) @ Rbar @ V)
    ds = d * s
    denom = ds[..., :, None] + ds[..., None, :]
    # dL/d(dU~_kl) = d_k (G^_kl - G^_lk) / (d_k s_k + d_l s_l), zero for k = l
    Ubar = d[..., :, None] * (Gh - np.swapaxes(Gh, -1, -2))
    off = ~np.eye(3, dtype=bool)
    Ubar = np.where(off, Ubar / np.where(off, denom, 1.0), 0.0)
    return U @ Ubar @ Vt


# ------------------------------------------------------------- forward -----

def mm_step(V, U, graph, X, nu_a, nu_r, alpha, beta, robust="welsch"):
    """One plain MM step: the minimiser of the surrogate built at X."""
    t = model.energy_terms(V, U, graph, X, nu_a, nu_r, robust=robust)
    K, B, parts = surrogate.normal_equations(V, U, graph, t, nu_a, nu_r, alpha, beta, robust=robust)
    Xn = np.asarray(scipy.linalg.cho_solve(scipy.linalg.cho_factor(K.toarray(), lower=True), B))
    return Xn.reshape(graph.N, 12), t, K, parts


def unrolled_forward(V, U, graph, X0, nu_a, nu_r, alpha, beta, n_steps, robust="welsch"):
    """X^(0..K) of K plain MM steps from X0 (the checkpoints of the backward)."""
    Xs = [np.asarray(X0, dtype=np.float64).reshape(graph.N, 12).copy()]
    for _ in range(n_steps):
        Xn, _, _, _ = mm_step(V, U, graph, Xs[-1], nu_a, nu_r, alpha, beta, robust)
        Xs.append(Xn)
    return Xs


# ------------------------------------------------------------ backward -----

def _rows4(M):
    """[4N, 3] <-> [N, 12] layout helpers."""
    return np.asarray(M).reshape(-1, 3)


def weight_slope(w, nu, robust):
    """d w / d(x^2) of a surrogate weight as a function of the squared
    residual: -w / (2 nu^2) for Welsch's function; 0 for the squared norm
    (and almost everywhere for its truncation)."""
    return -w / (2.0 * nu * nu) if robust == "welsch" else np.zeros_like(w)


def step_vjp(V, U, graph, Xk, Xn, gbar, nu_a, nu_r, alpha, beta, robust="welsch"):
    """Reverse-mode derivative of one MM step X' = Phi(X^k, V) at X^k with
    X' = Xn given: returns (dL/dX^k [N,12], dL/dV [P,3]) for dL/dX' = gbar.
    Every product below is a matrix-calculus identity on the matrices of
    Sec. 3.3.2 (F, Q, W_a, H, Y, W_r, J, Z)."""
    V = np.asarray(V, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    N = graph.N
    t = model.energy_terms(V, U, graph, Xk, nu_a, nu_r, robust=robust)
    K, B, parts = surrogate.normal_equations(V, U, graph, t, nu_a, nu_r, alpha, beta, robust=robust)
    F, Q, wa, H, Y, wr, Z = (parts[k] for k in ("F", "Q", "wa", "H", "Y", "wr", "Z"))
    Xp = _rows4(Xn)                                    # X' in [4N, 3]
    lam = scipy.linalg.cho_solve(scipy.linalg.cho_factor(K.toarray(), lower=True),
                                 _rows4(gbar))         # K lambda = gbar (K symmetric)
    # dL/dK = -lambda X'^T and dL/dB = lambda. With K = F^T W_a F + ..., the
    # derivative w.r.t. the diagonal weight w^a_i is
    #   f_i^T (dL/dK) f_i + f_i^T (dL/dB) Q_i = (F lambda)_i . (Q_i - (F X')_i)
    Fl = F @ lam
    FX = F @ Xp
    wa_bar = np.sum(Fl * (Q - FX), axis=1)
    if H.shape[0]:
        Hl = H @ lam
        HX = H @ Xp
        wr_bar = alpha * np.sum(Hl * (Y - HX), axis=1)
    # B's rotation part is beta J^T J Z: dL/dZ = beta J^T J lambda (rows 0..2)
    Jd = np.tile(np.array([1.0, 1.0, 1.0, 0.0]), N)
    Z_bar = beta * Jd[:, None] * lam

    # dL/dF at F's non-zeros: dL/dF = W_a F (dL/dK + dL/dK^T) + W_a Q (dL/dB)^T
    #                               = W_a (-(F lambda) X'^T - (F X') lambda^T + Q lambda^T)
    # and F_(i, 4j+c) = w_ij (v_i - p_j)_c for c < 3
    gV = np.zeros_like(V)
    lam_b = lam.reshape(N, 4, 3)
    Xp_b = Xp.reshape(N, 4, 3)
    for s in range(graph.nidx.shape[1]):
        j = graph.nidx[:, s]
        m = np.nonzero(j >= 0)[0]
        jj = j[m]
        # row i, block j of dL/dF: 4-vector
        Fbar_blk = wa[m, None] * (-np.einsum("nac,nc->na", Xp_b[jj], Fl[m])
                                  - np.einsum("nac,nc->na", lam_b[jj], FX[m])
                                  + np.einsum("nac,nc->na", lam_b[jj], Q[m]))
        gV[m] += graph.w[m, s][:, None] * Fbar_blk[:, :3]

    # chain through w^a_i(d_i^2) (slope: weight_slope), d_i^2 = |v_hat_i - u_i|^2
    d2_bar = wa_bar * weight_slope(wa, nu_a, robust)
    vh_bar = 2.0 * d2_bar[:, None] * (t["vhat"] - U[t["rho"]])
    # v_hat = F X^k + sum_j w_ij p_j: dL/dX^k += F^T vh_bar
    gX = np.asarray(F.T @ vh_bar)
    # d v_hat_i / d v_i = sum_j w_ij A_j
    A = model.A_of(Xk)
    for s in range(graph.nidx.shape[1]):
        j = graph.nidx[:, s]
        m = np.nonzero(j >= 0)[0]
        gV[m] += graph.w[m, s][:, None] * np.einsum("nab,na->nb", A[j[m]], vh_bar[m])
    # chain through w^r(|D|^2) (slope: weight_slope), D = H X^k - Y
    if H.shape[0]:
        Dk = t["D"]
        Dn2_bar = wr_bar * weight_slope(wr, nu_r, robust)
        gX += np.asarray(H.T @ (2.0 * Dn2_bar[:, None] * Dk))
    # chain through Z_j rows 0..2 = proj_R(A_j)^T
    Rbar = np.transpose(Z_bar.reshape(N, 4, 3)[:, :3, :], (0, 2, 1))
    Abar = proj_rotation_vjp(A, Rbar)
    gXb = gX.reshape(N, 4, 3)
    gXb[:, :3, :] += np.transpose(Abar, (0, 2, 1))
    return gXb.reshape(N, 12), gV


def unrolled_backward(V, U, graph, Xs, nu_a, nu_r, alpha, beta, cotangent=None, robust="welsch"):
    """Gradient of L(X^(K)) w.r.t. X^(0) and V through the K steps whose
    iterates are Xs = [X^(0), ..., X^(K)]. cotangent: dL/dX^(K) [N,12], or
    None for L = E(X^(K)) (Eq. objective_func with the closest points held
    at X^(K); its direct dependence on V is included).
    Returns (dL/dX^(0) [N,12], dL/dV [P,3])."""
    V = np.asarray(V, dtype=np.float64)
    if cotangent is None:
        g, gV = model.energy_gradient(V, U, graph, Xs[-1], nu_a, nu_r, alpha, beta, robust=robust)
    else:
        g = np.asarray(cotangent, dtype=np.float64).reshape(graph.N, 12).copy()
        gV = np.zeros_like(V)
    for k in range(len(Xs) - 2, -1, -1):
        g, gv_k = step_vjp(V, U, graph, Xs[k], Xs[k + 1], g, nu_a, nu_r, alpha, beta, robust)
        gV += gv_k
    return g, gV


def unrolled_loss(V, U, graph, X0, nu_a, nu_r, alpha, beta, n_steps, cotangent=None, robust="welsch"):
    """L(X^(K)) of the unrolled map (for finite-difference checks); also the
    closest points of every step (to detect flips)."""
    Xs = [np.asarray(X0, dtype=np.float64).reshape(graph.N, 12)]
    rhos = []
    for _ in range(n_steps):
        Xn, t, _, _ = mm_step(V, U, graph, Xs[-1], nu_a, nu_r, alpha, beta, robust)
        rhos.append(t["rho"])
        Xs.append(Xn)
    tK = model.energy_terms(V, U, graph, Xs[-1], nu_a, nu_r, robust=robust)
    rhos.append(tK["rho"])
    if cotangent is None:
        L = model.total_energy(tK, alpha, beta)
    else:
        L = float(np.sum(np.asarray(cotangent).reshape(graph.N, 12) * Xs[-1]))
    return L, rhos
