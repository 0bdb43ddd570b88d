"""Anderson acceleration of the MM fixed-point map (Sec. 3.3.4, Eq. AA_solution).

G is the MM map, F(X) = G(X) - X. With the last m_k differences
dF_j = F^(k-j+1) - F^(k-j) and dG_j = G^(k-j+1) - G^(k-j):

  theta = argmin |F^(k) - sum_j theta_j dF_j|^2,
  X_AA  = G^(k) - sum_j theta_j dG_j.

Readings (the paper is silent on them):
* m_k is the number of stored differences, min(#solves in the stage - 1, m);
  the first solve of a stage is a plain MM step.
* The least-squares problem carries a ridge lambda = 1e-10 trace(dF^T dF)/m_k,
  solved here as the augmented least-squares problem [dF; sqrt(lambda) I].
* If theta is not finite or |theta| > 1e4, the pass uses the plain MM step.
* The history is cleared at every stage start (nu changes the map G).
"""
from __future__ import annotations

import numpy as np

RIDGE = 1e-10
THETA_MAX = 1e4


class Anderson:
    def __init__(self, m: int):
        self.m = int(m)
        self.reset()

    def reset(self) -> None:
        self.dF: list[np.ndarray] = []
        self.dG: list[np.ndarray] = []
        self.F_prev = None
        self.G_prev = None
        self.last_theta = None

    def mix(self, G: np.ndarray, X: np.ndarray) -> np.ndarray:
        """Returns X^(k+1) from G^(k) = G(X^(k)) and X^(k) (any shape)."""
        shape = G.shape
        g = np.asarray(G, dtype=np.float64).ravel()
        f = g - np.asarray(X, dtype=np.float64).ravel()
        if self.F_prev is not None and self.m > 0:
            self.dF.append(f - self.F_prev)
            self.dG.append(g - self.G_prev)
            if len(self.dF) > self.m:
                self.dF.pop(0)
                self.dG.pop(0)
        self.F_prev, self.G_prev = f, g
        self.last_theta = None
        mk = len(self.dF)
        if mk == 0:
            return g.reshape(shape).copy()
        M = np.stack(self.dF, axis=1)                     # [n, mk]
        lam = RIDGE * float(np.sum(M * M)) / mk
        Aug = np.concatenate([M, np.sqrt(lam) * np.eye(mk)], axis=0)
        rhs = np.concatenate([f, np.zeros(mk)])
        theta, *_ = np.linalg.lstsq(Aug, rhs, rcond=None)
        if not np.all(np.isfinite(theta)) or np.linalg.norm(theta) > THETA_MAX:
            return g.reshape(shape).copy()
        self.last_theta = theta
        out = g - np.stack(self.dG, axis=1) @ theta
        return out.reshape(shape)
