"""The preliminary version's solver, as a comparison solver on the same
energy (Sec. 3.3.4, the Remark on the preliminary version; Sec. 4.3), in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper describes it as an outer loop that builds a non-quadratic
surrogate of E and minimises it with an inner L-BFGS solver whose line
search has a sufficient-decrease threshold and whose termination has two
parameters. Readings used here (the paper gives no further detail):

* Surrogate: S(X | X^k) = E(X) with the closest points held at rho(X^k).
  It majorises E (a closest-point distance is at most the distance to the
  held point and psi is increasing) and equals E at X^k; it keeps Welsch's
  functions and the rotation term, so it is not quadratic.
* Inner L-BFGS on S from X^k: history of m pairs (s, y), cleared at every
  outer iteration (each has its own surrogate); pairs with
  y^T s <= 1e-12 |y| |s| are not stored. Direction d = -H g by the two-loop
  recursion with H0 = gamma I, gamma = s^T y / y^T y of the newest pair,
  or gamma = 1 / |g| without pairs (a first step of unit length).
* Line search: backtracking from t = 1, halving, until the sufficient
  decrease S(X + t d) <= S(X) + c1 t g^T d (at most 30 halvings; if none
  is accepted the inner solve ends).
* Termination (the two parameters): |g| <= g_tol |g_0| or max_inner
  accepted steps.
* Outer loop: one outer iteration per pass; nu annealing, alpha, beta and
  the stopping tests (displacement eps, or the relative energy change
  between consecutive outer iterates when rel_energy_tol > 0, and I_max
  outer iterations per stage) are those of Algorithm 2 (oracle.solver).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import model
from .solver import Params, Registration


@dataclass
class LbfgsParams:
    m: int = 5                 # history pairs
    c1: float = 1e-4           # sufficient-decrease threshold of the line search
    g_tol: float = 1e-3        # |g| <= g_tol |g_0| ends the inner solve
    max_inner: int = 20        # accepted inner steps per outer iteration
    max_halvings: int = 30


def two_loop(g: np.ndarray, S: list, Y: list) -> np.ndarray:
    """d = -H g of L-BFGS (Nocedal and Wright, Algorithm 7.4) with the pairs
    (S[i], Y[i]) oldest first and H0 = gamma I."""
    q = np.array(g, dtype=np.float64)
    k = len(S)
    alpha = np.zeros(k)
    rho = np.array([1.0 / float(np.dot(Y[i], S[i])) for i in range(k)])
    for i in range(k - 1, -1, -1):
        alpha[i] = rho[i] * float(np.dot(S[i], q))
        q = q - alpha[i] * Y[i]
    if k:
        gamma = float(np.dot(S[-1], Y[-1])) / float(np.dot(Y[-1], Y[-1]))
    else:
        gamma = 1.0 / float(np.linalg.norm(g))
    r = gamma * q
    for i in range(k):
        b = rho[i] * float(np.dot(Y[i], r))
        r = r + (alpha[i] - b) * S[i]
    return -r


class LbfgsRegistration(Registration):
    """Algorithm 2's stage loop around the preliminary version's outer
    iteration (fixed closest points + inner L-BFGS). ``step`` runs one outer
    iteration and returns its record; ``inner`` holds, per outer iteration,
    the accepted steps and line-search halvings."""

    def __init__(self, src, tgt, params: Params | None = None, lb: LbfgsParams | None = None, graph=None):
        super().__init__(src, tgt, params, graph)
        self.lb = lb or LbfgsParams()
        self.inner = []

    def surrogate(self, X, rho):
        alpha, beta = self.weights()
        t = model.energy_terms(self.V, self.U, self.graph, X, self.nu_a, self.nu_r, rho=rho,
                               robust=self.p.robust)
        return model.total_energy(t, alpha, beta)

    def surrogate_grad(self, X, rho):
        alpha, beta = self.weights()
        gX, _ = model.energy_gradient(self.V, self.U, self.graph, X, self.nu_a, self.nu_r, alpha, beta,
                                      rho=rho, robust=self.p.robust)
        return gX

    def minimise_surrogate(self, X0, rho):
        lb = self.lb
        X = np.array(X0, dtype=np.float64)
        f = self.surrogate(X, rho)
        g = self.surrogate_grad(X, rho).ravel()
        g0 = float(np.linalg.norm(g))
        S, Y = [], []
        steps, halvings = 0, 0
        while steps < lb.max_inner and float(np.linalg.norm(g)) > lb.g_tol * g0:
            d = two_loop(g, S, Y)
            gd = float(np.dot(g, d))
            t = 1.0
            accepted = False
            for _ in range(lb.max_halvings + 1):
                Xt = X + t * d.reshape(X.shape)
                ft = self.surrogate(Xt, rho)
                if ft <= f + lb.c1 * t * gd:
                    accepted = True
                    break
                t *= 0.5
                halvings += 1
            if not accepted:
                break
            gt = self.surrogate_grad(Xt, rho).ravel()
            s = (Xt - X).ravel()
            y = gt - g
            if float(np.dot(y, s)) > 1e-12 * float(np.linalg.norm(y)) * float(np.linalg.norm(s)):
                S.append(s)
                Y.append(y)
                if len(S) > lb.m:
                    S.pop(0)
                    Y.pop(0)
            X, f, g = Xt, ft, gt
            steps += 1
        self.inner.append((steps, halvings))
        return X

    def step(self):
        """One outer iteration: closest points at X^k, the energy (stop
        tests as Algorithm 2), then the inner L-BFGS on the surrogate."""
        from .solver import PassRecord
        if self.done:
            return None
        alpha, beta = self.weights()
        t = self.terms()
        E = model.total_energy(t, alpha, beta)
        rec = PassRecord(E, t["E_align"], t["E_reg"], t["E_rot"], True, self.nu_a, self.nu_r, self.stage)
        if (self.p.rel_energy_tol > 0 and math.isfinite(self.E_prev)
                and abs(self.E_prev - E) < self.p.rel_energy_tol * abs(self.E_prev)):
            self.records.append(rec)
            self._end_stage()
            return rec
        self.E_prev = E
        X_new = self.minimise_surrogate(self.X, t["rho"])
        self.n_solves += 1
        self.n_solves_total += 1
        vh_new = model.deform(self.V, self.graph.nidx, self.graph.w, self.graph.p, X_new)
        rec.max_disp = float(np.max(np.linalg.norm(vh_new - t["vhat"], axis=1)))
        self.records.append(rec)
        self.X = X_new
        disp_stop = self.p.rel_energy_tol <= 0 and rec.max_disp < self.eps
        if disp_stop or self.n_solves == self.p.max_iters_per_stage:
            self._end_stage()
        return rec
