"""Algorithm 2: robust non-rigid registration with Welsch's function and
Anderson acceleration, in FP64.

One *pass* is one execution of the repeat body of Algorithm 2: closest
points and rotations at X^(k), the energy, the safeguard test, and (if the
iterate is kept) the weights, the solve of Eq. (surr_solution) and the AA mix.

Readings of Algorithm 2 used here:
* The safeguard compares with E_prev, the energy of the last kept iterate in
  the current stage, and rejects only if E > E_prev (ties are kept). After a
  rejection, X^(k) becomes the last MM result G^(k-1) and that iterate is kept
  unconditionally on its re-evaluation (MM descent holds in exact
  arithmetic; the unconditional keep rules out an endless loop caused by
  rounding). The AA history is kept across a rejection.
* The stopping test max_i |v_hat_i^(k+1) - v_hat_i^(k)| < eps compares the
  deformed source at the new iterate with the one at the kept iterate of
  the pass; I_max counts solves in the stage.
* Optional energy stopping test (off unless rel_energy_tol > 0): the stage
  ends when two consecutive kept energies differ by less than
  rel_energy_tol relative to the earlier one. It replaces the displacement
  test (a stage then ends on the energy test or I_max only): the
  depth-scale workload is run to a relative energy change below 1e-6.
* nu annealing: nu_a starts at the median initial closest-point distance of
  the undeformed source, nu_r at 3 l-bar; after each stage nu_a is halved
  (clamped at nu_a_min = l-bar / sqrt(3)) and nu_r is halved; the last stage
  is the one run with nu_a == nu_a_min. alpha and beta follow Eq.
  (WeightSettings) with the current nu values, |V| = P, |E_G| = undirected
  edge count, |V_G| = N, unless given explicitly.
* eps defaults to 1e-5 times the bbox diagonal of source and target (the
  paper's 1e-5 on inputs scaled to unit diagonal).
* Singular K (the paper is silent): when no point with a non-zero alignment
  weight is influenced by a connected component of the deformation graph
  (far from the target at a small nu_a, the Welsch weights underflow to 0),
  the surrogate does not depend on that component's common translation. G
  then keeps the component's summed translation of X^(k) (the minimiser
  whose update has no component along the null space), and the pass
  records the count of such components (PassRecord.n_singular).
* Variants of Sec. 4.2 (Params.robust, Params.nu_fixed): "l2" replaces both
  Welsch functions by squared norms (all weights 1) and runs one stage (its
  energy has no nu); "l2r" keeps the nu_a schedule and gives an alignment
  weight 0 once a distance reaches 3 nu_a (the MM weights of the truncated
  quadratic min(d^2, 9 nu_a^2)). For both, alpha = k_alpha |V| / |E_G| and
  beta = k_beta |V| / |V_G|: the factors nu_r^2/nu_a^2 and 1/(2 nu_a^2) of
  Eq. (WeightSettings) scale Welsch's curvature at 0 (psi_nu(x) ~ x^2 /
  (2 nu^2)), which the squared norms do not have. nu_fixed = "max" / "min" /
  "med" runs one stage at the first stage's (nu_a, nu_r), at the last
  stage's, or at their means, the stages being those the annealing would
  run.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import graph as graph_mod
from . import geodesic, model, surrogate
from .anderson import Anderson


@dataclass
class Params:
    radius: float = 0.0             # <= 0: 5 * l-bar (Sec. 4.1)
    max_influence: int = 8
    nu_a: float = 0.0               # <= 0: median initial NN distance
    nu_r: float = 0.0               # <= 0: 3 l-bar
    nu_a_min: float = 0.0           # <= 0: l-bar / sqrt(3)
    anneal: bool = True
    k_alpha: float = 100.0
    k_beta: float = 1.0
    alpha: float = -1.0             # >= 0 overrides k_alpha
    beta: float = -1.0              # >= 0 overrides k_beta
    aa_m: int = 5
    max_iters_per_stage: int = 100  # I_max
    max_total_passes: int = 100000
    eps: float = 0.0                # <= 0: 1e-5 * bbox diagonal
    rel_energy_tol: float = 0.0
    robust: str = "welsch"          # "welsch" | "l2" | "l2r" (Sec. 4.2 variants)
    nu_fixed: str = ""              # "" (anneal per `anneal`) | "max" | "min" | "med"


@dataclass
class PassRecord:
    E: float
    E_align: float
    E_reg: float
    E_rot: float
    kept: bool
    nu_a: float
    nu_r: float
    stage: int
    max_disp: float = float("nan")
    n_singular: int = 0             # free components of the pass's solve


class Registration:
    def __init__(self, src, tgt, params: Params | None = None, graph=None, faces=None):
        """``faces`` [F,3]: the source is a triangle mesh; the graph then uses
        geodesic distances and l-bar is the mean mesh edge length
        (``oracle.geodesic``)."""
        self.V = np.asarray(src, dtype=np.float64)
        self.U = np.asarray(tgt, dtype=np.float64)
        self.p = params or Params()
        need_lbar = (self.p.radius <= 0 or self.p.nu_r <= 0
                     or self.p.nu_a_min <= 0)
        if faces is not None:
            self.lbar = geodesic.mean_edge_length(self.V, faces)
        else:
            self.lbar = graph_mod.mean_spacing(self.V) if need_lbar else float("nan")
        R = self.p.radius if self.p.radius > 0 else 5.0 * self.lbar
        if graph is None and faces is not None:
            graph = geodesic.build_graph_mesh(self.V, faces, R, self.p.max_influence)
        self.graph = graph if graph is not None else graph_mod.build_graph(
            self.V, R, self.p.max_influence)
        both = np.concatenate([self.V, self.U])
        self.diag = float(np.linalg.norm(both.max(axis=0) - both.min(axis=0)))
        self.eps = self.p.eps if self.p.eps > 0 else 1e-5 * self.diag
        if self.p.nu_a > 0:
            nu_a0 = self.p.nu_a
        else:
            _, d2 = model.closest_points(self.V, self.U)
            nu_a0 = float(np.median(np.sqrt(d2)))
        self.nu_a_min = self.p.nu_a_min if self.p.nu_a_min > 0 else self.lbar / math.sqrt(3.0)
        self.nu_r = self.p.nu_r if self.p.nu_r > 0 else 3.0 * self.lbar
        if not self.p.anneal:
            self.nu_a_min = nu_a0
        self.nu_a = max(nu_a0, self.nu_a_min)
        if self.p.nu_fixed:
            # the stages the annealing would run: nu_a halves (clamped at
            # nu_a_min) and nu_r halves until nu_a == nu_a_min
            na, nr = self.nu_a, self.nu_r
            while na != self.nu_a_min:
                na = max(na / 2.0, self.nu_a_min)
                nr = nr / 2.0
            pick = {"max": (self.nu_a, self.nu_r), "min": (na, nr),
                    "med": ((self.nu_a + na) / 2.0, (self.nu_r + nr) / 2.0)}[self.p.nu_fixed]
            self.nu_a, self.nu_r = pick
            self.nu_a_min = self.nu_a
        if self.p.robust == "l2":
            self.nu_a_min = self.nu_a
        self.X = model.identity_X(self.graph.N)
        self.aa = Anderson(self.p.aa_m)
        self.records: list[PassRecord] = []
        self.stage = 0
        self.done = False
        self.n_solves_total = 0
        self.n_rejected = 0
        self._start_stage()

    # -- parameters -------------------------------------------------------
    def weights(self):
        P, N, E = self.V.shape[0], self.graph.N, max(self.graph.n_edges, 1)
        if self.p.robust == "welsch":
            alpha = self.p.k_alpha * P / E * self.nu_r ** 2 / self.nu_a ** 2
            beta = self.p.k_beta * P / max(N, 1) / (2.0 * self.nu_a ** 2)
        else:
            alpha = self.p.k_alpha * P / E
            beta = self.p.k_beta * P / max(N, 1)
        if self.p.alpha >= 0:
            alpha = self.p.alpha
        if self.p.beta >= 0:
            beta = self.p.beta
        return alpha, beta

    def _start_stage(self):
        self.E_prev = math.inf
        self.just_reverted = False
        self.n_solves = 0
        self.G_last = None
        self.aa.reset()

    def _end_stage(self):
        if self.nu_a == self.nu_a_min:
            self.done = True
            return
        self.nu_a = max(self.nu_a / 2.0, self.nu_a_min)
        self.nu_r = self.nu_r / 2.0
        self.stage += 1
        self._start_stage()

    # -- evaluation -------------------------------------------------------
    def terms(self, X=None, rho=None):
        return model.energy_terms(self.V, self.U, self.graph,
                                  self.X if X is None else X,
                                  self.nu_a, self.nu_r, rho=rho, robust=self.p.robust)

    def energy(self, X=None):
        t = self.terms(X)
        a, b = self.weights()
        return model.total_energy(t, a, b), t

    def mm_map(self, terms, X=None):
        """G(X^k): minimiser of the surrogate built at the state ``terms``
        (evaluated at X^k = ``X``, default the current iterate). Components
        of the graph without alignment weight keep their summed translation
        of X^k (surrogate.free_components); their count is left in
        ``self.last_free``."""
        alpha, beta = self.weights()
        K, B, parts = surrogate.normal_equations(self.V, self.U, self.graph, terms,
                                                 self.nu_a, self.nu_r, alpha, beta,
                                                 robust=self.p.robust)
        free = surrogate.free_components(self.graph, parts["wa"])
        self.last_free = len(free)
        return surrogate.solve_normal_equations(K, B, self.X if X is None else X, free)

    # -- one pass of Algorithm 2 -----------------------------------------
    def step(self) -> PassRecord | None:
        if self.done:
            return None
        alpha, beta = self.weights()
        t = self.terms()
        E = model.total_energy(t, alpha, beta)
        rec = PassRecord(E, t["E_align"], t["E_reg"], t["E_rot"], True,
                         self.nu_a, self.nu_r, self.stage)
        if E > self.E_prev and not self.just_reverted:
            rec.kept = False
            self.records.append(rec)
            self.n_rejected += 1
            self.X = self.G_last.copy()
            self.just_reverted = True
            return rec
        self.just_reverted = False
        if (self.p.rel_energy_tol > 0 and math.isfinite(self.E_prev)
                and abs(self.E_prev - E) < self.p.rel_energy_tol * abs(self.E_prev)):
            self.records.append(rec)
            self._end_stage()
            return rec
        self.E_prev = E
        G = self.mm_map(t)
        rec.n_singular = self.last_free
        self.G_last = G.copy()
        X_new = self.aa.mix(G, self.X)
        self.n_solves += 1
        self.n_solves_total += 1
        vh_new = model.deform(self.V, self.graph.nidx, self.graph.w,
                              self.graph.p, X_new)
        disp = float(np.max(np.linalg.norm(vh_new - t["vhat"], axis=1)))
        rec.max_disp = disp
        self.records.append(rec)
        self.X = X_new
        disp_stop = self.p.rel_energy_tol <= 0 and disp < self.eps
        if disp_stop or self.n_solves == self.p.max_iters_per_stage:
            self._end_stage()
        return rec

    def solve(self, max_passes: int | None = None):
        cap = self.p.max_total_passes if max_passes is None else max_passes
        n = 0
        while not self.done and n < cap:
            self.step()
            n += 1
        return self.X
