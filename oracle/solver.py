"""Algorithm 1 (PCG), the subset weighted mean and the Levenberg-Marquardt step.

* ``pcg``: Algorithm 1 (Sec. 3.3) step by step, in the paper's notation
  (b, M^-1, x, u, g, r, z, p, alpha, beta). The preconditioner is the Jacobi
  M^-1 = 1 / diag(J^T J), or a given positive diagonal D in its place.
* ``combine``: Eq. combine-pcg (Sec. 3.3), Delta = sum_i M_i Delta_i / sum_k M_k.
* ``lm_step``: Eq. norm-eq for the direction, Eq. tr-update for rho and the
  damping update, with gamma = 1 (no line search).

Readings where the paper is silent:
  - the loop "for i = 0 to n_iters" runs n_iters times after the initial product;
  - the LM update follows Ceres (Sec. 3.2), whose Levenberg-Marquardt strategy
    clamps the diagonal diag(J^T J) to [1e-6, 1e32] before using it; the
    clamped diagonal is used as the Jacobi preconditioner and in the damping
    term lambda * M, while the subset weights of Eq. combine-pcg keep the raw
    diagonal (they come from the derivation in Sec. B);
  - the break test compares ||r||^2 with break_rel2 * ||b||^2 (0 disables it);
  - a step is accepted when rho > 1e-5 and the predicted decrease is positive;
    lambda is multiplied by 1 - (2 rho - 1)^3 (accepted) or 2 (rejected), then
    clamped to [lambda_min, lambda_max];
  - the predicted decrease uses every subset's J_i and F_i at the old parameters.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import math

import numpy as np

from . import jacobian as jac
from . import residual as res


@dataclass
class PCGStats:
    iters: int = 0
    rel_residual: float = 0.0        # ||r|| / ||b|| (recursive r)
    breakdown: bool = False
    history: list = field(default_factory=list)   # ||r||^2 after each iteration


DIAG_MIN, DIAG_MAX = 1e-6, 1e32


def clamp_diag(diag: np.ndarray) -> np.ndarray:
    """diag(J^T J) clamped to [DIAG_MIN, DIAG_MAX] (Ceres' LM diagonal bounds)."""
    return np.clip(diag, DIAG_MIN, DIAG_MAX)


def jacobi_inverse(diag: np.ndarray) -> np.ndarray:
    """M^-1 of Algorithm 1 from the clamped diagonal."""
    return 1.0 / clamp_diag(diag)


def pcg(apply_JTJ, b: np.ndarray, M: np.ndarray, lam: float, n_iters: int = 8,
        break_rel2: float = 0.0, Minv: np.ndarray | None = None):
    """Algorithm 1. apply_JTJ(v) returns J^T J v; M is the raw diag(J^T J), clamped
    here for the preconditioner and the damping. Returns (x, stats)."""
    if Minv is None:
        Minv = jacobi_inverse(M)
    M = clamp_diag(M)
    st = PCGStats()
    bb = float(np.vdot(b, b))
    x = Minv * b                                   # x0 = M^-1 b
    g = apply_JTJ(x)                               # u0 = J x0; g0 = J^T u0
    r = b - (g + lam * M * x)                      # r0 = b - (g0 + lambda M x0)
    z = Minv * r                                   # z0 = M^-1 r0
    p = z.copy()                                   # p0 = z0
    rz = float(np.vdot(r, z))
    for i in range(n_iters):
        g = apply_JTJ(p)                           # u_i = J p_i; g_i = J^T u_i
        g = g + lam * M * p                        # g_i += lambda M p_i
        pg = float(np.vdot(p, g))
        if not np.isfinite(pg) or pg <= 0.0:
            st.breakdown = True
            break
        alpha = rz / pg                            # alpha_i = r^T z / p^T g
        x = x + alpha * p
        r = r - alpha * g
        z = Minv * r
        rz_new = float(np.vdot(r, z))
        beta = rz_new / rz if rz != 0.0 else 0.0
        p = z + beta * p
        rz = rz_new
        st.iters = i + 1
        rr = float(np.vdot(r, r))
        st.history.append(rr)
        if break_rel2 > 0.0 and rr < break_rel2 * bb:
            break
    st.rel_residual = float(np.sqrt(np.vdot(r, r) / bb)) if bb > 0 else 0.0
    return x, st


def combine(deltas: list, diags: list) -> np.ndarray:
    """Eq. combine-pcg: elementwise weighted mean with weights M_i = diag(J_i^T J_i)."""
    num = np.zeros_like(deltas[0])
    den = np.zeros_like(diags[0])
    for d, m in zip(deltas, diags):
        num += m * d
        den += m
    return np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), 0.0)


@dataclass
class SubsetSystem:
    cams: list
    lin: list
    F: np.ndarray        # L2: c - C; L1 + SSIM: e = (dr/dc) r summed over both residuals
    cost: float
    b: np.ndarray
    M: np.ndarray
    W: np.ndarray | None = None   # L1 + SSIM: (dr1/dc)^2 + (dr2/dc)^2 per pixel channel; None for L2


def objective_cost(img_flat: np.ndarray, tgt_flat: np.ndarray, cams: list, objective=None) -> float:
    """E at a rendered image: ||c - C||^2 (L2) or Eq. gn-loss (objective given)."""
    if objective is None:
        F = jac.residual(img_flat, tgt_flat)
        return jac.cost(F)
    return res.cost(img_flat, tgt_flat, cams, objective)


def build_subset(params: np.ndarray, cams: list, targets_flat: np.ndarray, smooth=False,
                 objective=None) -> SubsetSystem:
    """buildCache + diagJTJ of Algorithm 1: F, b = -J^T F and M = diag(J^T J) for one subset.
    objective: None for the sum-of-squares residual c - C, or a residual.Objective
    (L1 + SSIM, Eq. gn-loss), whose weights enter through (dr/dc) (Sec. C)."""
    lin = jac.linearise(params, cams, smooth)
    img = np.concatenate([vl.ras.image.ravel() for vl in lin])
    N = params.shape[0]
    if objective is None:
        F = jac.residual(img, targets_flat)
        return SubsetSystem(cams, lin, F, jac.cost(F), -jac.apply_JT(lin, F, N), jac.jacobi_diag(lin, N))
    wt = res.weights(img, targets_flat, cams, objective)
    b = -jac.apply_JT(lin, wt.e, N)                      # J^T F = (dc/dx)^T e
    M = jac.jacobi_diag(lin, N, weights=wt.w)
    return SubsetSystem(cams, lin, wt.e, wt.cost, b, M, wt.w)


def apply_JTJ(sys_: SubsetSystem, v: np.ndarray) -> np.ndarray:
    """J^T J v: (dc/dx)^T ((dc/dx) v), weighted by W between the two products when
    the residual is not L2 (Eq. apply-jtj-simplified-vec-vec)."""
    N = sys_.b.shape[0]
    u = jac.apply_J(sys_.lin, v, sys_.F.shape[0])
    if sys_.W is not None:
        u = sys_.W * u
    return jac.apply_JT(sys_.lin, u, N)


def solve_subset(sys_: SubsetSystem, lam: float, n_iters: int, break_rel2: float = 0.0, Minv=None):
    return pcg(lambda v: apply_JTJ(sys_, v), sys_.b, sys_.M, lam, n_iters, break_rel2, Minv)


@dataclass
class LMResult:
    params: np.ndarray
    lam: float
    accepted: bool
    rho: float
    cost: float
    cost_new: float
    pred: float
    delta: np.ndarray
    pcg: list
    gamma: float = 1.0
    ls_costs: list = None


def line_search_views(subsets: list, frac: float) -> list:
    """Views the line search renders: the first ceil(frac * V) of the step's V
    views, in subset order; returned as a count per subset (a prefix of each)."""
    total = sum(len(c) for c in subsets)
    n = int(math.ceil(frac * total))
    out = []
    for cams in subsets:
        k = min(len(cams), max(n, 0))
        out.append(k)
        n -= k
    return out


def line_search(params: np.ndarray, delta: np.ndarray, subsets: list, targets: list, steps: int, frac: float,
                smooth=False, objective=None):
    """Eq. line-search, min over gamma of E(x + gamma Delta), read as: evaluate the
    sum-of-squares cost on the line-search views at gamma = 1, 1/2, 1/4, ... (at
    most `steps` values), stop at the first value larger than the previous finite
    one, and return the best gamma (ties: the larger gamma) and the costs seen."""
    counts = line_search_views(subsets, frac)
    best_g, best_e, prev, costs = 1.0, math.inf, math.inf, []
    for k in range(steps):
        g = 0.5 ** k
        e = 0.0
        x = params + g * delta
        for cams, tg, nv in zip(subsets, targets, counts):
            if nv == 0:
                continue
            npx = sum(c.width * c.height * 3 for c in cams[:nv])
            e += objective_cost(jac.render(x, cams[:nv], smooth), tg[:npx], cams[:nv], objective)
        costs.append(e)
        if e < best_e:
            best_g, best_e = g, e
        if math.isfinite(prev) and e > prev:
            break
        prev = e
    return best_g, costs


def lm_step(params: np.ndarray, subsets: list, targets: list, lam: float, n_iters: int = 8,
            lambda_min: float = 1e-4, lambda_max: float = 1e4, break_rel2: float = 0.0,
            smooth=False, precond=None, ls_steps: int = 0, ls_frac: float = 0.3, objective=None) -> LMResult:
    """One LM iteration over image subsets (Sec. 3.2 and Eq. combine-pcg).

    subsets: list of camera lists; targets: list of flat target vectors (one per subset).
    precond: optional callable (SubsetSystem) -> D replacing M^-1 in Algorithm 1.
    ls_steps > 0: the step is scaled by the line search of Eq. line-search (see
    line_search); rho (Eq. tr-update) then uses gamma Delta.
    objective: None (sum of squares) or a residual.Objective (L1 + SSIM).
    """
    systems = [build_subset(params, cams, tg, smooth, objective) for cams, tg in zip(subsets, targets)]
    deltas, stats = [], []
    for s in systems:
        Minv = precond(s) if precond is not None else None
        d, st = solve_subset(s, lam, n_iters, break_rel2, Minv)
        deltas.append(d)
        stats.append(st)
    delta = combine(deltas, [s.M for s in systems])
    cost0 = sum(s.cost for s in systems)
    gamma, ls_costs = 1.0, None
    if ls_steps > 0:
        gamma, ls_costs = line_search(params, delta, subsets, targets, ls_steps, ls_frac, smooth, objective)
    pred = 0.0
    for s in systems:
        u = jac.apply_J(s.lin, delta, s.F.shape[0])
        if s.W is None:
            v = gamma * u + s.F
            pred += float(np.dot(v, v))
        else:   # the Gauss-Newton model E + 2 gamma e.u + gamma^2 W.u^2
            pred += s.cost + 2.0 * gamma * float(np.dot(s.F, u)) + gamma * gamma * float(np.dot(s.W, u * u))
    new = params + gamma * delta
    cost1 = 0.0
    for cams, tg in zip(subsets, targets):
        cost1 += objective_cost(jac.render(new, cams, smooth), tg, cams, objective)
    den = cost0 - pred
    rho = (cost0 - cost1) / den if den > 0 else -np.inf
    accepted = bool(den > 0 and rho > 1e-5)
    if accepted:
        lam = lam * (1.0 - (2.0 * rho - 1.0) ** 3)
        out = new
    else:
        lam = lam * 2.0
        out = params
    lam = float(min(max(lam, lambda_min), lambda_max))
    return LMResult(out, lam, accepted, float(rho), cost0, cost1, pred, delta, stats, gamma, ls_costs)
