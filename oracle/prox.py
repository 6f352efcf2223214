"""Algorithm 1 (Sec. III-B): the unbalanced Beckmann-OT proximal algorithm, FP64.

Computes prox^mu_{rho V}(p0, p1) of eq. (Prox_UOT):

    argmin_{x0, x1 >= 0, M, r}  ||M||_{2,1} + mu ||r||_p^p + (1/2rho) ||x - p||^2
    s.t.  D(M) - x0 + x1 = r

by the Chambolle-Pock iteration of eqs. (Prox_UOT_M)-(Prox_UOT_a), in the
order of Algorithm 1: M-step, x-step, r-step, b = 2K(z^{k+1}) - K(z^k),
a-step.

Modes (which arguments are variables):
  "prox"        -- x0 and x1 both free (eq. Prox_UOT);
  "fixed_first" -- x0 frozen at p0 = s, x1 free with centre p1: the special
                   case of eq. (Prox_UOT_specialcase), A := I and
                   K := D(M) - s + x - r;
  "eval"        -- x0 = p0 and x1 = p1 frozen: the iteration then solves the
                   regulariser V_mu(p0, p1) itself (eq. Unbal_OT_beckman).
``balanced`` drops r (r = 0), which gives the balanced Beckmann problem
(eq. OT_beckman) -- the paper's balanced comparison variant.
``p_exp`` = 1 is the paper's l1 growth/decay penalty; 2 is the "averaging
update" the paper mentions for p = 2 (Sec. III-B).

Readings where the paper is ambiguous (each also listed in the design notes):
  * x-step: the objective weights (1/2rho)||x - p||^2 (eqs. Prox_UOT and the
    prox definition of Sec. II-B) while the printed closed form is the
    minimiser for a (rho/2) weight.  We follow the objective:
    x = Pi_+((tau1 p + rho (x^k - tau1 A^T a^k)) / (rho + tau1)).
  * Constraint sign: D(M) - x0 + x1 = r with A = [-I, I] (eqs. Prox_UOT,
    Lagrangian), not the opposite sign of eq. (Unbal_OT_beckman); both give
    the same objective values.
  * Stopping: every ``check_every`` iterations, with s_p = max(||p||, 1e-30),
      res_pri = ||K(z^{k+1})|| / s_p
      res_fp  = ||(z^{k+1}, a^{k+1}) - (z^k, a^k)|| / max(||(z^{k+1}, a^{k+1})||, 1e-30)
    over the stored state (Mx, My, x0, x1, r, a; a frozen x is its input);
    converged when max(res_pri, res_fp) <= tol.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import grid


@dataclass
class ProxParams:
    mu: float = 8.0
    rho: float = 1.0
    tau1: float = 0.0           # <= 0: default 0.99 / sqrt(lambda_max + n_id)
    tau2: float = 0.0
    mode: str = "prox"          # "prox" | "fixed_first" | "eval"
    norm: str = "iso"           # "iso" | "aniso"
    balanced: bool = False
    p_exp: int = 1
    tol: float = 1e-5
    max_iter: int = 100000
    check_every: int = 10


@dataclass
class ProxState:
    Mx: np.ndarray
    My: np.ndarray
    x0: np.ndarray
    x1: np.ndarray
    r: np.ndarray
    a: np.ndarray

    def copy(self) -> "ProxState":
        return ProxState(*(v.copy() for v in self.tuple()))

    def tuple(self):
        return (self.Mx, self.My, self.x0, self.x1, self.r, self.a)


def frozen(mode: str) -> tuple[bool, bool]:
    """(x0 frozen, x1 frozen) for a mode."""
    return {"prox": (False, False), "fixed_first": (True, False), "eval": (True, True)}[mode]


def n_identity_blocks(prm: ProxParams) -> int:
    """Number of +-I blocks of K acting on free variables (x0, x1, r)."""
    f0, f1 = frozen(prm.mode)
    return int(not f0) + int(not f1) + int(not prm.balanced)


def default_steps(H: int, W: int, prm: ProxParams) -> ProxParams:
    """Fill tau1 = tau2 = 0.99 / sqrt(||K||^2) when not given, where
    ||K||^2 = lambda_max(D D*) + (number of identity blocks): the bound of
    Theorem 1 (lambda_max + 3 for the full problem)."""
    L = grid.lambda_max(H, W) + n_identity_blocks(prm)
    t = 0.99 / np.sqrt(max(L, 1e-300))
    return replace(prm, tau1=prm.tau1 if prm.tau1 > 0 else t, tau2=prm.tau2 if prm.tau2 > 0 else t)


def zero_state(p0: np.ndarray, p1: np.ndarray, mode: str) -> ProxState:
    """All-zero initial state (Algorithm 2 initialises the cached prox state
    to 0); frozen x take their input values."""
    z = np.zeros(np.shape(p0), np.float64)
    f0, f1 = frozen(mode)
    return ProxState(z.copy(), z.copy(),
                     np.array(p0, np.float64) if f0 else z.copy(),
                     np.array(p1, np.float64) if f1 else z.copy(),
                     z.copy(), z.copy())


def K_op(st: ProxState, prm: ProxParams) -> np.ndarray:
    """K(M, x, r) = D(M) + A x - r = D(M) - x0 + x1 - r (Sec. III-B); r = 0
    when balanced.  For a frozen x the stored value is the fixed argument."""
    k = grid.div(st.Mx, st.My) - st.x0 + st.x1
    if not prm.balanced:
        k = k - st.r
    return k


def shrink_l2(gx: np.ndarray, gy: np.ndarray, t: float):
    """Vector soft shrinkage max(||q|| - t, 0) q / ||q|| of each 2-vector
    (eq. Prox_UOT_M_prox); 0 where ||q|| = 0."""
    n = np.sqrt(gx * gx + gy * gy)
    safe = np.where(n > 0, n, 1.0)
    s = np.where(n > 0, np.maximum(n - t, 0.0) / safe, 0.0)
    return gx * s, gy * s


def shrink_l1(q: np.ndarray, t: float) -> np.ndarray:
    """sign(q) max(|q| - t, 0) (Sec. III-B, r-step)."""
    return np.sign(q) * np.maximum(np.abs(q) - t, 0.0)


def alg1_iteration(st: ProxState, p0: np.ndarray, p1: np.ndarray, prm: ProxParams) -> ProxState:
    """One pass of the while-loop body of Algorithm 1."""
    H, W = st.a.shape[-2:]
    t1, t2, rho, mu = prm.tau1, prm.tau2, prm.rho, prm.mu
    f0, f1 = frozen(prm.mode)
    # line 3: m_i <- shrink_{tau1}(m_i - tau1 D*(a)_i)
    gx, gy = grid.div_adj(st.a)
    qx = st.Mx - t1 * gx
    qy = st.My - t1 * gy
    if prm.norm == "iso":
        Mx, My = shrink_l2(qx, qy, t1)
    else:   # prox of sum |Mx| + |My|
        Mx, My = shrink_l1(qx, t1), shrink_l1(qy, t1)
    mx, my = grid.edge_masks(H, W)
    Mx = Mx * mx
    My = My * my
    # line 4: x <- Pi_+(...), A^T a = [-a; a]
    x0 = st.x0 if f0 else np.maximum((t1 * p0 + rho * (st.x0 - t1 * (-st.a))) / (rho + t1), 0.0)
    x1 = st.x1 if f1 else np.maximum((t1 * p1 + rho * (st.x1 - t1 * st.a)) / (rho + t1), 0.0)
    # line 5: r <- shrink_{mu tau1}(r + tau1 a)   (p = 1) or the p = 2 average
    if prm.balanced:
        r = np.zeros_like(st.r)
    elif prm.p_exp == 1:
        r = shrink_l1(st.r + t1 * st.a, mu * t1)
    else:
        r = (st.r + t1 * st.a) / (1.0 + 2.0 * mu * t1)
    new = ProxState(Mx, My, x0, x1, r, st.a)
    # line 6: b = 2 K(z^{k+1}) - K(z^k);  line 7: a <- a + tau2 b
    b = 2.0 * K_op(new, prm) - K_op(st, prm)
    new.a = st.a + t2 * b
    return new


def iterate(p0, p1, prm: ProxParams, n_iter: int, state: ProxState | None = None) -> ProxState:
    """Run ``n_iter`` iterations of Algorithm 1 with no stopping test (the
    inexact, warm-started use of Sec. III-B and Algorithm 3 line 11)."""
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    H, W = p0.shape[-2:]
    prm = default_steps(H, W, prm)
    st = zero_state(p0, p1, prm.mode) if state is None else state.copy()
    for _ in range(n_iter):
        st = alg1_iteration(st, p0, p1, prm)
    return st


def _sq(v) -> float:
    return float(np.sum(np.asarray(v, np.float64) ** 2))


def residuals(new: ProxState, old: ProxState, p0, p1, prm: ProxParams) -> tuple[float, float]:
    """(res_pri, res_fp) of the stopping rule described in the module header."""
    sp = max(np.sqrt(_sq(p0) + _sq(p1)), 1e-30)
    res_pri = np.sqrt(_sq(K_op(new, prm))) / sp
    d = sum(_sq(n - o) for n, o in zip(new.tuple(), old.tuple()))
    z = sum(_sq(n) for n in new.tuple())
    res_fp = np.sqrt(d) / max(np.sqrt(z), 1e-30)
    return float(res_pri), float(res_fp)


def objective(st: ProxState, p0, p1, prm: ProxParams) -> float:
    """||M||_{2,1} + mu ||r||_p^p + (1/2rho) ||x - p||^2 over the free x
    (eq. Prox_UOT); for "eval" this is the objective of eq. (Unbal_OT_beckman)."""
    f0, f1 = frozen(prm.mode)
    v = grid.l21(st.Mx, st.My, prm.norm)
    if not prm.balanced:
        v += prm.mu * (float(np.sum(np.abs(st.r))) if prm.p_exp == 1 else _sq(st.r))
    if not f0:
        v += _sq(st.x0 - p0) / (2.0 * prm.rho)
    if not f1:
        v += _sq(st.x1 - p1) / (2.0 * prm.rho)
    return float(v)


@dataclass
class SolveInfo:
    iters: int
    res_pri: float
    res_fp: float
    converged: bool
    history: list = field(default_factory=list)


def solve(p0, p1, prm: ProxParams, state: ProxState | None = None) -> tuple[ProxState, SolveInfo]:
    """Algorithm 1 until the stopping rule holds or ``max_iter`` iterations."""
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    H, W = p0.shape[-2:]
    prm = default_steps(H, W, prm)
    st = zero_state(p0, p1, prm.mode) if state is None else state.copy()
    info = SolveInfo(0, np.inf, np.inf, False)
    for k in range(1, prm.max_iter + 1):
        new = alg1_iteration(st, p0, p1, prm)
        if k % prm.check_every == 0 or k == prm.max_iter:
            rp, rf = residuals(new, st, p0, p1, prm)
            info.history.append((k, rp, rf))
            info.iters, info.res_pri, info.res_fp = k, rp, rf
            if max(rp, rf) <= prm.tol:
                info.converged = True
                return new, info
        st = new
    info.iters = prm.max_iter
    return st, info


def certificate(st: ProxState, p0, p1, prm: ProxParams) -> dict:
    """Duality-gap certificate for eq. (Prox_UOT), derived from its Lagrangian.

    The dual function g(a) = inf over (M, x, r) of the Lagrangian is finite
    only when ||(D* a)_i|| <= 1 for every i (dual norm of the flux norm) and,
    for p = 1, |a_i| <= mu.  A feasible dual point is obtained from the iterate
    by a_bar = clip(a / max(1, max_i ||(D*a)_i||), -mu, mu) (clipping is
    1-Lipschitz, so it keeps the flux condition).  Then
        g(a_bar) = sum over free x_k of min_{x >= 0} [(1/2rho)(x - p_k)^2 + c_k x]
                   + <a_bar, contribution of frozen x>  (- sum a^2/4mu for p = 2)
    with c = A^T a_bar = [-a_bar; a_bar].  A feasible primal point keeps (M, x)
    and sets r' = D(M) + A x; its objective P' >= optimum >= g(a_bar).
    Returns P', g, gap = P' - g and rel_gap = gap / max(|P'|, 1e-30).
    For the balanced problem r' must be zero, so no feasible primal point is
    available from an inexact iterate and the gap is not a bound
    (``gap_valid`` is False).
    """
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    f0, f1 = frozen(prm.mode)
    gx, gy = grid.div_adj(st.a)
    if prm.norm == "iso":
        nmax = float(np.max(np.sqrt(gx * gx + gy * gy)))
    else:
        nmax = float(max(np.max(np.abs(gx)), np.max(np.abs(gy))))
    ab = st.a / max(1.0, nmax)
    if not prm.balanced and prm.p_exp == 1:
        ab = np.clip(ab, -prm.mu, prm.mu)
    g = 0.0
    for frz, x, p, sgn in ((f0, st.x0, p0, -1.0), (f1, st.x1, p1, 1.0)):
        c = sgn * ab
        if frz:
            g += float(np.sum(c * x))
        else:
            xs = np.maximum(p - prm.rho * c, 0.0)
            g += float(np.sum((xs - p) ** 2 / (2.0 * prm.rho) + c * xs))
    if not prm.balanced and prm.p_exp == 2:
        g -= _sq(ab) / (4.0 * prm.mu)
    rprime = grid.div(st.Mx, st.My) - st.x0 + st.x1
    feas = replace(st.copy(), r=rprime)
    P = objective(feas, p0, p1, prm) if not prm.balanced else objective(st, p0, p1, prm)
    gap = P - g
    return {"primal": P, "dual": g, "gap": gap, "rel_gap": gap / max(abs(P), 1e-30),
            "dual_scale": max(1.0, nmax),
            "gap_valid": not prm.balanced}
