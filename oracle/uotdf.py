"""Algorithm 2 (UOT-DF ADMM, Sec. IV-A.1) with Phi = I, FP64.

Test infrastructure only: the CUDA path never imports this module.

Problem (eq. general_UOT-DF with Phi = I), for a batch of independent frames
[B, H, W]:
    min_{s >= 0}  1/2 ||y - s||^2 + R(s) + kappa V_mu(s, s0),
R = 0 (UOT-DF, eq. UOT-DF) or R = lambda ||s||_1 (BPDN+UOT-DF).
Splitting s = x = z with scaled duals a, b; one ADMM iteration (Algorithm 2,
in the order of its loop body):
    s <- argmin R(s) + i_+(s) + rho/2 ||s - (x + a)||^2 + rho/2 ||s - (z + b)||^2
       = max(q, 0), or max(q - lambda/(2 rho), 0),   q = (x + a + z + b) / 2
    x <- (y + rho (s - a)) / (1 + rho)
    z <- prox of (kappa/rho) V_mu(., s0) at s - b: Algorithm 1 in its
         fixed-first-argument form (eq. Prox_UOT_specialcase) with the
         argument s0 frozen, prox centre s - b and prox weight kappa/rho,
         ``n_inner`` warm-started iterations from the cached state
    a <- a + x - s
    b <- b + z - s
Readings:
  * the s-update: the printed line takes the prox at x + a alone, but s
    appears in both augmented terms of the printed Lagrangian; minimising it
    over s gives the prox (weight 1/(2 rho)) at the average of x + a and
    z + b.  With the printed line the iteration ignores z in s and settles at
    s = Pi_+(y) whatever kappa is;
  * the BPDN prox is printed as Pi_+(q - rho/lambda); the prox of
    lambda ||.||_1 + i_+ with weight 1/(2 rho) is Pi_+(q - lambda/(2 rho));
  * V_mu is symmetric in its two arguments (swap M -> -M, r -> -r), so the
    fixed argument s0 takes the frozen slot x0 and z the free slot x1;
  * stopping: the paper's primal and dual residuals
    ||(x - s, z - s)|| and rho ||(dx, dz)||, here relative to ||y||.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import prox as P


@dataclass
class UotdfParams:
    kappa: float = 0.5
    mu: float = 3.0
    rho: float = 1.0
    lam: float = 0.0            # 0: UOT-DF; > 0: BPDN+UOT-DF
    n_inner: int = 1
    norm: str = "iso"
    p_exp: int = 1
    tol: float = 1e-5
    max_iter: int = 20000


@dataclass
class UotdfState:
    s: np.ndarray
    x: np.ndarray
    a: np.ndarray
    b: np.ndarray
    prox: P.ProxState           # z = prox.x1; prox.x0 holds s0
    history: list = field(default_factory=list)

    @property
    def z(self) -> np.ndarray:
        return self.prox.x1


def line6_weight(prm: UotdfParams) -> float:
    """Line 6: z minimises kappa V_mu(s0, z) + rho/2 ||z - (s - b)||^2, the prox
    of eq. (Prox_UOT_specialcase) with weight kappa / rho."""
    return prm.kappa / prm.rho


def prox_params(prm: UotdfParams, H: int, W: int) -> P.ProxParams:
    """Line 6: prox of (kappa/rho) V_mu(., s0), the fixed-first form."""
    return P.default_steps(H, W, P.ProxParams(mu=prm.mu, rho=line6_weight(prm), mode="fixed_first",
                                              norm=prm.norm, p_exp=prm.p_exp))


def zero_state(s0: np.ndarray) -> UotdfState:
    """Line 2: all variables 0; the cached prox state is 0 with x0 = s0."""
    s0 = np.asarray(s0, np.float64)
    z = np.zeros_like(s0)
    return UotdfState(z.copy(), z.copy(), z.copy(), z.copy(), P.zero_state(s0, z, "fixed_first"))


def prox_R(q: np.ndarray, prm: UotdfParams) -> np.ndarray:
    """Line 4: prox of R + i_+ with weight 1/(2 rho) (two augmented terms)."""
    return np.maximum(q - prm.lam / (2.0 * prm.rho), 0.0) if prm.lam > 0 else np.maximum(q, 0.0)


def line5_x(y: np.ndarray, s: np.ndarray, a: np.ndarray, rho: float) -> np.ndarray:
    """Line 5 with Phi = I: x minimises 1/2 ||y - x||^2 + rho/2 ||x - s + a||^2."""
    return (y + rho * (s - a)) / (1.0 + rho)


def iteration(st: UotdfState, y: np.ndarray, s0: np.ndarray, prm: UotdfParams) -> tuple[UotdfState, float, float]:
    """One pass of Algorithm 2's loop body; returns the new state and the
    residuals (relative to ||y||)."""
    y = np.asarray(y, np.float64)
    s0 = np.asarray(s0, np.float64)
    H, W = y.shape[-2:]
    rho = prm.rho
    s = prox_R(0.5 * (st.x + st.a + st.prox.x1 + st.b), prm)   # line 4
    x = line5_x(y, s, st.a, rho)                       # line 5, Phi = I
    pp = prox_params(prm, H, W)
    pst = P.iterate(s0, s - st.b, pp, prm.n_inner, state=st.prox)   # line 6
    z_old = st.prox.x1
    z = pst.x1
    a = st.a + x - s                                   # line 7
    b = st.b + z - s                                   # line 8
    ny = max(np.sqrt(np.sum(y * y)), 1e-30)
    pri = np.sqrt(np.sum((x - s) ** 2) + np.sum((z - s) ** 2)) / ny
    dual = rho * np.sqrt(np.sum((x - st.x) ** 2) + np.sum((z - z_old) ** 2)) / ny
    return UotdfState(s, x, a, b, pst, st.history), float(pri), float(dual)


def solve(y, s0, prm: UotdfParams, state: UotdfState | None = None, max_iter: int | None = None):
    y = np.asarray(y, np.float64)
    s0 = np.asarray(s0, np.float64)
    st = zero_state(s0) if state is None else state
    n = prm.max_iter if max_iter is None else max_iter
    pri = dual = np.inf
    for it in range(1, n + 1):
        st, pri, dual = iteration(st, y, s0, prm)
        st.history.append((it, pri, dual))
        if max(pri, dual) <= prm.tol:
            return st, {"iters": it, "res_pri": pri, "res_dual": dual, "converged": True}
    return st, {"iters": n, "res_pri": pri, "res_dual": dual, "converged": False}


def objective(s: np.ndarray, y: np.ndarray, s0: np.ndarray, prm: UotdfParams, V: float) -> float:
    """1/2 ||y - s||^2 + R(s) + kappa V, with V = V_mu(s, s0) supplied by the caller."""
    s = np.asarray(s, np.float64)
    val = 0.5 * float(np.sum((np.asarray(y, np.float64) - s) ** 2)) + prm.kappa * V
    if prm.lam > 0:
        val += prm.lam * float(np.sum(np.abs(s)))
    return val
