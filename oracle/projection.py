"""The prox of eq. (Prox_UOT) by ADMM with an exact projection (FP64).

Not an algorithm of the paper: the paper solves eq. (Prox_UOT) with the fully
explicit Algorithm 1.  This is a second solver of the *same* problem, whose
only linear-algebra step is the grid-Laplacian solve that the DCT-II
diagonalises (the identity behind Theorem 1's proof: K K^T = D D^T + c I,
c = number of identity blocks of K).  Its minimiser is the one of
eq. (Prox_UOT): x and the objective value are unique, so they are what the two
solvers are compared on.

Splitting: minimise f(z) + g(w) s.t. z = w, with
    z = (M, free x, r),
    f(z) = ||M||_{2,1} + mu ||r||_p^p + (1/2rho) ||x - p||^2 + i_+(x),
    g(w) = indicator of {K w = k0},  K w = D(M) + A x - r,
    k0   = p0 (if x0 frozen) - p1 (if x1 frozen).
Scaled ADMM with penalty beta:
    z <- prox_{f/beta}(w - u)        (separable shrinks and a clipped average)
    w <- (z + u) - K^T (K K^T)^{-1} (K (z + u) - k0)
    u <- u + z - w
Stopping: res_pri = ||K z - k0|| / s_p and res_fp = relative change of
(z, w, u), checked every ``check_every`` iterations, as for Algorithm 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dct, grid
from .prox import ProxParams, ProxState, frozen, n_identity_blocks, shrink_l1, shrink_l2


def _names(prm: ProxParams) -> list[str]:
    f0, f1 = frozen(prm.mode)
    n = ["Mx", "My"]
    if not f0:
        n.append("x0")
    if not f1:
        n.append("x1")
    if not prm.balanced:
        n.append("r")
    return n


# coefficient of each block in K: D for M, -1 for x0, +1 for x1, -1 for r
_SIGN = {"x0": -1.0, "x1": 1.0, "r": -1.0}


def K_apply(v: dict, prm: ProxParams) -> np.ndarray:
    k = grid.div(v["Mx"], v["My"])
    for n in ("x0", "x1", "r"):
        if n in v:
            k = k + _SIGN[n] * v[n]
    return k


def KT_apply(y: np.ndarray, names: list[str]) -> dict:
    gx, gy = grid.div_adj(y)
    out = {"Mx": gx, "My": gy}
    for n in names[2:]:
        out[n] = _SIGN[n] * y
    return out


def rhs(p0, p1, prm: ProxParams) -> np.ndarray:
    f0, f1 = frozen(prm.mode)
    k0 = np.zeros_like(np.asarray(p0, np.float64))
    if f0:
        k0 = k0 + p0
    if f1:
        k0 = k0 - p1
    return k0


def project(v: dict, k0: np.ndarray, prm: ProxParams) -> dict:
    """Euclidean projection onto {K w = k0} using (D D* + cI)^{-1} (DCT-II)."""
    names = list(v.keys())
    c = float(n_identity_blocks(prm))
    y = dct.neumann_solve(K_apply(v, prm) - k0, c)
    kt = KT_apply(y, names)
    return {n: v[n] - kt[n] for n in names}


def prox_f(v: dict, p0, p1, prm: ProxParams, beta: float) -> dict:
    """argmin_z f(z) + (beta/2) ||z - v||^2, block by block."""
    out = {}
    H, W = v["Mx"].shape[-2:]
    mx, my = grid.edge_masks(H, W)
    if prm.norm == "iso":
        Mx, My = shrink_l2(v["Mx"], v["My"], 1.0 / beta)
    else:
        Mx, My = shrink_l1(v["Mx"], 1.0 / beta), shrink_l1(v["My"], 1.0 / beta)
    out["Mx"], out["My"] = Mx * mx, My * my
    for n, p in (("x0", p0), ("x1", p1)):
        if n in v:
            out[n] = np.maximum((p + prm.rho * beta * v[n]) / (1.0 + prm.rho * beta), 0.0)
    if "r" in v:
        if prm.p_exp == 1:
            out["r"] = shrink_l1(v["r"], prm.mu / beta)
        else:
            out["r"] = v["r"] / (1.0 + 2.0 * prm.mu / beta)
    return out


@dataclass
class AdmmState:
    z: dict
    w: dict
    u: dict


def zero_admm_state(p0, prm: ProxParams) -> AdmmState:
    z0 = np.zeros(np.shape(p0))
    names = _names(prm)
    return AdmmState({n: z0.copy() for n in names}, {n: z0.copy() for n in names},
                     {n: z0.copy() for n in names})


def admm_iteration(st: AdmmState, p0, p1, prm: ProxParams, beta: float, k0) -> AdmmState:
    names = list(st.z.keys())
    z = prox_f({n: st.w[n] - st.u[n] for n in names}, p0, p1, prm, beta)
    w = project({n: z[n] + st.u[n] for n in names}, k0, prm)
    u = {n: st.u[n] + z[n] - w[n] for n in names}
    return AdmmState(z, w, u)


def to_prox_state(st: AdmmState, p0, p1, prm: ProxParams) -> ProxState:
    """The z iterate as an Algorithm 1 state (frozen x take their inputs; the
    dual a is not produced by this solver and is left at 0)."""
    z = st.z
    zero = np.zeros(np.shape(p0))
    return ProxState(z["Mx"], z["My"], z.get("x0", np.asarray(p0, np.float64)),
                     z.get("x1", np.asarray(p1, np.float64)), z.get("r", zero), zero.copy())


def solve(p0, p1, prm: ProxParams, beta: float = 1.0, state: AdmmState | None = None):
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    k0 = rhs(p0, p1, prm)
    st = zero_admm_state(p0, prm) if state is None else state
    sp = max(np.sqrt(np.sum(p0 ** 2) + np.sum(p1 ** 2)), 1e-30)
    info = {"iters": 0, "res_pri": np.inf, "res_fp": np.inf, "converged": False}
    for k in range(1, prm.max_iter + 1):
        new = admm_iteration(st, p0, p1, prm, beta, k0)
        if k % prm.check_every == 0 or k == prm.max_iter:
            rp = np.sqrt(np.sum((K_apply(new.z, prm) - k0) ** 2)) / sp
            d = sum(np.sum((getattr(new, f)[n] - getattr(st, f)[n]) ** 2)
                    for f in ("z", "w", "u") for n in new.z)
            nz = sum(np.sum(getattr(new, f)[n] ** 2) for f in ("z", "w", "u") for n in new.z)
            rf = np.sqrt(d) / max(np.sqrt(nz), 1e-30)
            info.update(iters=k, res_pri=float(rp), res_fp=float(rf))
            if max(rp, rf) <= prm.tol:
                info["converged"] = True
                return new, info
        st = new
    return st, info
