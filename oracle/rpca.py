"""Algorithm 3 (RPCA+UOT-DF ADMM, Sec. IV-B.1) with Phi_t = I, FP64.

Frames are stored [T, H, W] (frame t = column t of the N x T matrices of the
paper).  Variables S, L, X, Tm (the paper's T), A, D are [T, H, W]; the OT
splitting variables z_t, w_{t+1} and their duals b_t, c_{t+1} are
[T-1, H, W] (entry t of Z, B pairs with entry t of W, C, i.e. frames t, t+1).
The T-1 prox problems of line 11 keep an Algorithm 1 state each (warm start,
``n_inner`` iterations per outer iteration, Sec. IV-B.2).

Readings where the printed algorithm is inconsistent with its own derivation:
  (i)   line 12: the augmented term ||X - S - L + A||^2 gives
        A <- A + X - S - L (the printed "+ L" is a sign slip);
  (ii)  line 9 with Phi = I: x_t = (y_t + rho (s_t + l_t - a_t)) / (1 + rho)
        (the printed line omits rho);
  (iii) line 7: S >= 0, so s_t = max(k_t / sigma_t - lambda / (rho sigma_t), 0);
  (v)   line 8: 1/2 inside or outside Pi_+ is the same.
Stopping (ADMM residuals of Boyd Sec. 3.3, relative to ||Y||):
  res_pri  = ||(X - S - L, L - Tm, z - s_t, w - s_{t+1})|| / ||Y||
  res_dual = rho ||(dX, dTm, dz, dw)|| / ||Y||
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import prox as P
from . import svt as SV


@dataclass
class RpcaParams:
    lam: float = 0.02
    gamma: float = 5.12
    kappa: float = 0.05
    mu: float = 3.0
    rho: float = 1.0
    n_inner: int = 1
    tol: float = 1e-5
    max_iter: int = 5000
    norm: str = "iso"           # flux norm of the inner prox ("aniso" for the LP/QP pins)


@dataclass
class RpcaState:
    S: np.ndarray
    L: np.ndarray
    X: np.ndarray
    Tm: np.ndarray
    A: np.ndarray
    D: np.ndarray
    B: np.ndarray
    C: np.ndarray
    prox: P.ProxState           # z = prox.x0, w = prox.x1 (the prox outputs)
    history: list = field(default_factory=list)


def zero_state(T: int, H: int, W: int) -> RpcaState:
    f = np.zeros((T, H, W))
    g = np.zeros((T - 1, H, W))
    return RpcaState(f.copy(), f.copy(), f.copy(), f.copy(), f.copy(), f.copy(), g.copy(), g.copy(),
                     P.ProxState(g.copy(), g.copy(), g.copy(), g.copy(), g.copy(), g.copy()))


def line7_s(k: np.ndarray, sigma: np.ndarray, lam: float, rho: float) -> np.ndarray:
    """Line 7: s_t minimises lambda sum(s) + (rho sigma_t / 2) ||s - k_t / sigma_t||^2
    over s >= 0 (the sigma_t augmented terms that contain s_t, collected)."""
    return np.maximum(k / sigma - lam / (rho * sigma), 0.0)


def line8_l(Tm: np.ndarray, D: np.ndarray, X: np.ndarray, S: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Line 8: L minimises rho/2 ||X - S - L + A||^2 + rho/2 ||L - Tm + D||^2
    over L >= 0 (the 1/2 outside or inside Pi_+ is the same)."""
    return 0.5 * np.maximum(Tm - D + X - S + A, 0.0)


def line9_x(Y: np.ndarray, S: np.ndarray, L: np.ndarray, A: np.ndarray, rho: float) -> np.ndarray:
    """Line 9 with Phi = I: X minimises 1/2 ||Y - X||^2 + rho/2 ||X - S - L + A||^2."""
    return (Y + rho * (S + L - A)) / (1.0 + rho)


def line10_theta(prm: RpcaParams) -> float:
    """Line 10: Tm minimises gamma ||Tm||_* + rho/2 ||L + D - Tm||^2, i.e. the
    SVT of L + D at gamma / rho."""
    return prm.gamma / prm.rho


def line11_weight(prm: RpcaParams) -> float:
    """Line 11: (z_t, w_{t+1}) minimise kappa V_mu(z, w) + rho/2 ||z - s_t + b_t||^2
    + rho/2 ||w - s_{t+1} + c_{t+1}||^2, the prox of eq. (Prox_UOT) with
    weight kappa / rho."""
    return prm.kappa / prm.rho


def line12_a(A: np.ndarray, X: np.ndarray, S: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Line 12: dual ascent on the constraint X - S - L = 0 of the augmented
    term ||X - S - L + A||^2 (the printed "+ L" is a sign slip)."""
    return A + X - S - L


def prox_params(prm: RpcaParams, H: int, W: int) -> P.ProxParams:
    """Line 11 evaluates prox^mu_{kappa/rho V}: the prox weight of eq.
    (Prox_UOT) is kappa / rho."""
    return P.default_steps(H, W, P.ProxParams(mu=prm.mu, rho=line11_weight(prm), mode="prox", norm=prm.norm))


def outer_iteration(st: RpcaState, Y: np.ndarray, prm: RpcaParams) -> tuple[RpcaState, float, float]:
    T, H, W = Y.shape
    rho, lam = prm.rho, prm.lam
    z, w = st.prox.x0, st.prox.x1
    # lines 4-7: omega, k_t, sigma_t, s_t
    om_z = np.array([1.0] * (T - 1) + [0.0])[:, None, None]
    om_w = np.array([0.0] + [1.0] * (T - 1))[:, None, None]
    zb = np.concatenate([z + st.B, np.zeros((1, H, W))], axis=0)     # z_t + b_t, t = 1..T-1
    wc = np.concatenate([np.zeros((1, H, W)), w + st.C], axis=0)     # w_t + c_t, t = 2..T
    k = (st.X - st.L + st.A) + om_z * zb + om_w * wc
    sigma = 1.0 + om_z + om_w
    S = line7_s(k, sigma, lam, rho)
    # line 8
    L = line8_l(st.Tm, st.D, st.X, S, st.A)
    # line 9 (Phi = I)
    X = line9_x(Y, S, L, st.A, rho)
    # line 10
    N = H * W
    Tm = SV.svt((L + st.D).reshape(T, N).T, line10_theta(prm)).T.reshape(T, H, W)
    # line 11: warm-started, n_inner Algorithm 1 iterations on the T-1 pairs
    pp = prox_params(prm, H, W)
    c0 = S[:-1] - st.B
    c1 = S[1:] - st.C
    pst = P.iterate(c0, c1, pp, prm.n_inner, state=st.prox)
    z_new, w_new = pst.x0, pst.x1
    # lines 12-15
    A = line12_a(st.A, X, S, L)
    D = st.D + L - Tm
    Bn = st.B + z_new - S[:-1]
    Cn = st.C + w_new - S[1:]
    ny = max(np.sqrt(np.sum(Y.astype(np.float64) ** 2)), 1e-30)
    pri = np.sqrt(np.sum((X - S - L) ** 2) + np.sum((L - Tm) ** 2)
                  + np.sum((z_new - S[:-1]) ** 2) + np.sum((w_new - S[1:]) ** 2)) / ny
    dual = rho * np.sqrt(np.sum((X - st.X) ** 2) + np.sum((Tm - st.Tm) ** 2)
                         + np.sum((z_new - z) ** 2) + np.sum((w_new - w) ** 2)) / ny
    new = RpcaState(S, L, X, Tm, A, D, Bn, Cn, pst, st.history)
    return new, float(pri), float(dual)


def solve(Y: np.ndarray, prm: RpcaParams, state: RpcaState | None = None, max_iter: int | None = None):
    Y = np.asarray(Y, np.float64)
    T, H, W = Y.shape
    st = zero_state(T, H, W) if state is None else state
    n = prm.max_iter if max_iter is None else max_iter
    pri = dual = np.inf
    for it in range(1, n + 1):
        st, pri, dual = outer_iteration(st, Y, prm)
        st.history.append((it, pri, dual))
        if max(pri, dual) <= prm.tol:
            return st, {"iters": it, "res_pri": pri, "res_dual": dual, "converged": True}
    return st, {"iters": n, "res_pri": pri, "res_dual": dual, "converged": False}
