"""RPCA+UOT-DF with a signed sparse component S = S+ - S- (eq.
RPCA_UOTDF_PN, Sec. IV-B, the real-video experiment), Phi_t = I, FP64.

Test infrastructure only: the CUDA path never imports this module.

Where the foreground may be darker or lighter than the background, the
paper drops S >= 0, writes S = S+ - S- with S+, S- >= 0 and gives each part
its own transport term:
    min_{S+, S-, L >= 0}  1/2 sum_t ||y_t - (s+_t - s-_t + l_t)||^2
        + lambda (||S+||_1 + ||S-||_1) + gamma ||L||_*
        + kappa sum_{t<T} ( V_mu(s+_t, s+_{t+1}) + V_mu(s-_t, s-_{t+1}) ).
It prints no algorithm for this objective.  Reading: the ADMM of Algorithm 3
with its splitting applied to each sign,
    X = S+ - S- + L,  Tm = L,  z±_t = s±_t,  w±_{t+1} = s±_{t+1},
scaled duals A, D, b±, c±, and the blocks updated in Algorithm 3's order with
S+ before S- (each sees the other's latest value in the data-split term).
Each sign's update is the exact minimiser of the augmented Lagrangian over
that block, a separable quadratic plus lambda s over s >= 0, as Algorithm 3's
line 7 is:
    s+ <- max(k+ / sigma - lambda / (rho sigma), 0),
          k+ = (X - L + A + S-) + omega_z (z+ + b+) + omega_w (w+ + c+)
    s- <- max(k- / sigma - lambda / (rho sigma), 0),
          k- = (S+ - X + L - A) + omega_z (z- + b-) + omega_w (w- + c-)
(omega and sigma as in Algorithm 3: the frames with a pair after / before
them).  Then, with S = S+ - S-, lines 8-10 of Algorithm 3 unchanged, line 11
for each sign (two sets of T - 1 prox problems, warm-started), lines 12-15
for each sign.  The readings of Algorithm 3's own garbles (oracle.rpca) carry
over.  Stopping: Algorithm 3's residuals with the terms of both signs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import prox as P
from . import rpca as R
from . import svt as SV


@dataclass
class PnParams(R.RpcaParams):
    norm: str = "iso"           # flux norm of the inner prox ("aniso" for the LP pins)


@dataclass
class PnState:
    Sp: np.ndarray              # S+
    Sm: np.ndarray              # S-
    L: np.ndarray
    X: np.ndarray
    Tm: np.ndarray
    A: np.ndarray
    D: np.ndarray
    Bp: np.ndarray              # duals of z+ = s+_t, w+ = s+_{t+1}
    Cp: np.ndarray
    Bm: np.ndarray              # duals of z- = s-_t, w- = s-_{t+1}
    Cm: np.ndarray
    prox_p: P.ProxState         # z+ = prox_p.x0, w+ = prox_p.x1
    prox_m: P.ProxState
    history: list = field(default_factory=list)

    @property
    def S(self) -> np.ndarray:
        return self.Sp - self.Sm


def zero_state(T: int, H: int, W: int) -> PnState:
    f = np.zeros((T, H, W))
    g = np.zeros((T - 1, H, W))

    def prox_zero():
        return P.ProxState(g.copy(), g.copy(), g.copy(), g.copy(), g.copy(), g.copy())
    return PnState(f.copy(), f.copy(), f.copy(), f.copy(), f.copy(), f.copy(), f.copy(),
                   g.copy(), g.copy(), g.copy(), g.copy(), prox_zero(), prox_zero())


def prox_params(prm: PnParams, H: int, W: int) -> P.ProxParams:
    """Line 11 for either sign: prox^mu_{kappa/rho V} (prox weight kappa/rho)."""
    return P.default_steps(H, W, P.ProxParams(mu=prm.mu, rho=prm.kappa / prm.rho, mode="prox", norm=prm.norm))


def s_update(target: np.ndarray, z, b, w, c, lam: float, rho: float) -> np.ndarray:
    """Line 7 for one sign: the data-split target plus the OT copies of the
    pairs before (w + c) and after (z + b) each frame."""
    T, H, W = target.shape
    om_z = np.array([1.0] * (T - 1) + [0.0])[:, None, None]
    om_w = np.array([0.0] + [1.0] * (T - 1))[:, None, None]
    zb = np.concatenate([z + b, np.zeros((1, H, W))], axis=0)
    wc = np.concatenate([np.zeros((1, H, W)), w + c], axis=0)
    k = target + om_z * zb + om_w * wc
    sigma = 1.0 + om_z + om_w
    return np.maximum(k / sigma - lam / (rho * sigma), 0.0)


def outer_iteration(st: PnState, Y: np.ndarray, prm: PnParams) -> tuple[PnState, float, float]:
    T, H, W = Y.shape
    rho, lam = prm.rho, prm.lam
    zp, wp, zm, wm = st.prox_p.x0, st.prox_p.x1, st.prox_m.x0, st.prox_m.x1
    # line 7, S+ then S-
    Sp = s_update(st.X - st.L + st.A + st.Sm, zp, st.Bp, wp, st.Cp, lam, rho)
    Sm = s_update(Sp - st.X + st.L - st.A, zm, st.Bm, wm, st.Cm, lam, rho)
    S = Sp - Sm
    # lines 8-10 with S = S+ - S-
    L = 0.5 * np.maximum(st.Tm - st.D + st.X - S + st.A, 0.0)
    X = (Y + rho * (S + L - st.A)) / (1.0 + rho)
    N = H * W
    Tm = SV.svt((L + st.D).reshape(T, N).T, prm.gamma / rho).T.reshape(T, H, W)
    # line 11 for each sign
    pp = prox_params(prm, H, W)
    pst_p = P.iterate(Sp[:-1] - st.Bp, Sp[1:] - st.Cp, pp, prm.n_inner, state=st.prox_p)
    pst_m = P.iterate(Sm[:-1] - st.Bm, Sm[1:] - st.Cm, pp, prm.n_inner, state=st.prox_m)
    # lines 12-15 for each sign
    A = st.A + X - S - L
    D = st.D + L - Tm
    Bp = st.Bp + pst_p.x0 - Sp[:-1]
    Cp = st.Cp + pst_p.x1 - Sp[1:]
    Bm = st.Bm + pst_m.x0 - Sm[:-1]
    Cm = st.Cm + pst_m.x1 - Sm[1:]
    ny = max(np.sqrt(np.sum(Y.astype(np.float64) ** 2)), 1e-30)
    pri = np.sqrt(np.sum((X - S - L) ** 2) + np.sum((L - Tm) ** 2)
                  + np.sum((pst_p.x0 - Sp[:-1]) ** 2) + np.sum((pst_p.x1 - Sp[1:]) ** 2)
                  + np.sum((pst_m.x0 - Sm[:-1]) ** 2) + np.sum((pst_m.x1 - Sm[1:]) ** 2)) / ny
    dual = rho * np.sqrt(np.sum((X - st.X) ** 2) + np.sum((Tm - st.Tm) ** 2)
                         + np.sum((pst_p.x0 - zp) ** 2) + np.sum((pst_p.x1 - wp) ** 2)
                         + np.sum((pst_m.x0 - zm) ** 2) + np.sum((pst_m.x1 - wm) ** 2)) / ny
    new = PnState(Sp, Sm, L, X, Tm, A, D, Bp, Cp, Bm, Cm, pst_p, pst_m, st.history)
    return new, float(pri), float(dual)


def solve(Y: np.ndarray, prm: PnParams, state: PnState | None = None, max_iter: int | None = None):
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
