"""Pins of the Algorithm 2 oracle (UOT-DF / BPDN+UOT-DF with Phi = I).

The problem min_{s >= 0} 1/2 ||y - s||^2 + lambda sum(s) + kappa V_mu(s, s0)
is strongly convex in s, so its minimiser is unique.  It is solved here a
second, independent way: V_mu with the anisotropic flux norm equals the
unbalanced transport LP with Manhattan ground cost (pinned in
test_oracle_prox.py), which turns the whole problem into one convex QP over
(s, plan, mass defects), handed to SciPy's interior-point solver.
"""
import numpy as np
import pytest
from scipy.optimize import Bounds, LinearConstraint, minimize

from oracle import uotdf as U


def qp_uotdf(y, s0, kappa, mu, lam):
    """min 1/2 ||y - s||^2 + lam sum s + kappa (<P, C> + mu sum(u+ + u- + v+ + v-))
    s.t. P 1 - u+ + u- = s, P^T 1 - v+ + v- = s0, all variables >= 0."""
    H, W = y.shape
    n = H * W
    coords = np.array([(i, j) for i in range(H) for j in range(W)])
    C = np.abs(coords[:, None, :] - coords[None, :, :]).sum(-1).astype(float)
    nv = n + n * n + 4 * n
    lin = np.concatenate([lam * np.ones(n), kappa * C.ravel(), kappa * mu * np.ones(4 * n)])
    yv = y.ravel()
    Hm = np.zeros((nv, nv))
    Hm[:n, :n] = np.eye(n)

    def f(v):
        return 0.5 * np.sum((yv - v[:n]) ** 2) + lin @ v

    def g(v):
        gr = lin.copy()
        gr[:n] += v[:n] - yv
        return gr

    Aeq = np.zeros((2 * n, nv))
    o = n + n * n
    for i in range(n):
        Aeq[i, n + i * n:n + (i + 1) * n] = 1.0        # row sums of the plan
        Aeq[n + i, n + i:n + n * n:n] = 1.0            # column sums
    Aeq[:n, :n] = -np.eye(n)
    Aeq[:n, o:o + n] = -np.eye(n)
    Aeq[:n, o + n:o + 2 * n] = np.eye(n)
    Aeq[n:, o + 2 * n:o + 3 * n] = -np.eye(n)
    Aeq[n:, o + 3 * n:] = np.eye(n)
    beq = np.concatenate([np.zeros(n), s0.ravel()])
    res = minimize(f, np.full(nv, 0.01), jac=g, hess=lambda v: Hm, method="trust-constr",
                   constraints=[LinearConstraint(Aeq, beq, beq)], bounds=Bounds(np.zeros(nv), np.full(nv, np.inf)),
                   options={"gtol": 1e-12, "xtol": 1e-14, "barrier_tol": 1e-12, "maxiter": 20000})
    return res.x[:n].reshape(H, W)


@pytest.mark.parametrize("lam,seed", [(0.0, 0), (0.1, 0), (0.0, 3)])
def test_admm_matches_independent_qp(lam, seed):
    rng = np.random.default_rng(seed)
    H, W = 3, 3
    s0 = rng.uniform(0, 1, (H, W)) * (rng.uniform(size=(H, W)) < 0.6)
    y = np.roll(s0, 1, axis=1) * 1.2 + 0.05 * rng.normal(size=(H, W))
    s_qp = qp_uotdf(y, s0, 0.5, 1.0, lam)
    prm = U.UotdfParams(kappa=0.5, mu=1.0, rho=1.0, lam=lam, n_inner=20, norm="aniso", tol=1e-10, max_iter=50000)
    st, info = U.solve(y[None], s0[None], prm)
    assert info["converged"]
    assert np.max(np.abs(st.s[0] - s_qp)) <= 1e-5
    # the splitting variables agree at the fixed point
    assert np.max(np.abs(st.x - st.s)) <= 1e-8 and np.max(np.abs(st.z - st.s)) <= 1e-8


def test_prediction_equal_to_data_is_the_solution():
    """y = s0 >= 0: both terms vanish at s = s0."""
    rng = np.random.default_rng(5)
    s0 = rng.uniform(0, 1, (2, 6, 7)) * (rng.uniform(size=(2, 6, 7)) < 0.5)
    prm = U.UotdfParams(kappa=0.7, mu=2.0, rho=1.0, n_inner=5, tol=1e-9, max_iter=20000)
    st, info = U.solve(s0, s0, prm)
    assert info["converged"]
    assert np.max(np.abs(st.s - s0)) <= 1e-6


@pytest.mark.parametrize("lam", [0.0, 0.15])
def test_vanishing_kappa_reduces_to_the_nonnegative_lasso(lam):
    """kappa -> 0: argmin 1/2 ||y - s||^2 + lam sum s over s >= 0 is max(y - lam, 0)."""
    rng = np.random.default_rng(7)
    y = rng.normal(0.3, 0.5, (1, 8, 8))
    s0 = rng.uniform(0, 1, (1, 8, 8))
    prm = U.UotdfParams(kappa=1e-7, mu=1.0, rho=1.0, lam=lam, n_inner=3, tol=1e-10, max_iter=20000)
    st, info = U.solve(y, s0, prm)
    assert info["converged"]
    assert np.max(np.abs(st.s - np.maximum(y - lam, 0.0))) <= 1e-5


def test_printed_s_update_would_ignore_the_transport_term():
    """A guard on the reading of line 4: taking the prox at x + a alone (as
    printed) converges to Pi_+(y) whatever kappa is, which the QP rejects."""
    rng = np.random.default_rng(0)
    H, W = 3, 3
    s0 = rng.uniform(0, 1, (H, W)) * (rng.uniform(size=(H, W)) < 0.6)
    y = np.roll(s0, 1, axis=1) * 1.2 + 0.05 * rng.normal(size=(H, W))
    s_qp = qp_uotdf(y, s0, 0.5, 1.0, 0.0)
    assert np.max(np.abs(s_qp - np.maximum(y, 0.0))) > 0.1
