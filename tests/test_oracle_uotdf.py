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
from qp_pins import qp_prox_pairs


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


@pytest.mark.parametrize("lam,seed,rho", [(0.0, 0, 1.0), (0.1, 0, 1.0), (0.0, 3, 1.0),
                                          (0.1, 0, 0.4), (0.1, 0, 2.5), (0.0, 3, 0.4), (0.0, 3, 2.5)])
def test_admm_matches_independent_qp(lam, seed, rho):
    """At rho = 1 a misplaced rho (lambda / (2 rho) of line 4, the rho of
    line 5, the prox weight kappa / rho of line 6) would not show; the fixed
    point does not depend on rho, so the same QP pins rho = 0.4 and 2.5."""
    rng = np.random.default_rng(seed)
    H, W = 3, 3
    s0 = rng.uniform(0, 1, (H, W)) * (rng.uniform(size=(H, W)) < 0.6)
    y = np.roll(s0, 1, axis=1) * 1.2 + 0.05 * rng.normal(size=(H, W))
    s_qp = qp_uotdf(y, s0, 0.5, 1.0, lam)
    prm = U.UotdfParams(kappa=0.5, mu=1.0, rho=rho, lam=lam, n_inner=20, norm="aniso", tol=1e-10, max_iter=50000)
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


def uotdf_block_violations(rho, seed=6, n_inner=6000):
    """One iteration of Algorithm 2 from a random, unconverged state; returns
    the blocks whose output does not minimise its subproblem of the augmented
    Lagrangian lam sum s + i_+(s) + 1/2 ||y - x||^2 + kappa V(s0, z)
    + rho/2 ||x - s + a||^2 + rho/2 ||z - s + b||^2 (written out here)."""
    rng = np.random.default_rng(seed)
    B, H, W = 2, 2, 3
    s0 = rng.uniform(0, 1, (B, H, W)) * (rng.uniform(size=(B, H, W)) < 0.7)
    y = rng.uniform(0, 1.2, (B, H, W))
    st = U.zero_state(s0)
    st.x = rng.uniform(0, 1, (B, H, W))
    st.a = rng.normal(0, 0.3, (B, H, W))
    st.b = rng.normal(0, 0.3, (B, H, W))
    st.prox.x1[...] = rng.uniform(0, 1, (B, H, W))
    x_old, a_old, b_old, z_old = st.x.copy(), st.a.copy(), st.b.copy(), st.prox.x1.copy()
    prm = U.UotdfParams(kappa=0.5, mu=1.0, rho=rho, lam=0.1, n_inner=n_inner, norm="aniso")
    new, _, _ = U.iteration(st, y, s0, prm)
    fails = []
    # line 4: lam sum s + rho/2 ||x - s + a||^2 + rho/2 ||z - s + b||^2 over s >= 0
    s = new.s
    g = prm.lam - rho * (x_old - s + a_old) - rho * (z_old - s + b_old)
    if s.min() < 0 or np.max(np.abs(g[s > 0]), initial=0.0) > 1e-10 or np.min(g[s == 0], initial=np.inf) < -1e-10:
        fails.append("line 4 (s)")
    # line 5: 1/2 ||y - x||^2 + rho/2 ||x - s + a||^2
    if np.max(np.abs((new.x - y) + rho * (new.x - s + a_old))) > 1e-10:
        fails.append("line 5 (x)")
    # line 6: kappa V(s0, z) + rho/2 ||z - (s - b)||^2 over z >= 0, by the QP
    _, z_qp = qp_prox_pairs(None, s - b_old, prm.kappa, prm.mu, rho, s0=s0)
    if np.max(np.abs(new.z - z_qp)) > 1e-6:
        fails.append("line 6 (z)")
    active = (s > 0).any() and (s == 0).any()
    return fails, active


@pytest.mark.parametrize("rho", [1.0, 0.4, 2.5])
def test_blocks_minimise_the_augmented_lagrangian(rho):
    fails, active = uotdf_block_violations(rho)
    assert fails == [] and active


UOTDF_MUTANTS = {
    "line 4: lambda / 2": ("prox_R", lambda q, prm: np.maximum(q - prm.lam / 2.0, 0.0)),
    "line 4: printed rho / lambda": ("prox_R", lambda q, prm: np.maximum(q - prm.rho / prm.lam, 0.0)),
    "line 5: without rho": ("line5_x", lambda y, s, a, rho: (y + s - a) / (1.0 + rho)),
    "line 6: kappa": ("line6_weight", lambda prm: prm.kappa),
}


@pytest.mark.parametrize("name", list(UOTDF_MUTANTS))
def test_planted_mistakes_are_rejected(monkeypatch, name):
    """Each mistake is planted in the oracle (on the CPU); the block checks at
    rho = 2.5 must reject it."""
    attr, mutant = UOTDF_MUTANTS[name]
    monkeypatch.setattr(U, attr, mutant)
    fails, _ = uotdf_block_violations(2.5, n_inner=3000)
    assert fails, name
