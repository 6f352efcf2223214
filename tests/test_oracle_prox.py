"""Pins of Algorithm 1 (oracle.prox) against closed forms, brute-force LPs and
the paper's own subproblem definitions (Sec. III-A/B).

Each pin is chosen so that a plausible slip in the oracle (a wrong sign in
D*, a dropped term in an update, the wrong rho convention, a transposed
stencil) breaks at least one of them.
"""
import numpy as np
import pytest
from scipy.optimize import linprog

from oracle import grid
from oracle import prox as P


def solve_eval(p0, p1, mu, norm="iso", balanced=False, tol=1e-11, max_iter=400000, check=50):
    prm = P.ProxParams(mu=mu, mode="eval", norm=norm, balanced=balanced, tol=tol,
                       max_iter=max_iter, check_every=check)
    st, info = P.solve(p0, p1, prm)
    prm = P.default_steps(*np.shape(p0)[-2:], prm)
    return st, info, prm


# ---------------------------------------------------------------- subproblems
def test_alg1_steps_minimise_the_paper_subproblems():
    """Lines 3-5 of Algorithm 1 are the minimisers of eqs. (Prox_UOT_M),
    (Prox_UOT_x), (Prox_UOT_r): check each by random perturbations of the
    subproblem objectives written with D itself (not D*)."""
    rng = np.random.default_rng(11)
    B, H, W = 1, 6, 7
    p0, p1 = rng.uniform(0, 1, (2, B, H, W))
    prm = P.default_steps(H, W, P.ProxParams(mu=0.3, rho=0.7))
    st = P.ProxState(*(rng.normal(size=(B, H, W)) for _ in range(6)))
    mx, my = grid.edge_masks(H, W)
    st.Mx *= mx
    st.My *= my
    new = P.alg1_iteration(st, p0, p1, prm)
    t1, rho, mu = prm.tau1, prm.rho, prm.mu

    def F_M(Mx, My):
        return (grid.l21(Mx, My) + np.sum(st.a * grid.div(Mx, My))
                + (np.sum((Mx - st.Mx) ** 2) + np.sum((My - st.My) ** 2)) / (2 * t1))

    def F_x(x0, x1):
        if np.any(x0 < 0) or np.any(x1 < 0):
            return np.inf
        return (np.sum((x0 - p0) ** 2 + (x1 - p1) ** 2) / (2 * rho) + np.sum(st.a * (-x0 + x1))
                + np.sum((x0 - st.x0) ** 2 + (x1 - st.x1) ** 2) / (2 * t1))

    def F_r(r):
        return mu * np.sum(np.abs(r)) + np.sum(st.a * (-r)) + np.sum((r - st.r) ** 2) / (2 * t1)

    fM, fx, fr = F_M(new.Mx, new.My), F_x(new.x0, new.x1), F_r(new.r)
    for s in (1e-2, 1e-4):
        for _ in range(60):
            dx, dy = rng.normal(size=(2, B, H, W)) * s
            assert F_M(new.Mx + dx * mx, new.My + dy * my) >= fM - 1e-12
            d0, d1 = rng.normal(size=(2, B, H, W)) * s
            assert F_x(np.maximum(new.x0 + d0, 0), np.maximum(new.x1 + d1, 0)) >= fx - 1e-12
            assert F_r(new.r + rng.normal(size=(B, H, W)) * s) >= fr - 1e-12
    # line 7: a^{k+1} = a^k + tau2 (2 K(z^{k+1}) - K(z^k)), K written out with D
    K_new = grid.div(new.Mx, new.My) - new.x0 + new.x1 - new.r
    K_old = grid.div(st.Mx, st.My) - st.x0 + st.x1 - st.r
    assert np.allclose(new.a, st.a + prm.tau2 * (2 * K_new - K_old), atol=1e-13)


def test_p2_r_step_minimises_its_subproblem():
    rng = np.random.default_rng(5)
    r0, a = rng.normal(size=(2, 1, 3, 4))
    prm = P.default_steps(3, 4, P.ProxParams(mu=0.8, p_exp=2))
    st = P.ProxState(np.zeros_like(r0), np.zeros_like(r0), np.zeros_like(r0), np.zeros_like(r0), r0, a)
    new = P.alg1_iteration(st, np.zeros_like(r0), np.zeros_like(r0), prm)
    # stationarity of mu r^2 - a r + (r - r0)^2 / (2 tau1)
    g = 2 * prm.mu * new.r - a + (new.r - r0) / prm.tau1
    assert np.max(np.abs(g)) <= 1e-12


def test_default_steps_satisfy_theorem1():
    for H, W in ((1, 5), (64, 64), (256, 256), (3, 1000)):
        prm = P.default_steps(H, W, P.ProxParams())
        assert prm.tau1 * prm.tau2 * (grid.lambda_max(H, W) + 3) < 1.0


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eval_1d_equals_cdf_l1(seed):
    """On a 1 x n grid with balanced masses and mu >= (n-1)/2 transport is never
    dearer than creation + destruction, and V_mu is the 1-D W1 distance:
    the l1 norm of the difference of the cumulative sums."""
    rng = np.random.default_rng(seed)
    n = 12
    p0 = np.zeros((1, 1, n))
    p1 = np.zeros((1, 1, n))
    p0[0, 0, rng.choice(n, 3, replace=False)] = rng.uniform(0.5, 1.0, 3)
    p1[0, 0, rng.choice(n, 4, replace=False)] = rng.uniform(0.5, 1.0, 4)
    p1 *= p0.sum() / p1.sum()
    closed = np.sum(np.abs(np.cumsum(p1[0, 0])[:-1] - np.cumsum(p0[0, 0])[:-1]))
    st, info, prm = solve_eval(p0, p1, mu=(n - 1) / 2 + 0.5)
    cert = P.certificate(st, p0, p1, prm)
    assert cert["dual"] - 1e-9 <= closed <= cert["primal"] + 1e-9
    assert abs(P.objective(st, p0, p1, prm) - closed) <= 1e-6 * closed


@pytest.mark.parametrize("d,mu,m0,m1", [(3, 10.0, 1.0, 1.0), (5, 1.5, 1.0, 1.0), (4, 10.0, 0.8, 0.5),
                                         (2, 0.6, 0.7, 1.0)])
def test_point_mass_cost(d, mu, m0, m1):
    """Mass m0 at (1, j) and m1 at (1, j + d): moving min(m0, m1) costs
    min(d, 2 mu) per unit and the surplus |m0 - m1| costs mu."""
    p0 = np.zeros((1, 3, 10))
    p1 = np.zeros((1, 3, 10))
    p0[0, 1, 2] = m0
    p1[0, 1, 2 + d] = m1
    closed = min(m0, m1) * min(d, 2 * mu) + mu * abs(m0 - m1)
    st, info, prm = solve_eval(p0, p1, mu=mu, tol=1e-12)
    cert = P.certificate(st, p0, p1, prm)
    assert cert["dual"] - 1e-8 <= closed <= cert["primal"] + 1e-8
    assert abs(P.objective(st, p0, p1, prm) - closed) <= 2e-6 * closed


def lp_unbalanced_manhattan(p, q, mu):
    """Eq. (Unbal_OT), p = 1, ground cost = Manhattan grid distance, as an LP:
    min <P, C> + mu (||P 1 - p||_1 + ||P^T 1 - q||_1), P >= 0 (HiGHS)."""
    H, W = p.shape
    n = H * W
    coords = np.array([(i, j) for i in range(H) for j in range(W)])
    C = np.abs(coords[:, None, :] - coords[None, :, :]).sum(-1).astype(float)
    # variables: P (n*n), u+ u- (n each), v+ v- (n each)
    nv = n * n + 4 * n
    c = np.concatenate([C.ravel(), mu * np.ones(4 * n)])
    Aeq = np.zeros((2 * n, nv))
    for i in range(n):
        Aeq[i, i * n:(i + 1) * n] = 1.0            # row sums
        Aeq[n + i, i:n * n:n] = 1.0                # column sums
    Aeq[:n, n * n:n * n + n] = -np.eye(n)
    Aeq[:n, n * n + n:n * n + 2 * n] = np.eye(n)
    Aeq[n:, n * n + 2 * n:n * n + 3 * n] = -np.eye(n)
    Aeq[n:, n * n + 3 * n:] = np.eye(n)
    beq = np.concatenate([p.ravel(), q.ravel()])
    res = linprog(c, A_eq=Aeq, b_eq=beq, bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("H,W,mu,seed", [(3, 3, 1.0, 0), (2, 4, 0.7, 1), (4, 4, 1.5, 2), (3, 4, 0.4, 3)])
def test_eval_aniso_equals_lp(H, W, mu, seed):
    """With the anisotropic flux norm, V_mu on the grid equals the unbalanced
    LP of eq. (Unbal_OT) (p = 1) with Manhattan ground cost; the isotropic
    value lies in [LP / sqrt(2), LP]."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0, 1, (H, W)) * (rng.uniform(size=(H, W)) < 0.6)
    q = rng.uniform(0, 1, (H, W)) * (rng.uniform(size=(H, W)) < 0.6)
    lp = lp_unbalanced_manhattan(p, q, mu)
    st, info, prm = solve_eval(p[None], q[None], mu=mu, norm="aniso", tol=1e-12)
    cert = P.certificate(st, p[None], q[None], prm)
    assert cert["dual"] - 1e-8 <= lp <= cert["primal"] + 1e-8
    assert abs(P.objective(st, p[None], q[None], prm) - lp) <= 1e-5 * max(lp, 1e-3)
    st_i, _, prm_i = solve_eval(p[None], q[None], mu=mu, norm="iso", tol=1e-10)
    v_iso = P.certificate(st_i, p[None], q[None], prm_i)
    assert lp / np.sqrt(2) - 1e-6 <= v_iso["dual"] and v_iso["dual"] <= lp + 1e-6


def test_balanced_limit():
    """Balanced masses and mu >= (H + W - 2) / 2: V_mu = W (the balanced
    Beckmann problem, eq. OT_beckman) -- the large-mu limit of Sec. III-A."""
    rng = np.random.default_rng(4)
    H, W = 5, 6
    p = rng.uniform(0, 1, (1, H, W))
    q = rng.uniform(0, 1, (1, H, W))
    q *= p.sum() / q.sum()
    mu = (H + W - 2) / 2 + 0.5
    st_u, _, prm_u = solve_eval(p, q, mu=mu, tol=1e-11)
    st_b, _, prm_b = solve_eval(p, q, mu=mu, balanced=True, tol=1e-11)
    vu = P.objective(st_u, p, q, prm_u)
    vb = P.objective(st_b, p, q, prm_b)
    assert abs(vu - vb) <= 1e-5 * vb
    assert np.max(np.abs(st_u.r)) <= 1e-6


# ---------------------------------------------------------------- prox special cases
def test_prox_identical_frames_is_identity():
    rng = np.random.default_rng(9)
    p = rng.uniform(0, 1, (2, 8, 9))
    st, info = P.solve(p, p, P.ProxParams(mu=2.0, rho=0.05, tol=1e-12, max_iter=20000))
    assert np.allclose(st.x0, p, atol=1e-9) and np.allclose(st.x1, p, atol=1e-9)
    assert np.max(np.abs(st.Mx)) <= 1e-9 and np.max(np.abs(st.r)) <= 1e-9


def test_prox_small_rho_keeps_x_near_p():
    rng = np.random.default_rng(10)
    p0, p1 = rng.uniform(0, 1, (2, 1, 8, 8))
    devs = []
    for rho in (1e-2, 1e-3, 1e-4):
        st, _ = P.solve(p0, p1, P.ProxParams(mu=1.0, rho=rho, tol=1e-10, max_iter=100000))
        devs.append(max(np.max(np.abs(st.x0 - p0)), np.max(np.abs(st.x1 - p1))))
    # |x - p| = rho |A^T a| <= rho * max|a| : shrinks linearly with rho
    assert devs[0] > devs[1] > devs[2]
    assert devs[2] <= 1e-4 * 2.0


@pytest.mark.parametrize("mode,balanced,p_exp", [("prox", False, 1), ("fixed_first", False, 1),
                                                  ("eval", False, 1), ("prox", True, 1), ("prox", False, 2)])
def test_duality_gap_nonnegative_and_vanishing(mode, balanced, p_exp):
    from synth import blob_pairs, rng_for
    p0, p1 = blob_pairs(rng_for(0, 3), 1, 20, 20)
    p0 = p0.astype(np.float64)
    p1 = p1.astype(np.float64)
    if balanced:
        p1 *= p0.sum() / p1.sum()
    prm = P.default_steps(20, 20, P.ProxParams(mu=3.0, rho=0.01, mode=mode, balanced=balanced,
                                               p_exp=p_exp, tol=1e-9,
                                               max_iter=20000 if mode == "eval" else 60000))
    st = P.zero_state(p0, p1, mode)
    gaps = []
    for k in range(1, prm.max_iter + 1):
        new = P.alg1_iteration(st, p0, p1, prm)
        if k % 500 == 0:
            c = P.certificate(new, p0, p1, prm)
            if c["gap_valid"]:
                gaps.append(c["gap"])
                assert c["gap"] >= -1e-9 * max(1.0, abs(c["primal"]))
            rp, rf = P.residuals(new, st, p0, p1, prm)
            if max(rp, rf) <= prm.tol:
                break
        st = new
    c = P.certificate(new, p0, p1, prm)
    if not balanced:
        # EVAL has no strongly convex term and converges sublinearly
        assert c["rel_gap"] <= (1e-4 if mode == "eval" else 1e-6)
        assert gaps[-1] <= max(1e-2 * gaps[0], 1e-9 * abs(c["primal"]))
    else:
        # balanced: the certificate needs K(z) = 0; check the constraint instead
        assert np.sqrt(np.sum(P.K_op(new, prm) ** 2)) <= 1e-7 * np.sqrt(np.sum(p0 ** 2))


def test_fixed_first_small_rho_tends_to_eval():
    """prox_{rho V_s}(p) with rho -> 0 returns x -> p and the objective -> V(s, p)."""
    rng = np.random.default_rng(12)
    s = rng.uniform(0, 1, (1, 5, 5))
    p = rng.uniform(0, 1, (1, 5, 5))
    st_e, _, prm_e = solve_eval(s, p, mu=1.0, tol=1e-11)
    ve = P.objective(st_e, s, p, prm_e)
    st_f, _ = P.solve(s, p, P.ProxParams(mu=1.0, rho=1e-5, mode="fixed_first", tol=1e-12, max_iter=400000))
    prm_f = P.default_steps(5, 5, P.ProxParams(mu=1.0, rho=1e-5, mode="fixed_first"))
    assert np.max(np.abs(st_f.x1 - p)) <= 1e-4
    assert abs(P.objective(st_f, s, p, prm_f) - ve) <= 1e-3 * ve
