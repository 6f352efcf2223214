"""Pins of the Algorithm 3 oracle (RPCA+UOT-DF, Phi = I, Sec. IV-B.1) with
rho away from 1.

At rho = 1 a rho in the wrong place (lambda / (rho sigma) of line 7, the
rho of line 9, gamma / rho of line 10, kappa / rho of line 11) changes
nothing, so every pin here runs at rho = 0.4 and 2.5 as well:

  * the whole solve against an independent QP: with gamma large the low-rank
    part is 0 and, with the anisotropic flux norm, Algorithm 3's objective is
    one convex QP over S, a transport plan and mass defects per frame pair
    (tests/qp_pins.py).  S is unique (strictly convex data term);
  * at a finite gamma, the converged state against the KKT conditions of
    the objective written out with the splitting's multipliers rho A, rho D,
    rho b, rho c: the splitting constraints, Y - X = rho A, the S block
    (lambda = rho (A + b + c) where S > 0, lambda >= that where S = 0), the L
    block (A = D where L > 0, A <= D where L = 0) and the nuclear-norm block
    (U^T D V = gamma / rho on the range of Tm, ||D||_2 <= gamma / rho);
  * one outer iteration from a random, unconverged state: each block's
    output against the optimality conditions of its own subproblem of the
    augmented Lagrangian, written out here from the objective and the
    constraints X = S + L, Tm = L, z = s_t, w = s_{t+1}; line 10 against
    LAPACK's SVD; line 11 against the independent QP of its prox problem;
  * planted mistakes: each rho misplaced in turn (and the printed sign of
    line 12) is put into the oracle here, on the CPU, and at least one of the
    checks above must reject it.
"""
import numpy as np
import pytest

from oracle import rpca as R
from qp_pins import qp_prox_pairs, qp_rpca_l0

RHOS = (0.4, 2.5)


def bright_video(seed, T, H, W, noise=0.03):
    """A spot moving one pixel a frame over a faint positive floor, plus noise."""
    rng = np.random.default_rng(seed)
    Y = 0.05 + noise * rng.normal(size=(T, H, W))
    for t in range(T):
        Y[t, t % H, (2 * t) % W] += 1.0
    return Y


# ---------------------------------------------------------------------------
# the whole solve against an independent QP (L = 0)

@pytest.mark.parametrize("rho", (1.0,) + RHOS)
def test_admm_matches_independent_qp(rho):
    Y = bright_video(0, T=3, H=2, W=3)
    kappa, mu, lam = 0.5, 1.0, 0.05
    S_qp = qp_rpca_l0(Y, kappa, mu, lam)
    prm = R.RpcaParams(lam=lam, gamma=1e6, kappa=kappa, mu=mu, rho=rho, n_inner=20, norm="aniso",
                       tol=1e-10, max_iter=50000)
    st, info = R.solve(Y, prm)
    assert info["converged"], info
    assert np.max(np.abs(st.Tm)) == 0.0 and np.max(np.abs(st.L)) <= 1e-8
    assert np.max(np.abs(st.S - S_qp)) <= 1e-5, np.max(np.abs(st.S - S_qp))
    # transport and the l1 term both act: S is neither Y's positive part nor 0
    assert np.max(np.abs(S_qp - np.maximum(Y - lam, 0))) > 1e-2 and S_qp.max() > 0.3


# ---------------------------------------------------------------------------
# KKT conditions of the converged state at a finite gamma

def kkt_violations(st, Y, prm, tol):
    """The converged ADMM state against the optimality conditions of
    Algorithm 3's objective; returns the names of the conditions that fail."""
    rho, lam, gamma = prm.rho, prm.lam, prm.gamma
    T, H, W = Y.shape
    ny = np.linalg.norm(Y)
    fails = []

    def check(name, ok):
        if not ok:
            fails.append(name)

    check("X = S + L", np.linalg.norm(st.X - st.S - st.L) <= tol * ny)
    check("Tm = L", np.linalg.norm(st.L - st.Tm) <= tol * ny)
    check("z = s_t", np.linalg.norm(st.prox.x0 - st.S[:-1]) <= tol * ny)
    check("w = s_t+1", np.linalg.norm(st.prox.x1 - st.S[1:]) <= tol * ny)
    check("S, L >= 0", st.S.min() >= 0 and st.L.min() >= 0)
    # X block: 0 = (X - Y) + rho A
    check("Y - X = rho A", np.linalg.norm(Y - st.X - rho * st.A) <= tol * ny)
    # S block: 0 in lambda - rho (A + b_t + c_{t-1}) + N_{S >= 0}
    g = lam - rho * st.A
    g[:-1] -= rho * st.B
    g[1:] -= rho * st.C
    on = st.S > 0
    scale = max(lam, 1e-30)
    check("S block, S > 0", np.max(np.abs(g[on]), initial=0.0) <= 1e3 * tol * scale)
    check("S block, S = 0", np.min(g[~on], initial=np.inf) >= -1e3 * tol * scale)
    # L block: 0 in rho (D - A) + N_{L >= 0}
    onl = st.L > 1e-6 * ny
    dscale = max(np.max(np.abs(st.D)), 1e-30)
    check("L block, L > 0", np.max(np.abs((st.A - st.D)[onl]), initial=0.0) <= 1e3 * tol * dscale)
    check("L block, L = 0", np.max((st.A - st.D)[~onl], initial=-np.inf) <= 1e3 * tol * dscale)
    # nuclear-norm block: rho D in gamma d||Tm||_* (frames as columns)
    Tmat = st.Tm.reshape(T, -1).T
    Dmat = st.D.reshape(T, -1).T
    U, s, Vt = np.linalg.svd(Tmat, full_matrices=False)
    r = int(np.sum(s > 1e-6 * max(s[0], 1e-30)))
    theta = gamma / rho
    check("||D||_2 <= gamma / rho", np.linalg.norm(Dmat, 2) <= theta * (1 + 1e3 * tol))
    if r:
        M = U[:, :r].T @ Dmat @ Vt[:r].T
        check("U^T D V = gamma / rho", np.max(np.abs(M - theta * np.eye(r))) <= 1e3 * tol * theta)
    return fails


def low_rank_video(seed, T, H, W):
    rng = np.random.default_rng(seed)
    bg = np.outer(rng.uniform(0.2, 1.0, T), rng.uniform(0, 1, H * W)).reshape(T, H, W)
    return bright_video(seed, T, H, W) + bg


def kkt_params(rho, **kw):
    base = dict(lam=0.05, gamma=1.0, kappa=0.3, mu=2.0, rho=rho, n_inner=5, tol=1e-9, max_iter=40000)
    base.update(kw)
    return R.RpcaParams(**base)


@pytest.mark.parametrize("rho", RHOS)
def test_converged_state_meets_the_kkt_conditions(rho):
    Y = low_rank_video(3, T=5, H=6, W=6)
    prm = kkt_params(rho)
    st, info = R.solve(Y, prm)
    assert info["converged"], info
    assert kkt_violations(st, Y, prm, 1e-7) == []
    # every block is active: low-rank part, foreground, and zeros in both
    assert np.linalg.norm(st.L) > 0.1 * np.linalg.norm(Y) and st.S.max() > 0.3
    assert (st.S == 0).any() and np.linalg.matrix_rank(st.Tm.reshape(5, -1), tol=1e-6) < 5


# ---------------------------------------------------------------------------
# every block of one outer iteration minimises its subproblem

def random_state(rng, T, H, W):
    st = R.zero_state(T, H, W)
    for name in ("S", "L"):
        setattr(st, name, rng.uniform(0, 1, (T, H, W)) * (rng.uniform(size=(T, H, W)) < 0.6))
    for name in ("X", "Tm", "A", "D"):
        setattr(st, name, rng.normal(0, 0.5, (T, H, W)))
    st.B = rng.normal(0, 0.3, (T - 1, H, W))
    st.C = rng.normal(0, 0.3, (T - 1, H, W))
    st.prox.x0[...] = rng.uniform(0, 1, (T - 1, H, W))
    st.prox.x1[...] = rng.uniform(0, 1, (T - 1, H, W))
    return st


def block_violations(rho, seed=4, n_inner=6000):
    """One outer iteration from a random state; returns the blocks whose
    output does not minimise its subproblem of the augmented Lagrangian."""
    rng = np.random.default_rng(seed)
    T, H, W = 3, 2, 3
    st = random_state(rng, T, H, W)
    old = R.RpcaState(*(getattr(st, f).copy() for f in ("S", "L", "X", "Tm", "A", "D", "B", "C")),
                      st.prox.copy())
    # gamma scales with rho so that the threshold gamma / rho = 1.4 splits the
    # singular values of L + D (about 1.74, 1.25, 1.04) at every rho
    prm = R.RpcaParams(lam=0.07, gamma=1.4 * rho, kappa=0.5, mu=1.0, rho=rho, n_inner=n_inner, norm="aniso")
    Y = rng.uniform(0, 1.5, (T, H, W))
    new, _, _ = R.outer_iteration(st, Y, prm)
    lam = prm.lam
    fails = []

    def nonneg_block(name, V, g, tol=1e-10):
        """0 in g + N_{V >= 0}: g = 0 where V > 0, g >= 0 where V = 0."""
        if V.min() < 0 or np.max(np.abs(g[V > 0]), initial=0.0) > tol or np.min(g[V == 0], initial=np.inf) < -tol:
            fails.append(name)

    # line 7: lambda sum S + rho/2 ||X - S - L + A||^2 + rho/2 ||z - s_t + b||^2 + rho/2 ||w - s_{t+1} + c||^2
    S = new.S
    g = lam - rho * (old.X - S - old.L + old.A)
    g[:-1] -= rho * (old.prox.x0 - S[:-1] + old.B)
    g[1:] -= rho * (old.prox.x1 - S[1:] + old.C)
    nonneg_block("line 7 (S)", S, g)
    # line 8: rho/2 ||X - S - L + A||^2 + rho/2 ||L - Tm + D||^2 over L >= 0
    L = new.L
    nonneg_block("line 8 (L)", L, -rho * (old.X - S - L + old.A) + rho * (L - old.Tm + old.D))
    # line 9: 1/2 ||Y - X||^2 + rho/2 ||X - S - L + A||^2
    gx = (new.X - Y) + rho * (new.X - S - L + old.A)
    if np.max(np.abs(gx)) > 1e-10:
        fails.append("line 9 (X)")
    # line 10: gamma ||Tm||_* + rho/2 ||L + D - Tm||^2, by LAPACK's SVD
    U, s, Vt = np.linalg.svd((L + old.D).reshape(T, -1).T, full_matrices=False)
    Tm_ref = ((U * np.maximum(s - prm.gamma / rho, 0.0)) @ Vt).T.reshape(T, H, W)
    if np.max(np.abs(new.Tm - Tm_ref)) > 1e-10:
        fails.append("line 10 (Tm)")
    # line 11: kappa V(z, w) + rho/2 ||z - (s_t - b)||^2 + rho/2 ||w - (s_{t+1} - c)||^2, by the QP
    z_qp, w_qp = qp_prox_pairs(S[:-1] - old.B, S[1:] - old.C, prm.kappa, prm.mu, rho)
    if max(np.max(np.abs(new.prox.x0 - z_qp)), np.max(np.abs(new.prox.x1 - w_qp))) > 1e-6:
        fails.append("line 11 (z, w)")
    # every block has both active and inactive entries (checked on the unmutated oracle)
    active = (S > 0).any() and (S == 0).any() and (L > 0).any() and (L == 0).any() \
        and 0 < np.sum(s > prm.gamma / rho) < len(s)
    return fails, active


@pytest.mark.parametrize("rho", (1.0,) + RHOS)
def test_blocks_minimise_the_augmented_lagrangian(rho):
    fails, active = block_violations(rho)
    assert fails == [] and active


# ---------------------------------------------------------------------------
# planted mistakes

MUTANTS = {
    "line 7: lambda / sigma": ("line7_s", lambda k, sigma, lam, rho: np.maximum(k / sigma - lam / sigma, 0.0)),
    "line 8: 1/2 dropped": ("line8_l", lambda Tm, D, X, S, A: np.maximum(Tm - D + X - S + A, 0.0)),
    "line 9: printed, without rho": ("line9_x", lambda Y, S, L, A, rho: (Y + S + L - A) / (1.0 + rho)),
    "line 10: gamma": ("line10_theta", lambda prm: prm.gamma),
    "line 11: kappa": ("line11_weight", lambda prm: prm.kappa),
    "line 11: kappa rho": ("line11_weight", lambda prm: prm.kappa * prm.rho),
    "line 12: printed + L": ("line12_a", lambda A, X, S, L: A + X - S + L),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistakes_are_rejected(monkeypatch, name):
    attr, mutant = MUTANTS[name]
    monkeypatch.setattr(R, attr, mutant)
    fails, _ = block_violations(2.5, n_inner=3000)
    if not fails:
        # a mistake outside the block updates (the dual ascent) shows at the fixed point
        Y = low_rank_video(3, T=4, H=4, W=4)
        prm = kkt_params(2.5, max_iter=4000)
        with np.errstate(all="ignore"):
            st, info = R.solve(Y, prm)
        fails = ["no convergence"] if not info["converged"] else kkt_violations(st, Y, prm, 1e-7)
    assert fails, name
