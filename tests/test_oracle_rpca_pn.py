"""Pins of the signed-foreground RPCA+UOT-DF oracle (eq. RPCA_UOTDF_PN, Phi = I).

The oracle's ADMM is a reading (the paper prints only the objective), so it
is pinned against the objective itself, solved other ways:
  * with gamma large the low-rank part vanishes (L = 0), and with the
    anisotropic flux norm V_mu is the unbalanced transport LP with Manhattan
    cost (pinned in test_oracle_prox.py), so the whole problem is one convex
    QP over (S+, S-, a plan and mass defects per frame pair and sign), given
    to SciPy's interior-point solver.  The data term is strictly convex in
    S = S+ - S-, so S is unique;
  * kappa -> 0 with L = 0 leaves min 1/2 ||y - S||^2 + lambda ||S||_1, whose
    minimiser is the signed soft threshold of y;
  * with L = 0 the objective is symmetric under y -> -y, S+ <-> S-, so the
    minimiser's S changes sign with y;
  * at convergence the splitting constraints and the data-term optimality
    (y - X = rho A) hold, and the low-rank block's (A = D where L > 0,
    A <= D where L = 0);
  * each sign's update is the exact minimiser, over its block, of the
    augmented Lagrangian of the splitting (written out in the test from the
    objective and the constraints X = S+ - S- + L, z = s_t, w = s_{t+1}),
    with S- seeing the new S+: checked element-wise by its optimality
    conditions on a random, unconverged state.
"""
import numpy as np
import pytest
from scipy.optimize import Bounds, LinearConstraint, minimize

from oracle import rpca_pn as PN


def qp_pn(Y, kappa, mu, lam):
    """min 1/2 sum_t ||y_t - s+_t + s-_t||^2 + lam sum (s+ + s-)
         + kappa sum_{sign, t} (<P, C> + mu sum(u+ + u- + v+ + v-))
    s.t. P 1 - u+ + u- = s_t, P^T 1 - v+ + v- = s_{t+1} (per sign and pair),
    all variables >= 0.  Returns S = S+ - S-."""
    T, H, W = Y.shape
    n = H * W
    coords = np.array([(i, j) for i in range(H) for j in range(W)])
    C = np.abs(coords[:, None, :] - coords[None, :, :]).sum(-1).astype(float).ravel()
    npair = n * n + 4 * n
    nsign = T * n + (T - 1) * npair
    nv = 2 * nsign
    lin = np.zeros(nv)
    for g in range(2):
        o = g * nsign
        lin[o:o + T * n] = lam
        for t in range(T - 1):
            q = o + T * n + t * npair
            lin[q:q + n * n] = kappa * C
            lin[q + n * n:q + npair] = kappa * mu
    yv = Y.reshape(T * n)
    Hm = np.zeros((nv, nv))
    I = np.eye(T * n)
    Hm[:T * n, :T * n] = I
    Hm[nsign:nsign + T * n, nsign:nsign + T * n] = I
    Hm[:T * n, nsign:nsign + T * n] = -I
    Hm[nsign:nsign + T * n, :T * n] = -I

    def resid(v):
        return yv - v[:T * n] + v[nsign:nsign + T * n]

    def f(v):
        return 0.5 * np.sum(resid(v) ** 2) + lin @ v

    def grad(v):
        g = lin.copy()
        r = resid(v)
        g[:T * n] -= r
        g[nsign:nsign + T * n] += r
        return g

    rows = []
    for g in range(2):
        o = g * nsign
        for t in range(T - 1):
            q = o + T * n + t * npair
            u = q + n * n
            for side in range(2):                      # row sums vs frame t, column sums vs frame t + 1
                A = np.zeros((n, nv))
                for i in range(n):
                    if side == 0:
                        A[i, q + i * n:q + (i + 1) * n] = 1.0
                    else:
                        A[i, q + i:q + n * n:n] = 1.0
                f0 = o + (t + side) * n
                A[:, f0:f0 + n] -= np.eye(n)
                A[:, u + 2 * side * n:u + (2 * side + 1) * n] -= np.eye(n)      # excess   (u+ / v+)
                A[:, u + (2 * side + 1) * n:u + (2 * side + 2) * n] += np.eye(n)  # shortfall (u- / v-)
                rows.append(A)
    Aeq = np.concatenate(rows)
    res = minimize(f, np.full(nv, 0.01), jac=grad, hess=lambda v: Hm, method="trust-constr",
                   constraints=[LinearConstraint(Aeq, 0.0, 0.0)], bounds=Bounds(np.zeros(nv), np.full(nv, np.inf)),
                   options={"gtol": 1e-12, "xtol": 1e-14, "barrier_tol": 1e-12, "maxiter": 20000})
    v = res.x
    return (v[:T * n] - v[nsign:nsign + T * n]).reshape(T, H, W)


def signed_video(seed, T, H, W, noise=0.03):
    """A bright and a dark spot moving one pixel a frame, plus noise."""
    rng = np.random.default_rng(seed)
    Y = noise * rng.normal(size=(T, H, W))
    for t in range(T):
        Y[t, 0, t % W] += 1.0
        Y[t, H - 1, (W - 1 - t) % W] -= 0.8
    return Y


def pn_params(**kw):
    base = dict(lam=0.05, gamma=1e6, kappa=0.5, mu=1.0, rho=1.0, n_inner=20, tol=1e-10, max_iter=50000)
    base.update(kw)
    return PN.PnParams(**base)


def test_admm_matches_independent_qp():
    Y = signed_video(0, T=3, H=2, W=3)
    S_qp = qp_pn(Y, kappa=0.5, mu=1.0, lam=0.05)
    st, info = PN.solve(Y, pn_params(norm="aniso"))
    assert info["converged"], info
    assert np.max(np.abs(st.L)) <= 1e-8
    assert np.max(np.abs(st.S - S_qp)) <= 1e-5, np.max(np.abs(st.S - S_qp))
    # both signs are used: the dark spot lands in S-
    assert st.Sm.max() > 0.3 and st.Sp.max() > 0.3


def test_vanishing_kappa_gives_the_signed_soft_threshold():
    Y = signed_video(1, T=4, H=6, W=5, noise=0.2)
    lam = 0.1
    st, info = PN.solve(Y, pn_params(kappa=1e-7, lam=lam, n_inner=3, max_iter=20000))
    assert info["converged"], info
    soft = np.sign(Y) * np.maximum(np.abs(Y) - lam, 0.0)
    assert np.max(np.abs(st.S - soft)) <= 1e-5
    assert np.max(np.abs(st.Sp - np.maximum(Y - lam, 0.0))) <= 1e-5
    assert np.max(np.abs(st.Sm - np.maximum(-Y - lam, 0.0))) <= 1e-5


def test_sign_of_the_data_flips_the_sign_of_S():
    Y = signed_video(2, T=4, H=6, W=6)
    prm = pn_params(kappa=0.3, mu=2.0, n_inner=5, tol=1e-9, max_iter=40000)
    st1, i1 = PN.solve(Y, prm)
    st2, i2 = PN.solve(-Y, prm)
    assert i1["converged"] and i2["converged"]
    assert np.max(np.abs(st1.S + st2.S)) <= 1e-6, np.max(np.abs(st1.S + st2.S))


@pytest.mark.parametrize("gamma", [1e6, 0.5])
def test_fixed_point_conditions(gamma):
    """At the fixed point the splitting constraints hold and y - X = rho A
    (line 9 with X = S + L); with a finite gamma the low-rank part is used."""
    rng = np.random.default_rng(3)
    T, H, W = 5, 6, 6
    bg = np.outer(rng.uniform(0.2, 1.0, T), rng.uniform(0, 1, H * W)).reshape(T, H, W)
    Y = signed_video(3, T, H, W) + bg
    prm = pn_params(gamma=gamma, kappa=0.3, mu=2.0, n_inner=5, tol=1e-9, max_iter=40000)
    st, info = PN.solve(Y, prm)
    assert info["converged"], info
    assert np.max(np.abs(st.X - st.S - st.L)) <= 1e-7
    assert np.max(np.abs(st.L - st.Tm)) <= 1e-7
    for sgn, pst in ((st.Sp, st.prox_p), (st.Sm, st.prox_m)):
        assert np.max(np.abs(pst.x0 - sgn[:-1])) <= 1e-7 and np.max(np.abs(pst.x1 - sgn[1:])) <= 1e-7
    assert np.max(np.abs(Y - st.X - prm.rho * st.A)) <= 1e-7
    assert st.Sp.min() >= 0 and st.Sm.min() >= 0 and st.L.min() >= 0
    # the L block: 0 in rho (D - A) + N_{L >= 0}(L) at X = S + L, Tm = L
    on = st.L > 1e-6
    if on.any():
        assert np.max(np.abs((st.A - st.D)[on])) <= 1e-6
    assert np.max((st.A - st.D)[~on], initial=-np.inf) <= 1e-6
    if gamma < 1:
        assert np.linalg.norm(st.L) > 0.1 * np.linalg.norm(bg)


def test_sign_updates_minimise_the_augmented_lagrangian():
    """One outer iteration from a random state: S+ minimises
        lambda sum S+ + rho/2 ||X - S+ + S- - L + A||^2
        + rho/2 ||z+ - S+_{1..T-1} + b+||^2 + rho/2 ||w+ - S+_{2..T} + c+||^2
    over S+ >= 0 (S-, X, L, A at their previous values), and S- minimises the
    same with the signs' roles swapped and S+ at its new value.  For these
    separable convex quadratics: gradient 0 where the minimiser is positive,
    gradient >= 0 where it is 0."""
    rng = np.random.default_rng(4)
    T, H, W = 4, 5, 6
    st = PN.zero_state(T, H, W)
    for name in ("Sp", "Sm", "L"):
        setattr(st, name, rng.uniform(0, 1, (T, H, W)) * (rng.uniform(size=(T, H, W)) < 0.5))
    for name in ("X", "Tm", "A", "D"):
        setattr(st, name, rng.normal(0, 0.5, (T, H, W)))
    for name in ("Bp", "Cp", "Bm", "Cm"):
        setattr(st, name, rng.normal(0, 0.3, (T - 1, H, W)))
    for pst in (st.prox_p, st.prox_m):
        pst.x0[...] = rng.uniform(0, 1, (T - 1, H, W))
        pst.x1[...] = rng.uniform(0, 1, (T - 1, H, W))
    old = PN.PnState(*(getattr(st, f).copy() for f in ("Sp", "Sm", "L", "X", "Tm", "A", "D", "Bp", "Cp", "Bm", "Cm")),
                     st.prox_p.copy(), st.prox_m.copy())
    prm = pn_params(lam=0.07, rho=1.3, gamma=0.4, kappa=0.2)
    Y = rng.normal(0, 1, (T, H, W))
    new, _, _ = PN.outer_iteration(st, Y, prm)
    rho, lam = prm.rho, prm.lam

    def grad(Sx, data_resid, sign, z, b, w, c):
        """d/dS of lambda sum S + rho/2 ||data_resid||^2 (data_resid linear in
        S with coefficient -sign) + the two OT-copy terms."""
        g = lam - sign * rho * data_resid
        g[:-1] += -rho * (z - Sx[:-1] + b)
        g[1:] += -rho * (w - Sx[1:] + c)
        return g

    Sp = new.Sp
    gp = grad(Sp, old.X - Sp + old.Sm - old.L + old.A, 1.0, old.prox_p.x0, old.Bp, old.prox_p.x1, old.Cp)
    Sm = new.Sm
    gm = grad(Sm, old.X - Sp + Sm - old.L + old.A, -1.0, old.prox_m.x0, old.Bm, old.prox_m.x1, old.Cm)
    for S_, g_ in ((Sp, gp), (Sm, gm)):
        assert S_.min() >= 0
        assert np.max(np.abs(g_[S_ > 0])) <= 1e-10
        assert np.min(g_[S_ == 0]) >= -1e-10
        assert (S_ > 0).any() and (S_ == 0).any()
