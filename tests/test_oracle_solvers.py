"""Pins of the projection-form prox, the SVT and Algorithm 3 oracles.

* The projection-form ADMM and Algorithm 1 are two different algorithms for
  the one problem eq. (Prox_UOT); its minimiser x and its optimal value are
  unique, so they must agree.  Its projection is checked against the
  definition of a Euclidean projection (feasibility + orthogonality).
* The Jacobi SVD is checked against LAPACK; SVT against its defining property.
* Algorithm 3: the ADMM residuals vanish, and at the fixed point every
  splitting constraint holds and S, L obey their own optimality conditions.
"""
import numpy as np
import pytest

from oracle import grid, projection, rpca, svt
from oracle import prox as P
from synth import blob_pairs, rng_for, rpca_video


@pytest.mark.parametrize("mode", ["prox", "fixed_first", "eval"])
def test_projection_is_euclidean_projection(mode):
    rng = np.random.default_rng(1)
    H, W = 5, 6
    prm = P.ProxParams(mode=mode)
    p0, p1 = rng.uniform(0, 1, (2, 1, H, W))
    names = projection._names(prm)
    v = {n: rng.normal(size=(1, H, W)) for n in names}
    mx, my = grid.edge_masks(H, W)
    v["Mx"] *= mx
    v["My"] *= my
    k0 = projection.rhs(p0, p1, prm)
    w = projection.project(v, k0, prm)
    # feasible: D(M) + A x - r = k0, written out with the paper's operator
    Kw = grid.div(w["Mx"], w["My"]) - w.get("x0", 0) + w.get("x1", 0) - w.get("r", 0)
    assert np.max(np.abs(Kw - k0)) <= 1e-12
    # orthogonal: <v - w, u - w> = 0 for any other feasible u (u - w in ker K)
    for _ in range(5):
        d = {n: rng.normal(size=(1, H, W)) for n in names}
        d["Mx"] *= mx
        d["My"] *= my
        dker = projection.project(d, np.zeros_like(k0), prm)
        ip = sum(np.sum((v[n] - w[n]) * dker[n]) for n in names)
        assert abs(ip) <= 1e-11


@pytest.mark.parametrize("mode,balanced", [("prox", False), ("fixed_first", False), ("prox", True)])
def test_projection_form_matches_algorithm1(mode, balanced):
    """The flux M is not unique (equal-cost routes tie), so both iterations
    approach the solution set slowly at tight tolerance; they are compared
    after a fixed number of iterations on what is unique: the objective value
    and x."""
    p0, p1 = blob_pairs(rng_for(0, 5), 1, 10, 10, sigma=2.0, max_shift=2)
    p0 = p0.astype(np.float64)
    p1 = p1.astype(np.float64)
    if balanced:
        p1 *= p0.sum() / p1.sum()
    prm = P.ProxParams(mu=3.0, rho=0.01, mode=mode, balanced=balanced, tol=1e-12, max_iter=20000)
    st, info = P.solve(p0, p1, prm)
    prm_d = P.default_steps(10, 10, prm)
    prm_a = P.ProxParams(mu=3.0, rho=0.01, mode=mode, balanced=balanced, tol=1e-12, max_iter=5000)
    ast, ainfo = projection.solve(p0, p1, prm_a, beta=1.0)
    ps = projection.to_prox_state(ast, p0, p1, prm)
    v1 = P.objective(st, p0, p1, prm_d)
    v2 = P.objective(ps, p0, p1, prm_d)
    assert abs(v1 - v2) <= 1e-6 * abs(v1)
    assert np.max(np.abs(ps.x0 - st.x0)) <= 1e-5 and np.max(np.abs(ps.x1 - st.x1)) <= 1e-5
    assert ainfo["res_pri"] <= 1e-6


def test_jacobi_svd_matches_lapack():
    rng = np.random.default_rng(2)
    for n, m in ((40, 6), (200, 9), (7, 7)):
        X = rng.normal(size=(n, m))
        U, s, V = svt.jacobi_svd(X)
        assert np.allclose(s, np.linalg.svd(X, compute_uv=False), atol=1e-12 * s[0])
        assert np.allclose((U * s) @ V.T, X, atol=1e-12 * s[0])
        assert np.allclose(V.T @ V, np.eye(m), atol=1e-12)
        assert np.allclose(U.T @ U, np.eye(m), atol=1e-11)


def test_svt_shrinks_singular_values():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(300, 3)) @ np.diag([50.0, 30.0, 12.0]) @ rng.normal(size=(3, 10)) / 10
    X = A + 0.01 * rng.normal(size=A.shape)
    theta = 1.0
    s_in = np.linalg.svd(X, compute_uv=False)
    Y = svt.svt(X, theta)
    s_out = np.linalg.svd(Y, compute_uv=False)
    assert np.allclose(s_out, np.maximum(s_in - theta, 0), atol=1e-10)
    assert np.linalg.matrix_rank(Y, tol=1e-8) == int(np.sum(s_in > theta))
    # SVT is the prox of theta ||.||_*: X - Y lies in theta * subdifferential (spectral norm <= theta)
    assert np.linalg.norm(X - Y, 2) <= theta + 1e-10
    # wide input goes through the transpose route
    assert np.allclose(svt.svt(X.T, theta), Y.T, atol=1e-10)


def test_rpca_fixed_point_conditions():
    Y, L0, S0 = rpca_video(rng_for(1, 7), T=6, H=12, W=12, n_blobs=2)
    prm = rpca.RpcaParams(lam=0.02, gamma=0.02 * 12, kappa=0.005, mu=3.0, rho=1.0, tol=1e-7, max_iter=20000)
    st, info = rpca.solve(Y, prm)
    assert info["converged"], info
    Yd = Y.astype(np.float64)
    ny = np.linalg.norm(Yd)
    # splitting constraints of Sec. IV-B.1 hold at the fixed point
    assert np.linalg.norm(st.X - st.S - st.L) <= 1e-6 * ny
    assert np.linalg.norm(st.L - st.Tm) <= 1e-6 * ny
    assert np.linalg.norm(st.prox.x0 - st.S[:-1]) <= 1e-6 * ny
    assert np.linalg.norm(st.prox.x1 - st.S[1:]) <= 1e-6 * ny
    assert np.min(st.S) >= 0 and np.min(st.L) >= 0
    # data term: X minimises 1/2||Y - X||^2 + <A rho, X>: Y - X = rho A  (Phi = I)
    assert np.linalg.norm((Yd - st.X) - prm.rho * st.A) <= 1e-5 * ny
    # the low-rank part is the SVT of (L + D): ||L + D - Tm||_2 <= gamma / rho
    T, H, W = Y.shape
    R = (st.L + st.D - st.Tm).reshape(T, -1).T
    assert np.linalg.norm(R, 2) <= prm.gamma / prm.rho * (1 + 1e-8)
    # residual history decreases overall
    h = np.array([max(a, b) for _, a, b in st.history])
    assert h[-1] <= 1e-3 * h[0]
