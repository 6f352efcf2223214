"""Pins of the grid operators, spectrum and DCT-II (oracle.grid, oracle.dct).

Sec. III-A defines D; Theorem 1 uses the spectrum of D D*.  Each check is
against something the oracle does not compute itself: the inner-product
definition of an adjoint, exact integer arithmetic, a LAPACK eigensolver on
the explicitly assembled matrix, and scipy's DCT.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import dct, grid

SHAPES = [(1, 1), (1, 7), (6, 1), (3, 5), (4, 4), (7, 10)]


def dense_laplacian(H, W):
    """Assemble D D* column by column from the operators."""
    n = H * W
    Lm = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        gx, gy = grid.div_adj(e.reshape(H, W))
        Lm[:, k] = grid.div(gx, gy).ravel()
    return Lm


@pytest.mark.parametrize("H,W", SHAPES)
def test_adjoint_identity(H, W):
    rng = np.random.default_rng(H * 100 + W)
    for _ in range(5):
        Mx, My, a = rng.normal(size=(3, 2, H, W))
        lhs = np.sum(grid.div(Mx, My) * a)
        gx, gy = grid.div_adj(a)
        rhs = np.sum(Mx * gx + My * gy)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("H,W", SHAPES)
def test_mass_conservation_exact(H, W):
    rng = np.random.default_rng(7)
    Mx = rng.integers(-50, 50, size=(H, W)).astype(np.float64)
    My = rng.integers(-50, 50, size=(H, W)).astype(np.float64)
    assert np.sum(grid.div(Mx, My)) == 0.0


def test_divergence_stencil_by_hand():
    # one unit of flux on the edge (1,2)-(2,2): source at (1,2), sink at (2,2)
    Mx = np.zeros((4, 5))
    My = np.zeros((4, 5))
    Mx[1, 2] = 1.0
    d = grid.div(Mx, My)
    assert d[1, 2] == 1.0 and d[2, 2] == -1.0 and np.count_nonzero(d) == 2
    # flux on a boundary slot that does not exist is ignored (zero flux)
    Mx2 = np.zeros((4, 5))
    Mx2[3, 0] = 5.0
    assert np.count_nonzero(grid.div(Mx2, My)) == 0


@pytest.mark.parametrize("H,W", SHAPES)
def test_laplacian_spectrum_closed_form(H, W):
    Lm = dense_laplacian(H, W)
    assert np.allclose(Lm, Lm.T, atol=0)
    ev = np.linalg.eigvalsh(Lm)
    closed = np.sort((grid.neumann_eigenvalues(H)[:, None] + grid.neumann_eigenvalues(W)[None, :]).ravel())
    assert np.allclose(ev, closed, atol=1e-10)
    assert abs(grid.lambda_max(H, W) - ev[-1]) <= 1e-10
    assert grid.lambda_max(H, W) < 8.0


@pytest.mark.parametrize("n", [1, 2, 5, 8, 17])
def test_dct_matrix_matches_scipy(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=(n, 3))
    ours = dct.dct2_matrix(n) @ x
    ref = scipy.fft.dct(x, type=2, norm="ortho", axis=0)
    assert np.allclose(ours, ref, atol=1e-13)
    C = dct.dct2_matrix(n)
    assert np.allclose(C @ C.T, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("H,W", [(3, 5), (4, 4), (6, 3)])
def test_dct_diagonalises_laplacian(H, W):
    Lm = dense_laplacian(H, W)
    CH, CW = dct.dct2_matrix(H), dct.dct2_matrix(W)
    Ckron = np.kron(CH, CW)              # row-major vectorisation of C_H X C_W^T
    lam = dct.laplacian_spectrum(H, W).ravel()
    assert np.allclose(Ckron.T @ np.diag(lam) @ Ckron, Lm, atol=1e-12)
    assert np.allclose(dct.dct2(np.eye(H * W)[0].reshape(H, W)).ravel(),
                       scipy.fft.dctn(np.eye(H * W)[0].reshape(H, W), type=2, norm="ortho").ravel(), atol=1e-13)


@pytest.mark.parametrize("c", [3.0, 2.0, 1.0, 0.0])
@pytest.mark.parametrize("H,W", [(1, 9), (5, 7), (8, 8)])
def test_neumann_solve_residual(H, W, c):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(2, H, W))
    if c == 0.0:
        X -= X.mean(axis=(-2, -1), keepdims=True)     # range of the singular operator
    Y = dct.neumann_solve(X, c)
    gx, gy = grid.div_adj(Y)
    R = grid.div(gx, gy) + c * Y - X
    assert np.max(np.abs(R)) <= 1e-12 * max(1.0, np.max(np.abs(X)))
    if c == 0.0:
        assert np.max(np.abs(Y.mean(axis=(-2, -1)))) <= 1e-13
