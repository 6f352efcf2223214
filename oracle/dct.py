"""Orthonormal DCT-II and the Neumann-Laplacian solve it diagonalises (FP64).

The grid Laplacian D D* of Theorem 1 (zero-flux, i.e. Neumann, boundary) is a
Kronecker sum of two path-graph Laplacians.  The path-graph Laplacian on n
nodes has eigenvectors given by the DCT-II basis
    C[k, m] = s_k cos(pi (m + 1/2) k / n),  s_0 = sqrt(1/n),  s_k = sqrt(2/n),
with eigenvalues 4 sin^2(pi k / 2n).  Hence, for c >= 0,
    (D D* + c I)^{-1} X = C_H^T [ (C_H X C_W^T) / (lam_k + lam_l + c) ] C_W,
the zero mode (k = l = 0) being dropped when c = 0 (pseudo-inverse).

The transform is written out from its definition (matrix of cosines, direct
sums); no FFT is used.
"""
from __future__ import annotations

import numpy as np

from . import grid


def dct2_matrix(n: int) -> np.ndarray:
    """n x n orthonormal DCT-II matrix from its defining cosine sums."""
    C = np.zeros((n, n))
    for k in range(n):
        s = np.sqrt(1.0 / n) if k == 0 else np.sqrt(2.0 / n)
        for m in range(n):
            C[k, m] = s * np.cos(np.pi * (m + 0.5) * k / n)
    return C


def dct2(X: np.ndarray) -> np.ndarray:
    """2-D orthonormal DCT-II of [..., H, W]: C_H X C_W^T."""
    H, W = X.shape[-2:]
    return dct2_matrix(H) @ X @ dct2_matrix(W).T


def idct2(Y: np.ndarray) -> np.ndarray:
    """Inverse of ``dct2``: C_H^T Y C_W."""
    H, W = Y.shape[-2:]
    return dct2_matrix(H).T @ Y @ dct2_matrix(W)


def laplacian_spectrum(H: int, W: int) -> np.ndarray:
    """lam_k + lam_l on the H x W grid of DCT coefficients."""
    return grid.neumann_eigenvalues(H)[:, None] + grid.neumann_eigenvalues(W)[None, :]


def neumann_solve(X: np.ndarray, c: float) -> np.ndarray:
    """(D D* + c I)^{-1} X for c > 0; the pseudo-inverse (zero mean kept at 0)
    for c = 0."""
    H, W = X.shape[-2:]
    lam = laplacian_spectrum(H, W) + c
    Xh = dct2(np.asarray(X, np.float64))
    inv = np.where(lam > 0, 1.0 / np.where(lam > 0, lam, 1.0), 0.0)
    return idct2(Xh * inv)
