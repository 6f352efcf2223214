"""Grid operators of the Beckmann formulation (Sec. III-A) in float64.

Layout: arrays are [..., H, W]; paper index i (the "x" direction) is the row,
j ("y") is the column.  The flux field M is stored as two planes Mx, My.

Zero-flux boundary (reading of Sec. III-A): flux lives on the edges between
grid points.  Mx[i, j] carries mass between (i, j) and (i+1, j), so it exists
for i < H-1; My[i, j] carries mass between (i, j) and (i, j+1), so it exists
for j < W-1.  The slots Mx[H-1, :] and My[:, W-1] are identically zero.  With
this reading sum(D(M)) = 0 for every M (no mass leaves the grid) and D D* is
the Neumann graph Laplacian that Theorem 1's proof relies on.
"""
from __future__ import annotations

import numpy as np


def edge_masks(H: int, W: int) -> tuple[np.ndarray, np.ndarray]:
    """1 where an edge flux exists, 0 on the outer slots Mx[H-1,:], My[:,W-1]."""
    mx = np.ones((H, W))
    my = np.ones((H, W))
    mx[H - 1, :] = 0.0
    my[:, W - 1] = 0.0
    return mx, my


def div(Mx: np.ndarray, My: np.ndarray) -> np.ndarray:
    """Divergence D(M)[i,j] = (Mx[i,j] - Mx[i-1,j]) + (My[i,j] - My[i,j-1]),
    with zero flux outside the support (Sec. III-A)."""
    H, W = Mx.shape[-2:]
    mx, my = edge_masks(H, W)
    Mx = Mx * mx
    My = My * my
    out = np.zeros(np.broadcast_shapes(Mx.shape, My.shape))
    for i in range(H):
        out[..., i, :] += Mx[..., i, :]
        if i > 0:
            out[..., i, :] -= Mx[..., i - 1, :]
    for j in range(W):
        out[..., :, j] += My[..., :, j]
        if j > 0:
            out[..., :, j] -= My[..., :, j - 1]
    return out


def div_adj(a: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Adjoint D* of ``div`` (used in eq. Prox_UOT_M_prox):
    (D*a)_x[i,j] = a[i,j] - a[i+1,j] for i < H-1, (D*a)_y[i,j] = a[i,j] - a[i,j+1]
    for j < W-1, and 0 on the slots where no edge exists."""
    H, W = a.shape[-2:]
    gx = np.zeros_like(a, dtype=np.float64)
    gy = np.zeros_like(a, dtype=np.float64)
    for i in range(H - 1):
        gx[..., i, :] = a[..., i, :] - a[..., i + 1, :]
    for j in range(W - 1):
        gy[..., :, j] = a[..., :, j] - a[..., :, j + 1]
    return gx, gy


def l21(Mx: np.ndarray, My: np.ndarray, norm: str = "iso") -> float:
    """||M||_{2,1} = sum_ij sqrt(Mx^2 + My^2) (Sec. III-A); ``aniso`` is the
    l1 variant sum |Mx| + |My| used only for the LP pins."""
    if norm == "iso":
        return float(np.sum(np.sqrt(Mx * Mx + My * My)))
    return float(np.sum(np.abs(Mx)) + np.sum(np.abs(My)))


def neumann_eigenvalues(n: int) -> np.ndarray:
    """Eigenvalues 4 sin^2(pi k / 2n), k = 0..n-1, of the 1-D Neumann Laplacian
    (path graph on n nodes)."""
    k = np.arange(n, dtype=np.float64)
    return 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2


def lambda_max(H: int, W: int) -> float:
    """Largest eigenvalue of the grid Laplacian D D* (Theorem 1):
    4 sin^2(pi (H-1) / 2H) + 4 sin^2(pi (W-1) / 2W)."""
    return float(neumann_eigenvalues(H)[-1] + neumann_eigenvalues(W)[-1])
