"""Singular-value thresholding (Algorithm 3 line 10, Sec. IV-B.1), FP64.

shrink*_theta(X) = U shrink^{l1}_theta(Sigma) V^T for any SVD X = U Sigma V^T.

The SVD is computed here by one-sided (Hestenes) Jacobi: plane rotations of
column pairs of X until all columns are mutually orthogonal; the column norms
are then the singular values and the accumulated rotations are V.  This is
deliberately a different route from the GPU's (Gram matrix + eigensolver).
"""
from __future__ import annotations

import numpy as np


def jacobi_svd(X: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Thin SVD of X (n x m, n >= m): returns U (n x m), s (m,), V (m x m),
    s sorted in decreasing order."""
    Uc = np.array(X, np.float64, copy=True)
    n, m = Uc.shape
    V = np.eye(m)
    for _ in range(max_sweeps):
        off = 0.0
        for p in range(m - 1):
            for q in range(p + 1, m):
                alpha = float(Uc[:, p] @ Uc[:, p])
                beta = float(Uc[:, q] @ Uc[:, q])
                gamma = float(Uc[:, p] @ Uc[:, q])
                if alpha == 0.0 or beta == 0.0:
                    continue
                c_rel = abs(gamma) / np.sqrt(alpha * beta)
                off = max(off, c_rel)
                if c_rel <= tol:
                    continue
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.sign(zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta)) if zeta != 0 else 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                up = Uc[:, p].copy()
                Uc[:, p] = c * up - s * Uc[:, q]
                Uc[:, q] = s * up + c * Uc[:, q]
                vp = V[:, p].copy()
                V[:, p] = c * vp - s * V[:, q]
                V[:, q] = s * vp + c * V[:, q]
        if off <= tol:
            break
    sv = np.sqrt(np.sum(Uc * Uc, axis=0))
    order = np.argsort(-sv)
    sv = sv[order]
    V = V[:, order]
    Uc = Uc[:, order]
    U = np.where(sv[None, :] > 0, Uc / np.where(sv > 0, sv, 1.0)[None, :], 0.0)
    return U, sv, V


def svt(X: np.ndarray, theta: float) -> np.ndarray:
    """shrink*_theta(X): singular values below theta are dropped, the others
    reduced by theta.  X is N x T (frames as columns)."""
    X = np.asarray(X, np.float64)
    tall = X.shape[0] >= X.shape[1]
    U, s, V = jacobi_svd(X if tall else X.T)
    s_new = np.maximum(s - theta, 0.0)
    Y = (U * s_new[None, :]) @ V.T
    return Y if tall else Y.T
