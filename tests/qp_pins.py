"""Independent convex programs behind the pins of the Algorithm 2 and 3 oracles.

With the anisotropic flux norm, V_mu is the unbalanced transport LP with
Manhattan ground cost (pinned against HiGHS in test_oracle_prox.py):

    V_mu(x0, x1) = min <P, C> + mu sum(u+ + u- + v+ + v-)
                   s.t.  P 1 - u+ + u- = x0,   P^T 1 - v+ + v- = x1,
                         P, u+-, v+- >= 0.

Every problem here is written out from its objective as one convex QP over
the densities, a plan and the mass defects of each frame pair, and handed to
SciPy's interior-point solver.  Nothing here imports the oracle.
"""
import numpy as np
from scipy.optimize import Bounds, LinearConstraint, minimize


def manhattan(H, W):
    coords = np.array([(i, j) for i in range(H) for j in range(W)])
    return np.abs(coords[:, None, :] - coords[None, :, :]).sum(-1).astype(float)


def solve_qp(Q, q, lin, Aeq, beq):
    """min 1/2 v^T Q v - q^T v + lin^T v  s.t.  Aeq v = beq, v >= 0."""
    nv = len(lin)

    def f(v):
        return 0.5 * v @ (Q @ v) - q @ v + lin @ v

    def g(v):
        return Q @ v - q + lin

    res = minimize(f, np.full(nv, 0.01), jac=g, hess=lambda v: Q, method="trust-constr",
                   constraints=[LinearConstraint(Aeq, beq, beq)], bounds=Bounds(np.zeros(nv), np.full(nv, np.inf)),
                   options={"gtol": 1e-12, "xtol": 1e-14, "barrier_tol": 1e-12, "maxiter": 20000})
    v = res.x
    # polish: an interior point stops a little inside the bounds.  First try
    # the active set it points to (entries near 0): the optimum then solves
    # the equality-constrained KKT system on the free entries exactly; where
    # the plan is not unique that system is singular, and an active-set SQP
    # (SLSQP) started from the interior point finishes the job instead
    for rel in (1e-6, 1e-7, 1e-8):
        free = v > rel * max(np.max(v), 1e-30)
        nf = int(free.sum())
        Af = Aeq[:, free]
        K = np.block([[Q[np.ix_(free, free)], Af.T], [Af, np.zeros((len(beq), len(beq)))]])
        rhs = np.concatenate([(q - lin)[free], beq])
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
        w = np.zeros(nv)
        w[free] = sol[:nf]
        if (w.min() >= -1e-12 and np.max(np.abs(Aeq @ w - beq)) <= 1e-11
                and np.max(np.abs(K @ sol - rhs)) <= 1e-10 and f(np.maximum(w, 0)) <= f(v) + 1e-13):
            return np.maximum(w, 0)
    r = minimize(f, v, jac=g, method="SLSQP", bounds=[(0, None)] * nv,
                 constraints=[{"type": "eq", "fun": lambda x: Aeq @ x - beq, "jac": lambda x: Aeq}],
                 options={"ftol": 1e-16, "maxiter": 2000})
    w = np.maximum(r.x, 0)
    if np.max(np.abs(Aeq @ w - beq)) <= 1e-11 and f(w) <= f(v):
        return w
    return v


class _Layout:
    """Column layout: density blocks of n entries, then per pair a plan
    (n x n) and four defect vectors (u+, u-, v+, v-)."""

    def __init__(self, n, n_dens, n_pairs):
        self.n, self.n_dens, self.n_pairs = n, n_dens, n_pairs
        self.pair_len = n * n + 4 * n
        self.nv = n_dens * n + n_pairs * self.pair_len

    def dens(self, i):
        return slice(i * self.n, (i + 1) * self.n)

    def pair(self, t):
        return self.n_dens * self.n + t * self.pair_len

    def transport_rows(self, t, first, second, kappa_cost, mu, lin, fixed=None):
        """Marginal rows of pair t between densities ``first`` and ``second``
        (an index into the density blocks, or None with the values given in
        ``fixed`` = (rhs_first, rhs_second)); fills the pair's costs into lin."""
        n = self.n
        q = self.pair(t)
        lin[q:q + n * n] = kappa_cost
        lin[q + n * n:q + self.pair_len] = mu
        rows, rhs = [], []
        for side, dens in enumerate((first, second)):
            A = np.zeros((n, self.nv))
            for i in range(n):
                if side == 0:
                    A[i, q + i * n:q + (i + 1) * n] = 1.0
                else:
                    A[i, q + i:q + n * n:n] = 1.0
            u = q + n * n + 2 * side * n
            A[:, u:u + n] -= np.eye(n)              # excess over the density
            A[:, u + n:u + 2 * n] += np.eye(n)      # shortfall
            if dens is None:
                rhs.append(np.asarray(fixed[side], float).ravel())
            else:
                A[:, self.dens(dens)] -= np.eye(n)
                rhs.append(np.zeros(n))
            rows.append(A)
        return rows, rhs


def qp_rpca_l0(Y, kappa, mu, lam):
    """Algorithm 3's objective with L = 0 and S >= 0 (eq. RPCA_UOTDF with
    Phi = I), anisotropic flux norm:
        min_{S >= 0} 1/2 ||Y - S||^2 + lam sum S + kappa sum_t V_mu(s_t, s_{t+1})."""
    T, H, W = Y.shape
    n = H * W
    lay = _Layout(n, T, T - 1)
    C = manhattan(H, W).ravel()
    lin = np.zeros(lay.nv)
    lin[:T * n] = lam
    Q = np.zeros((lay.nv, lay.nv))
    Q[:T * n, :T * n] = np.eye(T * n)
    q = np.zeros(lay.nv)
    q[:T * n] = Y.ravel()
    rows, rhs = [], []
    for t in range(T - 1):
        r, b = lay.transport_rows(t, t, t + 1, kappa * C, kappa * mu, lin)
        rows += r
        rhs += b
    v = solve_qp(Q, q, lin, np.concatenate(rows), np.concatenate(rhs))
    return v[:T * n].reshape(T, H, W)


def qp_prox_pairs(c0, c1, kappa, mu, rho, s0=None):
    """For every pair independently, the prox problem of Algorithm 3 line 11
    (or, with ``s0`` given, Algorithm 2 line 6, whose first argument is fixed):
        min_{z, w >= 0} kappa V_mu(z, w) + rho/2 ||z - c0||^2 + rho/2 ||w - c1||^2.
    Arrays are [B, H, W]; returns (z, w) (z = s0 when fixed)."""
    c0 = np.asarray(c0, float)
    c1 = np.asarray(c1, float)
    B, H, W = c1.shape
    n = H * W
    C = manhattan(H, W).ravel()
    z_out, w_out = np.zeros_like(c1), np.zeros_like(c1)
    for b in range(B):
        n_dens = 1 if s0 is not None else 2
        lay = _Layout(n, n_dens, 1)
        lin = np.zeros(lay.nv)
        Q = np.zeros((lay.nv, lay.nv))
        q = np.zeros(lay.nv)
        Q[:n_dens * n, :n_dens * n] = rho * np.eye(n_dens * n)
        if s0 is None:
            q[lay.dens(0)] = rho * c0[b].ravel()
            q[lay.dens(1)] = rho * c1[b].ravel()
            rows, rhs = lay.transport_rows(0, 0, 1, kappa * C, kappa * mu, lin)
        else:
            q[lay.dens(0)] = rho * c1[b].ravel()
            rows, rhs = lay.transport_rows(0, None, 0, kappa * C, kappa * mu, lin, fixed=(s0[b], None))
        v = solve_qp(Q, q, lin, np.concatenate(rows), np.concatenate(rhs))
        if s0 is None:
            z_out[b] = v[lay.dens(0)].reshape(H, W)
            w_out[b] = v[lay.dens(1)].reshape(H, W)
        else:
            z_out[b] = s0[b]
            w_out[b] = v[lay.dens(0)].reshape(H, W)
    return z_out, w_out
