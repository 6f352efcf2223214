"""GPU parity of Algorithm 2 (UOT-DF / BPDN+UOT-DF, Phi = I) against the FP64
oracle.

The fused elementwise passes are exact to FP32 rounding and the inner
Algorithm 1 iterations are the kernels tested in test_gpu_prox.py; the dual
accumulators a += x - s and b += z - s add differences of nearly equal
operands, so every variable is measured against the data norm ||y||.  Over k
iterations of a nonexpansive scheme the FP32 rounding accumulates at most
linearly: the bound is 1e-5 max(1, k/20).
"""
import numpy as np
import pytest

from oracle import uotdf as U
from synth import blob_pairs, rng_for

pytestmark = pytest.mark.gpu

VARS = {"s": "s", "x": "x", "a": "a", "b": "b", "z": "z"}


def inputs(B, H, W, seed):
    p0, p1 = blob_pairs(rng_for(3, seed), B, H, W, n_blobs=3, sigma=2.5, max_shift=3)
    rng = np.random.default_rng(seed)
    y = (p1 + 0.02 * rng.normal(size=p1.shape)).astype(np.float32)
    return y, p0.astype(np.float32)


def oracle_run(y, s0, prm, k):
    st = U.zero_state(s0.astype(np.float64))
    res = None
    for _ in range(k):
        st, pri, dual = U.iteration(st, y.astype(np.float64), s0.astype(np.float64), prm)
        res = (pri, dual)
    return st, res


CASES = [dict(lam=0.0, norm="iso", p_exp=1, n_inner=1),
         dict(lam=0.05, norm="iso", p_exp=1, n_inner=3),
         dict(lam=0.0, norm="aniso", p_exp=2, n_inner=2)]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("k", [1, 10, 50])
@pytest.mark.parametrize("rho", [1.0, 0.4, 2.5])
def test_uotdf_trajectory_parity(lib, case, k, rho):
    """rho != 1 as well: at rho = 1 a misplaced rho (lambda/(2 rho), the
    x-update's rho, the prox weight kappa/rho) would not show."""
    B, H, W = 2, 24, 30
    c = CASES[case]
    y, s0 = inputs(B, H, W, 10 + case)
    prm = U.UotdfParams(kappa=0.5, mu=3.0, rho=rho, **c)
    with lib.Uotdf(B, H, W, kappa=0.5, mu=3.0, rho=rho, **c) as u:
        u.set_input(y, s0)
        res = u.iterate_checked(k)
        got = {n: u.get(n).double().cpu().numpy() for n in VARS}
    st, (pri, dual) = oracle_run(y, s0, prm, k)
    ny = np.linalg.norm(y.astype(np.float64))
    for n, attr in VARS.items():
        e = np.linalg.norm(got[n] - getattr(st, attr)) / ny
        assert e <= 1e-5 * max(1, k / 20), (n, e)
    assert abs(res["res_pri"] - pri) <= 1e-3 * pri + 1e-7
    assert abs(res["res_dual"] - dual) <= 1e-3 * dual + 1e-7
    assert np.min(got["s"]) >= 0


@pytest.mark.parametrize("rho", [1.0, 2.5])
def test_uotdf_solve_matches_oracle(lib, rho):
    B, H, W = 3, 20, 20
    y, s0 = inputs(B, H, W, 21)
    prm = U.UotdfParams(kappa=0.5, mu=3.0, rho=rho, n_inner=1, tol=1e-6, max_iter=20000)
    with lib.Uotdf(B, H, W, kappa=0.5, mu=3.0, rho=rho, n_inner=1, tol=1e-6, max_iter=20000) as u:
        u.set_input(y, s0)
        res = u.solve()
        s = u.get("s").double().cpu().numpy()
    assert res["status"] == 0, res
    st, info = U.solve(y, s0, prm)
    assert info["converged"]
    ny = np.linalg.norm(y.astype(np.float64))
    assert np.linalg.norm(s - st.s) <= 1e-3 * ny
    # the transport term moved the estimate off the plain projection Pi_+(y)
    assert np.linalg.norm(s - np.maximum(y, 0)) > 1e-2 * ny


def test_uotdf_full_size_sampled(lib):
    """63 frames of 256 x 256 (a 64-frame video's pairs as independent
    tracking steps), two iterations; the oracle checks two frames alone."""
    B, H, W = 63, 256, 256
    y, s0 = inputs(B, H, W, 30)
    with lib.Uotdf(B, H, W, kappa=0.5, mu=3.0, rho=1.0) as u:
        u.set_input(y, s0)
        u.iterate_checked(2)
        s = u.get("s").double().cpu().numpy()
    prm = U.UotdfParams(kappa=0.5, mu=3.0, rho=1.0)
    for b in (0, 62):
        st, _ = oracle_run(y[b:b + 1], s0[b:b + 1], prm, 2)
        assert np.linalg.norm(s[b] - st.s[0]) <= 1e-5 * np.linalg.norm(y[b].astype(np.float64))


def test_uotdf_rejects_bad_input(lib):
    y, s0 = inputs(1, 8, 8, 1)
    y[0, 3, 3] = np.nan
    with lib.Uotdf(1, 8, 8) as u:
        with pytest.raises(lib.OtError):
            u.set_input(y, s0)
    with pytest.raises(lib.OtError):
        lib.Uotdf(1, 8, 8, kappa=-1.0)
