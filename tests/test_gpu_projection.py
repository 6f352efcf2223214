"""GPU parity of the DCT-II Neumann solve and of the projection-form prox
(ADMM with an exact projection) against the FP64 oracle.

Tolerance of the solve.  Each DCT transform is a GEMM with K = H or W; in
FP32 its relative error is about u sqrt(K) per transform, and the diagonal
scaling amplifies it by at most the condition number (lam_max + c) / (lam_min
+ c) of the shifted Laplacian (for c = 0 the smallest non-zero eigenvalue).
The test bound is 8 u sqrt(max(H, W)) times that condition number, floored at
1e-5.

Split-BF16 precision (tensor cores, "split_bf16").  Every GEMM operand is held as two BF16
pieces, x = hi + lo with |x - hi - lo| <= 2^-18 |x|, and the lo*lo product is
dropped (another 2^-18 per term).  Along the four transforms the input and
the three intermediates are re-split (four representation errors) and each
GEMM drops one product: at most eight contributions of 2^-18 relative, which
the orthonormal transforms carry over in l2 norm.  Only the scaling between
the second and third transform amplifies, and only components along small
eigenvalues; for c >= 1 (the projection form's shifts) the test bound is
8 * 2^-18 * sqrt(cond), about 1.1e-4 at c = 1.  One projection iteration is
firmly nonexpansive, so over k iterations the trajectory error grows at most
like k times the per-solve bound.  The 3-piece split ("split_bf16_3": an
exact representation, six products down to 2^-16, the correction products in
their own accumulator) is held to the FP32 solve's bound per solve and to an
eighth of the 2-piece bound: what remains is the tensor cores' FP32
accumulation.
"""
import numpy as np
import pytest
import torch

from oracle import dct, grid, projection
from oracle import prox as P
from synth import blob_pairs, rng_for

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def solve_bound(H, W, c):
    lam = dct.laplacian_spectrum(H, W) + c
    nz = lam[lam > 1e-12]
    cond = nz.max() / nz.min()
    return max(1e-5, 8 * U32 * np.sqrt(max(H, W)) * cond)


@pytest.mark.parametrize("B,H,W", [(3, 17, 30), (1, 64, 64), (2, 256, 256), (2, 96, 130), (1, 1, 9)])
@pytest.mark.parametrize("c", [3.0, 2.0, 1.0, 0.0])
def test_neumann_solve_matches_oracle(lib, B, H, W, c):
    rng = np.random.default_rng(B * 1000 + H + W)
    X = rng.normal(size=(B, H, W))
    if c == 0.0:
        X -= X.mean(axis=(1, 2), keepdims=True)
    if c == 0.0 and H * W > 4096:
        pytest.skip("pseudo-inverse of a 256x256 Laplacian is too ill-conditioned for an FP32 bound")
    Xf = X.astype(np.float32)
    ref = dct.neumann_solve(Xf.astype(np.float64), c)
    Y = lib.neumann_solve(torch.from_numpy(Xf).cuda(), c, "fp32").double().cpu().numpy()
    err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert err <= solve_bound(H, W, c), err
    # residual of the defining equation with the oracle's operators
    gx, gy = grid.div_adj(Y)
    R = grid.div(gx, gy) + c * Y - Xf.astype(np.float64)
    assert np.linalg.norm(R) <= 1e-5 * np.linalg.norm(X) * max(1.0, 8.0 / max(c, 1.0))


def split_bound(H, W, c):
    lam = dct.laplacian_spectrum(H, W) + c
    return 8 * 2.0 ** -18 * np.sqrt(lam.max() / lam.min())


@pytest.mark.parametrize("B,H,W", [(3, 17, 30), (1, 64, 64), (2, 256, 256), (2, 96, 130), (1, 1, 9), (5, 200, 72)])
@pytest.mark.parametrize("c", [3.0, 2.0, 1.0])
def test_neumann_solve_split_bf16_matches_oracle(lib, B, H, W, c):
    rng = np.random.default_rng(B * 1000 + H + W + 7)
    X = rng.normal(size=(B, H, W)).astype(np.float32)
    ref = dct.neumann_solve(X.astype(np.float64), c)
    Y = lib.neumann_solve(torch.from_numpy(X).cuda(), c, "split_bf16").double().cpu().numpy()
    err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert err <= split_bound(H, W, c), err
    # every problem of the batch, separately (the batch is folded into the GEMM rows)
    for b in range(B):
        eb = np.linalg.norm(Y[b] - ref[b]) / np.linalg.norm(ref[b])
        assert eb <= 2 * split_bound(H, W, c), (b, eb)


@pytest.mark.parametrize("B,H,W", [(3, 17, 30), (1, 64, 64), (2, 256, 256), (2, 96, 130), (1, 1, 9), (5, 200, 72),
                                   (2, 1024, 1024)])
@pytest.mark.parametrize("c", [3.0, 1.0])
def test_neumann_solve_split_bf16_3_matches_fp32_bound(lib, B, H, W, c):
    """The exact 3-piece split with six products: the FP32 solve's bound
    (the dropped products are below 2^-24 of each term), well under the
    2-piece split's."""
    rng = np.random.default_rng(B * 1000 + H + W + 9)
    X = rng.normal(size=(B, H, W)).astype(np.float32)
    ref = dct.neumann_solve(X.astype(np.float64), c) if H * W <= 256 * 256 else None
    Y = lib.neumann_solve(torch.from_numpy(X).cuda(), c, "split_bf16_3").double().cpu().numpy()
    if ref is None:   # 1024 x 1024: one problem by the oracle
        ref = dct.neumann_solve(X[:1].astype(np.float64), c)
        Y = Y[:1]
    err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert err <= solve_bound(H, W, c), err
    assert err <= split_bound(H, W, c) / 8, err


def test_neumann_solve_split_bf16_large_batch_sampled(lib):
    """63 problems of 256 x 256 (the batch of a 64-frame sequence); the oracle
    checks a sample of problems one by one."""
    B, H, W, c = 63, 256, 256, 3.0
    rng = np.random.default_rng(11)
    X = rng.normal(size=(B, H, W)).astype(np.float32)
    Y = lib.neumann_solve(torch.from_numpy(X).cuda(), c, "split_bf16").double().cpu().numpy()
    for b in (0, 31, 62):
        ref = dct.neumann_solve(X[b:b + 1].astype(np.float64), c)[0]
        assert np.linalg.norm(Y[b] - ref) / np.linalg.norm(ref) <= split_bound(H, W, c)


def test_neumann_solve_in_place(lib):
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.normal(size=(2, 40, 50)).astype(np.float32)).cuda()
    Y = lib.neumann_solve(X.clone(), 2.0, "fp32")
    Xi = X.clone()
    lib.neumann_solve(Xi, 2.0, "fp32", out=Xi)
    assert torch.equal(Y, Xi)


BETA = 1.0


def oracle_admm(p0, p1, prm, n):
    p0 = p0.astype(np.float64)
    p1 = p1.astype(np.float64)
    k0 = projection.rhs(p0, p1, prm)
    st = projection.zero_admm_state(p0, prm)
    for _ in range(n):
        st = projection.admm_iteration(st, p0, p1, prm, BETA, k0)
    return st


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "split_bf16_3"])
@pytest.mark.parametrize("mode,balanced", [("prox", False), ("fixed_first", False), ("eval", False), ("prox", True)])
@pytest.mark.parametrize("k", [1, 10, 60])
def test_projection_form_trajectory(lib, mode, balanced, k, precision):
    B, H, W = 2, 24, 36
    p0, p1 = blob_pairs(rng_for(0, 70), B, H, W, n_blobs=2, sigma=2.0, max_shift=2)
    if balanced:
        p1 = (p1 * (p0.sum(axis=(1, 2), keepdims=True) / p1.sum(axis=(1, 2), keepdims=True))).astype(np.float32)
    prm = P.ProxParams(mu=3.0, rho=0.01, mode=mode, balanced=balanced)
    with lib.OtProx(B, H, W, mu=3.0, rho=0.01, mode=mode, balanced=balanced, algorithm="projection",
                    precision=precision, beta=BETA) as s:
        s.set_input(p0, p1)
        s.step(k)
        g = {n: v.double().cpu().numpy() for n, v in s.get_state().items()}
    st = oracle_admm(p0, p1, prm, k)
    z = st.z
    scale = np.linalg.norm(p0)
    n_id = P.n_identity_blocks(prm)
    # split-BF16: the rounding error is relative to the whole iterate (the
    # projection mixes all blocks), so it is measured against ||z||, not the
    # norm of one (possibly still tiny) block
    z_norm = np.sqrt(sum(np.linalg.norm(v) ** 2 for v in z.values()))
    # the 3-piece split's per-solve error is that of the tensor cores' FP32
    # accumulation, within split_bound / 8 (test_neumann_solve_split_bf16_3...)
    per_solve = {"split_bf16": split_bound(H, W, float(n_id)), "split_bf16_3": split_bound(H, W, float(n_id)) / 8}
    tol = max(1e-5, k * per_solve[precision]) if precision in per_solve else 1e-5 * max(1, k / 20)
    for name in ("Mx", "My", "x0", "x1", "r"):
        if name not in z:
            continue
        o = z[name]
        den = z_norm if precision in per_solve else np.linalg.norm(o)
        e = np.linalg.norm(g[name] - o) / max(den, 1e-3 * scale)
        assert e <= tol, (name, e)


def test_projection_form_solves_the_same_prox(lib):
    """At convergence the projection form and Algorithm 1 agree on what is
    unique: the objective value and x (eq. Prox_UOT is strongly convex in x)."""
    B, H, W = 2, 32, 32
    p0, p1 = blob_pairs(rng_for(0, 71), B, H, W)
    res = {}
    states = {}
    for alg in ("alg1", "projection"):
        with lib.OtProx(B, H, W, mu=3.0, rho=0.01, algorithm=alg, precision="fp32", beta=BETA, tol=1e-5,
                        max_iter=60000) as s:
            s.set_input(p0, p1)
            res[alg] = s.solve()
            states[alg] = {n: v.double().cpu().numpy() for n, v in s.get_state().items()}
    assert res["projection"]["status"] == 0 and res["alg1"]["status"] == 0, res
    o1, o2 = res["alg1"]["objective"], res["projection"]["objective"]
    assert abs(o1 - o2) <= 1e-3 * o1
    for n in ("x0", "x1"):
        assert np.max(np.abs(states["alg1"][n] - states["projection"][n])) <= 2e-3 * np.max(p0)
    # the multiplier a = beta y certifies the projection form's solution
    assert res["projection"]["rel_gap"] <= 1e-3
