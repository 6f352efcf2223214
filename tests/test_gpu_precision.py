"""The precision forms on a 128 x 128 crop of the 32-frame 1024 x 1024 blob
video (one frame pair, solved as its own problem), against the FP64 oracle.

Per result: plain FP32 Algorithm 1 and the projection form (R8) with its
DCT-II Neumann solves in FP32 and in split BF16 on the tensor cores, each
after the same number of iterations as the oracle running the same
algorithm in FP64 from the same start (the iterate error of the number
format alone), and each solved to the 1e-5 rule against the oracle's
optimum (the objective error of a solve).  The printed summary is the
per-result error table of the precision form.
"""
import numpy as np
import pytest
import torch

from oracle import projection as PJ
from oracle import prox as P
from synth import blob_video, rng_for

pytestmark = pytest.mark.gpu

PRM = dict(mu=8.0, rho=1.0)          # where the projection form converges quickly


def crop_pair(size=128, at=448):
    """Frames 0 and 1 of the precision workload's video, cut to a window
    (the full video: rng_for(4, 0), 32 frames of 1024 x 1024, 32 blobs)."""
    v = blob_video(rng_for(4, 0), 2, 1024, 1024, n_blobs=32)
    w = v[:, at:at + size, at:at + size]
    return np.ascontiguousarray(w[:1]), np.ascontiguousarray(w[1:])


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def test_crop_iterates_and_objective_per_form(lib):
    p0, p1 = crop_pair()
    assert p0.sum() > 1.0 and p1.sum() > 1.0      # the window holds mass
    H, W = p0.shape[-2:]
    prm = P.default_steps(H, W, P.ProxParams(mode="prox", **PRM))
    # the optimum: FP64 Algorithm 1 far past the rule
    ref, info = P.solve(p0.astype(np.float64), p1.astype(np.float64),
                        P.ProxParams(mode="prox", tol=1e-10, max_iter=200000, **PRM))
    assert info.converged
    f_ref = P.objective(ref, p0, p1, prm)
    rows = {}
    # iterate errors after k iterations of the same algorithm
    k1 = 200
    with lib.OtProx(1, H, W, kernel="tiled", **PRM) as s:
        s.set_input(p0, p1)
        s.step(k1)
        g = {n: t.double().cpu().numpy() for n, t in s.get_state().items()}
    o = P.iterate(p0, p1, P.ProxParams(mode="prox", **PRM), k1)
    rows["alg1_fp32"] = {"iterate_err": max(rel(g[n], getattr(o, n)) for n in ("x0", "x1", "Mx", "My", "a"))}
    k2 = 10
    pp = P.ProxParams(mode="prox", **PRM)
    k0 = PJ.rhs(p0.astype(np.float64), p1.astype(np.float64), pp)
    o2 = PJ.zero_admm_state(p0.astype(np.float64), pp)
    for _ in range(k2):
        o2 = PJ.admm_iteration(o2, p0.astype(np.float64), p1.astype(np.float64), pp, 1.0, k0)
    z = o2.z
    z_norm = np.sqrt(sum(np.linalg.norm(v) ** 2 for v in z.values()))
    for prec in ("fp32", "split_bf16", "split_bf16_3"):
        with lib.OtProx(1, H, W, algorithm="projection", precision=prec, beta=1.0, **PRM) as s:
            s.set_input(p0, p1)
            s.step(k2)
            g = {n: t.double().cpu().numpy() for n, t in s.get_state().items()}
        # the projection mixes every block, so its rounding is relative to ||z||
        rows["projection_" + prec] = {"iterate_err": max(float(np.linalg.norm(g[n] - z[n])) / z_norm
                                                         for n in ("Mx", "My", "x0", "x1", "r"))}
    # solved to the 1e-5 rule: objective and x against the optimum
    for name, kw in (("alg1_fp32", {}),
                     ("projection_fp32", dict(algorithm="projection", precision="fp32", beta=1.0)),
                     ("projection_split_bf16", dict(algorithm="projection", precision="split_bf16", beta=1.0)),
                     ("projection_split_bf16_3", dict(algorithm="projection", precision="split_bf16_3", beta=1.0))):
        with lib.OtProx(1, H, W, tol=1e-5, max_iter=2000, **PRM, **kw) as s:
            s.set_input(p0, p1)
            r = s.solve()
            g = {n: t.double().cpu().numpy() for n, t in s.get_state().items()}
        st = P.ProxState(g["Mx"], g["My"], g["x0"], g["x1"], g["r"], g["a"])
        rows[name].update({"iters": r["iters"], "status": r["status"],
                           "objective_err": abs(P.objective(st, p0, p1, prm) - f_ref) / abs(f_ref),
                           "x_err": max(rel(g["x0"], ref.x0), rel(g["x1"], ref.x1))})
    print("\nprecision forms on the 128x128 crop:", {k: {a: (f"{b:.2e}" if isinstance(b, float) else b)
                                                        for a, b in v.items()} for k, v in rows.items()})
    # the number format's own error along the same iterations
    assert rows["alg1_fp32"]["iterate_err"] <= 1e-5
    assert rows["projection_fp32"]["iterate_err"] <= 1e-5
    assert rows["projection_split_bf16_3"]["iterate_err"] <= 1e-5
    assert rows["projection_split_bf16"]["iterate_err"] <= 1e-4
    # every form but the 2-piece split reaches the 1e-5 rule; the 2-piece
    # split's solves (about 1e-5 of their result each) keep the primal
    # residual near 1e-5 and it stalls there (status OT_ENOTCONV)
    for name in ("alg1_fp32", "projection_fp32", "projection_split_bf16_3"):
        row = rows[name]
        assert row["status"] == 0, (name, row)
        assert row["objective_err"] <= 1e-4 and row["x_err"] <= 1e-4, (name, row)
    assert rows["projection_split_bf16"]["status"] in (0, -4)
    assert rows["projection_split_bf16"]["objective_err"] <= 1e-4
