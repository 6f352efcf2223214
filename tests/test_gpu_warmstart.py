"""Warm start of Algorithm 1 from a predicted state, and the trained network's
gain over a cold start.

``ot_prox_warm_start`` writes (Mx, My, r, a) from a [B, 4, H, W] prediction
and sets each free x at its step's fixed point given a,
x0 = max(p0 + rho a, 0), x1 = max(p1 - rho a, 0) (the optimality condition of
the (1/2 rho)||x - p||^2 term).  From the converged state itself the solver
must stop at its first check; from the trained network's prediction it must
need fewer iterations than from zero.
"""
import numpy as np
import pytest
import torch

from synth import blob_pairs, rng_for

pytestmark = pytest.mark.gpu

KW = dict(mode="prox", mu=3.0, rho=0.01, tol=1e-5, max_iter=100000)


def pairs(seed, n, S, nb=None):
    rng = rng_for(5, seed)
    p0s, p1s = [], []
    for k in range(0, n, 16):
        m = min(16, n - k)
        a, b = blob_pairs(rng, m, S, S, n_blobs=nb or int(rng.integers(3, 9)))
        p0s.append(a)
        p1s.append(b)
    return np.concatenate(p0s), np.concatenate(p1s)


def test_warm_start_gate_keeps_the_prediction_only_near_mass(lib):
    """gate > 0: where p0 + p1 stays at or below the gate in the 5 x 5
    neighbourhood the state is that of a zero prediction (x = p); elsewhere
    the prediction's."""
    B, H, W, rho, gate = 2, 24, 32, 0.01, 1e-3
    p0 = np.zeros((B, H, W), np.float32)
    p1 = np.zeros((B, H, W), np.float32)
    p0[:, 5, 6] = 1.0
    p1[:, 15, 20] = 0.5
    p1[:, 20, 3] = 0.5 * gate          # below the gate: no effect
    pred = np.random.default_rng(1).normal(size=(B, 4, H, W)).astype(np.float32)
    with lib.OtProx(B, H, W, mode="prox", mu=3.0, rho=rho) as s:
        s.set_input(p0, p1)
        s.warm_start(torch.from_numpy(pred).cuda(), gate)
        st = {k: v.cpu().numpy() for k, v in s.get_state().items()}
    near = np.zeros((B, H, W), bool)
    for (i, j) in ((5, 6), (15, 20)):
        near[:, max(i - 2, 0):i + 3, max(j - 2, 0):j + 3] = True
    assert np.array_equal(st["a"], np.where(near, pred[:, 3], 0))
    assert np.array_equal(st["r"], np.where(near, pred[:, 2], 0))
    mx = np.where(near, pred[:, 0], 0)
    mx[:, H - 1, :] = 0
    assert np.array_equal(st["Mx"], mx)
    assert np.array_equal(st["x0"][~near], p0[~near]) and np.array_equal(st["x1"][~near], p1[~near])


@pytest.mark.parametrize("mode", ["prox", "fixed_first", "eval"])
def test_warm_start_writes_the_state(lib, mode):
    B, H, W, rho = 3, 21, 34, 0.37
    p0, p1 = pairs(1, B, 40)
    p0, p1 = p0[:, :H, :W].copy(), p1[:, :H, :W].copy()
    rng = np.random.default_rng(0)
    pred = rng.normal(size=(B, 4, H, W)).astype(np.float32)
    with lib.OtProx(B, H, W, mode=mode, mu=3.0, rho=rho) as s:
        s.set_input(p0, p1)
        s.warm_start(torch.from_numpy(pred).cuda())
        st = {k: v.cpu().numpy() for k, v in s.get_state().items()}
    mx = pred[:, 0].copy()
    mx[:, H - 1, :] = 0
    my = pred[:, 1].copy()
    my[:, :, W - 1] = 0
    assert np.array_equal(st["Mx"], mx) and np.array_equal(st["My"], my)
    assert np.array_equal(st["r"], pred[:, 2]) and np.array_equal(st["a"], pred[:, 3])
    r32 = np.float32(rho)
    x0 = np.maximum(p0.astype(np.float64) + np.float64(r32) * pred[:, 3], 0).astype(np.float32)
    x1 = np.maximum(p1.astype(np.float64) - np.float64(r32) * pred[:, 3], 0).astype(np.float32)
    # one FMA on the GPU; the FP64 sum rounded to FP32 is within one ulp
    def ulp_equal(got, want):
        return np.all(np.abs(got - want) <= np.spacing(np.abs(want)))
    assert ulp_equal(st["x0"], x0) if mode == "prox" else np.array_equal(st["x0"], p0)
    assert ulp_equal(st["x1"], x1) if mode != "eval" else np.array_equal(st["x1"], p1)


def test_warm_start_from_the_converged_state_stops_at_once(lib):
    B, S = 8, 64
    p0, p1 = pairs(2, B, S, nb=4)
    with lib.OtProx(B, S, S, **KW) as s:
        s.set_input(p0, p1)
        cold = s.solve()
        st = s.get_state()
    pred = torch.stack([st[k] for k in ("Mx", "My", "r", "a")], 1).contiguous()
    with lib.OtProx(B, S, S, **KW) as s:
        s.set_input(p0, p1)
        s.warm_start(pred)
        warm = s.solve()
    assert cold["status"] == 0 and warm["status"] == 0
    assert cold["iters"] > 500
    assert warm["iters"] == 10, warm


def test_warm_start_rejects_a_wrong_prediction_tensor(lib):
    with lib.OtProx(2, 16, 16, **KW) as s:
        with pytest.raises(ValueError):
            s.warm_start(torch.zeros((2, 3, 16, 16), device="cuda"))
        with pytest.raises(ValueError):
            s.warm_start(torch.zeros((2, 4, 16, 16)))


def test_trained_network_needs_fewer_iterations_than_a_cold_start(lib):
    """Train the U-Net (library kernels) on 2048 pairs solved by the plain
    method, then solve 128 held-out pairs from its prediction and from zero,
    both to the same 1e-5 stopping rule."""
    from paper_1909_00149_gb300 import warmstart as WS
    S, base, batch = 128, 32, 16
    p0, p1 = pairs(0, 2048, S)
    X, T, _ = WS.solve_targets(p0, p1, **KW)
    net = lib.UNet(S, S, batch, base)
    net.init(0)
    losses = WS.train(net, X, T, epochs=6, batch=batch, lr=1e-3)
    assert losses[-1] < 0.2 * losses[0]
    ev = lib.UNet(S, S, 128, base)
    ev.set_params(net.get_params())
    q0, q1 = pairs(99, 128, S)
    cold = WS.solve(q0, q1, **KW)
    warm = WS.solve(q0, q1, net=ev, gate=1e-3, **KW)
    print(f"\ncold {cold['iters']} iterations, warm {warm['iters']} iterations")
    assert cold["status"] == 0 and warm["status"] == 0
    assert warm["res_pri"] <= 1e-5 and warm["res_fp"] <= 1e-5
    assert warm["iters"] < 0.95 * cold["iters"], (cold["iters"], warm["iters"])
