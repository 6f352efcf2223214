"""GPU parity of Algorithm 1 (libotprox, tiled and resident kernels) against
the FP64 oracle on the same seeded inputs.

Tolerances.  The kernels compute in FP32 (unit roundoff u = 6e-8); the oracle
in FP64.  One iteration is a short chain of FMAs per value, so one step from
an identical FP32 state agrees to ~1e-7 relative (tested at 1e-6).  Over k
iterations the Chambolle-Pock map is non-expansive, so rounding differences
add up at most linearly and in practice like a random walk: the bar for
trajectory parity is the stated 1e-5 relative l2 error per variable.
Support masks (flux ||m|| > 0, source r != 0, x > 0) must agree bit for bit
wherever the oracle's pre-threshold value is farther than a guard band from
the threshold; inside the band FP32 and FP64 may legitimately round to
different sides.
"""
import numpy as np
import pytest
import torch

from oracle import grid
from oracle import prox as P
from synth import blob_pairs, blob_pair_64x64, rng_for

pytestmark = pytest.mark.gpu

MU, RHO = 3.0, 0.01
NAMES = ("Mx", "My", "x0", "x1", "r", "a")


def rel_err(g, o, scale):
    no = np.linalg.norm(o)
    return np.linalg.norm(g - o) / max(no, 1e-3 * scale)


def gpu_iterate(lib, p0, p1, n, state=None, **kw):
    B, H, W = p0.shape
    with lib.OtProx(B, H, W, **kw) as s:
        s.set_input(torch.from_numpy(p0).cuda(), torch.from_numpy(p1).cuda())
        if state is not None:
            s.set_state(**{k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in state.items()})
        s.step(n)
        st = s.get_state()
    return {k: v.double().cpu().numpy() for k, v in st.items()}


def oracle_params(**kw):
    keys = ("mu", "rho", "mode", "norm", "balanced", "p_exp", "tau1", "tau2")
    d = {k: v for k, v in kw.items() if k in keys}
    d.setdefault("mu", MU)
    d.setdefault("rho", RHO)
    return P.ProxParams(**d)


def check_state(g, o: P.ProxState, tol, scale):
    for name in NAMES:
        e = rel_err(g[name], getattr(o, name), scale)
        assert e <= tol, f"{name}: relative error {e:.3e} > {tol:g}"


@pytest.mark.parametrize("kernel", ["tiled", "resident", "tma"])
@pytest.mark.parametrize("k,tol", [(1, 1e-6), (10, 1e-5), (500, 1e-5)])
def test_trajectory_parity_64x64_pair(lib, kernel, k, tol):
    """The 64x64 frame pair: 3 blobs, shifts in [-4, 4], one blob rescaled."""
    p0, p1 = blob_pair_64x64()
    g = gpu_iterate(lib, p0, p1, k, mu=MU, rho=RHO, kernel=kernel)
    o = P.iterate(p0.astype(np.float64), p1.astype(np.float64), oracle_params(), k)
    check_state(g, o, tol, np.linalg.norm(p0))


SHAPES = [(1, 1, 1), (1, 1, 9), (2, 5, 3), (1, 17, 130), (3, 33, 257), (2, 16, 128), (1, 129, 5)]
VARIANTS = [dict(), dict(mode="fixed_first"), dict(mode="eval"), dict(balanced=True),
            dict(norm="aniso"), dict(p_exp=2), dict(mode="eval", balanced=True)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", range(len(VARIANTS)))
@pytest.mark.parametrize("kernel", ["tiled", "resident", "tma"])
def test_shapes_and_modes(lib, shape, variant, kernel):
    B, H, W = shape
    kw = dict(mu=1.5, rho=0.02, **VARIANTS[variant])
    if kw.get("mode") == "eval" and kw.get("balanced") and H * W == 1:
        pytest.skip("1x1 balanced EVAL has no variables")
    if kernel == "resident" and 10 * H * ((W + 3) // 4 * 4) * 4 > 200 * 1024:
        pytest.skip("does not fit the resident kernel")
    rng = rng_for(0, 1000 + H * 7 + W)
    p0, p1 = blob_pairs(rng, B, H, W, n_blobs=2, sigma=max(1.0, min(H, W) / 8), max_shift=2)
    if kw.get("balanced"):
        p1 = (p1 * (p0.sum(axis=(1, 2), keepdims=True) / np.maximum(p1.sum(axis=(1, 2), keepdims=True), 1e-30))).astype(np.float32)
    n = 25
    g = gpu_iterate(lib, p0, p1, n, kernel=kernel, **kw)
    o = P.iterate(p0.astype(np.float64), p1.astype(np.float64), oracle_params(**kw), n)
    check_state(g, o, 1e-5, max(np.linalg.norm(p0), 1e-3))


def _oracle_state_f32(p0, p1, n, prm):
    st = P.iterate(p0.astype(np.float64), p1.astype(np.float64), prm, n)
    return {k: getattr(st, k).astype(np.float32) for k in NAMES}


def _masks_and_margins(st: dict, p0, p1, prm):
    """Masks after one iteration from state st (FP64) and each mask's
    pre-threshold margin."""
    prm = P.default_steps(*p0.shape[-2:], prm)
    s = P.ProxState(*(st[k].astype(np.float64) for k in NAMES))
    gx, gy = grid.div_adj(s.a)
    qx, qy = s.Mx - prm.tau1 * gx, s.My - prm.tau1 * gy
    mx, my = grid.edge_masks(*p0.shape[-2:])
    qx, qy = qx * mx, qy * my
    m_margin = np.sqrt(qx * qx + qy * qy) - prm.tau1
    qr = s.r + prm.tau1 * s.a
    r_margin = np.abs(qr) - prm.mu * prm.tau1
    x0_pre = (prm.tau1 * p0 + prm.rho * (s.x0 + prm.tau1 * s.a)) / (prm.rho + prm.tau1)
    x1_pre = (prm.tau1 * p1 + prm.rho * (s.x1 - prm.tau1 * s.a)) / (prm.rho + prm.tau1)
    new = P.alg1_iteration(s, p0.astype(np.float64), p1.astype(np.float64), prm)
    return new, {"M": (m_margin, prm.tau1), "r": (r_margin, prm.mu * prm.tau1),
                 "x0": (x0_pre, 0.0), "x1": (x1_pre, 0.0)}


def _gpu_masks(g):
    return {"M": np.hypot(g["Mx"], g["My"]) > 0, "r": g["r"] != 0, "x0": g["x0"] > 0, "x1": g["x1"] > 0}


@pytest.mark.parametrize("kernel", ["tiled", "resident", "tma"])
def test_support_masks_bit_exact_one_step(lib, kernel):
    """One iteration from an identical FP32 state: the flux, source and
    non-negativity masks agree bit for bit outside a 1e-5 guard band."""
    p0, p1 = blob_pair_64x64()
    prm = oracle_params()
    st = _oracle_state_f32(p0, p1, 300, prm)
    g = gpu_iterate(lib, p0, p1, 1, state=st, mu=MU, rho=RHO, kernel=kernel)
    new, margins = _masks_and_margins(st, p0, p1, prm)
    ref = {"M": np.hypot(new.Mx, new.My) > 0, "r": new.r != 0, "x0": new.x0 > 0, "x1": new.x1 > 0}
    gm = _gpu_masks(g)
    n_support = 0
    for key, (margin, thr) in margins.items():
        outside = np.abs(margin) > 1e-5 * max(1.0, thr)
        mism = (gm[key] != ref[key]) & outside
        assert not mism.any(), f"{key}: {int(mism.sum())} mask mismatches outside the guard band"
        n_support += int(ref[key].sum())
    assert int(ref["M"].sum()) > 100 and int(ref["r"].sum()) > 50   # the masks are not trivial


@pytest.mark.parametrize("kernel", ["tiled", "resident", "tma"])
def test_support_masks_after_500_iterations(lib, kernel):
    p0, p1 = blob_pair_64x64()
    prm = oracle_params()
    g = gpu_iterate(lib, p0, p1, 500, mu=MU, rho=RHO, kernel=kernel)
    st499 = _oracle_state_f32(p0, p1, 499, prm)
    new, margins = _masks_and_margins(st499, p0, p1, prm)
    ref = {"M": np.hypot(new.Mx, new.My) > 0, "r": new.r != 0, "x0": new.x0 > 0, "x1": new.x1 > 0}
    gm = _gpu_masks(g)
    for key, (margin, thr) in margins.items():
        outside = np.abs(margin) > 1e-4 * max(1.0, thr)
        mism = (gm[key] != ref[key]) & outside
        assert not mism.any(), f"{key}: {int(mism.sum())} mismatches outside the 1e-4 band"


@pytest.mark.parametrize("kernel", ["tiled", "resident", "tma"])
def test_solve_matches_oracle(lib, kernel):
    """ot_prox_solve to 1e-5: same stopping rule as the oracle's; compare the
    state after the iterations the GPU ran, and the reported quantities."""
    p0, p1 = blob_pairs(rng_for(0, 11), 2, 32, 48)
    with lib.OtProx(2, 32, 48, mu=MU, rho=RHO, kernel=kernel, tol=1e-5, check_every=10) as s:
        s.set_input(torch.from_numpy(p0).cuda(), torch.from_numpy(p1).cuda())
        res = s.solve()
        g = {k: v.double().cpu().numpy() for k, v in s.get_state().items()}
    assert res["status"] == 0 and res["iters"] % 10 == 0
    prm = P.default_steps(32, 48, oracle_params())
    o = P.iterate(p0.astype(np.float64), p1.astype(np.float64), prm, res["iters"])
    check_state(g, o, 1e-5, np.linalg.norm(p0))
    o_prev = P.iterate(p0.astype(np.float64), p1.astype(np.float64), prm, res["iters"] - 1)
    rp, rf = P.residuals(o, o_prev, p0.astype(np.float64), p1.astype(np.float64), prm)
    assert max(rp, rf) <= 1.2e-5
    assert abs(res["res_pri"] - rp) <= 0.05 * rp + 1e-9
    assert abs(res["res_fp"] - rf) <= 0.05 * rf + 1e-9
    obj = P.objective(o, p0.astype(np.float64), p1.astype(np.float64), prm)
    assert abs(res["objective"] - obj) <= 1e-5 * obj
    cert = P.certificate(o, p0.astype(np.float64), p1.astype(np.float64), prm)
    assert abs(res["primal_feasible"] - cert["primal"]) <= 1e-5 * abs(cert["primal"])
    assert abs(res["dual_obj"] - cert["dual"]) <= 1e-5 * abs(cert["primal"])


def test_evaluate_matches_oracle_certificate(lib):
    p0, p1 = blob_pair_64x64()
    prm = P.default_steps(64, 64, oracle_params())
    st = _oracle_state_f32(p0, p1, 200, prm)
    with lib.OtProx(1, 64, 64, mu=MU, rho=RHO) as s:
        s.set_input(p0, p1)
        s.set_state(**st)
        res = s.evaluate()
    o = P.ProxState(*(st[k].astype(np.float64) for k in NAMES))
    cert = P.certificate(o, p0.astype(np.float64), p1.astype(np.float64), prm)
    obj = P.objective(o, p0.astype(np.float64), p1.astype(np.float64), prm)
    assert abs(res["objective"] - obj) <= 1e-9 * obj
    assert abs(res["primal_feasible"] - cert["primal"]) <= 1e-9 * cert["primal"]
    assert abs(res["dual_obj"] - cert["dual"]) <= 1e-9 * cert["primal"]
    assert abs(res["rel_gap"] - cert["rel_gap"]) <= 1e-8


@pytest.mark.parametrize("kernel", ["tiled", "resident", "tma"])
def test_warm_restart_is_bit_exact(lib, kernel):
    """Checkpoint/resume: 500 iterations == 250 + get_state/set_state + 250."""
    p0, p1 = blob_pair_64x64()
    a = gpu_iterate(lib, p0, p1, 500, mu=MU, rho=RHO, kernel=kernel)
    h = gpu_iterate(lib, p0, p1, 250, mu=MU, rho=RHO, kernel=kernel)
    b = gpu_iterate(lib, p0, p1, 250, state={k: v.astype(np.float32) for k, v in h.items()}, mu=MU, rho=RHO,
                    kernel=kernel)
    for k in NAMES:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("other", ["resident", "tma"])
def test_kernels_agree(lib, other):
    p0, p1 = blob_pair_64x64()
    a = gpu_iterate(lib, p0, p1, 200, mu=MU, rho=RHO, kernel="tiled")
    b = gpu_iterate(lib, p0, p1, 200, mu=MU, rho=RHO, kernel=other)
    for k in NAMES:
        assert rel_err(a[k], b[k], np.linalg.norm(p0)) <= 1e-6, k


def test_tma_and_tiled_bit_identical(lib):
    """Same arithmetic in the same order: the TMA pipeline changes only how
    the inputs reach shared memory, so its iterates equal the tiled kernel's."""
    from synth import blob_video
    v = blob_video(rng_for(1, 4), 9, 200, 300, n_blobs=5)
    p0, p1 = np.ascontiguousarray(v[:-1]), np.ascontiguousarray(v[1:])
    a = gpu_iterate(lib, p0, p1, 30, mu=MU, rho=RHO, kernel="tiled")
    b = gpu_iterate(lib, p0, p1, 30, mu=MU, rho=RHO, kernel="tma")
    for k in NAMES:
        assert np.array_equal(a[k], b[k]), k


def test_host_pointers_equal_device_pointers(lib):
    p0, p1 = blob_pairs(rng_for(0, 12), 2, 20, 30)
    outs = []
    for host in (False, True):
        with lib.OtProx(2, 20, 30, mu=MU, rho=RHO) as s:
            if host:
                s.set_input(p0, p1)           # numpy: pageable host memory
            else:
                s.set_input(torch.from_numpy(p0).cuda(), torch.from_numpy(p1).cuda())
            s.step(40)
            outs.append(s.get_state(device="cpu" if host else "cuda"))
    for k in NAMES:
        assert torch.equal(outs[0][k].cpu(), outs[1][k].cpu()), k


def test_nonfinite_input_is_reported(lib):
    p0, p1 = blob_pairs(rng_for(0, 13), 1, 16, 16)
    p0[0, 3, 4] = np.nan
    with lib.OtProx(1, 16, 16, mu=MU, rho=RHO, max_iter=50) as s:
        s.set_input(p0, p1)
        with pytest.raises(lib.OtError) as ei:
            s.solve()
    assert ei.value.code == -5


def test_max_iter_reports_not_converged(lib):
    p0, p1 = blob_pair_64x64()
    with lib.OtProx(1, 64, 64, mu=MU, rho=RHO, max_iter=20, tol=1e-12) as s:
        s.set_input(p0, p1)
        res = s.solve()
    assert res["status"] == -4 and res["iters"] == 20


def test_full_size_video_batch_parity(lib):
    """The 63 frame pairs of a 64-frame 256x256 sequence, TMA kernel with the
    CUDA-graph check loop as in the benchmark: the whole state after 20
    iterations (two check intervals) against the oracle."""
    from synth import blob_video
    v = blob_video(rng_for(1, 3), 64, 256, 256, n_blobs=8)
    p0, p1 = np.ascontiguousarray(v[:-1]), np.ascontiguousarray(v[1:])
    with lib.OtProx(63, 256, 256, mu=MU, rho=RHO, kernel="tma", use_graph=True, max_iter=20, tol=0.0) as s:
        s.set_input(torch.from_numpy(p0).cuda(), torch.from_numpy(p1).cuda())
        res = s.solve()
        g = {k: v.double().cpu().numpy() for k, v in s.get_state().items()}
    assert res["iters"] == 20
    o = P.iterate(p0.astype(np.float64), p1.astype(np.float64), oracle_params(), 20)
    check_state(g, o, 1e-5, np.linalg.norm(p0))
    obj = P.objective(o, p0.astype(np.float64), p1.astype(np.float64), P.default_steps(256, 256, oracle_params()))
    assert abs(res["objective"] - obj) <= 1e-5 * obj


def test_resident_handles_of_different_sizes_coexist(lib):
    """The shared-memory limit of the one-CTA-per-problem kernel belongs to
    the kernel: a later handle with a smaller state must not lower it under
    an earlier, larger handle."""
    big = (3, 64, 64)
    small = (2, 24, 24)
    p_big = blob_pairs(rng_for(3, 91), *big, n_blobs=2)
    p_small = blob_pairs(rng_for(3, 92), *small, n_blobs=2)
    with lib.OtProx(*big, kernel="resident", mu=3.0, rho=0.01) as a, \
            lib.OtProx(*small, kernel="resident", mu=3.0, rho=0.01) as b:
        a.set_input(*p_big)
        b.set_input(*p_small)
        a.step(20)
        b.step(20)
        a.step(20)
        st = a.get_state()
    with lib.OtProx(*big, kernel="resident", mu=3.0, rho=0.01) as c:
        c.set_input(*p_big)
        c.step(40)
        ref = c.get_state()
    for k in ("Mx", "a"):
        assert torch.equal(st[k], ref[k]), k
