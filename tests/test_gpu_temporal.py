"""Temporal blocking of Algorithm 1 (kernel "temporal"): tb_depth iterations
(lines 3-7, Sec. III-B) per pass over the state.

The kernel runs the tiled kernel's per-pixel arithmetic in the same order on
a tile grown by a halo, so every iterate must equal the tiled kernel's bit for
bit: for each depth (2, 3, 4), each split of a call into passes, each mode
and shape (several tiles and ragged tails in both directions, widths that are
not a multiple of 4, images smaller than the halo).  Against the FP64 oracle
the trajectory then meets the 1e-5 bar of the other kernels, checked directly
on the 64 x 64 pair and the full 63-pair 256 x 256 batch.
"""
import numpy as np
import pytest
import torch

from oracle import prox as P
from synth import blob_pair_64x64, blob_pairs, rng_for
from test_gpu_prox import NAMES, check_state, gpu_iterate, oracle_params

pytestmark = pytest.mark.gpu

MU, RHO = 3.0, 0.01

# (B, H, W): the extended tile is 45 rows (own rows 37 at depth 3-4, 41 at
# depth 2) by 136 columns (128 own)
SHAPES = [(1, 1, 1), (2, 5, 3), (1, 17, 130), (3, 33, 257), (2, 100, 300), (1, 41, 129), (1, 38, 256),
          (2, 75, 128), (1, 129, 5)]
VARIANTS = [dict(), dict(mode="fixed_first"), dict(mode="eval"), dict(balanced=True),
            dict(norm="aniso"), dict(p_exp=2), dict(mode="eval", balanced=True)]


def inputs(B, H, W, balanced=False):
    rng = rng_for(0, 2000 + H * 7 + W)
    p0, p1 = blob_pairs(rng, B, H, W, n_blobs=2, sigma=max(1.0, min(H, W) / 8), max_shift=2)
    if balanced:
        p1 = (p1 * (p0.sum(axis=(1, 2), keepdims=True) /
                    np.maximum(p1.sum(axis=(1, 2), keepdims=True), 1e-30))).astype(np.float32)
    return p0, p1


def assert_identical(a, b):
    for k in NAMES:
        assert np.array_equal(a[k], b[k]), (k, np.max(np.abs(a[k] - b[k])))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", range(len(VARIANTS)))
def test_bit_identical_to_tiled(lib, shape, variant):
    """11 iterations: depth 4 runs passes of 4, 4, 3; depth 3 of 3, 3, 3, 2;
    depth 2 of 2 x 5 and 1."""
    B, H, W = shape
    kw = dict(mu=1.5, rho=0.02, **VARIANTS[variant])
    if kw.get("mode") == "eval" and kw.get("balanced") and H * W == 1:
        pytest.skip("1x1 balanced EVAL has no variables")
    p0, p1 = inputs(B, H, W, kw.get("balanced", False))
    ref = gpu_iterate(lib, p0, p1, 11, kernel="tiled", **kw)
    for depth in (2, 3, 4):
        assert_identical(gpu_iterate(lib, p0, p1, 11, kernel="temporal", tb_depth=depth, **kw), ref)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9, 13])
def test_every_pass_split_is_bit_identical(lib, n):
    """Odd pass counts leave x0, x1, r in the second copy: get_state must
    read the current one."""
    p0, p1 = inputs(2, 90, 200)
    ref = gpu_iterate(lib, p0, p1, n, kernel="tiled", mu=MU, rho=RHO)
    for depth in (2, 4):
        assert_identical(gpu_iterate(lib, p0, p1, n, kernel="temporal", tb_depth=depth, mu=MU, rho=RHO), ref)


@pytest.mark.parametrize("k,tol", [(1, 1e-6), (10, 1e-5), (500, 1e-5)])
def test_trajectory_parity_64x64_pair(lib, k, tol):
    p0, p1 = blob_pair_64x64()
    g = gpu_iterate(lib, p0, p1, k, mu=MU, rho=RHO, kernel="temporal")
    o = P.iterate(p0.astype(np.float64), p1.astype(np.float64), oracle_params(), k)
    check_state(g, o, tol, np.linalg.norm(p0))


def test_check_sums_match_tiled(lib):
    """The stopping-check sums come from the last iteration of the last pass:
    the same per-pixel terms as the tiled kernel, summed in another order."""
    p0, p1 = inputs(3, 70, 260)
    out = []
    for kernel in ("tiled", "temporal"):
        with lib.OtProx(3, 70, 260, mu=MU, rho=RHO, kernel=kernel, use_graph=False) as s:
            s.set_input(p0, p1)
            s.step(17)
            out.append(s.check_interval(10))
    for key in ("res_pri", "res_fp", "objective"):
        assert abs(out[0][key] - out[1][key]) <= 1e-6 * abs(out[0][key]), key


def test_solve_graph_replay_and_restart(lib):
    """solve() with CUDA-graph replay of the check interval stops where the
    tiled kernel stops, with the same state; a checkpoint taken after an odd
    number of passes resumes bit for bit."""
    p0, p1 = blob_pairs(rng_for(0, 21), 2, 48, 160)
    res, st = [], []
    for kernel in ("tiled", "temporal"):
        with lib.OtProx(2, 48, 160, mu=MU, rho=RHO, kernel=kernel, tol=1e-5, check_every=10, use_graph=True,
                        stream=torch.cuda.Stream()) as s:
            s.set_input(p0, p1)
            res.append(s.solve())
            st.append({k: v.double().cpu().numpy() for k, v in s.get_state().items()})
    assert res[0]["iters"] == res[1]["iters"] and res[1]["status"] == 0
    assert_identical(st[0], st[1])
    full = gpu_iterate(lib, p0, p1, 18, mu=MU, rho=RHO, kernel="temporal")
    half = gpu_iterate(lib, p0, p1, 9, mu=MU, rho=RHO, kernel="temporal")
    resumed = gpu_iterate(lib, p0, p1, 9, state={k: v.astype(np.float32) for k, v in half.items()}, mu=MU,
                          rho=RHO, kernel="temporal")
    assert_identical(full, resumed)


def test_full_size_video_batch(lib):
    """The 63 frame pairs of a 64-frame 256x256 sequence: 20 iterations (five
    passes of 4) equal the TMA kernel's bit for bit and the oracle's to 1e-5."""
    from synth import blob_video
    v = blob_video(rng_for(1, 3), 64, 256, 256, n_blobs=8)
    p0, p1 = np.ascontiguousarray(v[:-1]), np.ascontiguousarray(v[1:])
    a = gpu_iterate(lib, p0, p1, 20, mu=MU, rho=RHO, kernel="tma")
    b = gpu_iterate(lib, p0, p1, 20, mu=MU, rho=RHO, kernel="temporal", tb_depth=4)
    assert_identical(a, b)
    o = P.iterate(p0.astype(np.float64), p1.astype(np.float64), oracle_params(), 20)
    check_state(b, o, 1e-5, np.linalg.norm(p0))


def _run_sequence(lib, kernel, p0, p1, pred):
    """After an odd number of passes (x0, x1, r in the second copy under
    temporal blocking): a warm start, more iterations, the certificate, a
    reset and a fresh run."""
    B, H, W = p0.shape
    kw = dict(mu=MU, rho=RHO, kernel=kernel, use_graph=False)
    if kernel == "temporal":
        kw["tb_depth"] = 4
    with lib.OtProx(B, H, W, **kw) as s:
        s.set_input(p0, p1)
        s.step(5)                    # temporal: passes of 3 and 2
        s.step(3)                    # one pass: the parity is odd now
        s.warm_start(pred, 1e-3)
        s.step(7)
        ev = s.evaluate()
        st1 = {k: v.double().cpu().numpy() for k, v in s.get_state().items()}
        s.reset()
        s.step(6)
        st2 = {k: v.double().cpu().numpy() for k, v in s.get_state().items()}
    return ev, st1, st2


def test_warm_start_evaluate_reset_follow_the_parity(lib):
    """warm_start writes x0, x1 (and M, r, a) into the current copy, the
    certificate reads it, and reset returns to the first copy: every result
    equals the tiled kernel's."""
    p0, p1 = inputs(2, 60, 140)
    g = torch.Generator(device="cpu").manual_seed(5)
    pred = (1e-3 * torch.randn((2, 4, 60, 140), generator=g)).cuda()
    ev_a, a1, a2 = _run_sequence(lib, "tiled", p0, p1, pred)
    ev_b, b1, b2 = _run_sequence(lib, "temporal", p0, p1, pred)
    assert_identical(a1, b1)
    assert_identical(a2, b2)
    for key in ("objective", "primal_feasible", "dual_obj", "rel_gap"):
        assert ev_a[key] == ev_b[key], key
