"""The batched Algorithm 1 over sequences of uneven size.

Every pixel of a sequence goes through the same arithmetic as the
one-problem tiled kernel (the same tile body, whatever the tile height), so
the batched iterates must equal OtProx(kernel="tiled") on each sequence bit
for bit, and the per-sequence stopping decisions must coincide.  Every
sequence is also checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

from oracle import prox as P
from synth import blob_pairs, rng_for

pytestmark = pytest.mark.gpu

SIZES = [(3, 24, 40), (1, 64, 64), (2, 17, 130), (5, 33, 9), (1, 96, 128)]
KW = dict(mu=3.0, rho=0.01)


def seq_inputs(k, b, h, w):
    p0, p1 = blob_pairs(rng_for(4, k), b, h, w, n_blobs=2, sigma=2.0, max_shift=2)
    return p0, p1


def single_state(lib, b, h, w, p0, p1, n, **kw):
    with lib.OtProx(b, h, w, kernel="tiled", **KW, **kw) as s:
        s.set_input(p0, p1)
        s.step(n)
        return s.get_state()


@pytest.mark.parametrize("config", [("tma", 16, 1), ("tiled", 8, 2), ("tiled", 16, 2)])
@pytest.mark.parametrize("mode", ["prox", "fixed_first", "eval"])
def test_batch_iterates_equal_single_problem_bit_for_bit(lib, config, mode):
    n = 7
    ins = [seq_inputs(k, *sz) for k, sz in enumerate(SIZES)]
    with lib.ProxBatch(SIZES, mode=mode, **KW) as bt:
        bt.set_config(*config)
        for k, (p0, p1) in enumerate(ins):
            bt.set_input(k, p0, p1)
        bt.step(n)
        got = [bt.get_state(k) for k in range(len(SIZES))]
    for k, (sz, (p0, p1)) in enumerate(zip(SIZES, ins)):
        ref = single_state(lib, *sz, p0, p1, n, mode=mode)
        for name in ("Mx", "My", "x0", "x1", "r", "a"):
            assert torch.equal(got[k][name], ref[name]), (k, name)


@pytest.mark.parametrize("kernel", ["tma", "tiled"])
def test_batch_solve_matches_single_problem_solves(lib, kernel):
    ins = [seq_inputs(10 + k, *sz) for k, sz in enumerate(SIZES)]
    with lib.ProxBatch(SIZES, tol=1e-5, max_iter=40000, **KW) as bt:
        bt.set_config(kernel, 16, 2)
        for k, (p0, p1) in enumerate(ins):
            bt.set_input(k, p0, p1)
        res, launches = bt.solve()
        states = [bt.get_state(k) for k in range(len(SIZES))]
    assert launches > 0
    for k, (sz, (p0, p1)) in enumerate(zip(SIZES, ins)):
        with lib.OtProx(*sz, kernel="tiled", tol=1e-5, max_iter=40000, check_every=10, **KW) as s:
            s.set_input(p0, p1)
            r = s.solve()
            ref = s.get_state()
        assert res[k]["status"] == 0 and r["status"] == 0, (k, res[k], r)
        assert res[k]["iters"] == r["iters"], (k, res[k]["iters"], r["iters"])
        # the one-problem solve re-evaluates its final residual in a separate
        # FP64 pass; the batch reports the check sums of its last interval
        assert res[k]["res_pri"] == pytest.approx(r["res_pri"], rel=1e-4, abs=0)
        for name in ("Mx", "x0", "a"):
            assert torch.equal(states[k][name], ref[name]), (k, name)


@pytest.mark.parametrize("mode", ["prox", "fixed_first"])
def test_batch_sequences_match_oracle(lib, mode):
    """Every sequence of the uneven batch against the FP64 oracle trajectory
    (its own size, hence its own step sizes from Theorem 1's lambda_max)."""
    n = 40
    ins = [seq_inputs(20 + k, *sz) for k, sz in enumerate(SIZES)]
    with lib.ProxBatch(SIZES, mode=mode, **KW) as bt:
        for k, (p0, p1) in enumerate(ins):
            bt.set_input(k, p0, p1)
        bt.step(n)
        got = [{k: v.double().cpu().numpy() for k, v in bt.get_state(q).items()} for q in range(len(SIZES))]
    for q, (p0, p1) in enumerate(ins):
        st = P.iterate(p0.astype(np.float64), p1.astype(np.float64), P.ProxParams(mode=mode, **KW), n)
        for name in ("Mx", "My", "x0", "x1", "r", "a"):
            o = getattr(st, name)
            e = np.linalg.norm(got[q][name] - o) / max(np.linalg.norm(o), 1e-3 * np.linalg.norm(p0))
            assert e <= 1e-5 * max(1, n / 20), (q, name, e)


def test_batch_autotune_keeps_results(lib):
    ins = [seq_inputs(30 + k, *sz) for k, sz in enumerate(SIZES)]
    with lib.ProxBatch(SIZES, **KW) as bt:
        for k, (p0, p1) in enumerate(ins):
            bt.set_input(k, p0, p1)
        cfg = bt.autotune()
        assert cfg["kernel"] in ("tma", "tiled") and cfg["tile_rows"] in (8, 16)
        assert cfg["ctas_per_sm"] in (1, 2, 4) and cfg["ms_per_iter"] > 0
        bt.reset()
        bt.step(5)
        got = bt.get_state(2)
    ref = single_state(lib, *SIZES[2], *ins[2], 5)
    assert torch.equal(got["Mx"], ref["Mx"]) and torch.equal(got["a"], ref["a"])


def test_batch_rejects_bad_parameters(lib):
    with pytest.raises(lib.OtError):
        lib.ProxBatch(SIZES, check_every=7, **KW)
    with pytest.raises(lib.OtError):
        lib.ProxBatch(SIZES, tau1=0.1, **KW)
    with pytest.raises(lib.OtError):
        lib.ProxBatch([(1, 0, 5)], **KW)
