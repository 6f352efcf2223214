"""Pins of the U-Net oracle: the convolution against SciPy's correlation,
pooling/upsampling against their definitions, and the whole backward pass
against central finite differences of the loss."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import unet as U


def test_conv2d_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv2d(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, c], w[o, c], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def test_pool_and_upsample_are_adjoint():
    """<up2(a), b> = 4 <a, avgpool2(b)>: the two are adjoint up to the factor 4."""
    rng = np.random.default_rng(1)
    a = rng.normal(size=(2, 3, 4, 5))
    b = rng.normal(size=(2, 3, 8, 10))
    assert np.isclose(np.sum(U.up2(a) * b), 4 * np.sum(a * U.avgpool2(b)))
    assert np.allclose(U.avgpool2(U.up2(a)), a)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    base = 2
    params = U.init_params(rng, base)
    # non-zero biases so that every ReLU pattern is exercised
    params = {k: (w, rng.normal(0, 0.1, b.shape)) for k, (w, b) in params.items()}
    x = rng.normal(size=(2, 2, 8, 8))
    t = rng.normal(size=(2, 4, 8, 8))
    out, cache = U.forward(params, x)
    _, g = U.mse(out, t)
    grads = U.backward(params, cache, g)
    eps = 1e-6
    for name in ("enc0a", "bottb", "dec1a", "head"):
        w, b = params[name]
        for idx in [tuple(rng.integers(0, s) for s in w.shape) for _ in range(3)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            pp = dict(params)
            pp[name] = (wp, b)
            lp = U.mse(U.forward(pp, x)[0], t)[0]
            pp[name] = (wm, b)
            lm = U.mse(U.forward(pp, x)[0], t)[0]
            fd = (lp - lm) / (2 * eps)
            assert abs(grads[name][0][idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, idx, grads[name][0][idx], fd)
        k = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[k] += eps
        bm[k] -= eps
        pp = dict(params)
        pp[name] = (w, bp)
        lp = U.mse(U.forward(pp, x)[0], t)[0]
        pp[name] = (w, bm)
        lm = U.mse(U.forward(pp, x)[0], t)[0]
        assert abs(grads[name][1][k] - (lp - lm) / (2 * eps)) <= 1e-6 * max(1.0, abs((lp - lm) / (2 * eps)))


def test_round_bf16_matches_torch_conversion():
    """The oracle's bfloat16 rounding against PyTorch's float32 -> bfloat16
    conversion (round to nearest even) on values of many magnitudes."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = (rng.normal(size=20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.round_bf16(x), want)


def test_round_bf16_ties_go_to_even():
    one = 1.0
    assert U.round_bf16(one + 2.0 ** -8) == 1.0                 # halfway to 1 + 2^-7: even is 1
    assert U.round_bf16(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # halfway: even is 1 + 2^-6
    assert U.round_bf16(-(one + 2.0 ** -8)) == -1.0
    assert U.round_bf16(0.0) == 0.0
    v = np.array([0.5, 1.0 + 2.0 ** -7, -3.0, 2.0 ** -100])
    assert np.array_equal(U.round_bf16(v), v)                   # already 8 significant bits
    assert U.round_bf16(1.0 + 2.0 ** -9) == 1.0


def test_rounded_network_stays_near_fp64():
    """Storage rounding perturbs the output by about the bfloat16 unit
    roundoff (2^-9) per stored tensor: visibly, but far below O(1)."""
    rng = np.random.default_rng(4)
    params = U.init_params(rng, 2)
    params = {k: (w, rng.normal(0, 0.1, b.shape)) for k, (w, b) in params.items()}
    x = rng.normal(size=(2, 2, 16, 16))
    y64, _ = U.forward(params, x)
    y16, _ = U.forward(params, x, rnd=U.round_bf16)
    e = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < e < 2e-2
