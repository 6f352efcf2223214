"""The warm-start U-Net's CUDA kernels against the FP64 oracle network.

The oracle runs with the same BF16-rounded weights the kernels multiply by
(biases stay FP32 on both sides) and rounds every stored activation and
activation gradient to bfloat16 where the kernels do (``rnd=round_bf16``).
What remains is FP32 against FP64 accumulation: it moves some values across
a bfloat16 rounding boundary (one bfloat16 unit, 2^-8 relative, each), and a
random network amplifies these flips layer by layer.  The test measures that
floor on the oracle itself: the same network with every stored value first
perturbed by a relative 2^-22 (below the FP32 accumulation error of these
sums) and then rounded.  The GPU must agree with the oracle within three
times that spread (at least 2e-3), norm-wise per tensor; a wrong tap,
channel, layout or mask gives errors of order one.  Sizes are ragged on
purpose: 24 x 40 pixels is not a multiple of the 16 x 8 tensor-core tile
(the coarsest level is 3 x 5 pixels, smaller than one tile) nor of the
16 x 16 weight-gradient tile.
"""
import numpy as np
import pytest
import torch

from oracle import unet as U

pytestmark = pytest.mark.gpu

H, W, BASE, N = 24, 40, 32, 3


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def random_params(seed, base):
    rng = np.random.default_rng(seed)
    params = U.init_params(rng, base)
    return {k: (w.astype(np.float32).astype(np.float64), rng.normal(0, 0.1, b.shape).astype(np.float32).astype(np.float64))
            for k, (w, b) in params.items()}


def flat(params, base):
    parts = []
    for name, _, _, _ in U.layer_specs(base):
        w, b = params[name]
        parts += [w.ravel(), b.ravel()]
    return np.concatenate(parts).astype(np.float32)


def unflat(vec, base):
    out, off = {}, 0
    for name, ci, co, k in U.layer_specs(base):
        nw = co * ci * k * k
        out[name] = (vec[off:off + nw].reshape(co, ci, k, k), vec[off + nw:off + nw + co])
        off += nw + co
    assert off == vec.size
    return out


def inputs(seed, n=N, h=H, w=W):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 2, h, w)).astype(np.float32)
    t = (rng.normal(size=(n, 4, h, w)) * 0.5).astype(np.float32)
    return x, t


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


def perturbed_rounding(seed):
    """bfloat16 rounding after a relative 2^-22 Gaussian perturbation."""
    rng = np.random.default_rng(seed)

    def rnd(v):
        return U.round_bf16(v * (1.0 + 2.0 ** -22 * rng.standard_normal(np.shape(v))))
    return rnd


def tol(noisy, ref):
    return max(3.0 * rel(noisy, ref), 2e-3)


def test_layer_order_matches_oracle(lib):
    assert [s for s in lib.unet_layer_specs(BASE)] == U.layer_specs(BASE)
    with lib.UNet(H, W, N, BASE) as net:
        assert net.n_params == sum(co * ci * k * k + co for _, ci, co, k in U.layer_specs(BASE))


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_matches_oracle(lib, seed):
    params = random_params(seed, BASE)
    x, _ = inputs(seed)
    with lib.UNet(H, W, N, BASE) as net:
        net.set_params(flat(params, BASE))
        got = net.forward(x).cpu().numpy()
    ref = {k: (bf16(w), b) for k, (w, b) in params.items()}
    out, _ = U.forward(ref, x.astype(np.float64), rnd=U.round_bf16)
    noisy, _ = U.forward(ref, x.astype(np.float64), rnd=perturbed_rounding(seed))
    assert rel(got, out) <= tol(noisy, out), (rel(got, out), rel(noisy, out))


@pytest.mark.parametrize("seed", [2, 3])
def test_gradients_match_oracle(lib, seed):
    params = random_params(seed, BASE)
    x, t = inputs(seed)
    with lib.UNet(H, W, N, BASE) as net:
        net.set_params(flat(params, BASE))
        loss, g = net.gradients(x, t)
    ref = {k: (bf16(w), b) for k, (w, b) in params.items()}

    def oracle(rnd):
        out, cache = U.forward(ref, x.astype(np.float64), rnd=rnd)
        l_ref, g_out = U.mse(out, t.astype(np.float64))
        return l_ref, U.backward(ref, cache, g_out, rnd=rnd)
    l_ref, grads = oracle(U.round_bf16)
    l_noisy, noisy = oracle(perturbed_rounding(seed))
    assert abs(loss - l_ref) <= max(3 * abs(l_noisy - l_ref), 1e-3 * l_ref)
    got = unflat(g, BASE)
    for name, _, _, _ in U.layer_specs(BASE):
        for j in (0, 1):
            e, bound = rel(got[name][j], grads[name][j]), tol(noisy[name][j], grads[name][j])
            assert e <= bound, (name, j, e, bound)


def test_gradients_are_deterministic_and_batch_independent(lib):
    """Fixed summation order: identical calls give identical bits; a larger
    handle (more splits available) gives the same loss on the same batch."""
    params = random_params(4, BASE)
    x, t = inputs(4)
    with lib.UNet(H, W, N, BASE) as net:
        net.set_params(flat(params, BASE))
        l1, g1 = net.gradients(x, t)
        l2, g2 = net.gradients(x, t)
    assert l1 == l2 and np.array_equal(g1, g2)
    with lib.UNet(H, W, 8, BASE) as net:
        net.set_params(flat(params, BASE))
        l3, _ = net.gradients(x, t)
    assert l3 == pytest.approx(l1, rel=1e-6)


def test_first_adam_step_is_a_signed_step(lib):
    """After one Adam step from zero moments, m_hat = g and v_hat = g^2, so
    every parameter moves by -lr g / (|g| + eps)."""
    params = random_params(5, BASE)
    x, t = inputs(5)
    lr = 1e-3
    with lib.UNet(H, W, N, BASE) as net:
        p0 = flat(params, BASE)
        net.set_params(p0)
        _, g = net.gradients(x, t)
        net.train_step(x, t, lr)
        p1 = net.get_params()
    want = p0.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, want, rtol=1e-6, atol=1e-6 * lr)


def test_training_reduces_loss(lib):
    rng = np.random.default_rng(6)
    x, _ = inputs(6, n=4, h=32, w=32)
    # a target the network can represent: smooth functions of the input
    t = np.concatenate([x[:, :1] - x[:, 1:], 0.5 * x[:, :1], x[:, 1:] ** 2, np.sin(3 * x[:, :1])], axis=1)
    t = t.astype(np.float32) + 0.01 * rng.normal(size=t.shape).astype(np.float32)
    with lib.UNet(32, 32, 4, 32) as net:
        net.init(seed=0)
        losses = [net.train_step(x, t, 2e-3) for _ in range(60)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def test_unet_rejects_bad_arguments(lib):
    with pytest.raises(lib.OtError):
        lib.UNet(20, 24, 1, 32)         # H not a multiple of 8
    with pytest.raises(lib.OtError):
        lib.UNet(16, 16, 0, 32)
    with pytest.raises(lib.OtError):
        lib.UNet(16, 16, 1, 16)         # the tensor-core tiles take 32 base channels
    with lib.UNet(16, 16, 2, 32) as net:
        x = np.zeros((3, 2, 16, 16), np.float32)
        with pytest.raises(lib.OtError):
            net.forward(x)              # batch above max_batch


def one_hot_params(seed, base):
    """Each output channel copies one input channel at one tap with weight
    +-1 (a quarter negative, so ReLU clips), biases in multiples of 2^-6.
    With inputs in multiples of 2^-6 every sum the network forms is exact in
    FP32 (all values are multiples of 2^-12 below 8), so the bfloat16
    roundings see identical values on both sides."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co, k in U.layer_specs(base):
        w = np.zeros((co, ci, k, k))
        for o in range(co):
            w[o, rng.integers(0, ci), rng.integers(0, k), rng.integers(0, k)] = -1.0 if rng.random() < 0.25 else 1.0
        params[name] = (w, rng.integers(0, 8, co) * 2.0 ** -6)
    return params


def test_exact_network_forward_is_bit_identical(lib):
    params = one_hot_params(7, BASE)
    rng = np.random.default_rng(7)
    x = (rng.integers(16, 64, size=(N, 2, H, W)) / 64.0).astype(np.float32)
    with lib.UNet(H, W, N, BASE) as net:
        net.set_params(flat(params, BASE))
        got = net.forward(x).cpu().numpy().astype(np.float64)
    out, _ = U.forward(params, x.astype(np.float64), rnd=U.round_bf16)
    assert np.count_nonzero(out) > out.size // 4
    assert np.array_equal(got, out), np.max(np.abs(got - out))


def test_exact_network_gradients(lib):
    """Target 0 and 4 n H W a power of two make the loss gradient exact too;
    the data gradients (sums of a few bfloat16 values) then match bit for bit
    and the weight gradients differ only by FP32 summation over the pixels."""
    n, h, w = 2, 8, 128
    params = one_hot_params(8, BASE)
    rng = np.random.default_rng(8)
    x = (rng.integers(16, 64, size=(n, 2, h, w)) / 64.0).astype(np.float32)
    t = np.zeros((n, 4, h, w), np.float32)
    with lib.UNet(h, w, n, BASE) as net:
        net.set_params(flat(params, BASE))
        loss, g = net.gradients(x, t)
    out, cache = U.forward(params, x.astype(np.float64), rnd=U.round_bf16)
    l_ref, g_out = U.mse(out, t.astype(np.float64))
    grads = U.backward(params, cache, g_out, rnd=U.round_bf16)
    assert loss == pytest.approx(l_ref, rel=1e-6)
    got = unflat(g, BASE)
    for name, _, _, _ in U.layer_specs(BASE):
        for j in (0, 1):
            assert rel(got[name][j], grads[name][j]) <= 1e-4, (name, j, rel(got[name][j], grads[name][j]))


def test_bias_free_training_keeps_zero_biases_and_a_zero_far_field(lib):
    """Bias-free: every bias gradient is reported as 0, so Adam leaves the
    zero biases alone, and an all-zero neighbourhood maps to exactly 0."""
    S = 256
    rng = np.random.default_rng(9)
    x = np.zeros((2, 2, S, S), np.float32)
    x[:, :, :24, :24] = rng.random((2, 2, 24, 24))
    t = rng.normal(size=(2, 4, S, S)).astype(np.float32) * (x[:, :1] > 0)
    with lib.UNet(S, S, 2, BASE, bias_free=True) as net:
        net.init(seed=1)
        for _ in range(3):
            net.train_step(x, t, 1e-3)
        params = unflat(net.get_params(), BASE)
        y = net.forward(x).cpu().numpy()
    assert all(np.all(b == 0) for _, b in params.values())
    assert np.count_nonzero(y[:, :, :24, :24]) > 0
    assert np.all(y[:, :, 128:, :] == 0) and np.all(y[:, :, :, 128:] == 0)
