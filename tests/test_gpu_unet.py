"""The warm-start U-Net's CUDA kernels against the FP64 oracle network.

The oracle runs with the same BF16-rounded weights the kernels multiply by
(biases stay FP32 on both sides), so the only differences are FP32
accumulation and rounding of activations: the forward output, the loss and
every parameter's gradient agree to a relative ``1e-4`` (norm-wise per
layer).  Sizes are ragged on purpose: 24 x 40 pixels is not a multiple of the
16 x 16 pixel tile, 20 base channels are not a multiple of the 16-channel
output block nor of the 8-channel input stage.
"""
import numpy as np
import pytest
import torch

from oracle import unet as U

pytestmark = pytest.mark.gpu

H, W, BASE, N = 24, 40, 20, 2


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
    out, _ = U.forward(ref, x.astype(np.float64))
    assert rel(got, out) <= 1e-4
    assert np.max(np.abs(got - out)) <= 1e-4 * np.max(np.abs(out))


@pytest.mark.parametrize("seed", [2, 3])
def test_gradients_match_oracle(lib, seed):
    params = random_params(seed, BASE)
    x, t = inputs(seed)
    with lib.UNet(H, W, N, BASE) as net:
        net.set_params(flat(params, BASE))
        loss, g = net.gradients(x, t)
    ref = {k: (bf16(w), b) for k, (w, b) in params.items()}
    out, cache = U.forward(ref, x.astype(np.float64))
    l_ref, g_out = U.mse(out, t.astype(np.float64))
    grads = U.backward(ref, cache, g_out)
    assert loss == pytest.approx(l_ref, rel=1e-5)
    got = unflat(g, BASE)
    for name, _, _, _ in U.layer_specs(BASE):
        assert rel(got[name][0], grads[name][0]) <= 1e-4, name
        assert rel(got[name][1], grads[name][1]) <= 1e-4, name


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
    with lib.UNet(32, 32, 4, 8) as net:
        net.init(seed=0)
        losses = [net.train_step(x, t, 2e-3) for _ in range(60)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def test_unet_rejects_bad_arguments(lib):
    with pytest.raises(lib.OtError):
        lib.UNet(20, 24, 1, 4)          # H not a multiple of 8
    with pytest.raises(lib.OtError):
        lib.UNet(16, 16, 0, 4)
    with lib.UNet(16, 16, 2, 4) as net:
        x = np.zeros((3, 2, 16, 16), np.float32)
        with pytest.raises(lib.OtError):
            net.forward(x)              # batch above max_batch
