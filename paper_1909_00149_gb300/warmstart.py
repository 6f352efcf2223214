"""Learned warm start of Algorithm 1: data, training and the warm solve.

Sec. III-B warm-starts Algorithm 1 from cached iterates.  Here the cache is
predicted by the U-Net of ``ot_unet_*`` from the frame pair alone, trained on
states that the plain solver reaches at its stopping rule.  From the
predicted state the plain iterations run to the same stopping rule, so the
network changes the iteration count, never the answer's tolerance.

Everything numerical runs in the library's kernels (the solver, the
network's forward and backward passes, Adam, the state write of
``ot_prox_warm_start``); this module only moves tensors into the layouts the
C calls take: the pair as [n, 2, H, W] and the state as [n, 4, H, W] in the
order (Mx, My, r, a).
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import OtProx, UNet

STATE_CHANNELS = ("Mx", "My", "r", "a")


def pair_tensor(p0, p1):
    """(p0, p1) [n, H, W] each, host or device -> [n, 2, H, W] CUDA tensor."""
    import torch
    p0 = torch.as_tensor(p0, dtype=torch.float32).cuda()
    p1 = torch.as_tensor(p1, dtype=torch.float32).cuda()
    return torch.stack([p0, p1], 1).contiguous()


def solve_targets(p0, p1, chunk: int = 128, **params):
    """Solve every pair with the plain method (cold start) in chunks of
    ``chunk`` problems; returns (inputs [n, 2, H, W], targets [n, 4, H, W],
    iterations per chunk), tensors on the GPU."""
    import torch
    n, H, W = np.shape(p0)
    X = torch.empty((n, 2, H, W), dtype=torch.float32, device="cuda")
    T = torch.empty((n, 4, H, W), dtype=torch.float32, device="cuda")
    iters = []
    for k in range(0, n, chunk):
        m = min(chunk, n - k)
        with OtProx(m, H, W, **params) as s:
            s.set_input(p0[k:k + m], p1[k:k + m])
            r = s.solve()
            st = s.get_state()
        iters.append(r["iters"])
        X[k:k + m] = pair_tensor(p0[k:k + m], p1[k:k + m])
        for c, name in enumerate(STATE_CHANNELS):
            T[k:k + m, c] = st[name]
    return X, T, iters


def train(net: UNet, X, T, epochs: int, batch: int, lr: float = 1e-3, seed: int = 0) -> list[float]:
    """Adam on the MSE between net(X) and T, cosine-decayed learning rate,
    shuffled mini-batches; returns the mean loss of each epoch."""
    import torch
    n = X.shape[0]
    g = torch.Generator().manual_seed(seed)
    steps = epochs * (n // batch)
    step = 0
    out = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        losses = []
        for k in range(0, n - batch + 1, batch):
            idx = perm[k:k + batch]
            rate = lr * 0.5 * (1.0 + np.cos(np.pi * step / max(steps, 1)))
            losses.append(net.train_step(X[idx].contiguous(), T[idx].contiguous(), rate))
            step += 1
        out.append(float(np.mean(losses)))
    return out


def solve(p0, p1, net: UNet | None = None, gate: float = 0.0, **params) -> dict:
    """Solve the pairs [B, H, W] to the stopping rule, from the network's
    prediction when ``net`` is given (its max_batch must cover B; ``gate`` as
    in ``OtProx.warm_start``), cold otherwise.  Returns the solver's result
    plus ``seconds`` (host time around prediction + solve, inputs already on
    the device)."""
    import torch
    B, H, W = np.shape(p0)
    x = pair_tensor(p0, p1) if net is not None else None
    with OtProx(B, H, W, **params) as s:
        s.set_input(p0, p1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if net is not None:
            s.warm_start(net.forward(x), gate)
        r = s.solve()
        torch.cuda.synchronize()
        r["seconds"] = time.perf_counter() - t0
    return r


# ---------------------------------------------------------------- trained weights
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_warmstart_256.npz")


def fold_output_scale(net: UNet, channel: int, factor: float) -> None:
    """Multiply output ``channel`` of the network by ``factor``: the last
    layer is a 1x1 convolution (weights [4, base], then biases [4]), so its
    weights and bias of that channel are scaled."""
    params = net.get_params().astype(np.float32)
    c = net.base
    off = params.size - (4 * c + 4)
    params[off + channel * c:off + (channel + 1) * c] *= factor
    params[off + 4 * c + channel] *= factor
    net.set_params(params)


def save_params(net: UNet, path: str, **meta) -> None:
    """The network's FP32 parameters (``ot_unet_get_params`` order) and the
    training record, as a compressed .npz."""
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path, params=net.get_params(), base_channels=net.base,
                        **{k: np.asarray(v) for k, v in meta.items()})


def load_params(net: UNet, path: str = WEIGHTS) -> dict:
    """Load parameters written by ``save_params`` into ``net``; returns the
    training record."""
    with np.load(path) as d:
        if int(d["base_channels"]) != net.base:
            raise ValueError(f"{path}: base_channels {int(d['base_channels'])} != {net.base}")
        net.set_params(d["params"].astype(np.float32))
        return {k: d[k].tolist() for k in d.files if k not in ("params", "base_channels")}


def main(argv=None) -> None:
    """Train the warm-start network and write its parameters:

        python -m paper_1909_00149_gb300.warmstart --pairs 20000 --size 256 \\
            --epochs 4 --out paper_1909_00149_gb300/weights/unet_warmstart_256.npz

    The training pairs come from the seeded blob-video generator of
    ``synth.warmstart_pairs`` (run from the repository root); their targets
    are the states the plain solver reaches at the 1e-5 stopping rule
    (mu = 3, rho = 0.01, the library's defaults)."""
    import argparse
    import sys
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--a-weight", type=float, default=1.0,
                    help="train on this multiple of the dual a (its squared error weighs a-weight^2 in the "
                         "loss); the factor is divided out of the output layer before saving")
    ap.add_argument("--normalize", action="store_true",
                    help="train on targets scaled to unit RMS per channel (equal relative errors); the scales "
                         "are divided out of the output layer before saving")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.getcwd())
    from synth import rng_for, warmstart_pairs
    kw = dict(mode="prox", mu=3.0, rho=0.01, tol=1e-5, max_iter=100000, check_every=10)
    t0 = time.perf_counter()
    p0, p1 = warmstart_pairs(rng_for(5, a.seed), a.pairs, a.size)
    X, T, its = solve_targets(p0, p1, **kw)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    del p0, p1
    rms = [float(torch.sqrt(torch.mean(T[:, c] ** 2))) for c in range(len(STATE_CHANNELS))]
    scale = [1.0 / max(r, 1e-30) if a.normalize else 1.0 for r in rms]
    scale[STATE_CHANNELS.index("a")] *= a.a_weight
    for c, f in enumerate(scale):
        if f != 1.0:
            T[:, c] *= f
    net = UNet(a.size, a.size, a.batch, 32)
    net.init(seed=0)
    t0 = time.perf_counter()
    losses = train(net, X, T, epochs=a.epochs, batch=a.batch, lr=a.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for c, f in enumerate(scale):
        if f != 1.0:
            fold_output_scale(net, c, 1.0 / f)
    save_params(net, a.out, pairs=a.pairs, size=a.size, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed,
                mu=kw["mu"], rho=kw["rho"], tol=kw["tol"], loss_per_epoch=np.array(losses),
                solve_seconds=t_solve, train_seconds=t_train, target_iters=np.array(its),
                a_weight=a.a_weight, normalized=a.normalize, target_rms=np.array(rms))
    print({"out": a.out, "loss_per_epoch": losses, "solve_s": round(t_solve, 1), "train_s": round(t_train, 1)},
          flush=True)


if __name__ == "__main__":
    main()
