"""Seeded synthetic inputs for the unbalanced Beckmann-OT proximal path.

This module only draws random numbers and lays out images; it holds none of
the method's arithmetic, so the FP64 oracle and the CUDA path can both read
its output without sharing any part of the computation they are compared on.

Every generator returns float32 arrays: the GPU consumes them as they are and
the oracle promotes the same rounded values to float64, so the two sides start
from bit-identical inputs.

Workloads (sizes and distributions follow the paper's synthetic setups of
Sec. IV-A.2 and Sec. IV-B.3: Gaussian targets moving on a pixel grid, mass
growth/decay on the interval [0.5, 1.5], a low-rank non-negative clutter):

* ``blob_pairs``  -- frame pairs (p0, p1) of Gaussian blobs, the second frame
  shifted by integer offsets, one blob's amplitude rescaled (unbalanced).
* ``blob_video``  -- a T-frame sequence of moving blobs (the pair batch of a
  video is frames t, t+1).
* ``rpca_video``  -- Y = L + S + noise: rank-3 smooth background, moving sparse
  blobs that appear and disappear, i.i.d. Gaussian noise.
* ``uneven_sequences`` -- many sequences of uneven H, W, T.
"""
from __future__ import annotations

import numpy as np

SEED0 = 190900149


def rng_for(workload: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator seeded from a workload number (and an optional stream)."""
    return np.random.Generator(np.random.PCG64([SEED0 + workload, stream]))


def _blob(H: int, W: int, cy: float, cx: float, amp: float, sigma: float) -> np.ndarray:
    ii = np.arange(H, dtype=np.float64)[:, None]
    jj = np.arange(W, dtype=np.float64)[None, :]
    return amp * np.exp(-((ii - cy) ** 2 + (jj - cx) ** 2) / (2.0 * sigma * sigma))


def blob_pairs(rng: np.random.Generator, B: int, H: int, W: int, n_blobs: int = 3,
               sigma: float = 3.0, max_shift: int = 4) -> tuple[np.ndarray, np.ndarray]:
    """B independent frame pairs [B, H, W] (float32, non-negative).

    p0: ``n_blobs`` Gaussian blobs (std ``sigma`` px, amplitude U[0.5, 1]),
    centres uniform in the central 5/8 of the frame.  p1: the same blobs moved
    by integer offsets drawn from {-max_shift..max_shift}^2, and one blob's
    amplitude multiplied by U[0.5, 1.5].
    """
    p0 = np.zeros((B, H, W), np.float64)
    p1 = np.zeros((B, H, W), np.float64)
    for b in range(B):
        cy = rng.uniform(0.1875 * H, 0.8125 * H, n_blobs)
        cx = rng.uniform(0.1875 * W, 0.8125 * W, n_blobs)
        amp = rng.uniform(0.5, 1.0, n_blobs)
        dy = rng.integers(-max_shift, max_shift + 1, n_blobs)
        dx = rng.integers(-max_shift, max_shift + 1, n_blobs)
        k = int(rng.integers(0, n_blobs))
        scale = rng.uniform(0.5, 1.5)
        for n in range(n_blobs):
            p0[b] += _blob(H, W, cy[n], cx[n], amp[n], sigma)
            a1 = amp[n] * (scale if n == k else 1.0)
            p1[b] += _blob(H, W, cy[n] + dy[n], cx[n] + dx[n], a1, sigma)
    return p0.astype(np.float32), p1.astype(np.float32)


def blob_video(rng: np.random.Generator, T: int, H: int, W: int, n_blobs: int = 3,
               sigma: float = 3.0, max_step: int = 4) -> np.ndarray:
    """T frames [T, H, W] of blobs taking integer steps in [-max_step, max_step]^2
    per frame (reflected at the borders); each frame one blob's amplitude is
    multiplied by U[0.5, 1.5] (clamped to [0.25, 2])."""
    cy = rng.uniform(0.1875 * H, 0.8125 * H, n_blobs)
    cx = rng.uniform(0.1875 * W, 0.8125 * W, n_blobs)
    amp = rng.uniform(0.5, 1.0, n_blobs)
    out = np.zeros((T, H, W), np.float64)
    for t in range(T):
        for n in range(n_blobs):
            out[t] += _blob(H, W, cy[n], cx[n], amp[n], sigma)
        cy = cy + rng.integers(-max_step, max_step + 1, n_blobs)
        cx = cx + rng.integers(-max_step, max_step + 1, n_blobs)
        cy = np.where(cy < 0, -cy, cy)
        cy = np.where(cy > H - 1, 2 * (H - 1) - cy, cy)
        cx = np.where(cx < 0, -cx, cx)
        cx = np.where(cx > W - 1, 2 * (W - 1) - cx, cx)
        k = int(rng.integers(0, n_blobs))
        amp[k] = float(np.clip(amp[k] * rng.uniform(0.5, 1.5), 0.25, 2.0))
    return out.astype(np.float32)


def warmstart_pairs(rng: np.random.Generator, n: int, S: int):
    """n consecutive-frame pairs [n, S, S] (p0, p1) cut from 17-frame S x S
    blob videos with 3 to 8 blobs each (sigma 3 px, amplitude U[0.5, 1],
    integer moves in [-4, 4]^2 a frame, one amplitude rescaled a frame):
    the 64x64 pair's generator scaled up, for training the warm start."""
    p0s, p1s = [], []
    for k in range(0, n, 16):
        v = blob_video(rng, 17, S, S, n_blobs=int(rng.integers(3, 9)))
        m = min(16, n - k)
        p0s.append(v[:m])
        p1s.append(v[1:m + 1])
    return np.concatenate(p0s), np.concatenate(p1s)


def _smooth_pattern(rng: np.random.Generator, H: int, W: int, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    g = gaussian_filter(rng.uniform(0.0, 1.0, (H, W)), sigma=sigma, mode="wrap")
    g = g - g.min()
    return g / max(g.max(), 1e-30)


def rpca_video(rng: np.random.Generator, T: int = 64, H: int = 256, W: int = 256,
               rank: int = 3, n_blobs: int = 8, noise: float = 0.02,
               sigma_bg: float = 16.0, sigma_blob: float = 3.0, max_speed: float = 2.0):
    """Y = L + S + eta, each [T, H, W] float32.

    L: sum of ``rank`` smooth spatial patterns (Gaussian-filtered U[0,1]
    noise, normalised to [0, 1]) times temporal coefficients U[0.2, 1].
    S: ``n_blobs`` Gaussian blobs (amplitude U[0.5, 1]) moving at a constant
    velocity of at most ``max_speed`` px/frame, each present on a random
    sub-interval of frames.  eta: i.i.d. N(0, noise^2).
    Returns (Y, L, S).
    """
    L = np.zeros((T, H, W), np.float64)
    for _ in range(rank):
        P = _smooth_pattern(rng, H, W, sigma_bg)
        c = rng.uniform(0.2, 1.0, T)
        L += P[None, :, :] * c[:, None, None]
    S = np.zeros((T, H, W), np.float64)
    for _ in range(n_blobs):
        cy, cx = rng.uniform(0.15 * H, 0.85 * H), rng.uniform(0.15 * W, 0.85 * W)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        spd = rng.uniform(0.0, max_speed)
        vy, vx = spd * np.sin(ang), spd * np.cos(ang)
        amp = rng.uniform(0.5, 1.0)
        t0 = int(rng.integers(0, max(T // 2, 1)))
        t1 = int(rng.integers(t0 + 1, T + 1))
        for t in range(t0, t1):
            S[t] += _blob(H, W, cy + vy * (t - t0), cx + vx * (t - t0), amp, sigma_blob)
    eta = rng.normal(0.0, noise, (T, H, W))
    Y = L + S + eta
    return Y.astype(np.float32), L.astype(np.float32), S.astype(np.float32)


def signed_rpca_video(rng: np.random.Generator, T: int = 64, H: int = 256, W: int = 256,
                      rank: int = 3, n_blobs: int = 8, noise: float = 0.02, **kw):
    """As ``rpca_video``, but every second blob is darker than the
    background (its amplitude negated): the foreground of the signed
    variant, S = S+ - S-.  The background is lifted by 1 so that Y stays
    positive under the dark blobs.  Returns (Y, L, S)."""
    rng2 = np.random.Generator(np.random.PCG64(rng.integers(0, 2**63)))
    Y, L, S = rpca_video(rng, T, H, W, rank=rank, n_blobs=0, noise=noise, **kw)
    Sd = np.zeros((T, H, W), np.float64)
    sigma_blob, max_speed = kw.get("sigma_blob", 3.0), kw.get("max_speed", 2.0)
    for k in range(n_blobs):
        cy, cx = rng2.uniform(0.15 * H, 0.85 * H), rng2.uniform(0.15 * W, 0.85 * W)
        ang = rng2.uniform(0.0, 2.0 * np.pi)
        spd = rng2.uniform(0.0, max_speed)
        vy, vx = spd * np.sin(ang), spd * np.cos(ang)
        amp = rng2.uniform(0.5, 1.0) * (1.0 if k % 2 == 0 else -1.0)
        t0 = int(rng2.integers(0, max(T // 2, 1)))
        t1 = int(rng2.integers(t0 + 1, T + 1))
        for t in range(t0, t1):
            Sd[t] += _blob(H, W, cy + vy * (t - t0), cx + vx * (t - t0), amp, sigma_blob)
    L1 = L.astype(np.float64) + 1.0
    Y = Y.astype(np.float64) + 1.0 + Sd
    return Y.astype(np.float32), L1.astype(np.float32), Sd.astype(np.float32)


def uneven_sequences(rng: np.random.Generator, n_seq: int = 48,
                     sizes=(96, 128, 192, 256, 384), t_range=(8, 64)):
    """``n_seq`` blob videos with H, W drawn independently from ``sizes`` and
    T uniform in ``t_range`` (inclusive).  Returns a list of [T, H, W] arrays."""
    seqs = []
    for _ in range(n_seq):
        H = int(rng.choice(sizes))
        W = int(rng.choice(sizes))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        seqs.append(blob_video(rng, T, H, W, n_blobs=3))
    return seqs


def blob_pair_64x64(H: int = 64, W: int = 64):
    """Single 64x64 frame pair: 3 blobs, integer shifts in [-4, 4], one blob
    rescaled by U[0.5, 1.5].  Returns (p0, p1) shaped [1, H, W]."""
    return blob_pairs(rng_for(0), 1, H, W, n_blobs=3)


def rpca_video_64x256x256(T: int = 64, H: int = 256, W: int = 256):
    """The 64-frame 256x256 RPCA video (rank-3 clutter, 8 moving blobs,
    noise 0.02).  Returns (Y, L, S)."""
    return rpca_video(rng_for(1), T, H, W)
