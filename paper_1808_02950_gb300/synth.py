"""Seeded synthetic inputs standing in for the paper's image and video data.

The paper's still-image experiment (§6.1) uses 44 USC-SIPI images (average
inter-pixel correlation about 0.86) and its video experiment (§6.2) uses the
HEVC common-test-condition sequences; neither is available here.  These
generators produce inputs with the same shapes and statistics: separable
first-order Markov (AR(1)) fields, the model under which the paper assesses
transforms (§4.2, rho = 0.95), with optional step edges, and video frames
made of a moving AR(1) texture plus noise, whose frame differences are the
int16 residual planes.

This module holds no arithmetic of the codec.  It is shared by the CUDA
tests, the benchmark and the oracle tests: both sides of every comparison
consume the same generated bytes.  Fields are drawn with torch on the device
they are generated on (CPU for small cases, CUDA for the large workloads);
the bytes depend on that device, so a comparison always copies one
generation to the other side rather than regenerating.

AR(1) field: e ~ N(0, 1) i.i.d.; along each row x_0 = e_0 / sqrt(1 - rho^2),
x_j = rho x_{j-1} + e_j; the same recursion along each column of the
result.  The stationary standard deviation is sigma = 1 / (1 - rho^2).
Pixel = clamp(round_half_even(mean + std * f / sigma), 0, 255).
"""
from __future__ import annotations

import math

import numpy as np
import torch

WORKLOADS = {
    "single_512": "one 512x512 u8 AR(1) image (rho 0.95), r = 10",
    "sweep_64x512": "64 u8 512x512 AR(1) images, rho ~ U[0.85, 0.98], half with step edges, r = 1..64",
    "batch_1024x1024": "1024 u8 1024x1024 AR(1) images (rho 0.95), r = 16",
    "ragged_2000": "2000 u8 images, H and W ~ U{64, 72, ..., 4096}, rho ~ U[0.85, 0.98], r ~ U{4, 8, 16, 32}",
    "video_600x1080p": "599 int16 residual frames of 1920x1080 4:2:0 video (Y r = 16, U/V r = 8)",
}


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _ar1_scan(x: torch.Tensor, rho: torch.Tensor, dim: int) -> torch.Tensor:
    """x_j <- sum_{m <= j} rho^(j - m) x_m along `dim` (log-depth scan)."""
    n = x.shape[dim]
    p = rho.clone()
    s = 1
    while s < n:
        head = x.narrow(dim, 0, n - s)
        tail = x.narrow(dim, s, n - s)
        upd = tail + p * head
        x = torch.cat([x.narrow(dim, 0, s), upd], dim=dim)
        p = p * p
        s *= 2
    return x


def ar1_fields(B: int, H: int, W: int, rho, gen: torch.Generator, device) -> torch.Tensor:
    """B separable AR(1) fields of size H x W, unit stationary variance (float32)."""
    rho_t = torch.as_tensor(rho, dtype=torch.float32, device=device).reshape(-1, 1, 1)
    if rho_t.shape[0] == 1 and B > 1:
        rho_t = rho_t.expand(B, 1, 1)
    e = torch.randn((B, H, W), generator=gen, device=device, dtype=torch.float32)
    a = torch.sqrt(1.0 - rho_t * rho_t)
    e[:, :, 0:1] = e[:, :, 0:1] / a
    x = _ar1_scan(e, rho_t, dim=2)
    x[:, 0:1, :] = x[:, 0:1, :] / a
    x = _ar1_scan(x, rho_t, dim=1)
    sigma = 1.0 / (1.0 - rho_t * rho_t)
    return x / sigma


def to_u8(f: torch.Tensor, mean: float = 128.0, std: float = 40.0) -> torch.Tensor:
    return torch.clamp(torch.round(mean + std * f), 0, 255).to(torch.uint8)


def ar1_images(B: int, H: int, W: int, rho, seed: int, device="cpu", chunk: int = 64) -> torch.Tensor:
    """B u8 AR(1) images (mean 128, std 40), generated in chunks of images."""
    out = torch.empty((B, H, W), dtype=torch.uint8, device=device)
    rho_all = np.broadcast_to(np.asarray(rho, dtype=np.float64), (B,))
    for c0 in range(0, B, chunk):
        c1 = min(B, c0 + chunk)
        g = _gen(seed * 100003 + c0, device)
        out[c0:c1] = to_u8(ar1_fields(c1 - c0, H, W, rho_all[c0:c1].astype(np.float32), g, device))
    return out


# ---- the five workloads ---------------------------------------------------------


def single_512(device="cpu", seed: int = 1):
    """One 512x512 u8 AR(1) image, rho 0.95 (4096 blocks); r = 10."""
    return ar1_images(1, 512, 512, 0.95, seed, device)[0], 10


def sweep_64x512(device="cpu", seed: int = 2, n: int = 64):
    """64 u8 512x512 AR(1) images, rho ~ U[0.85, 0.98]; images n/2.. get 3-10 step edges.

    Each edge: axis h or v, position ~ U{1, ..., dim - 1}, integer amplitude
    ~ U{40, ..., 120} with a random sign, added to every sample on the far
    side of the position; clamping to [0, 255] after all edges.
    """
    rs = np.random.default_rng(seed)
    rho = rs.uniform(0.85, 0.98, size=n)
    f = torch.empty((n, 512, 512), dtype=torch.float32, device=device)
    g = _gen(seed, device)
    for c0 in range(0, n, 16):
        c1 = min(n, c0 + 16)
        f[c0:c1] = 128.0 + 40.0 * ar1_fields(c1 - c0, 512, 512, rho[c0:c1].astype(np.float32), g, device)
    f = torch.round(f)
    for i in range(n // 2, n):
        for _ in range(int(rs.integers(3, 11))):
            axis = int(rs.integers(0, 2))
            pos = int(rs.integers(1, 512))
            amp = float(rs.integers(40, 121)) * (1.0 if rs.integers(0, 2) else -1.0)
            if axis == 0:
                f[i, pos:, :] += amp
            else:
                f[i, :, pos:] += amp
    imgs = torch.clamp(f, 0, 255).to(torch.uint8)
    return imgs, rho


def batch_1024x1024(device="cuda", seed: int = 3, n: int = 1024):
    """n u8 1024x1024 AR(1) images, rho 0.95, as one [n, 1024, 1024] tensor; r = 16."""
    return ar1_images(n, 1024, 1024, 0.95, seed, device, chunk=32), 16


def ragged_2000_params(seed: int = 4, n: int = 2000):
    """Per-image (H, W, rho, r) of the ragged batch."""
    rs = np.random.default_rng(seed)
    H = 8 * rs.integers(8, 513, size=n)
    W = 8 * rs.integers(8, 513, size=n)
    rho = rs.uniform(0.85, 0.98, size=n)
    r = rs.choice(np.array([4, 8, 16, 32]), size=n)
    return H.astype(np.int64), W.astype(np.int64), rho, r.astype(np.int64)


def ragged_2000(device="cuda", seed: int = 4, n: int = 2000, indices=None):
    """The ragged batch packed into one flat u8 buffer (tight pitch = W).

    Returns (buffer, offsets, H, W, r) with plane i at buffer[offsets[i]:],
    offsets 256-byte aligned.  ``indices`` restricts generation to a subset
    (the other planes stay zero).
    """
    H, W, rho, r = ragged_2000_params(seed, n)
    sizes = H * W
    offs = np.zeros(n, dtype=np.int64)
    acc = 0
    for i in range(n):
        offs[i] = acc
        acc += (int(sizes[i]) + 255) // 256 * 256
    buf = torch.zeros(acc, dtype=torch.uint8, device=device)
    for i in (range(n) if indices is None else indices):
        g = _gen(seed * 100003 + i, device)
        img = to_u8(ar1_fields(1, int(H[i]), int(W[i]), float(rho[i]), g, device))[0]
        buf[offs[i]: offs[i] + sizes[i]] = img.reshape(-1)
    return buf, offs, H, W, r


def video_600x1080p(device="cuda", seed: int = 5, frames: int = 600):
    """int16 residual planes of a synthetic 1920x1080 4:2:0 sequence.

    A 2160x3840 luma texture (AR(1), rho 0.95, mean 128, std 40) and two
    1080x1920 chroma textures (std 20) are read toroidally at an integer
    offset that random-walks by U{-8..8}^2 per frame (chroma at half the
    offset, floored); N(0, 3^2) noise is added per sample, rounded half to
    even and clamped to [0, 255].  Residual t = F_t - F_{t-1}, t = 1..599
    (the first frame is intra, not a residual).  Returns
    (Y [599,1080,1920], U [599,540,960], V [599,540,960]) int16 tensors.
    """
    rs = np.random.default_rng(seed)
    steps = rs.integers(-8, 9, size=(frames, 2))
    steps[0] = 0
    off = np.cumsum(steps, axis=0)
    g = _gen(seed, device)
    texY = 128.0 + 40.0 * ar1_fields(1, 2160, 3840, 0.95, g, device)[0]
    texU = 128.0 + 20.0 * ar1_fields(1, 1080, 1920, 0.95, g, device)[0]
    texV = 128.0 + 20.0 * ar1_fields(1, 1080, 1920, 0.95, g, device)[0]

    def frame(tex, oy, ox, h, w):
        ys = (torch.arange(h, device=device) + int(oy)) % tex.shape[0]
        xs = (torch.arange(w, device=device) + int(ox)) % tex.shape[1]
        f = tex.index_select(0, ys).index_select(1, xs)
        f = f + 3.0 * torch.randn((h, w), generator=g, device=device, dtype=torch.float32)
        return torch.clamp(torch.round(f), 0, 255).to(torch.int16)

    Y = torch.empty((frames - 1, 1080, 1920), dtype=torch.int16, device=device)
    U = torch.empty((frames - 1, 540, 960), dtype=torch.int16, device=device)
    V = torch.empty((frames - 1, 540, 960), dtype=torch.int16, device=device)
    prev = None
    for t in range(frames):
        oy, ox = off[t]
        cur = (
            frame(texY, oy, ox, 1080, 1920),
            frame(texU, math.floor(oy / 2), math.floor(ox / 2), 540, 960),
            frame(texV, math.floor(oy / 2), math.floor(ox / 2), 540, 960),
        )
        if prev is not None:
            Y[t - 1] = cur[0] - prev[0]
            U[t - 1] = cur[1] - prev[1]
            V[t - 1] = cur[2] - prev[2]
        prev = cur
    return Y, U, V


def adversarial_blocks(device="cpu") -> torch.Tensor:
    """8x8 u8 blocks at the extremes: constants, checkerboards and the sign
    patterns of the outer products of the rows of T1 (which maximise |Z| and
    the intermediate magnitudes), as one [8, 8 * count] plane."""
    t1 = np.array(
        [[1, 1, 1, 1, 1, 1, 1, 1], [2, 2, 1, 0, 0, -1, -2, -2], [2, 1, -1, -2, -2, -1, 1, 2],
         [1, 0, -2, -2, 2, 2, 0, -1], [1, -1, -1, 1, 1, -1, -1, 1], [2, -2, 0, 1, -1, 0, 2, -2],
         [1, -2, 2, -1, -1, 2, -2, 1], [0, -1, 2, -2, 2, -2, 1, 0]])
    blocks = [np.zeros((8, 8)), np.full((8, 8), 255), np.full((8, 8), 128), np.full((8, 8), 127)]
    cb = (np.indices((8, 8)).sum(0) % 2) * 255
    blocks += [cb, 255 - cb]
    for i in range(8):
        for j in range(8):
            s = np.sign(np.outer(t1[i], t1[j]))
            blocks.append(np.where(s > 0, 255, 0))
            blocks.append(np.where(s >= 0, 255, 0))
    arr = np.concatenate([b.astype(np.uint8) for b in blocks], axis=1)
    return torch.from_numpy(np.ascontiguousarray(arr)).to(device)
