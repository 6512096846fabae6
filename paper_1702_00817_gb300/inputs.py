"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds none of the codec's arithmetic: it only draws images.  The
paper evaluates on 45 greyscale 512x512 photographs from a public image bank
(Sec. 3), which are not available here; these generated images stand in for
them.  Recipe (one independent stream per image, seed = base + index):

    X(y, x) = clamp(rint(128 + sum_{k=1..8} A_k cos(2 pi (fx_k x / W + fy_k y / H) + phi_k))
                    + n(y, x), 0, 255)
    A_k ~ U[4, 24], fx_k, fy_k ~ U{0..8} cycles per image, phi_k ~ U[0, 2 pi),
    n ~ U{-16..16} per pixel.

Multi-channel images draw each channel in turn from the same stream.  The
cosine sum is evaluated through cos(a + b) = cos a cos b - sin a sin b as one
[H, 16] x [16, W] product so that large batches generate quickly.
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

BASE_SEED = 1702


def _cosine_plane(rng: np.random.Generator, height: int, width: int) -> np.ndarray:
    amp = rng.uniform(4.0, 24.0, 8)
    fx = rng.integers(0, 9, 8)
    fy = rng.integers(0, 9, 8)
    phi = rng.uniform(0.0, 2.0 * math.pi, 8)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[:, None]
    a = 2.0 * math.pi * fy[None, :] * ys / height + phi[None, :]  # [H, 8]
    b = 2.0 * math.pi * fx[None, :] * xs / width  # [W, 8]
    left = np.concatenate([np.cos(a) * amp, -np.sin(a) * amp], axis=1)  # [H, 16]
    right = np.concatenate([np.cos(b), np.sin(b)], axis=1)  # [W, 16]
    smooth = 128.0 + left @ right.T
    noise = rng.integers(-16, 17, size=(height, width))
    return np.clip(np.rint(smooth) + noise, 0, 255).astype(np.uint8)


def synth_image(height: int, width: int, seed: int, channels: int = 1) -> np.ndarray:
    """One image, [channels, height, width] uint8."""
    rng = np.random.default_rng(seed)
    return np.stack([_cosine_plane(rng, height, width) for _ in range(channels)])


def synth_image_device(height: int, width: int, seed: int, channels: int = 1, device="cuda"):
    """Same recipe evaluated on a CUDA device in float32 (for large benchmark
    batches): the per-image parameters come from the same numpy stream as
    synth_image; the noise comes from a torch generator seeded with `seed`.
    Returns a uint8 tensor [channels, height, width] on `device`."""
    import torch
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    ys = torch.arange(height, device=device, dtype=torch.float32)[:, None]
    xs = torch.arange(width, device=device, dtype=torch.float32)[:, None]
    out = torch.empty((channels, height, width), dtype=torch.uint8, device=device)
    for c in range(channels):
        amp = torch.tensor(rng.uniform(4.0, 24.0, 8), dtype=torch.float32, device=device)
        fx = torch.tensor(rng.integers(0, 9, 8), dtype=torch.float32, device=device)
        fy = torch.tensor(rng.integers(0, 9, 8), dtype=torch.float32, device=device)
        phi = torch.tensor(rng.uniform(0.0, 2.0 * math.pi, 8), dtype=torch.float32, device=device)
        a = 2.0 * math.pi * fy[None, :] * ys / height + phi[None, :]
        b = 2.0 * math.pi * fx[None, :] * xs / width
        left = torch.cat([torch.cos(a) * amp, -torch.sin(a) * amp], dim=1)
        right = torch.cat([torch.cos(b), torch.sin(b)], dim=1)
        smooth = 128.0 + left @ right.T
        noise = torch.randint(-16, 17, (height, width), generator=gen, device=device, dtype=torch.int16)
        out[c] = (torch.round(smooth) + noise).clamp_(0, 255).to(torch.uint8)
    return out


def synth_batch(n: int, height: int, width: int, base_seed: int = BASE_SEED, channels: int = 1,
                threads: int = 8) -> np.ndarray:
    """A uniform batch, [n, channels, height, width] uint8, image i seeded base_seed + i."""
    out = np.empty((n, channels, height, width), np.uint8)

    def one(i):
        out[i] = synth_image(height, width, base_seed + i, channels)

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(one, range(n)))
    return out


def ragged_sizes(n: int, seed: int = BASE_SEED, lo_log2: float = 6.0, hi_log2: float = 12.0,
                 ) -> list[tuple[int, int]]:
    """Sizes of a ragged batch: height and width each 8 * round(2^U[lo, hi] / 8),
    drawn independently (log-uniform 64..4096 by default)."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_log2, hi_log2, size=(n, 2))
    hw = np.maximum(8, 8 * np.rint(np.exp2(e) / 8.0)).astype(np.int64)
    return [(int(h), int(w)) for h, w in hw]


def ragged_batch(sizes, channels: int = 3, base_seed: int = BASE_SEED, threads: int = 8):
    """List of [channels, H, W] uint8 images, image i seeded base_seed + i."""
    out = [None] * len(sizes)

    def one(i):
        h, w = sizes[i]
        out[i] = synth_image(h, w, base_seed + i, channels)

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(one, range(len(sizes))))
    return out


def step_table(s: float) -> np.ndarray:
    """The step table Q_ij = 1 + floor(s (1 + i + j)), uint16 [8, 8]."""
    i = np.arange(8)[:, None]
    j = np.arange(8)[None, :]
    return (1 + np.floor(s * (1 + i + j))).astype(np.uint16)


def normal_batch(shape, seed: int = BASE_SEED) -> np.ndarray:
    """float32 N(0, 1) tensor of the given shape."""
    return np.random.default_rng(seed).standard_normal(shape, dtype=np.float32)
