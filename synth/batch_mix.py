"""Seeded shapes of uneven problem mixes, and device-side generation of their
data (large mixes do not fit a host-side generator's time budget).

No arithmetic of the method here: only random shapes and random matrices.
"""
from __future__ import annotations

import math

import numpy as np

DIMS = (64, 128, 256, 512, 1024)
KS = (1, 5, 10, 20)


def batch_mix(count: int = 64, n_range=(1e4, 2e6), seed: int = 0):
    """`count` CCA shapes (n, dx, dy, k): n log-uniform in n_range, dx and dy
    uniform over DIMS, k uniform over KS (the uneven batched workload)."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(lo, hi))))
        dx = int(rng.choice(DIMS))
        dy = int(rng.choice(DIMS))
        k = int(rng.choice(KS))
        out.append((n, dx, dy, k))
    return out


def serving_mix(count: int = 512, n_range=(1e4, 4e6), d_range=(64, 1024), cca_share: float = 0.7,
                bf16_share: float = 0.5, seed: int = 0):
    """`count` requests of a serving stream: kind ('cca' with probability
    cca_share, else 'lda'), n log-uniform in n_range, views' widths
    log-uniform in d_range (rounded to multiples of 8), storage 'bf16' with
    probability bf16_share else 'f32' (FDA requests are FP32), k in KS
    capped by the problem (FDA: l - 1 with l classes in 2..21)."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    dlo, dhi = math.log(d_range[0]), math.log(d_range[1])
    out = []
    for _ in range(count):
        kind = "cca" if rng.uniform() < cca_share else "lda"
        n = int(round(math.exp(rng.uniform(lo, hi))))
        d0 = max(8, int(round(math.exp(rng.uniform(dlo, dhi)) / 8)) * 8)
        d1 = max(8, int(round(math.exp(rng.uniform(dlo, dhi)) / 8)) * 8)
        k = int(rng.choice(KS))
        if kind == "cca":
            dt = "bf16" if rng.uniform() < bf16_share else "f32"
            out.append(dict(kind="cca", n=n, dx=d0, dy=d1, k=min(k, d0, d1), dtype=dt))
        else:
            l = int(rng.integers(2, 22))
            out.append(dict(kind="lda", n=n, d=d0, l=l, k=max(1, min(k, l - 1, d0)), dtype="f32"))
    return out


def latent_views_device(n: int, dx: int, dy: int, seed: int, latent: int = 24, noise: float = 0.5,
                        decay: float = 1.5, dtype: str = "bf16", device: str = "cuda"):
    """X = Z Ax + noise Ex, Y = Z Ay + noise Ey (Z n x latent with column j
    scaled by 10^(-decay j / (latent - 1)), so the canonical correlations are
    spread apart; Ax, Ay, Ex, Ey i.i.d. N(0, 1)) drawn on the device by
    torch's seeded generator, stored in `dtype`; generated in row chunks to
    bound the temporaries."""
    import torch
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32}[dtype]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    scale = torch.tensor(10.0 ** (-decay * np.arange(latent) / (latent - 1)), dtype=torch.float32, device=device)
    Ax = torch.randn(latent, dx, generator=g, device=device) * scale[:, None]
    Ay = torch.randn(latent, dy, generator=g, device=device) * scale[:, None]
    X = torch.empty(n, dx, dtype=tdt, device=device)
    Y = torch.empty(n, dy, dtype=tdt, device=device)
    chunk = 1 << 18
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        Z = torch.randn(r1 - r0, latent, generator=g, device=device)
        X[r0:r1] = (Z @ Ax + noise * torch.randn(r1 - r0, dx, generator=g, device=device)).to(tdt)
        Y[r0:r1] = (Z @ Ay + noise * torch.randn(r1 - r0, dy, generator=g, device=device)).to(tdt)
    return X, Y


def lda_views_device(n: int, d: int, l: int, seed: int, mean_std: float = 2.0, device: str = "cuda"):
    """FP32 class-structured data on the device: class means ~ N(0, mean_std^2
    I), unit within-class noise, labels in random order, balanced classes."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    means = mean_std * torch.randn(l, d, generator=g, device=device)
    y = (torch.arange(n, device=device) % l).to(torch.int32)
    y = y[torch.randperm(n, generator=g, device=device)].contiguous()
    X = means[y.long()] + torch.randn(n, d, generator=g, device=device)
    return X.contiguous(), y
