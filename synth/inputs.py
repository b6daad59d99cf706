"""Seeded generators for the synthetic workloads.

Shapes and value distributions follow the workloads the library is measured
on (regularized CCA on two tall views sharing a low-dimensional latent
signal; Fisher LDA on class-structured data) and the paper's synthetic
experiment (Sec. 6.2: tall, ill-conditioned views).  The real-data sets of the
paper's Sec. 6.1 (MNIST, MEDIAMILL, COVTYPE) are not available; these inputs
stand in for them by shape only.

Nothing here computes any part of the method.  Storage conversion to bf16 is
round-to-nearest-even on the fp32 bit pattern.
"""
from __future__ import annotations

import numpy as np

# Workload table: name -> keyword arguments of the generator that builds it.
CONFIGS = {
    # Plain FP64 CCA (the small parity workload): latent 10, noise 0.5, no scaling.
    "cca_small_fp64": dict(kind="cca", n=2000, dx=50, dy=40, k=5, latent=10,
                           noise=0.5, colscale=None, lam=1e-3, dtype="f64",
                           sketch="countsketch", s=4 * (50 + 40), seed=0),
    # Tall ill-conditioned CCA: columns scaled geometrically 1 -> 1e-4; the
    # 20 latent factors have strengths 10^(-2 j / 19), j = 0..19, so the
    # canonical correlations decay (0.9995 ... 0.79) and the top 10 are
    # separated from the rest (sigma_10 - sigma_11 ~ 0.02).
    "cca_tall_bf16": dict(kind="cca", n=262144, dx=512, dy=512, k=10, latent=20,
                          noise=0.5, colscale=(1.0, 1e-4), lam=1e-4, dtype="bf16",
                          sketch="srht", s=4 * (512 + 512), seed=0, latent_decay=2.0),
    "cca_tall_f32": dict(kind="cca", n=262144, dx=512, dy=512, k=10, latent=20,
                         noise=0.5, colscale=(1.0, 1e-4), lam=1e-4, dtype="f32",
                         sketch="srht", s=4 * (512 + 512), seed=0, latent_decay=2.0),
    # The same with the scaled columns rotated by a Haar-random orthogonal
    # matrix per view (X = (Z Ax + 0.5 Ex) diag(c) Qx^T), so that Sxx is not
    # diagonally dominant and every stored column mixes all scales.
    "cca_tall_bf16_mixed": dict(kind="cca", n=262144, dx=512, dy=512, k=10, latent=20,
                                noise=0.5, colscale=(1.0, 1e-4), lam=1e-4, dtype="bf16",
                                sketch="srht", s=4 * (512 + 512), seed=0, latent_decay=2.0,
                                mix=True),
    # Fisher LDA: 10 classes, 784 features, means N(0, 4I), within-class
    # variances log-uniform in [1e-4, 1].
    "lda_f32": dict(kind="lda", n=100000, d=784, l=10, k=9, dtype="f32",
                    sketch="countsketch", s=3 * 784, seed=0),
    # The same with the within-class covariance Q diag(e) Q^T, Q Haar-random.
    "lda_f32_mixed": dict(kind="lda", n=100000, d=784, l=10, k=9, dtype="f32",
                          sketch="countsketch", s=3 * 784, seed=0, mix=True),
}


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """fp32 -> bf16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    lsb = (u >> np.uint32(16)) & np.uint32(1)
    r = (u + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    """bf16 bit patterns (uint16) -> fp32 (exact)."""
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def _store(a: np.ndarray, dtype: str):
    """Return (storage array, exact float64 view of the stored values)."""
    if dtype == "f64":
        s = np.ascontiguousarray(a, dtype=np.float64)
        return s, s
    if dtype == "f32":
        s = np.ascontiguousarray(a, dtype=np.float32)
        return s, s.astype(np.float64)
    if dtype == "bf16":
        s = f32_to_bf16_bits(np.asarray(a, dtype=np.float32))
        return s, bf16_bits_to_f32(s).astype(np.float64)
    raise ValueError(dtype)


def _colscale(d: int, colscale):
    if colscale is None:
        return None
    hi, lo = colscale
    if d == 1:
        return np.array([hi], dtype=np.float64)
    j = np.arange(d, dtype=np.float64)
    return hi * (lo / hi) ** (j / (d - 1))


def latent_scales(latent: int, decay: float):
    """Strengths 10^(-decay j / (latent - 1)) of the latent factors."""
    if latent == 1:
        return np.ones(1)
    return 10.0 ** (-decay * np.arange(latent) / (latent - 1))


def make_workload(name: str, n: int | None = None, seed: int | None = None):
    """Build the named workload (optionally with fewer rows n or another seed)."""
    c = dict(CONFIGS[name])
    if n is not None:
        c["n"] = n
    if seed is not None:
        c["seed"] = seed
    if c["kind"] == "cca":
        ls = latent_scales(c["latent"], c["latent_decay"]) if c.get("latent_decay") else None
        P = cca_latent_problem(c["n"], c["dx"], c["dy"], latent=c["latent"], noise=c["noise"],
                               colscale=c["colscale"], dtype=c["dtype"], seed=c["seed"], latent_scale=ls,
                               mix=c.get("mix", False))
    else:
        P = lda_problem(c["n"], c["d"], c["l"], dtype=c["dtype"], seed=c["seed"], mix=c.get("mix", False))
    P["config"] = c
    return P


def haar_orthogonal(d: int, rng) -> np.ndarray:
    """Haar-distributed d x d orthogonal matrix: QR of a Gaussian matrix with
    the signs of R's diagonal moved into Q."""
    Q, R = np.linalg.qr(rng.standard_normal((d, d)))
    return Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]


def cca_latent_problem(n: int, dx: int, dy: int, latent: int = 10, noise: float = 0.5,
                       colscale=None, dtype: str = "f64", seed: int = 0, chunk: int = 65536,
                       latent_scale=None, mix: bool = False):
    """Two views sharing a latent signal: X = (Z Ax + noise Ex) diag(c), same for Y.

    Z (n x latent), Ax, Ay, Ex, Ey are i.i.d. N(0, 1).  ``colscale=(1, 1e-4)``
    multiplies column j by 10^(-4 j / (d - 1)), which makes X^T X
    ill-conditioned (kappa ~ 1e8) without mixing the columns.
    ``latent_scale`` (length latent) multiplies the latent columns, which
    spreads the canonical correlations apart (equal scales give near-equal
    correlations).  ``mix=True`` rotates the scaled columns of each view by a
    Haar-random orthogonal matrix (X <- X Qx^T), which keeps the spectrum of
    X^T X and spreads every scale over all stored columns.
    Returns dict(X, Y, X64, Y64) where X/Y are in the storage dtype (uint16
    bit patterns for bf16) and X64/Y64 are the stored values in float64.
    """
    rng = np.random.default_rng(seed)
    Ax = rng.standard_normal((latent, dx))
    Ay = rng.standard_normal((latent, dy))
    cx, cy = _colscale(dx, colscale), _colscale(dy, colscale)
    Qx = haar_orthogonal(dx, rng).T if mix else None
    Qy = haar_orthogonal(dy, rng).T if mix else None
    big = n * (dx + dy) > 4_000_000
    wdt = np.float32 if (big and dtype != "f64") else np.float64
    X = np.empty((n, dx), dtype=wdt)
    Y = np.empty((n, dy), dtype=wdt)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        m = r1 - r0
        Z = rng.standard_normal((m, latent))
        if latent_scale is not None:
            Z = Z * np.asarray(latent_scale, dtype=np.float64)[None, :]
        Ex = rng.standard_normal((m, dx), dtype=wdt)
        Ey = rng.standard_normal((m, dy), dtype=wdt)
        xb = (Z @ Ax).astype(wdt) + wdt(noise) * Ex
        yb = (Z @ Ay).astype(wdt) + wdt(noise) * Ey
        if cx is not None:
            xb *= cx.astype(wdt)
            yb *= cy.astype(wdt)
        if mix:
            xb = xb @ Qx.astype(wdt)
            yb = yb @ Qy.astype(wdt)
        X[r0:r1] = xb
        Y[r0:r1] = yb
    Xs, X64 = _store(X, dtype)
    Ys, Y64 = _store(Y, dtype)
    return dict(X=Xs, Y=Ys, X64=X64, Y64=Y64)


def random_tall(n: int, d: int, dtype: str = "f64", seed: int = 0, scale: float = 1.0):
    """Plain i.i.d. N(0, scale^2) tall matrix; returns (storage, float64 view)."""
    rng = np.random.default_rng(seed)
    a = scale * rng.standard_normal((n, d))
    return _store(a, dtype)


def lda_problem(n: int, d: int, l: int, dtype: str = "f32", seed: int = 0,
                mean_std: float = 2.0, var_range=(1e-4, 1.0), chunk: int = 65536, mix: bool = False):
    """Class-structured data for Fisher LDA.

    Class means m_k ~ N(0, mean_std^2 I).  Balanced classes (n_k = n / l, the
    remainder spread over the first classes), labels in random order.
    Within-class noise has independent coordinates with variances e_j drawn
    log-uniformly in ``var_range``; with ``mix=True`` the noise is rotated by
    a Haar-random orthogonal Q, so the within-class covariance is
    Q diag(e) Q^T.  Returns dict(X, X64, y, l).
    """
    rng = np.random.default_rng(seed)
    means = mean_std * rng.standard_normal((l, d))
    e = 10.0 ** rng.uniform(np.log10(var_range[0]), np.log10(var_range[1]), size=d)
    counts = np.full(l, n // l)
    counts[: n % l] += 1
    y = np.repeat(np.arange(l, dtype=np.int32), counts)
    rng.shuffle(y)
    big = n * d > 4_000_000
    wdt = np.float32 if (big and dtype != "f64") else np.float64
    X = np.empty((n, d), dtype=wdt)
    sd = np.sqrt(e).astype(wdt)
    Qt = haar_orthogonal(d, rng).T.astype(wdt) if mix else None
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        g = rng.standard_normal((r1 - r0, d), dtype=wdt) * sd
        if mix:
            g = g @ Qt
        X[r0:r1] = means[y[r0:r1]].astype(wdt) + g
    Xs, X64 = _store(X, dtype)
    return dict(X=Xs, X64=X64, y=y, l=l)


def countsketch_draws(n: int, s: int, seed: int = 0):
    """CountSketch randomness (Sec. 3): bucket h(i) uniform on [0, s), sign g(i) = +-1."""
    rng = np.random.default_rng(seed + 0x5EED)
    h = rng.integers(0, s, size=n, dtype=np.int64).astype(np.int32)
    g = np.where(rng.integers(0, 2, size=n) == 1, 1, -1).astype(np.int8)
    return h, g


def srht_draws(n_pad: int, s: int, seed: int = 0):
    """SRHT randomness (App. A): n_pad random signs, s rows sampled without replacement."""
    rng = np.random.default_rng(seed + 0x5487)
    D = np.where(rng.integers(0, 2, size=n_pad) == 1, 1, -1).astype(np.int8)
    rows = rng.choice(n_pad, size=s, replace=False).astype(np.int32)
    return D, rows
