"""Counter-based random numbers used when the library draws the sketch itself.

TEST INFRASTRUCTURE ONLY (see package docstring).

When a caller passes no explicit sketch randomness, the library derives every
random quantity of a sketch from (seed, index) with SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so any
entry can be regenerated independently.  This module restates that published
generator and the derived quantities so the GPU draws can be checked bit for
bit:

  sm64(seed, i)        the i-th output of a SplitMix64 stream started at seed:
                       z = seed + (i + 1) * 0x9E3779B97F4A7C15, then the
                       published finalizer (xor-shift 30, multiply, xor-shift
                       27, multiply, xor-shift 31), all mod 2^64.
  CountSketch (Sec. 3) r = sm64(seed, i): bucket h(i) = ((r >> 32) * s) >> 32,
                       sign g(i) = -1 if r & 1 else +1.
  SRHT (Def. A.1)      D_i from bit 0 of sm64(seed ^ SALT_D, i); the s sampled
                       rows are pi(0..s-1) for a 4-round Feistel permutation pi
                       of [0, 2^m) (Luby-Rackoff) with round function
                       F_r(x) = sm64(seed ^ SALT_R, r ^ (x << 8)) masked to the
                       half width; odd m works on m + 1 bits by cycle walking.

Parity: the generator is pinned by its published reference sequence for
seed 0 (tests/golden/splitmix64_seed0.txt), its distributional properties
and the bijectivity of the permutation (tests/test_oracle_sketch.py);
bucket/sign/row values are integer and compared bit-exactly with the GPU.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
SALT_D = np.uint64(0xD1B54A32D192ED03)
SALT_R = np.uint64(0x8CB92BA72F3D8DD7)
FEISTEL_ROUNDS = 4


def sm64(seed, i):
    """i-th SplitMix64 output of the stream seeded with ``seed`` (vectorised in i)."""
    with np.errstate(over="ignore"):
        i = np.asarray(i, dtype=np.uint64)
        z = np.uint64(seed) + (i + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def countsketch_hash(n: int, s: int, seed: int):
    """Bucket h (int32 in [0, s)) and sign g (int8 +-1) for rows 0..n-1."""
    r = sm64(seed, np.arange(n, dtype=np.uint64))
    with np.errstate(over="ignore"):
        h = ((r >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)
    g = np.where((r & np.uint64(1)) == 1, -1, 1).astype(np.int8)
    return h.astype(np.int32), g


def srht_signs(n_pad: int, seed: int):
    r = sm64(np.uint64(seed) ^ SALT_D, np.arange(n_pad, dtype=np.uint64))
    return np.where((r & np.uint64(1)) == 1, -1, 1).astype(np.int8)


def _feistel_even(x, bits: int, seed: int):
    """Balanced Feistel network on ``bits`` (even) bits, applied to array x."""
    half = bits // 2
    mask = np.uint64((1 << half) - 1)
    L = (x >> np.uint64(half)) & mask
    R = x & mask
    key = np.uint64(seed) ^ SALT_R
    for r in range(FEISTEL_ROUNDS):
        with np.errstate(over="ignore"):
            F = sm64(key, np.uint64(r) ^ (R << np.uint64(8))) & mask
        L, R = R, L ^ F
    return (L << np.uint64(half)) | R


def feistel_perm(m: int, seed: int, j):
    """pi(j) for the pseudo-random permutation of [0, 2^m)."""
    j = np.asarray(j, dtype=np.uint64)
    bits = m if m % 2 == 0 else m + 1
    lim = np.uint64(1) << np.uint64(m)
    y = _feistel_even(j, bits, seed)
    # cycle walking: re-apply until the value lands in [0, 2^m)
    for _ in range(1 << bits):
        bad = y >= lim
        if not bad.any():
            break
        y = np.where(bad, _feistel_even(y, bits, seed), y)
    return y.astype(np.int64)


def srht_rows(n_pad: int, s: int, seed: int):
    m = int(n_pad).bit_length() - 1
    assert (1 << m) == n_pad
    return feistel_perm(m, seed, np.arange(s, dtype=np.uint64)).astype(np.int32)
