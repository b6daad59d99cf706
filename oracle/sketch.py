"""Sketching transforms S (s x n) applied to a tall Z (n x d).

TEST INFRASTRUCTURE ONLY (see package docstring).

CountSketch (Sec. 3, the paragraph defining CountSketch): a hash h mapping the
n rows to s buckets and a sign g(i) = +-1; (S x)_b = sum over rows i with
h(i) = b of g(i) x_i.  Column i of S has the single nonzero g(i) in row h(i).
The paper writes h, g on {1..d}; the construction of S (s x n, one nonzero per
column) fixes their domain as the n rows, which is the reading used here.

SRHT (App. A, Def. A.1): S = c R H D with D random signs, H the normalized
Walsh-Hadamard matrix of order n = 2^m, R a choice of s of the n rows without
replacement.  The definition prints c = sqrt(s/n); with a normalized H that
gives E[S^T S] = (s/n)^2 I, at odds with the subspace-embedding use in
Lemma A.2, so c = sqrt(n/s) is used (E[S^T S] = I).  n that is not a power of
two is padded with zero rows (Z^T Z is unchanged).

Parity: pinned by brute force with the dense S on small n, by E[S^T S] = I
over seeds, and by the Lemma 3.1 eigenvalue bracket (tests/test_oracle_sketch.py).
"""
from __future__ import annotations

import numpy as np


def countsketch_dense(h: np.ndarray, g: np.ndarray, s: int) -> np.ndarray:
    """The s x n matrix S itself (tiny n only)."""
    n = h.shape[0]
    S = np.zeros((s, n))
    S[h, np.arange(n)] = g
    return S


def countsketch_apply(Z: np.ndarray, h: np.ndarray, g: np.ndarray, s: int) -> np.ndarray:
    """S Z by the defining sum: row i of Z, times g(i), added into row h(i)."""
    Z = np.asarray(Z, dtype=np.float64)
    out = np.zeros((s, Z.shape[1]))
    np.add.at(out, h, g.astype(np.float64)[:, None] * Z)
    return out


def hadamard_dense(n: int) -> np.ndarray:
    """Unnormalized Sylvester Walsh-Hadamard matrix: H[a, i] = (-1)^popcount(a & i)."""
    a = np.arange(n)[:, None] & np.arange(n)[None, :]
    pc = np.zeros_like(a)
    while a.any():
        pc += a & 1
        a >>= 1
    return np.where(pc % 2 == 0, 1.0, -1.0)


def fwht(Z: np.ndarray) -> np.ndarray:
    """Unnormalized Walsh-Hadamard transform along axis 0 (length a power of two),
    by the standard butterfly recursion H_{2m} = [[H_m, H_m], [H_m, -H_m]]."""
    A = np.array(Z, dtype=np.float64, copy=True)
    n = A.shape[0]
    assert n & (n - 1) == 0
    h = 1
    while h < n:
        A = A.reshape(n // (2 * h), 2, h, -1)
        a = A[:, 0].copy()
        b = A[:, 1].copy()
        A[:, 0] = a + b
        A[:, 1] = a - b
        A = A.reshape(n, -1)
        h *= 2
    return A


def next_pow2(n: int) -> int:
    return 1 << max(0, int(n - 1).bit_length())


def srht_apply(Z: np.ndarray, D: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """S Z with S = sqrt(n'/s) R H D, H normalized (so S = R H_unnorm D / sqrt(s))."""
    Z = np.asarray(Z, dtype=np.float64)
    n, d = Z.shape
    n_pad = D.shape[0]
    s = rows.shape[0]
    Zp = np.zeros((n_pad, d))
    Zp[:n] = Z
    HDZ = fwht(D.astype(np.float64)[:, None] * Zp)
    return HDZ[rows] / np.sqrt(s)


def srht_dense(D: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """The s x n' matrix sqrt(n'/s) R H D with normalized H (tiny n' only)."""
    n_pad = D.shape[0]
    s = rows.shape[0]
    H = hadamard_dense(n_pad) / np.sqrt(n_pad)
    return np.sqrt(n_pad / s) * H[rows] * D.astype(np.float64)[None, :]
