"""The per-iteration data products, as plain explicit matrix products.

TEST INFRASTRUCTURE ONLY (see package docstring).

One Riemannian-CG iteration of the paper's CCA needs products of the data with
the current point and search direction (Table 2: O(ndp) per component; Cor. 4.6
counts them as O(p (nnz X + nnz Y)) per iteration).  The library computes all
of them in one sweep over the rows; this module states what that sweep must
return, for Phi_x = [U, eta_U] (dx x 2k) and Phi_y = [V, eta_V] (dy x 2k):

  W   = [X Phi_x, Y Phi_y]          (n x 4k, never stored by the library)
  Gx  = X^T W                        (dx x 4k)
  Gy  = Y^T W                        (dy x 4k)
  Gram = W^T W                       (4k x 4k)

For FDA (Sec. 5.1, Cor. 5.6) with Phi = [W, eta] (d x 2k) and Xhat the
class-centred data: P = Xhat Phi, outputs Xhat^T P (= S_w Phi) and P^T P.

Parity: pinned (tests/test_oracle_fused.py) to the pinned covariance forms
of oracle.cca.sigmas (Gx = [(Sxx - lx I) Phi_x, Sxy Phi_y], Gy likewise, the
Gram = Phi_bd^T Sigma Phi_bd) and the within-class scatter of
oracle.lda.scatters (Xhat^T P = S_w Phi), and by row-by-row loops on tiny
inputs; a planted swap of the W blocks is caught.
"""
from __future__ import annotations

import numpy as np

from .lda import class_stats


def cca_pass(X, Y, Phix, Phiy):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    W = np.hstack([X @ Phix, Y @ Phiy])
    return X.T @ W, Y.T @ W, W.T @ W


def lda_pass(X, y, l, Phi):
    _, _, _, _, Xhat = class_stats(X, y, l)
    P = Xhat @ Phi
    return Xhat.T @ P, P.T @ P
