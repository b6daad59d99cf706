"""CCA and FDA as Riemannian problems: costs and Euclidean gradients.

TEST INFRASTRUCTURE ONLY (see package docstring).

CCA (Sec. 4.2): on St_Sxx(p, dx) x St_Syy(p, dy),
  f_CCA(U, V) = -1/2 tr(Z^T [[0, Sxy], [Sxy^T, 0]] Z N) = -tr(U^T Sxy V N),
  Euclidean gradient (-Sxy V N, -Sxy^T U N); the Riemannian gradient is the
  componentwise projection of M^{-1} times it (Eq. for grad f_CCA).
FDA (Sec. 5.2): on St_{S_w + lambda I}(p, d),
  f_FDA(W) = -1/2 tr(W^T S_B W N), Euclidean gradient -S_B W N.

Each problem is a list of manifold factors (B_i) plus cost / egrad acting on a
list of points, so one Riemannian CG serves both.

Parity: pinned through the geometry tests (finite-difference directional
derivatives) and the closed forms the reference solver converges to.
"""
from __future__ import annotations

import numpy as np


class CCAProblem:
    def __init__(self, Sxx, Syy, Sxy, mu):
        self.Bs = [Sxx, Syy]
        self.Sxy = Sxy
        self.N = np.diag(mu)

    def cost(self, pts):
        U, V = pts
        return -float(np.trace(U.T @ self.Sxy @ V @ self.N))

    def egrad(self, pts):
        U, V = pts
        return [-(self.Sxy @ V @ self.N), -(self.Sxy.T @ U @ self.N)]


class FDAProblem:
    def __init__(self, SB, Swl, mu):
        self.Bs = [Swl]
        self.SB = SB
        self.N = np.diag(mu)

    def cost(self, pts):
        (W,) = pts
        return -0.5 * float(np.trace(W.T @ self.SB @ W @ self.N))

    def egrad(self, pts):
        (W,) = pts
        return [-(self.SB @ W @ self.N)]
