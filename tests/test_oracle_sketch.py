"""Pins of the sketching oracle (CountSketch, SRHT) and the preconditioner factor."""
import numpy as np
import scipy.linalg as sl

from oracle import precond as P
from oracle import sketch as S
from oracle import rng as R
from synth import countsketch_draws, srht_draws


def test_countsketch_matches_dense_S():
    rng = np.random.default_rng(0)
    Z = rng.standard_normal((97, 5))
    h, g = countsketch_draws(97, 13, seed=2)
    Sd = S.countsketch_dense(h, g, 13)
    assert np.all((Sd != 0).sum(axis=0) == 1)  # one nonzero per column
    assert np.max(np.abs(S.countsketch_apply(Z, h, g, 13) - Sd @ Z)) < 1e-13


def test_hadamard_is_library_hadamard_and_fwht():
    for n in (1, 2, 8, 64):
        H = S.hadamard_dense(n)
        assert np.array_equal(H, sl.hadamard(n))
        Z = np.random.default_rng(n).standard_normal((n, 3))
        assert np.max(np.abs(S.fwht(Z) - H @ Z)) < 1e-12


def test_srht_matches_dense_and_is_orthogonal_when_full():
    rng = np.random.default_rng(1)
    n, n_pad = 27, 32
    Z = rng.standard_normal((n, 4))
    D, rows = srht_draws(n_pad, 9, seed=3)
    Sd = S.srht_dense(D, rows)
    Zp = np.vstack([Z, np.zeros((n_pad - n, 4))])
    assert np.max(np.abs(S.srht_apply(Z, D, rows) - Sd @ Zp)) < 1e-12
    # s = n': S = H D is orthogonal, so S^T S = I exactly (fixes the scale sqrt(n'/s))
    D2, rows2 = srht_draws(n_pad, n_pad, seed=4)
    Sf = S.srht_dense(D2, rows2)
    assert np.max(np.abs(Sf.T @ Sf - np.eye(n_pad))) < 1e-12


def test_sketch_second_moment_is_identity():
    """diag(S^T S) = 1 exactly for both transforms; off-diagonal mean -> 0."""
    n, s, trials = 16, 6, 3000
    acc_cs = np.zeros((n, n))
    acc_sr = np.zeros((n, n))
    for t in range(trials):
        h, g = countsketch_draws(n, s, seed=t)
        Sc = S.countsketch_dense(h, g, s)
        D, rows = srht_draws(n, s, seed=t)
        Sr = S.srht_dense(D, rows)
        Gc, Gr = Sc.T @ Sc, Sr.T @ Sr
        assert np.allclose(np.diag(Gc), 1) and np.allclose(np.diag(Gr), 1)
        acc_cs += Gc
        acc_sr += Gr
    off = ~np.eye(n, dtype=bool)
    assert np.max(np.abs(acc_cs[off] / trials)) < 0.12
    assert np.max(np.abs(acc_sr[off] / trials)) < 0.12


def test_lemma31_bracket():
    """Lemma 3.1: with s >= 20 s_lambda^2 / delta the pencil (Z^T Z + lam I,
    Z^T S^T S Z + lam I) has all eigenvalues in [1/2, 3/2] w.p. >= 1 - delta."""
    rng = np.random.default_rng(7)
    n, d, lam, delta = 30000, 3, 1.0, 0.25
    Z = rng.standard_normal((n, d)) @ np.diag([30.0, 3.0, 0.3])
    B = Z.T @ Z + lam * np.eye(d)
    s_lam = np.trace(np.linalg.solve(B, Z.T @ Z))
    s = int(np.ceil(20 * s_lam ** 2 / delta))
    assert s < n
    fails = 0
    trials = 60
    for t in range(trials):
        h, g = countsketch_draws(n, s, seed=100 + t)
        SZ = S.countsketch_apply(Z, h, g, s)
        M = SZ.T @ SZ + lam * np.eye(d)
        ev = sl.eigh(B, M, eigvals_only=True)
        if ev.min() < 0.5 or ev.max() > 1.5:
            fails += 1
    assert fails <= delta * trials


def test_precond_R_is_cholesky_of_M():
    rng = np.random.default_rng(2)
    SZ = rng.standard_normal((40, 7)) @ np.diag([1, 1e-1, 1e-2, 1e-3, 1, 2, 3])
    lam = 1e-4
    Rf = P.precond_R(SZ, lam)
    M = SZ.T @ SZ + lam * np.eye(7)
    assert np.allclose(np.tril(Rf, -1), 0)
    assert np.all(np.diag(Rf) > 0)
    assert np.max(np.abs(Rf.T @ Rf - M)) < 1e-12 * np.max(np.abs(M))
    assert np.max(np.abs(Rf - np.linalg.cholesky(M).T)) < 1e-9 * np.max(np.abs(Rf))
    V = rng.standard_normal((7, 3))
    assert np.max(np.abs(M @ P.apply_Minv(Rf, V) - V)) < 1e-8


def test_counter_based_draws():
    """Library-side sketch draws: buckets uniform, signs balanced, rows distinct."""
    n, s = 200000, 64
    h, g = R.countsketch_hash(n, s, seed=9)
    assert h.min() >= 0 and h.max() < s
    cnt = np.bincount(h, minlength=s)
    chi2 = np.sum((cnt - n / s) ** 2 / (n / s))
    assert chi2 < 130  # 63 dof, far tail
    assert abs(g.astype(int).sum()) < 4 * np.sqrt(n)
    # sign independent of bucket parity
    assert abs(g[h % 2 == 0].astype(int).mean()) < 0.02
    D = R.srht_signs(1 << 16, seed=9)
    assert abs(D.astype(int).sum()) < 4 * 256


def test_feistel_is_a_permutation():
    for m in range(1, 13):
        p = R.feistel_perm(m, seed=m * 7 + 1, j=np.arange(1 << m, dtype=np.uint64))
        assert p.min() >= 0 and p.max() < (1 << m)
        assert np.unique(p).size == (1 << m)
    rows = R.srht_rows(1 << 18, 4096, seed=3)
    assert np.unique(rows).size == 4096


def test_splitmix64_reference_sequence():
    """The counter form sm64(0, i) reproduces the generator's published
    reference outputs for seed 0 (tests/golden/splitmix64_seed0.txt)."""
    import os
    from oracle import rng
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64_seed0.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for idx, val in rows:
        assert int(rng.sm64(0, int(idx))) == int(val, 16)
