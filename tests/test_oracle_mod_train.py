"""Pins of the oracle's MOD update, training loop and Algorithm 1 steps.

MOD (Sec. 1) has a closed form, so it is checked against numpy's least-squares
solver and the normal equations; Proposition 1 (Sec. 1, proof in Appendix A) is
checked per signal, both its bound and the exact identity its proof rests on.
"""
import numpy as np
import pytest

import oracle
import sdl_inputs as si


def _sparse_codes(rng, n, K, s):
    idx = np.stack([rng.choice(K, s, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, s))
    return idx, val


def _dense(idx, val, K):
    X = np.zeros((K, idx.shape[0]))
    for i in range(idx.shape[0]):
        for a in range(idx.shape[1]):
            if idx[i, a] >= 0:
                X[idx[i, a], i] = val[i, a]
    return X


def test_mod_matches_lstsq_and_normal_equations():
    rng = np.random.default_rng(10)
    m, K, n, s = 16, 24, 300, 3
    Y = rng.standard_normal((n, m))
    idx, val = _sparse_codes(rng, n, K, s)
    Dprev = rng.standard_normal((K, m))
    D, usage, ridge, st = oracle.mod(Y, idx, val, Dprev, normalise=False)
    assert st == 0 and not ridge
    X = _dense(idx, val, K)
    assert (usage == (X != 0).sum(axis=1)).all() and (usage > 0).all()
    # numpy lstsq: min ||Y^T - X^T D^T||
    Dl, *_ = np.linalg.lstsq(X.T, Y, rcond=None)
    np.testing.assert_allclose(D, Dl, rtol=1e-10, atol=1e-12)
    # normal equations (Y - D X) X^T = 0
    R = (Y.T - D.T @ X) @ X.T
    assert np.abs(R).max() <= 1e-10 * np.abs(Y.T @ X.T).max()


def test_mod_recovers_generating_dictionary_and_normalises():
    rng = np.random.default_rng(11)
    m, K, n, s = 10, 20, 400, 4
    D0 = si.unit_gaussian_atoms(rng, m, K)
    idx, val = _sparse_codes(rng, n, K, s)
    Y = (D0.T @ _dense(idx, val, K)).T
    D, usage, ridge, st = oracle.mod(Y, idx, val, rng.standard_normal((K, m)), normalise=True)
    np.testing.assert_allclose(D, D0, rtol=0, atol=1e-10)
    # normalisation alone: scaled generator is still recovered as unit atoms
    D, *_ = oracle.mod(3.0 * Y, idx, val, rng.standard_normal((K, m)), normalise=True)
    np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(D, D0, atol=1e-10)


def test_mod_unused_atoms_keep_previous_value():
    rng = np.random.default_rng(12)
    m, K, n, s = 8, 12, 100, 2
    Y = rng.standard_normal((n, m))
    idx, val = _sparse_codes(rng, n, 8, s)      # atoms 8..11 never used
    Dprev = rng.standard_normal((K, m))
    D, usage, ridge, st = oracle.mod(Y, idx, val, Dprev, normalise=True)
    assert (usage[8:] == 0).all()
    np.testing.assert_array_equal(D[8:], Dprev[8:])
    X = _dense(idx, val, K)[:8]
    Dl, *_ = np.linalg.lstsq(X.T, Y, rcond=None)
    Dl /= np.linalg.norm(Dl, axis=1, keepdims=True)
    np.testing.assert_allclose(D[:8], Dl, atol=1e-10)


def test_mod_zero_column_keeps_previous_atom():
    """Atom 0 is used but every signal that uses it has its coefficient on a
    direction orthogonal to the data, so B's column is 0 and the solved atom is
    the zero vector: the previous atom is kept."""
    m, K = 4, 3
    Y = np.array([[0, 1, 0, 0], [0, 0, 1, 0], [0, 1, 1, 0.0]])
    idx = np.array([[1, -1], [2, -1], [1, 2]], np.int32)
    val = np.array([[1, 0], [1, 0], [1, 1.0]])
    # add atom 0 to a fourth signal that is zero
    Y = np.vstack([Y, np.zeros(4)])
    idx = np.vstack([idx, [[0, -1]]]).astype(np.int32)
    val = np.vstack([val, [[2.0, 0]]])
    Dprev = np.arange(12, dtype=np.float64).reshape(3, 4) + 1
    D, usage, ridge, st = oracle.mod(Y, idx, val, Dprev, normalise=True)
    assert usage.tolist() == [1, 2, 2]
    np.testing.assert_array_equal(D[0], Dprev[0])
    np.testing.assert_allclose(D[1], [0, 1, 0, 0], atol=1e-14)
    np.testing.assert_allclose(D[2], [0, 0, 1, 0], atol=1e-14)


def test_mod_ridge_retry_on_rank_deficient_codes():
    """Atoms 0 and 1 are always used together with equal coefficients: X X^T is
    singular, the factor breaks down and the documented ridge is applied.  The
    result must equal numpy's dense solve of (A_UU + lambda I) D^T = B^T."""
    rng = np.random.default_rng(13)
    m, K, n = 6, 5, 50
    Y = rng.standard_normal((n, m))
    third = rng.integers(2, K, size=n)
    idx = np.stack([np.zeros(n), np.ones(n), third], axis=1).astype(np.int32)
    c = rng.standard_normal(n)
    val = np.stack([c, c, rng.standard_normal(n)], axis=1)
    Dprev = rng.standard_normal((K, m))
    D, usage, ridge, st = oracle.mod(Y, idx, val, Dprev, normalise=False)
    assert st == 0 and ridge
    X = _dense(idx, val, K)
    A, B = X @ X.T, X @ Y
    lam = 1e-10 * np.trace(A) / K
    Ar = A + lam * np.eye(K)
    # cond(Ar) ~ 1e10: compare backward residuals, not two solvers' digits
    assert np.abs(Ar @ D - B).max() <= 1e-12 * np.abs(B).max() * np.abs(Ar).max()
    Dr = np.linalg.solve(Ar, B)
    assert np.abs(Ar @ Dr - B).max() <= 1e-12 * np.abs(B).max() * np.abs(Ar).max()
    np.testing.assert_allclose(D[0], D[1], rtol=1e-5)      # the tied atoms stay tied
    np.testing.assert_allclose(D[2:], Dr[2:], rtol=1e-4, atol=1e-6)


def test_train_config0_recovers_most_atoms():
    """Standard MOD/OMP on the FP64 synthetic workload (m=64, K=128, s=5,
    N=10,000, noise 0.01, atoms initialised from 128 random signals, 10
    iterations): the loop must reduce the RMSE towards the noise floor and
    recover most generating atoms (Sec. 3.1 criterion |d_i^T dhat_j| >= 0.98)."""
    c = si.config0()
    Y, D0 = c["Y"], c["D0"]
    Dinit = Y[c["pick"]] / np.linalg.norm(Y[c["pick"]], axis=1, keepdims=True)
    r = oracle.train(Y, Dinit, c["s"], c["iters"])
    rmse = r["rmse"]
    assert rmse[-1] < 0.5 * rmse[0]
    assert rmse[-1] < 0.05
    rec = oracle.recovery(D0, r["D"])
    # MOD from random-signal atoms converges to a local optimum (about 111 of 128
    # atoms after 30+ iterations on this draw): a soft pin, not parity.
    assert rec >= 0.75 * 128, rec


def test_train_started_at_generator_stays_at_noise_floor():
    """Started from the generating dictionary, OMP finds the true supports and the
    residual is the noise projected off s atoms: E||r||^2 = sigma^2 (m - s), so the
    RMSE is sigma sqrt((m - s)/m) (about 0.0096 for sigma=0.01, m=64, s=5) and every
    atom stays recovered."""
    c = si.config0()
    Y, D0 = c["Y"], c["D0"]
    r = oracle.train(Y, D0, c["s"], 3)
    want = 0.01 * np.sqrt((64 - 5) / 64)
    assert np.all(np.abs(r["rmse"] - want) < 0.03 * want), r["rmse"]
    assert oracle.recovery(D0, r["D"]) == 128


def test_train_rmse_matches_independent_residual():
    rng = np.random.default_rng(14)
    D0 = si.unit_gaussian_atoms(rng, 12, 24)
    Y, _, _ = si.sparse_signals(rng, D0, 500, 3, 0.05)
    Dinit = si.unit_gaussian_atoms(rng, 12, 24)
    r1 = oracle.train(Y, Dinit, 3, 1)
    # rmse of the single coding pass, recomputed with numpy from the returned codes
    X = _dense(r1["idx"], r1["val"], 24)
    rm = np.linalg.norm(Y.T - Dinit.T @ X) / np.sqrt(Y.size)
    assert abs(rm - r1["rmse"][0]) < 1e-12
    assert abs(r1["xfro"] - np.linalg.norm(r1["val"])) < 1e-12


def test_split_is_a_permutation_gather():
    rng = np.random.default_rng(15)
    Y = rng.standard_normal((50, 5))
    perm, offsets = si.random_partition(rng, [10, 15, 25])
    np.testing.assert_array_equal(oracle.split(Y, perm), Y[perm])
    assert sorted(perm.tolist()) == list(range(50)) and offsets.tolist() == [0, 10, 25, 50]


def test_local_train_is_independent_per_subset():
    rng = np.random.default_rng(16)
    m, K1, s1 = 8, 10, 2
    Y = rng.standard_normal((90, m))
    offsets = np.array([0, 20, 50, 90])
    D0 = np.stack([si.unit_gaussian_atoms(rng, m, K1) for _ in range(3)])
    r = oracle.local_train(Y, offsets, D0, s1, 4)
    for t in range(3):
        one = oracle.train(Y[offsets[t]:offsets[t + 1]], D0[t], s1, 4, nthreads=1)
        np.testing.assert_array_equal(r["D"][t], one["D"])
        np.testing.assert_array_equal(r["rmse"][t], one["rmse"])
        assert r["xfro"][t] == one["xfro"]


def test_merge_builds_scaled_stack_and_normalised_init():
    rng = np.random.default_rng(17)
    L, K1, m, K = 3, 5, 6, 4
    Dloc = rng.standard_normal((L, K1, m))
    xfro = np.array([2.0, 0.5, 3.0])
    pick = np.array([0, 7, 11, 14], np.int32)
    r = oracle.merge(Dloc, xfro, pick, K, 2, 0)
    Yt = (Dloc * xfro[:, None, None]).reshape(L * K1, m)
    np.testing.assert_allclose(r["Ytilde"], Yt, rtol=0, atol=0)
    np.testing.assert_allclose(r["D"], Yt[pick] / np.linalg.norm(Yt[pick], axis=1, keepdims=True),
                               atol=1e-15)


def test_proposition1_bound_and_identity():
    """Prop. 1: y = Dt x1 + e1 and Dt = D Z + E give y - D Z x1 = E x1 + e1 exactly,
    ||y - D Z x1|| <= K eps2 + eps1 with eps2 = ||x1|| max_j ||e_j||, and
    ||Z x1||_0 <= s1 s2."""
    rng = np.random.default_rng(18)
    m, K, K1, s1, s2 = 16, 32, 24, 3, 2
    D = si.unit_gaussian_atoms(rng, m, K)
    Dt = si.unit_gaussian_atoms(rng, m, K1) * 1.7
    Y = rng.standard_normal((200, m))
    c1 = oracle.omp(Dt, Y, s1, nthreads=2)
    cz = oracle.omp(D, Dt, s2, nthreads=2)
    Z = _dense(cz["idx"], cz["val"], K)                   # K x K1
    E = Dt.T - D.T @ Z                                    # m x K1
    for i in range(Y.shape[0]):
        x1 = np.zeros(K1)
        nz = c1["idx"][i] >= 0
        x1[c1["idx"][i][nz]] = c1["val"][i][nz]
        e1 = Y[i] - Dt.T @ x1
        lhs = Y[i] - D.T @ (Z @ x1)
        np.testing.assert_allclose(lhs, E @ x1 + e1, rtol=0, atol=1e-12)
        eps1 = np.linalg.norm(e1)
        assert abs(eps1 ** 2 - c1["resid2"][i]) < 1e-10
        eps2 = np.linalg.norm(x1) * np.linalg.norm(E, axis=0).max()
        assert np.linalg.norm(lhs) <= K * eps2 + eps1 + 1e-12
        assert np.count_nonzero(np.abs(Z @ x1) > 0) <= s1 * s2


def test_residual_and_recovery_closed_forms():
    rng = np.random.default_rng(19)
    D = si.unit_gaussian_atoms(rng, 8, 12)
    idx, val = _sparse_codes(rng, 30, 12, 3)
    Y = (D.T @ _dense(idx, val, 12)).T
    r2, y2 = oracle.residual(Y, D, idx, val)
    assert r2 < 1e-26 and abs(y2 - (Y * Y).sum()) < 1e-12
    r2, y2 = oracle.residual(2 * Y, D, idx, val)          # half explained: -6.02 dB
    assert abs(20 * np.log10(np.sqrt(r2 / y2)) - 20 * np.log10(0.5)) < 1e-12
    Dp = -D[rng.permutation(12)]
    assert oracle.recovery(D, Dp) == 12
    Dq = D.copy()
    Dq[0] = si.unit_gaussian_atoms(rng, 8, 1)[0]
    assert oracle.recovery(D, Dq, 0.98) == 11 + int(np.abs(D[0] @ Dq.T).max() >= 0.98)
