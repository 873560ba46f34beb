"""Pins of the oracle's OMP (Sec. 1, Sec. 3.2.2) to facts fixed outside it.

Each check uses an independent route -- hand-derived values, a coherence
theorem, numpy's least-squares solver, brute force -- so that a dropped term,
a wrong sign, a transposed operand or a wrong tie-break in the oracle fails.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    with open(os.path.join(HERE, "golden", "omp_worked_examples.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _golden()["cases"], ids=lambda c: c["name"])
def test_worked_examples(case):
    D = np.array(_golden()["D"], dtype=np.float64)
    r = oracle.omp(D, np.array([case["y"]], dtype=np.float64), case["s"], case["eps"], nthreads=1)
    assert r["idx"][0].tolist() == case["idx"]
    assert int(r["nnz"][0]) == case["nnz"]
    np.testing.assert_allclose(r["val"][0], case["val"], rtol=0, atol=1e-14)
    assert abs(r["resid2"][0] - case["resid2"]) < 1e-14
    gap = [None if not np.isfinite(g) else float(g) for g in r["gap"][0]]
    for g, want in zip(gap, case["gap"]):
        assert (g is None and want is None) or abs(g - want) < 1e-14


def _hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


def _identity_hadamard_dictionary():
    """24 atoms in R^16: the identity plus 8 normalised Hadamard rows.  Mutual
    coherence mu = 1/4, so mu (2s - 1) < 1 for s = 2 (Tropp's exact-recovery
    condition): OMP must recover every 2-sparse signal exactly."""
    H = _hadamard(16)[:8] / 4.0
    D = np.vstack([np.eye(16), H])
    G = np.abs(D @ D.T - np.eye(24))
    assert abs(G.max() - 0.25) < 1e-15
    return D


def test_exact_recovery_under_erc():
    D = _identity_hadamard_dictionary()
    rng = np.random.default_rng(1)
    supports = list(itertools.combinations(range(24), 2))
    X = rng.standard_normal((len(supports), 2))
    X += np.sign(X) * 0.1          # keep coefficients away from 0
    Y = np.stack([X[q, 0] * D[a] + X[q, 1] * D[b] for q, (a, b) in enumerate(supports)])
    r = oracle.omp(D, Y, 2, nthreads=2)
    for q, (a, b) in enumerate(supports):
        got = dict(zip(r["idx"][q].tolist(), r["val"][q].tolist()))
        assert set(got) == {a, b}
        assert abs(got[a] - X[q, 0]) < 1e-12 and abs(got[b] - X[q, 1]) < 1e-12
    assert r["resid2"].max() < 1e-24


def test_brute_force_best_subset_agrees_on_sparse_signals():
    """On 2-sparse signals under the recovery condition the exhaustive search over
    all C(24,2) supports (numpy lstsq on each) finds the same support OMP returns."""
    D = _identity_hadamard_dictionary()
    rng = np.random.default_rng(2)
    for _ in range(20):
        a, b = rng.choice(24, 2, replace=False)
        y = rng.standard_normal() * D[a] + rng.standard_normal() * D[b]
        y += 1e-4 * rng.standard_normal(16)       # small noise: still unique best subset
        best, best_err = None, np.inf
        for S in itertools.combinations(range(24), 2):
            x, *_ = np.linalg.lstsq(D[list(S)].T, y, rcond=None)
            err = np.linalg.norm(y - D[list(S)].T @ x)
            if err < best_err:
                best, best_err = set(S), err
        r = oracle.omp(D, y[None], 2, nthreads=1)
        assert set(r["idx"][0].tolist()) == best
        assert abs(np.sqrt(r["resid2"][0]) - best_err) < 1e-12


def _random_problem(seed, m=20, K=40, n=200):
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((K, m))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    Y = rng.standard_normal((n, m))
    return D, Y


def test_coefficients_are_least_squares_and_residual_orthogonal():
    D, Y = _random_problem(3)
    s = 7
    r = oracle.omp(D, Y, s, nthreads=4)
    for i in range(Y.shape[0]):
        S = r["idx"][i][: r["nnz"][i]]
        assert r["nnz"][i] == s and len(set(S.tolist())) == s
        x, *_ = np.linalg.lstsq(D[S].T, Y[i], rcond=None)
        np.testing.assert_allclose(r["val"][i][: len(S)], x, rtol=1e-10, atol=1e-12)
        res = Y[i] - D[S].T @ r["val"][i][: len(S)]
        assert np.abs(D[S] @ res).max() <= 1e-12 * np.linalg.norm(Y[i])
        assert abs(res @ res - r["resid2"][i]) <= 1e-12 * (Y[i] @ Y[i])


def test_greedy_choice_and_monotone_residual():
    """Step k picks the atom with the largest |d_j^T r_{k-1}| (lowest index on a
    tie), r_{k-1} recomputed here by numpy lstsq on the first k-1 atoms; the
    residual norm never increases; the recorded gap is the top-two gap."""
    D, Y = _random_problem(4, m=12, K=30, n=100)
    s = 6
    r = oracle.omp(D, Y, s, nthreads=2)
    for i in range(Y.shape[0]):
        S = r["idx"][i].tolist()
        prev = np.inf
        for k in range(s):
            if k == 0:
                res = Y[i].copy()
            else:
                x, *_ = np.linalg.lstsq(D[S[:k]].T, Y[i], rcond=None)
                res = Y[i] - D[S[:k]].T @ x
            nr = np.linalg.norm(res)
            assert nr <= prev + 1e-12
            prev = nr
            c = np.abs(D @ res)
            c[S[:k]] = -1
            order = np.argsort(-c, kind="stable")
            assert c[S[k]] >= c[order[0]] - 1e-12
            assert abs(r["gap"][i][k] - (c[order[0]] - c[order[1]])) < 1e-10


def test_eps_stop_is_prefix_of_sparsity_stop():
    D, Y = _random_problem(5)
    full = oracle.omp(D, Y, 10, eps=0.0, nthreads=2)
    eps = 0.6 * np.median(np.linalg.norm(Y, axis=1))
    part = oracle.omp(D, Y, 10, eps=eps, nthreads=2)
    for i in range(Y.shape[0]):
        k = part["nnz"][i]
        assert np.sqrt(part["resid2"][i]) <= eps or k == 10
        assert part["idx"][i][:k].tolist() == full["idx"][i][:k].tolist()
        assert (part["idx"][i][k:] == -1).all() and (part["val"][i][k:] == 0).all()
        if k > 0:   # one atom fewer would not have met eps
            x, *_ = np.linalg.lstsq(D[full["idx"][i][:k - 1]].T, Y[i], rcond=None) if k > 1 else (None,)
            prev = Y[i] - (D[full["idx"][i][:k - 1]].T @ x if k > 1 else 0)
            assert np.linalg.norm(prev) > eps
    big = oracle.omp(D, Y, 10, eps=1e9, nthreads=1)
    assert (big["nnz"] == 0).all() and (big["idx"] == -1).all()


def test_support_never_exceeds_dimension():
    """When s > m the residual vanishes after m atoms; every further atom lies in
    span(D_S) and must be refused, so nnz <= m."""
    D, Y = _random_problem(6, m=3, K=8, n=50)
    r = oracle.omp(D, Y, 6, nthreads=1)
    assert (r["nnz"] <= 3).all() and (r["nnz"] == 3).all()
    assert r["resid2"].max() < 1e-25


def test_zero_signal_and_empty_batch():
    D, _ = _random_problem(7)
    r = oracle.omp(D, np.zeros((3, D.shape[1])), 4, nthreads=1)
    assert (r["nnz"] == 0).all() and (r["idx"] == -1).all()
    r = oracle.omp(D, np.zeros((0, D.shape[1])), 4, nthreads=1)
    assert r["idx"].shape == (0, 4)
