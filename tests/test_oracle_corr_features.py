"""Pins of the oracle's dictionary-conditioned proposer input F = |D_t^T y|
(the magnitudes OMP's first greedy step ranks, Sec. 1), each fixed by
something other than the formula itself: scaled identity dictionaries (which
also pin the routing of rows to subsets, empty subsets included), Parseval's
identity for orthonormal dictionaries, the sign symmetries, atom permutations,
and the first atom of the pinned OMP oracle."""
import numpy as np

import oracle
import sdl_inputs as si


def test_scaled_identity_dictionaries_route_each_subset():
    rng = np.random.default_rng(900)
    m = 12
    scale = np.array([1.0, 2.0, 0.5, -3.0])
    sizes = [5, 0, 1, 7]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    D = np.stack([c * np.eye(m) for c in scale])
    Y = rng.standard_normal((int(off[-1]), m))
    F = oracle.corr_features(D, off, Y)
    for t in range(len(sizes)):
        a, b = off[t], off[t + 1]
        np.testing.assert_array_equal(F[a:b], np.abs(scale[t]) * np.abs(Y[a:b]))


def test_parseval_for_orthonormal_dictionaries():
    rng = np.random.default_rng(901)
    m = 16
    Q = np.stack([np.linalg.qr(rng.standard_normal((m, m)))[0].T for _ in range(3)])
    off = np.array([0, 40, 41, 90], np.int64)
    Y = rng.standard_normal((90, m))
    F = oracle.corr_features(Q, off, Y)
    np.testing.assert_allclose((F ** 2).sum(axis=1), (Y ** 2).sum(axis=1), rtol=1e-12)


def test_signs_and_atom_order():
    rng = np.random.default_rng(902)
    m, K = 10, 24
    D = si.unit_gaussian_atoms(rng, m, K)[None]
    off = np.array([0, 30], np.int64)
    Y = rng.standard_normal((30, m))
    F = oracle.corr_features(D, off, Y)
    assert (F >= 0).all()
    np.testing.assert_array_equal(oracle.corr_features(D, off, -Y), F)
    np.testing.assert_array_equal(oracle.corr_features(-D, off, Y), F)
    perm = rng.permutation(K)
    np.testing.assert_array_equal(oracle.corr_features(D[:, perm], off, Y), F[:, perm])


def test_largest_feature_is_omps_first_pick():
    rng = np.random.default_rng(903)
    m, K = 20, 60
    D = si.unit_gaussian_atoms(rng, m, K)
    Y = rng.standard_normal((200, m))
    F = oracle.corr_features(D[None], np.array([0, 200], np.int64), Y)
    first = oracle.omp(D, Y, 1)["idx"][:, 0]
    np.testing.assert_array_equal(np.argmax(F, axis=1), first)
