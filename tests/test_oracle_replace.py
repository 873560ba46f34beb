"""Pins of the oracle's atom replacement, an alternative dictionary-update
policy that the paper does not have (its MOD keeps unused atoms): after the
MOD update, every atom used by fewer than min_use signals, in increasing atom
index, becomes the unit vector along the training signal with the largest
squared residual of the coding pass (lower signal index on ties), each signal
used once, only signals with a positive residual.  The hand-worked cases are
chosen so that a reversed order, the other tie rule, a reused signal, a
missing normalisation or an off-by-one threshold each fail one of them."""
import numpy as np

import oracle
import sdl_inputs as si

Y = np.array([[3.0, 4.0], [1.0, 0.0], [0.0, 2.0], [0.0, 0.0], [5.0, 12.0]])
R2 = np.array([1.0, 4.0, 4.0, 0.0, 2.0])
D = np.array([[0.6, 0.8], [0.0, 1.0], [1.0, 0.0], [0.8, 0.6]])


def test_two_unused_atoms_take_the_two_worst_signals_lower_index_first():
    Dn, rep, cnt = oracle.replace_atoms(Y, [3, 0, 1, 0], R2, 1, D)
    want = D.copy()
    want[1] = [1.0, 0.0]   # signal 1: residual 4, tied with signal 2, lower index
    want[3] = [0.0, 1.0]   # signal 2 = (0, 2) normalised
    np.testing.assert_array_equal(Dn, want)
    assert rep.tolist() == [-1, 1, -1, 2] and cnt == 2


def test_threshold_is_strict():
    """usage[0] == min_use keeps atom 0; atoms 1, 2, 3 (usage 0, 1, 0 < 2) are
    replaced by signals 1, 2 and 4 (residuals 4, 4, 2)."""
    Dn, rep, cnt = oracle.replace_atoms(Y, [2, 0, 1, 0], R2, 2, D)
    assert rep.tolist() == [-1, 1, 2, 4] and cnt == 3
    np.testing.assert_array_equal(Dn[0], D[0])
    np.testing.assert_allclose(Dn[3], [5 / 13, 12 / 13], rtol=0, atol=1e-15)


def test_atoms_keep_their_value_once_no_signal_is_left():
    r2 = np.array([0.0, 0.0, 0.5, 0.0, 0.0])
    Dn, rep, cnt = oracle.replace_atoms(Y, [0, 0, 0, 0], r2, 1, D)
    assert rep.tolist() == [2, -1, -1, -1] and cnt == 1
    np.testing.assert_array_equal(Dn[0], [0.0, 1.0])
    np.testing.assert_array_equal(Dn[1:], D[1:])


def test_min_use_zero_replaces_nothing():
    Dn, rep, cnt = oracle.replace_atoms(Y, [0, 0, 0, 0], R2, 0, D)
    assert cnt == 0 and (rep == -1).all()
    np.testing.assert_array_equal(Dn, D)


def test_duplicated_atom_is_revived_by_the_worst_coded_signal():
    """Atom 7 duplicates atom 2, so OMP (lowest index on ties) never picks it and
    MOD keeps it.  With replacement, one training iteration equals MOD followed
    by overwriting atom 7 with the signal whose least-squares residual on its
    OMP support (computed here with numpy's lstsq) is largest."""
    rng = np.random.default_rng(71)
    m, K, n, s = 12, 16, 300, 3
    D0 = si.unit_gaussian_atoms(rng, m, K)
    D0[7] = D0[2]
    Ys, _, _ = si.sparse_signals(rng, D0, n, s, 0.05)
    codes = oracle.omp(D0, Ys, s)
    assert not (codes["idx"] == 7).any()
    r2 = np.empty(n)
    for i in range(n):
        S = codes["idx"][i][: codes["nnz"][i]]
        x, *_ = np.linalg.lstsq(D0[S].T, Ys[i], rcond=None)
        r2[i] = np.sum((Ys[i] - D0[S].T @ x) ** 2)
    worst = int(np.argmax(r2))
    Dmod, usage, _, _ = oracle.mod(Ys, codes["idx"], codes["val"], D0)
    assert usage[7] == 0 and (usage[np.arange(K) != 7] > 0).all()

    kept = oracle.train(Ys, D0, s, 1)["D"]
    np.testing.assert_allclose(kept, Dmod, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(kept[7], D0[7])

    got = oracle.train(Ys, D0, s, 1, min_use=1)["D"]
    want = Dmod.copy()
    want[7] = Ys[worst] / np.linalg.norm(Ys[worst])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
