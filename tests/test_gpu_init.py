"""Initial atoms (Sec. 3.1: atoms taken from the training vectors, scaled to unit
norm; Algorithm 1 step 2 starts every local dictionary this way) through the C
ABI's sdl_init_dict, against numpy.

Column c of the output is Y[pick[c]] / ||Y[pick[c]]||, or fill[c] / ||fill[c]||
where pick[c] < 0 (a subset with fewer than K1 signals: all of its signals,
then Gaussian fill columns); a zero column stays zero.  The kernel forms the
norm and the quotient in FP64 and rounds once, so FP32 output is within one
unit in the last place of numpy's FP64 quotient rounded to FP32, and FP64
output within a few units of 2^-53.
"""
import numpy as np
import pytest
import torch

import paper_1403_4781_gb300 as sdl
import sdl_inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _expected(Y, pick, fill):
    src = np.where(pick[:, None] >= 0, Y[np.maximum(pick, 0)], fill)
    nrm = np.linalg.norm(src, axis=1, keepdims=True)
    return np.divide(src, nrm, out=np.zeros_like(src), where=nrm > 0)


@pytest.mark.parametrize("dtype,tol", [(np.float32, 2.0 ** -23), (np.float64, 8 * 2.0 ** -53)])
def test_init_dict_matches_numpy_with_fill_for_small_subsets(dtype, tol):
    rng = np.random.default_rng(950)
    m, K1 = 37, 64
    sizes = [200, 10, 64, 63, 1, 130]       # subsets of 10, 63 and 1 signals need fill columns
    perm, offsets = si.random_partition(rng, sizes)
    Y = rng.standard_normal((offsets[-1], m))
    Y[perm[int(offsets[1])]] = 0.0           # a zero signal in the 10-signal subset: a zero atom
    picks = si.init_picks(rng, offsets, K1)
    fill = si.init_fill(rng, len(sizes), K1, m)
    fill[1, 20] = 0.0                        # a zero fill column stays zero
    assert (picks[1] < 0).sum() == K1 - 10 and (picks[3] < 0).sum() == 1 and (picks[4] < 0).sum() == K1 - 1
    Yg = sdl.split(_t(Y.astype(dtype)), _t(perm))
    Yp = Yg.cpu().numpy()
    np.testing.assert_array_equal(Yp, Y.astype(dtype)[perm])           # the split gather, bit-exact
    D = sdl.init_dict(Yg, _t(picks.reshape(-1)), _t(fill.reshape(-1, m).astype(dtype))).cpu().numpy()
    ref = _expected(Yp.astype(np.float64), picks.reshape(-1), fill.reshape(-1, m).astype(dtype).astype(np.float64))
    assert D.dtype == dtype and D.shape == (len(sizes) * K1, m)
    err = np.abs(D.astype(np.float64) - ref).max()
    assert err <= tol, err
    # picked columns are the picked signals' directions exactly (up to rounding), fill columns the fill's
    zero = np.linalg.norm(ref, axis=1) == 0
    assert zero.sum() >= 1 and (D[zero] == 0).all()
    np.testing.assert_allclose(np.linalg.norm(D[~zero].astype(np.float64), axis=1), 1.0, atol=4 * tol * np.sqrt(m))


def test_init_dict_without_fill_needs_every_pick():
    rng = np.random.default_rng(951)
    Y = rng.standard_normal((300, 16)).astype(np.float32)
    pick = rng.choice(300, 40, replace=False).astype(np.int64)
    D = sdl.init_dict(_t(Y), _t(pick)).cpu().numpy()
    ref = _expected(Y.astype(np.float64), pick, np.zeros((40, 16)))
    assert np.abs(D - ref).max() <= 2.0 ** -23
