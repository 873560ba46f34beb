"""The large image-patch workload (16 x 16 patches, m=256; local K1=512, s1=4;
merge to K=1024, s2=4; final s=16; overcomplete DCT initial dictionaries) and
the merge from a given initial dictionary, against the oracle.

Full size (4,194,304 patches, 256 subsets of 16,384), FP32 path:
  * two sampled subsets, two local iterations, each starting the GPU and the
    oracle from the GPU's dictionary: codes under the FP32 parity rule, the
    iteration's RMSE within 1e-3, the updated atoms against the oracle's MOD of
    the GPU's codes within 2e-5;
  * one merge iteration from the DCT on the GPU's stack of trained local
    atoms: codes of 4,000 sampled stacked atoms under the FP32 rule, the
    updated atoms against the oracle's MOD of the GPU's codes;
  * 4,000 sampled final codings (s=16, K=1024) under the FP32 rule.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_overcomplete_dct_atoms_are_unit_and_span():
    D = si.overcomplete_dct(16, 16, 32)
    assert D.shape == (512, 256)
    np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-12)
    assert np.linalg.matrix_rank(D) == 256
    # separable: atom (a, b) reshaped to 16 x 16 has rank one
    assert np.linalg.matrix_rank(D[37].reshape(16, 16)) == 1


@pytest.mark.gpu
def test_merge_from_given_initial_dictionary_matches_oracle():
    rng = np.random.default_rng(800)
    L, K1, m, K, s2, iters = 5, 40, 16, 32, 3, 4
    Dloc = np.stack([si.unit_gaussian_atoms(rng, m, K1) for _ in range(L)])
    xfro = rng.uniform(5, 20, size=L)
    D0 = si.unit_gaussian_atoms(rng, m, K)
    D, rmse = sdl.merge(_t(Dloc), _t(xfro), None, K, s2, iters, D_init=_t(D0))
    Yt = (Dloc * xfro[:, None, None]).reshape(-1, m)
    o = oracle.train(Yt, D0, s2, iters)
    np.testing.assert_allclose(rmse.cpu().numpy(), o["rmse"], rtol=1e-9)
    np.testing.assert_allclose(D.cpu().numpy(), o["D"], rtol=0, atol=1e-9)


def _check_codes(D, Y, idx, val, nnz, r2, s):
    orc = oracle.omp(D.astype(np.float64), Y.astype(np.float64), s)
    compare_codes(D.astype(np.float64), Y.astype(np.float64), idx, val, nnz, r2, orc,
                  fp32_gap_tol(D.shape[1], np.linalg.norm(Y.astype(np.float64), axis=1)), 1e-4)


@pytest.mark.gpu
def test_patches_full_size_sampled():
    p = si.config4(iters_local=2, iters_merge=1)
    rng = np.random.default_rng(801)
    Yg = _t(p.Y)
    Yp = sdl.split(Yg, _t(p.perm))
    Dl = sdl.init_dict(Yp, _t(p.picks.reshape(-1)), _t(p.fill.reshape(-1, p.m))).reshape(p.L, p.K1, p.m)
    np.testing.assert_allclose(Dl[0].cpu().numpy(), p.extra["D_local0"], atol=1e-6)
    sample = sorted(map(int, rng.choice(p.L, 2, replace=False)))
    Ypn = Yp.cpu().numpy()
    for it in range(p.iters_local):
        before = Dl.cpu().numpy()
        idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp_batched(Dl, Yp, p.offsets, p.s1))
        _, rmse = sdl.local_train(Yp, p.offsets, Dl, p.s1, 1)
        rmse, after = rmse.cpu().numpy()[:, 0], Dl.cpu().numpy()
        for t in sample:
            a, b = p.offsets[t], p.offsets[t + 1]
            Dt = before[t].astype(np.float64)
            _check_codes(before[t], Ypn[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], p.s1)
            o = oracle.train(Ypn[a:b].astype(np.float64), Dt, p.s1, 1)
            assert abs(rmse[t] - o["rmse"][0]) < 1e-3 * o["rmse"][0], (it, t)
            Dm, *_ = oracle.mod(Ypn[a:b].astype(np.float64), idx[a:b], val[a:b].astype(np.float64), Dt, True)
            np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5)
    # the rest of the local phase runs untested here; one merge iteration from the DCT
    xfro, _ = sdl.local_train(Yp, p.offsets, Dl, p.s1, 1, with_rmse=False)
    Dm0 = p.extra["D_merge0"]
    Dn = Dl.cpu().numpy().astype(np.float64)
    Yt = (Dn * xfro.cpu().numpy()[:, None, None]).reshape(-1, p.m).astype(np.float32)
    Ytg = _t(Yt)
    ci, cv, cn, cr = (x.cpu().numpy() for x in sdl.omp(_t(Dm0), Ytg, p.s2))
    Dg, _ = sdl.merge(Dl, xfro, None, p.K, p.s2, 1, D_init=_t(Dm0))
    pick = rng.choice(len(Yt), 4000, replace=False)
    _check_codes(Dm0, Yt[pick], ci[pick], cv[pick], cn[pick], cr[pick], p.s2)
    Dmod, *_ = oracle.mod(Yt.astype(np.float64), ci, cv.astype(np.float64), Dm0.astype(np.float64), True)
    np.testing.assert_allclose(Dg.cpu().numpy(), Dmod, rtol=0, atol=2e-5)
    # final coding with the merged dictionary, sampled
    sF = p.extra["s_final"]
    Df = Dg.cpu().numpy()
    pick = rng.choice(p.N, 4000, replace=False)
    fi, fv, fn, fr = (x.cpu().numpy() for x in sdl.omp(Dg, _t(p.Y[pick]), sF))
    _check_codes(Df, p.Y[pick], fi, fv, fn, fr, sF)
