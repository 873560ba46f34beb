"""FP32-accurate tensor-core path (SDL_PREC_F32X3) through the C ABI against the
FP64 oracle, held to the FP32 parity bar.

The path forms the correlations alpha0 = D^T y (Sec. 1 greedy choice) and the
Gram D^T D on the tensor cores from a two-term TF32 split of both operands
(x = hi + lo, hi = tf32(x), lo = tf32(x - hi)) with the three products
hi hi + hi lo + lo hi accumulated in FP32; the selection loop, refit and
refinement step are the FP32 path's.  Bound: e = x3_unit(m) = 3 2^-22 +
gamma_m(2^-23) of sum_i |x_i z_i| per correlation or Gram entry
(tests/_parity.py).  Tolerances:
  * Gram: |G - D D^T| <= e |D| |D|^T entrywise (plus 1e-30);
  * codes: supports identical except near-ties under the FP32 gap rule with e
    in place of gamma_m, at most 0.2 % of signals excused (the FP32 cap),
    coefficients within 1e-4 relative (the FP32 bar);
  * training: per-iteration RMSE within 1e-3 relative of the oracle's, MOD
    atoms within 2e-5 of the oracle's MOD of the GPU's own codes.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, x3_gap_tol, x3_unit

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
X3 = sdl.PREC_F32X3


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _problem(seed, m, K, n, s, sigma):
    rng = np.random.default_rng(seed)
    D0 = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    Y, _, _ = si.sparse_signals(rng, D0.astype(np.float64), n, s, sigma, dtype=np.float32)
    return D0, Y


def _check(D, Y, gi, gv, gn, gr, s, eps=0.0, max_excused=0.002):
    D64, Y64 = D.astype(np.float64), Y.astype(np.float64)
    orc = oracle.omp(D64, Y64, s, eps)
    m = D.shape[1]
    st = compare_codes(D64, Y64, gi, gv, gn, gr, orc, x3_gap_tol(m, np.linalg.norm(Y64, axis=1)), 1e-4,
                       eps=eps if eps > 0 else None, max_excused=max_excused, e=x3_unit(m))
    return st


def _omp(D, Y, s, eps=0.0):
    out = sdl.omp(_t(D), _t(Y), s, eps, prec=X3)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out]


GRAM_SHAPES = [(64, 256, 3), (144, 512, 2), (30, 60, 4), (256, 1024, 1), (8, 16, 5), (37, 130, 2), (64, 300, 2)]


@pytest.mark.parametrize("m,K,L", GRAM_SHAPES)
def test_gram_within_split_bound(m, K, L):
    rng = np.random.default_rng(850 + m + K + L)
    D = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(L)]).astype(np.float32)
    G = sdl.gram(_t(D), prec=X3).cpu().numpy().astype(np.float64)
    D64 = D.astype(np.float64)
    want = np.einsum("lkm,ljm->lkj", D64, D64)
    bound = x3_unit(m) * np.einsum("lkm,ljm->lkj", np.abs(D64), np.abs(D64)) + 1e-30
    err = np.abs(G - want)
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert (err <= bound).all(), (worst, err[worst], bound[worst])
    # the split is what holds the bound: one TF32 product errs ~2^-11
    assert err.max() < 2.0 ** -16


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5017])
def test_omp_tiles_and_ragged_tail(n):
    D, Y = _problem(860 + n, 64, 256, n, 6, 0.01)
    gi, gv, gn, gr = _omp(D, Y, 6)
    _check(D, Y, gi, gv, gn, gr, 6)


@pytest.mark.parametrize("m,K,s", [(30, 60, 6), (37, 130, 5), (16, 100, 3), (8, 16, 6), (64, 300, 8),
                                   (144, 512, 10), (256, 1024, 16), (256, 1000, 12)])
def test_omp_odd_and_extreme_shapes(m, K, s):
    """m not a multiple of 4 (scalar row loads), K not a multiple of 128 (a
    partial chunk) or of 256 (a partial pass), the largest shape."""
    D, Y = _problem(870 + m + K, m, K, 900, min(s, 4), 0.02)
    gi, gv, gn, gr = _omp(D, Y, s)
    st = _check(D, Y, gi, gv, gn, gr, s)
    print(f"m={m} K={K} s={s}: {st}")


def test_omp_error_constrained_stop():
    D, Y = _problem(880, 64, 256, 3000, 6, 0.05)
    eps = 0.5 * float(np.median(np.linalg.norm(Y.astype(np.float64), axis=1)))
    gi, gv, gn, gr = _omp(D, Y, 10, eps)
    _check(D, Y, gi, gv, gn, gr, 10, eps)
    assert ((np.sqrt(gr) <= eps * (1 + 1e-5)) | (gn == 10)).all()


def test_omp_zero_signals():
    D, Y = _problem(881, 32, 64, 300, 3, 0.0)
    Y[::3] = 0
    gi, gv, gn, gr = _omp(D, Y, 4)
    assert (gn[::3] == 0).all() and (gi[::3] == -1).all()
    _check(D, Y, gi, gv, gn, gr, 4)


def test_omp_batched_uneven_with_empty_subsets():
    rng = np.random.default_rng(882)
    m, K, s = 64, 256, 5
    sizes = [0, 300, 1000, 0, 129, 1]
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    Ys = [si.sparse_signals(rng, Ds[t].astype(np.float64), n, 4, 0.02, dtype=np.float32)[0] if n else
          np.zeros((0, m), np.float32) for t, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Y = np.concatenate(Ys)
    out = sdl.omp_batched(_t(Ds), _t(Y), offsets, s, prec=X3)
    gi, gv, gn, gr = (x.cpu().numpy() for x in out)
    for t in range(len(sizes)):
        a, b = offsets[t], offsets[t + 1]
        if b > a:
            _check(Ds[t], Y[a:b], gi[a:b], gv[a:b], gn[a:b], gr[a:b], s)


def test_local_train_uneven_subsets():
    p = si.split_merge_problem("t", 64, 256, 6, 6, 2, 256, [1300, 3000, 700], 4, 4, 0.02,
                               np.random.default_rng(883))
    Yp = p.Y[p.perm]
    Dinit = np.stack([Yp[q] / np.linalg.norm(Yp[q], axis=1, keepdims=True) for q in p.picks]).astype(np.float32)
    Dg = _t(Dinit)
    Ypg = _t(Yp.astype(np.float32))
    for it in range(4):
        before = Dg.cpu().numpy()
        gi, gv, gn, gr = (x.cpu().numpy() for x in sdl.omp_batched(Dg, Ypg, p.offsets, p.s1, prec=X3))
        _, rmse = sdl.local_train(Ypg, p.offsets, Dg, p.s1, 1, prec=X3)
        rmse, after = rmse.cpu().numpy()[:, 0], Dg.cpu().numpy()
        for t in range(p.L):
            a, b = p.offsets[t], p.offsets[t + 1]
            Yt = Yp[a:b].astype(np.float64)
            _check(before[t], Yp[a:b], gi[a:b], gv[a:b], gn[a:b], gr[a:b], p.s1)
            o = oracle.train(Yt, before[t].astype(np.float64), p.s1, 1)
            assert abs(rmse[t] - o["rmse"][0]) < 1e-3 * o["rmse"][0], (it, t)
            Dm, *_ = oracle.mod(Yt, gi[a:b], gv[a:b].astype(np.float64), before[t].astype(np.float64), True)
            np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5, err_msg=f"iteration {it} subset {t}")


def test_merge_matches_oracle():
    rng = np.random.default_rng(884)
    L, K1, m, K = 6, 40, 16, 32
    Dloc = np.stack([si.unit_gaussian_atoms(rng, m, K1) for _ in range(L)]).astype(np.float32)
    xfro = rng.uniform(5, 20, size=L)
    pick = si.merge_pick(rng, L * K1, K)
    D, rmse = sdl.merge(_t(Dloc), _t(xfro), _t(pick), K, 3, 8, prec=X3)
    orc = oracle.merge(Dloc.astype(np.float64), xfro, pick, K, 3, 8)
    rel = np.abs(rmse.cpu().numpy() - orc["rmse"]) / orc["rmse"]
    assert rel.max() < 1e-3, rel


def test_bounded_waits_run_out_and_context_stays_usable():
    """The loader role of the TF32 kernels leaves before its first copy
    (SDL_OPT_WAIT_TEST), so the MMA issuer's first wait for a dictionary chunk
    can never complete: with a short limit every role gives up, the call
    returns SDL_ETIMEOUT, and the next call on the same context matches the
    oracle."""
    ctx = sdl.context(0)
    D, Y = _problem(885, 64, 256, 700, 4, 0.02)
    ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 12)
    ctx.set_option(sdl.OPT_WAIT_TEST, 1)
    try:
        with pytest.raises(sdl.SdlError) as err:
            _omp(D, Y, 5)
        assert err.value.status == 3, err.value   # SDL_ETIMEOUT
    finally:
        ctx.set_option(sdl.OPT_WAIT_TEST, 0)
        ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 24)
    gi, gv, gn, gr = _omp(D, Y, 5)
    _check(D, Y, gi, gv, gn, gr, 5)


def test_patches_full_size_sampled():
    """The image-patch workload at full size (4,194,304 patches, 256 subsets of
    16,384; local K1=512, s1=4 from the overcomplete DCT; final coding K=1024,
    s=16) in the launch configuration the bench times: one batched local
    coding and one local iteration over all subsets, two sampled subsets
    compared in full (codes, RMSE, MOD of the GPU's codes); the final coding of
    all patches with the 1024-atom DCT, 4,000 sampled codes compared."""
    p = si.config4(iters_local=1, iters_merge=1)
    rng = np.random.default_rng(886)
    Yg = _t(p.Y)
    Yp = sdl.split(Yg, _t(p.perm))
    Dl = sdl.init_dict(Yp, _t(p.picks.reshape(-1)), _t(p.fill.reshape(-1, p.m))).reshape(p.L, p.K1, p.m)
    before = Dl.cpu().numpy()
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp_batched(Dl, Yp, p.offsets, p.s1, prec=X3))
    _, rmse = sdl.local_train(Yp, p.offsets, Dl, p.s1, 1, prec=X3)
    rmse, after = rmse.cpu().numpy()[:, 0], Dl.cpu().numpy()
    Ypn = Yp.cpu().numpy()
    for t in sorted(map(int, rng.choice(p.L, 2, replace=False))):
        a, b = p.offsets[t], p.offsets[t + 1]
        Dt = before[t].astype(np.float64)
        st = _check(before[t], Ypn[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], p.s1)
        print(f"subset {t}: {st}")
        o = oracle.train(Ypn[a:b].astype(np.float64), Dt, p.s1, 1)
        assert abs(rmse[t] - o["rmse"][0]) < 1e-3 * o["rmse"][0], t
        Dm, *_ = oracle.mod(Ypn[a:b].astype(np.float64), idx[a:b], val[a:b].astype(np.float64), Dt, True)
        np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5)
    del Yp
    Dm0 = p.extra["D_merge0"]
    sF = p.extra["s_final"]
    fi, fv, fn, fr = (x.cpu().numpy() for x in sdl.omp(_t(Dm0), Yg, sF, prec=X3))
    pick = np.sort(rng.choice(p.N, 4000, replace=False))
    st = _check(Dm0, p.Y[pick], fi[pick], fv[pick], fn[pick], fr[pick], sF)
    print(f"final coding: {st}")
