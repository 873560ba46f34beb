"""GPU OMP (sdl_omp / sdl_omp_batched through the C ABI) against the FP64 oracle.

Tolerances: FP32 path -- supports identical except near-ties (tests/_parity.py,
gap below max(1e-6, 2 gamma_m ||y||)), coefficients within 1e-4 relative;
FP64 path -- gap below 1e-6, coefficients within 1e-9 relative.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _problem(seed, m, K, n, s, sigma, dtype=np.float32):
    rng = np.random.default_rng(seed)
    D0 = si.unit_gaussian_atoms(rng, m, K).astype(dtype)
    Y, _, _ = si.sparse_signals(rng, D0.astype(np.float64), n, s, sigma, dtype=dtype)
    return D0, Y


def _run(D, Y, s, eps=0.0):
    Dg, Yg = torch.from_numpy(D).to(DEV), torch.from_numpy(Y).to(DEV)
    idx, val, nnz, r2 = sdl.omp(Dg, Yg, s, eps)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), val.cpu().numpy(), nnz.cpu().numpy(), r2.cpu().numpy()


def _check(D, Y, s, eps, fp64=False):
    gi, gv, gn, gr = _run(D, Y, s, eps)
    D64, Y64 = D.astype(np.float64), Y.astype(np.float64)
    orc = oracle.omp(D64, Y64, s, eps)
    if fp64:
        tol, rtol = 1e-6, 1e-9
    else:
        tol, rtol = fp32_gap_tol(D.shape[1], np.linalg.norm(Y64, axis=1)), 1e-4
    st = compare_codes(D64, Y64, gi, gv, gn, gr, orc, tol, rtol)
    assert st["excused"] <= max(2, 0.002 * len(Y)), st
    return st


@pytest.mark.parametrize("n", [1, 31, 32, 33, 5017])
def test_fp32_splitmerge_shape_tiles_and_ragged_tail(n):
    D, Y = _problem(100 + n, 64, 256, n, 6, 0.01)
    _check(D, Y, 6, 0.0)


def test_fp32_error_constrained_stop():
    D, Y = _problem(101, 64, 256, 3000, 6, 0.05)
    eps = 0.5 * float(np.median(np.linalg.norm(Y.astype(np.float64), axis=1)))
    st = _check(D, Y, 10, eps)
    gi, gv, gn, gr = _run(D, Y, 10, eps)
    assert ((np.sqrt(gr) <= eps * (1 + 1e-5)) | (gn == 10)).all()
    small = np.linalg.norm(Y.astype(np.float64), axis=1) <= eps
    assert (gn[small] == 0).all() and (gn[~small] > 0).all() and (gn < 10).any()


def test_fp64_standard_shape():
    D, Y = _problem(102, 64, 128, 3001, 5, 0.01, dtype=np.float64)
    _check(D, Y, 5, 0.0, fp64=True)


@pytest.mark.parametrize("m,K,s", [(30, 60, 6), (16, 100, 3), (8, 16, 6), (256, 1024, 16), (144, 512, 10)])
def test_fp32_odd_and_extreme_shapes(m, K, s):
    D, Y = _problem(103 + m + K, m, K, 700, min(s, 4), 0.02)
    _check(D, Y, s, 0.0)


def test_zero_signals_and_empty_batch():
    D, Y = _problem(104, 32, 64, 40, 3, 0.0)
    Y[::3] = 0
    gi, gv, gn, gr = _run(D, Y, 4)
    assert (gn[::3] == 0).all() and (gi[::3] == -1).all() and (gv[::3] == 0).all()
    gi, gv, gn, gr = _run(D, Y[:0], 4)
    assert gi.shape == (0, 4)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_golden_worked_examples(dtype):
    with open(os.path.join(os.path.dirname(__file__), "golden", "omp_worked_examples.json")) as f:
        gold = json.load(f)
    D = np.array(gold["D"], dtype=dtype)
    for case in gold["cases"]:
        Y = np.array([case["y"]], dtype=dtype)
        Dg, Yg = torch.from_numpy(D).to(DEV), torch.from_numpy(Y).to(DEV)
        idx, val, nnz, r2 = sdl.omp(Dg, Yg, case["s"], case["eps"])
        assert idx.cpu().numpy()[0].tolist() == case["idx"], case["name"]
        assert int(nnz.cpu()[0]) == case["nnz"]
        np.testing.assert_allclose(val.cpu().numpy()[0], case["val"], atol=1e-6)
        assert abs(float(r2.cpu()[0]) - case["resid2"]) < 1e-6


def test_batched_uneven_subsets_each_with_its_own_dictionary():
    rng = np.random.default_rng(105)
    m, K, s = 64, 256, 6
    sizes = [700, 0, 33, 1500, 1]
    L = len(sizes)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(L)]).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Y = rng.standard_normal((offsets[-1], m)).astype(np.float32)
    Dg, Yg = torch.from_numpy(Ds).to(DEV), torch.from_numpy(Y).to(DEV)
    idx, val, nnz, r2 = sdl.omp_batched(Dg, Yg, offsets, s)
    idx, val, nnz, r2 = (t.cpu().numpy() for t in (idx, val, nnz, r2))
    for t in range(L):
        a, b = offsets[t], offsets[t + 1]
        if a == b:
            continue
        D64, Y64 = Ds[t].astype(np.float64), Y[a:b].astype(np.float64)
        orc = oracle.omp(D64, Y64, s)
        compare_codes(D64, Y64, idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc,
                      fp32_gap_tol(m, np.linalg.norm(Y64, axis=1)), 1e-4)


def test_full_size_final_coding_sampled():
    """200,000 signals, m=64, K=256, s=6 (the final global coding of the
    split-and-merge workload), checked on 2,000 sampled signals."""
    D, Y = _problem(106, 64, 256, 200_000, 6, 0.01)
    gi, gv, gn, gr = _run(D, Y, 6)
    pick = np.random.default_rng(0).choice(len(Y), 2000, replace=False)
    D64, Y64 = D.astype(np.float64), Y[pick].astype(np.float64)
    orc = oracle.omp(D64, Y64, 6)
    compare_codes(D64, Y64, gi[pick], gv[pick], gn[pick], gr[pick], orc,
                  fp32_gap_tol(64, np.linalg.norm(Y64, axis=1)), 1e-4)


def test_invalid_arguments_raise():
    D, Y = _problem(107, 16, 32, 10, 2, 0.0)
    Dg, Yg = torch.from_numpy(D).to(DEV), torch.from_numpy(Y).to(DEV)
    with pytest.raises(sdl.SdlError):
        sdl.omp(Dg, Yg, 0)           # s = 0
    with pytest.raises(sdl.SdlError):
        sdl.omp(Dg, Yg, 17)          # s > m
    with pytest.raises(sdl.SdlError):
        sdl.omp(Dg, Yg, 2, eps=-1.0)
