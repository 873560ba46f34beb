"""Atom replacement (an alternative dictionary-update policy; the paper keeps
unused atoms) through the C ABI against the oracle.

Which atom takes which signal is integer work decided by comparisons of the
residuals, so it is compared bit for bit; the oracle takes those decisions on
the same values (the GPU's FP32 residuals widen to FP64 exactly).  The new
atoms are y / ||y||, within 1e-6 in FP32 and 1e-14 in FP64.  The training test
runs the FP64 loop with the option on against the oracle's loop with the same
policy."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dtype,atol", [(np.float32, 1e-6), (np.float64, 1e-14)])
@pytest.mark.parametrize("K,min_use", [(24, 1), (24, 3), (1024, 2)])
def test_replacement_matches_oracle_on_given_inputs(dtype, atol, K, min_use):
    rng = np.random.default_rng(500 + K + min_use)
    m = 20
    sizes = [300, 0, 1, 517, 64]
    L = len(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    Y = rng.standard_normal((n, m)).astype(dtype)
    r2 = rng.uniform(0.0, 1.0, n).astype(dtype)
    r2[::10] = 0.0          # perfectly coded signals never qualify
    r2[3::7] = 0.5          # ties: the lower signal index wins
    usage = rng.integers(0, 4, (L, K)).astype(np.int32)
    D = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(L)]).astype(dtype)
    Dg = _t(D)
    rep = sdl.replace_atoms(_t(Y), off, _t(usage), _t(r2), min_use, Dg).cpu().numpy()
    Dg = Dg.cpu().numpy()
    replaced = 0
    for t in range(L):
        a, b = off[t], off[t + 1]
        Do, rep_o, cnt = oracle.replace_atoms(Y[a:b].astype(np.float64), usage[t], r2[a:b].astype(np.float64),
                                              min_use, D[t].astype(np.float64))
        want = np.where(rep_o >= 0, rep_o + a, -1)
        np.testing.assert_array_equal(rep[t], want)
        np.testing.assert_allclose(Dg[t], Do, rtol=0, atol=atol)
        replaced += cnt
    assert replaced > 0


def test_min_use_zero_changes_nothing():
    rng = np.random.default_rng(510)
    m, K = 8, 16
    Y = rng.standard_normal((40, m)).astype(np.float32)
    D = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)[None]
    Dg = _t(D)
    rep = sdl.replace_atoms(_t(Y), [0, 40], _t(np.zeros((1, K), np.int32)),
                            _t(np.ones(40, np.float32)), 0, Dg)
    assert (rep.cpu().numpy() == -1).all()
    np.testing.assert_array_equal(Dg.cpu().numpy(), D)


def test_local_training_with_replacement_fp64():
    """Three subsets (each several times K signals, so every MOD system is well
    conditioned) whose initial dictionaries repeat atoms (OMP never picks the
    repeat, so MOD alone would keep it forever): four FP64 iterations with
    SDL_OPT_REPLACE = 1 follow the oracle's loop with the same policy, and the
    dictionaries differ from the run without it."""
    rng = np.random.default_rng(511)
    m, K, s, iters = 16, 32, 3, 4
    sizes = [400, 250, 160]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    D0 = si.unit_gaussian_atoms(rng, m, K)
    Y, _, _ = si.sparse_signals(rng, D0, int(off[-1]), s, 0.05)
    Dinit = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes])
    Dinit[:, 5] = Dinit[:, 1]
    Dinit[:, 9] = Dinit[:, 3]
    Dinit[:, 30] = Dinit[:, 0]
    ctx = sdl.context(0)
    out = {}
    try:
        for mu in (0, 1):
            ctx.set_option(sdl.OPT_REPLACE, mu)
            Dg = _t(Dinit)
            _, rmse = sdl.local_train(_t(Y), off, Dg, s, iters)
            out[mu] = (Dg.cpu().numpy(), rmse.cpu().numpy())
    finally:
        ctx.set_option(sdl.OPT_REPLACE, 0)
    orc = oracle.local_train(Y, off, Dinit, s, iters, min_use=1)
    np.testing.assert_allclose(out[1][0], orc["D"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out[1][1], orc["rmse"], rtol=1e-9, atol=0)
    assert np.abs(out[1][0] - out[0][0]).max() > 0.1
    orc0 = oracle.local_train(Y, off, Dinit, s, iters)
    np.testing.assert_allclose(out[0][0], orc0["D"], rtol=0, atol=1e-9)
