"""The checked mixed-precision MOD solve for FP32 data (SDL_OPT_MOD_MIXED)
against the oracle's MOD (Sec. 1: D = Y X^T (X X^T)^{-1} over the used atoms,
then unit columns, Sec. 3.1) and against the FP64 solve.

The FP32 pass factors and solves in FP32; a check estimates every used atom's
error from random-sign probes of the FP64 residual and hands any subset whose
estimated error norm exceeds 2e-5 of the atom's norm (or whose FP32 squared pivot fell to
1e-3 of its diagonal) to the FP64 solve.  Tolerances: every atom within 2e-5
absolute of the oracle's (the FP32 atom tolerance); unused atoms bit-exact;
a subset the check hands on matches the FP64 solve's result to 1e-6 (the same
tiled kernel, tile and cluster size; the runs differ only in the accumulation
order of A and B)."""
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


@pytest.fixture
def ctx():
    c = sdl.context(0)
    yield c
    c.set_option(sdl.OPT_MOD_SOLVE, 0)
    c.set_option(sdl.OPT_CLUSTER, 0)
    c.set_option(sdl.OPT_MOD_TILE, 0)
    c.set_option(sdl.OPT_AUTOTUNE, 1)
    c.set_option(sdl.OPT_MOD_MIXED, 1)
    c.set_option(sdl.OPT_MOD_CHECK_TOL, 20000)
    c.profile(False)


def _problem(seed, sizes, m, K, s, unused=3):
    rng = np.random.default_rng(seed)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    Y = rng.standard_normal((n, m)).astype(np.float32)
    hi = K - unused
    idx = np.stack([rng.choice(hi, s, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, s)).astype(np.float32)
    idx[::5, -1] = -1
    val[::5, -1] = 0
    D0 = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    return offsets, Y, idx, val, D0


def _oracle(offsets, Y, idx, val, D0):
    out = []
    for t in range(len(offsets) - 1):
        a, b = offsets[t], offsets[t + 1]
        Do, *_ = oracle.mod(Y[a:b].astype(np.float64), idx[a:b], val[a:b].astype(np.float64),
                            D0[t].astype(np.float64), True)
        out.append(Do)
    return np.stack(out)


def _run(ctx, mixed, ts, C, offsets, Y, idx, val, D0, autotune=0):
    ctx.set_option(sdl.OPT_MOD_SOLVE, 0)
    ctx.set_option(sdl.OPT_AUTOTUNE, autotune)
    ctx.set_option(sdl.OPT_MOD_TILE, ts)
    ctx.set_option(sdl.OPT_CLUSTER, C)
    ctx.set_option(sdl.OPT_MOD_MIXED, mixed)
    ctx.profile(True)
    ctx.profile_reset()
    Dg = _t(D0.copy())
    sdl.mod_update_batched(_t(Y), offsets, _t(idx), _t(val), Dg)
    prof = ctx.profile_read()
    ctx.profile(False)
    return Dg.cpu().numpy(), prof


@pytest.mark.parametrize("K,m,s", [(60, 30, 4), (97, 33, 5), (256, 64, 6), (512, 256, 4), (130, 70, 3)])
@pytest.mark.parametrize("ts,C", [(16, 1), (16, 4), (32, 2), (32, 16), (64, 1), (64, 4), (64, 16)])
def test_mixed_matches_oracle(ctx, ts, C, K, m, s):
    """The FP32 pass with every tile edge (64: the 4 x 4 register micro-tiled
    products, with K and m that leave partial tiles and rows not a multiple of
    4) and cluster size, checked and renormalised, against the oracle."""
    offsets, Y, idx, val, D0 = _problem(900 + K, [3 * K, 5 * K, 4 * K], m, K, s)
    want = _oracle(offsets, Y, idx, val, D0)
    got, prof = _run(ctx, 1, ts, C, offsets, Y, idx, val, D0)
    assert "mod_solve_fp32" in prof and "mod_check" in prof, prof
    np.testing.assert_array_equal(got[:, K - 3:], D0[:, K - 3:])   # unused atoms: bit-exact
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5)


@pytest.mark.parametrize("ts", [32, 64])
def test_mixed_single_system_K1024(ctx, ts):
    """One subset, K=1024, m=256 (the image-patch merge shape), clusters of 16."""
    offsets, Y, idx, val, D0 = _problem(910, [6000], 256, 1024, 4, unused=0)
    want = _oracle(offsets, Y, idx, val, D0)
    got, prof = _run(ctx, 1, ts, 16, offsets, Y, idx, val, D0)
    assert "mod_solve_fp32_single" in prof, prof
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5)


def _near_dependent(seed, rho, n=3000, m=48, K=64):
    """Three subsets; in subset 1 atoms 0 and 1 are used by the same signals
    with coefficients c and c (1 + delta), so their rows of X X^T have squared
    cosine about 1 - rho (the second pivot about rho of its diagonal)."""
    offsets, Y, idx, val, D0 = _problem(seed, [n, n, n], m, K, 3, unused=0)
    rng = np.random.default_rng(seed + 1)
    a, b = offsets[1], offsets[2]
    c = rng.standard_normal(b - a).astype(np.float32)
    delta = (np.sqrt(rho) * rng.standard_normal(b - a)).astype(np.float32)
    idx[a:b, 0], idx[a:b, 1] = 0, 1
    idx[a:b, 2] = rng.integers(2, K, size=b - a)
    val[a:b, 0], val[a:b, 1] = c, c * (1 + delta)
    return offsets, Y, idx, val, D0


@pytest.mark.parametrize("ts", [16, 64])
def test_breakdown_goes_to_fp64(ctx, ts):
    """In subset 1 the squared pivot of atom 1 is about 1e-5 of its diagonal:
    the FP32 factorisation breaks down (below 1e-3) and that subset comes out
    of the FP64 solve: within 1e-6 of the FP64-only run (the two runs differ
    only by the accumulation order of A and B, set by atomics, and the FP32
    rounding of the atoms); the whole result within 2e-5 of the oracle."""
    offsets, Y, idx, val, D0 = _near_dependent(920, 1e-5)
    want = _oracle(offsets, Y, idx, val, D0)
    mixed, prof = _run(ctx, 1, ts, 2, offsets, Y, idx, val, D0)
    fp64, prof64 = _run(ctx, 0, 16, 2, offsets, Y, idx, val, D0)
    assert "mod_check" in prof and "mod_check" not in prof64
    np.testing.assert_allclose(mixed[1], fp64[1], rtol=0, atol=1e-6)
    np.testing.assert_allclose(mixed, want, rtol=0, atol=2e-5)


@pytest.mark.parametrize("K,m", [(97, 33), (512, 256)])
def test_check_at_tiny_tolerance_sends_every_subset_to_fp64(ctx, K, m):
    """With the check's tolerance at 1e-9 of each atom's norm no FP32 solution
    passes, so every subset comes out of the FP64 solve (within 1e-6 of the
    FP64-only run); at the default tolerance the FP32 solutions are kept, and
    both are within 2e-5 of the oracle."""
    offsets, Y, idx, val, D0 = _problem(925 + K, [3 * K, 4 * K], m, K, 4)
    want = _oracle(offsets, Y, idx, val, D0)
    fp64, _ = _run(ctx, 0, 32, 2, offsets, Y, idx, val, D0)
    ctx.set_option(sdl.OPT_MOD_CHECK_TOL, 1)
    strict, prof = _run(ctx, 1, 32, 2, offsets, Y, idx, val, D0)
    ctx.set_option(sdl.OPT_MOD_CHECK_TOL, 20000)
    assert "mod_check" in prof
    np.testing.assert_allclose(strict, fp64, rtol=0, atol=1e-6)
    kept, _ = _run(ctx, 1, 32, 2, offsets, Y, idx, val, D0)
    err32 = np.abs(kept - want).max()
    print(f"K={K} m={m}: FP32 solutions kept, max atom error {err32:.2e}; FP64 {np.abs(fp64 - want).max():.2e}")
    np.testing.assert_allclose(kept, want, rtol=0, atol=2e-5)


def test_autotuned_choice_matches_oracle(ctx):
    """The autotuner times the checked FP32 pass beside the FP64 candidates and
    caches its choice; two calls give the same atoms."""
    offsets, Y, idx, val, D0 = _problem(930, [2048] * 24, 64, 256, 4)
    want = _oracle(offsets, Y, idx, val, D0)
    first, _ = _run(ctx, 1, 0, 0, offsets, Y, idx, val, D0, autotune=1)
    again, prof = _run(ctx, 1, 0, 0, offsets, Y, idx, val, D0, autotune=1)
    print(sorted(prof))
    # the accumulation of A and B visits each atom's signals in an order set by
    # atomics: repeated calls agree to rounding level, not bit for bit
    np.testing.assert_allclose(first, again, rtol=0, atol=1e-6)
    np.testing.assert_allclose(first, want, rtol=0, atol=2e-5)
    np.testing.assert_allclose(again, want, rtol=0, atol=2e-5)


def test_local_training_with_mixed_solve_matches_oracle(ctx):
    """FP32 local training (OMP + MOD, 5 iterations) with the checked FP32
    solve forced: per-iteration RMSE within 1e-3 of the oracle's."""
    ctx.set_option(sdl.OPT_AUTOTUNE, 0)
    ctx.set_option(sdl.OPT_MOD_MIXED, 1)
    p = si.split_merge_problem("t", 16, 32, 4, 2, 2, 32, [300, 900, 450, 66, 1000], 5, 5, 0.02,
                               np.random.default_rng(940))
    Yp = p.Y[p.perm]
    Dinit = np.stack([Yp[q] / np.linalg.norm(Yp[q], axis=1, keepdims=True) for q in p.picks])
    Dg = _t(Dinit.astype(np.float32))
    xfro, rmse = sdl.local_train(_t(Yp.astype(np.float32)), p.offsets, Dg, p.s1, 5)
    orc = oracle.local_train(Yp.astype(np.float64), p.offsets, Dinit.astype(np.float64), p.s1, 5)
    rel = np.abs(rmse.cpu().numpy() - orc["rmse"]) / orc["rmse"]
    assert rel.max() < 1e-3, rel
