"""The FP64 MOD solve implementations against the oracle's MOD (Sec. 1:
D = Y X^T (X X^T)^{-1} over the used atoms, then unit columns, Sec. 3.1).

Every implementation the context can select is forced in turn: the tiled
cluster solve with each tile edge and cluster size (ragged shapes whose K and m
are not multiples of the tile), the distributed-shared-memory cluster solve and
the one-block factorisation + separate solve; the autotuned default is checked
for a cached, repeatable choice.  FP64 path: atoms within 1e-10 absolute (unit
atoms, condition numbers of these normal equations below 1e3); FP32 path:
2e-5.
"""
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
    c.set_option(sdl.OPT_SM_BLOCKS, 0)
    c.set_option(sdl.OPT_AUTOTUNE, 1)


def _problem(seed, sizes, m, K, s, dtype, unused=3):
    rng = np.random.default_rng(seed)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    Y = rng.standard_normal((n, m)).astype(dtype)
    hi = K - unused                                # the last `unused` atoms stay unused
    idx = np.stack([rng.choice(hi, s, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, s)).astype(dtype)
    idx[::5, -1] = -1                              # ragged nnz
    val[::5, -1] = 0
    D0 = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(dtype)
    return offsets, Y, idx, val, D0


def _oracle_batched(offsets, Y, idx, val, D0):
    out = []
    for t in range(len(offsets) - 1):
        a, b = offsets[t], offsets[t + 1]
        Do, _, _, st = oracle.mod(Y[a:b].astype(np.float64), idx[a:b], val[a:b].astype(np.float64),
                                  D0[t].astype(np.float64), True)
        assert st == 0
        out.append(Do)
    return np.stack(out)


def _run(ctx, path, ts, C, offsets, Y, idx, val, D0, cap=0):
    ctx.set_option(sdl.OPT_MOD_SOLVE, path)
    ctx.set_option(sdl.OPT_MOD_TILE, ts)
    ctx.set_option(sdl.OPT_CLUSTER, C)
    ctx.set_option(sdl.OPT_SM_BLOCKS, cap)
    Dg = _t(D0.copy())
    sdl.mod_update_batched(_t(Y), offsets, _t(idx), _t(val), Dg)
    return Dg.cpu().numpy()


@pytest.mark.parametrize("K,m,s", [(60, 30, 4), (97, 33, 5), (256, 64, 6)])
@pytest.mark.parametrize("ts,C,cap", [(16, 1, 0), (16, 3, 2), (16, 16, 0), (32, 1, 1), (32, 2, 0), (32, 8, 3),
                                      (32, 16, 0)])
def test_tiled_solve_fp64_matches_oracle(ctx, ts, C, cap, K, m, s):
    offsets, Y, idx, val, D0 = _problem(300 + K, [3 * K, 5 * K, 4 * K], m, K, s, np.float64)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    got = _run(ctx, 3, ts, C, offsets, Y, idx, val, D0, cap)
    np.testing.assert_array_equal(got[:, K - 3:], D0[:, K - 3:])   # unused atoms: bit-exact
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


@pytest.mark.parametrize("ts,C", [(16, 1), (16, 4), (32, 2)])
def test_tiled_solve_ridge_retry(ctx, ts, C):
    """Atoms 0 and 1 always appear together with equal coefficients, so
    X X^T is singular and the factorisation breaks down; the retry with
    A + lambda I on the used atoms matches the oracle, which takes the same
    retry."""
    rng = np.random.default_rng(301)
    m, K, n = 6, 5, 50
    Y = rng.standard_normal((n, m))
    third = rng.integers(2, K, size=n)
    idx = np.stack([np.zeros(n), np.ones(n), third], axis=1).astype(np.int32)
    c = rng.standard_normal(n)
    val = np.stack([c, c, rng.standard_normal(n)], axis=1)
    Dprev = si.unit_gaussian_atoms(rng, m, K)
    Do, _, ridge, st = oracle.mod(Y, idx, val, Dprev, True)
    assert ridge and st == 0
    got = _run(ctx, 3, ts, C, np.array([0, n], np.int64), Y, idx, val, Dprev[None])
    np.testing.assert_allclose(got[0], Do, atol=1e-5)


def test_tiled_solve_merge_shape_K1024(ctx):
    """One subset with K=1024, m=256 (the large image-patch merge shape), 32 x 32
    tiles over a cluster of 16 blocks, FP32 atoms."""
    offsets, Y, idx, val, D0 = _problem(302, [6000], 256, 1024, 4, np.float32, unused=0)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    got = _run(ctx, 3, 32, 16, offsets, Y, idx, val, D0)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5)


def test_all_paths_agree_fp32(ctx):
    offsets, Y, idx, val, D0 = _problem(303, [700, 512, 1100, 900], 64, 256, 3, np.float32)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    for path in (1, 2, 3):
        got = _run(ctx, path, 0, 0, offsets, Y, idx, val, D0)
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-5, err_msg=f"path {path}")


def test_autotuned_choice_matches_oracle(ctx):
    """The first call tunes (every candidate runs on the call's inputs), later
    calls reuse the cached choice; all agree with the oracle.  Repeated calls
    agree to rounding level, not bit for bit: the accumulation of A and B
    visits each atom's signals in an order set by atomics."""
    offsets, Y, idx, val, D0 = _problem(304, [800, 900, 1000, 700, 600], 64, 128, 4, np.float64)
    ctx.set_option(sdl.OPT_AUTOTUNE, 0)
    ctx.set_option(sdl.OPT_AUTOTUNE, 1)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    for _ in range(3):
        got = _run(ctx, 0, 0, 0, offsets, Y, idx, val, D0)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


@pytest.mark.parametrize("K,m,s", [(60, 30, 4), (97, 33, 5), (256, 64, 6)])
@pytest.mark.parametrize("ts,G", [(16, 1), (16, 7), (16, 100), (32, 40)])
def test_wide_solve_fp64_matches_oracle(ctx, ts, G, K, m, s):
    """The wide form (option 4): each subset's tile tasks over G blocks of a
    cooperative launch meeting at barriers in global memory; the same steps as
    the cluster form, so the same 1e-10 FP64 bound, unused atoms bit-exact."""
    offsets, Y, idx, val, D0 = _problem(310 + K, [3 * K, 5 * K, 4 * K], m, K, s, np.float64)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    got = _run(ctx, 4, ts, G, offsets, Y, idx, val, D0)
    np.testing.assert_array_equal(got[:, K - 3:], D0[:, K - 3:])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


@pytest.mark.parametrize("ts,G", [(16, 8), (16, 64), (32, 30)])
def test_wide_solve_ridge_retry(ctx, ts, G):
    rng = np.random.default_rng(311)
    m, K, n = 6, 5, 50
    Y = rng.standard_normal((n, m))
    third = rng.integers(2, K, size=n)
    idx = np.stack([np.zeros(n), np.ones(n), third], axis=1).astype(np.int32)
    c = rng.standard_normal(n)
    val = np.stack([c, c, rng.standard_normal(n)], axis=1)
    Dprev = si.unit_gaussian_atoms(rng, m, K)
    Do, _, ridge, st = oracle.mod(Y, idx, val, Dprev, True)
    assert ridge and st == 0
    got = _run(ctx, 4, ts, G, np.array([0, n], np.int64), Y, idx, val, Dprev[None])
    np.testing.assert_allclose(got[0], Do, atol=1e-5)


@pytest.mark.parametrize("K,m,n", [(256, 64, 25600), (1024, 256, 12000)])
def test_wide_solve_single_system_merge_shapes(ctx, K, m, n):
    """The merge phase's single systems (K=256, m=64: the split-and-merge
    workload; K=1024, m=256: the image-patch workload), FP32 atoms, against the
    oracle; the wide form over every SM and the 16-block cluster form are timed
    side by side (printed)."""
    offsets, Y, idx, val, D0 = _problem(312 + K, [n], m, K, 4, np.float32, unused=0)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    import time
    times = {}
    for path, ts, G in ((3, 16 if K <= 256 else 32, 16), (4, 16, 152), (4, 32, 152), (4, 16, 304)):
        got = _run(ctx, path, ts, G, offsets, Y, idx, val, D0)
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-5, err_msg=f"path {path} ts {ts} G {G}")
        Dg = _t(D0.copy())
        Yg, ig, vg = _t(Y), _t(idx), _t(val)
        sdl.mod_update_batched(Yg, offsets, ig, vg, Dg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            sdl.mod_update_batched(Yg, offsets, ig, vg, Dg)
        torch.cuda.synchronize()
        times[(path, ts, G)] = (time.perf_counter() - t0) / 5 * 1e3
    print(f"K={K} m={m}: MOD update ms (accumulate + solve) by (path, tile, blocks): "
          + ", ".join(f"{k}: {v:.3f}" for k, v in times.items()))


def test_autotuned_single_system_matches_oracle(ctx):
    """One subset: the autotuner times the cluster candidates and the wide
    form; its cached choice agrees with the oracle on every call."""
    offsets, Y, idx, val, D0 = _problem(313, [4000], 64, 256, 4, np.float64, unused=0)
    ctx.set_option(sdl.OPT_AUTOTUNE, 0)
    ctx.set_option(sdl.OPT_AUTOTUNE, 1)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    for _ in range(3):
        got = _run(ctx, 0, 0, 0, offsets, Y, idx, val, D0)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


def test_wide_solve_bounded_wait_runs_out_and_context_stays_usable(ctx):
    """A device-side wait made to run out: one block of each wide-solve group
    leaves at once (SDL_OPT_WAIT_TEST), so the other blocks' first barrier can
    never complete.  With a short limit (2^14 polls of 64 ns) they give up, the
    call returns SDL_ETIMEOUT and leaves the atoms unchanged, and the next call
    on the same context matches the oracle."""
    offsets, Y, idx, val, D0 = _problem(314, [3000], 64, 256, 4, np.float64, unused=0)
    ctx.set_option(sdl.OPT_MOD_SOLVE, 4)
    ctx.set_option(sdl.OPT_MOD_TILE, 16)
    ctx.set_option(sdl.OPT_CLUSTER, 8)
    ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 14)
    ctx.set_option(sdl.OPT_WAIT_TEST, 1)
    Dg = _t(D0.copy())
    try:
        with pytest.raises(sdl.SdlError) as err:
            sdl.mod_update_batched(_t(Y), offsets, _t(idx), _t(val), Dg)
        assert err.value.status == 3, err.value   # SDL_ETIMEOUT
    finally:
        ctx.set_option(sdl.OPT_WAIT_TEST, 0)
        ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 24)
    np.testing.assert_array_equal(Dg.cpu().numpy(), D0)
    want = _oracle_batched(offsets, Y, idx, val, D0)
    got = _run(ctx, 4, 16, 8, offsets, Y, idx, val, D0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)
