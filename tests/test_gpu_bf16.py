"""BF16 tensor-core path (SDL_PREC_BF16: tcgen05 correlations and Gram, FP32 refit)
against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic): BF16 rounds each operand to 8
significant bits (round to nearest, u = 2^-9), products are exact and
accumulate in FP32, so alpha0_j = d_j^T y is off by at most
e sum_i |d_ji y_i|, e = 2u + u^2 + gamma_m.  The selection compares running
correlations alpha0_j - g_j^T G_SS^-1 alpha0_S (FP32 Gram from a BF16 hi/lo
split, about 2^-16), which inherit that error as delta_j - w_j^T delta_S with
w_j the coefficients of d_j on the support so far.  A support may differ from
the oracle's only at a step where the oracle's top-two gap, and the amount by
which the GPU's atom trails the oracle's under the oracle's own residual, are
both below 1.25 (E_o + E_g), E the per-atom bound (tests/_parity.py); each test
caps the share of signals that differ.  Whatever support the GPU chose, its
coefficients are corrected in FP32 on that support (residual from D and y), so they must
equal the exact least-squares fit on that support within the BF16 coefficient
tolerance 2e-2, and the reported residual must be that fit's residual.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import check_bf16_codes, check_rmse, compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
# Share of signals allowed to differ at near-ties that are not at rounding
# level, about twice what these seeded inputs gave (2.2 %, 0.9 %, 28 %, 1.8 %,
# 50 %).  The signals hold at most 6 atoms: coding them with s = 10 or 16 atoms
# spends the last picks on noise whose largest correlations lie within the
# BF16 bound of one another, hence the two high shares.
CAPS = {(64, 256): 0.04, (64, 128): 0.02, (144, 512): 0.40, (30, 60): 0.04, (256, 1024): 0.65}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _problem(seed, m, K, n, s, sigma):
    rng = np.random.default_rng(seed)
    D0 = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    Y, _, _ = si.sparse_signals(rng, D0.astype(np.float64), n, s, sigma, dtype=np.float32)
    return D0, Y


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("m,K,n,s", [(64, 256, 4133, 6), (64, 128, 700, 5), (144, 512, 1500, 10),
                                     (30, 60, 333, 6), (256, 1024, 300, 16)])
def test_bf16_omp_matches_oracle(m, K, n, s, form):
    """The BF16 forms (1: Batch-OMP selection from alpha0; 3: the same with a
    half-precision Gram copy in the running update; 2: residual form) under the
    Batch-OMP rule with the half-precision term, whose bound covers all three."""
    D, Y = _problem(400 + m + K, m, K, n, min(s, 6), 0.01)
    ctx = sdl.context(0)
    ctx.set_option(sdl.OPT_BF16_FORM, form)
    try:
        idx, val, nnz, r2 = sdl.omp(_t(D), _t(Y), s, prec=sdl.PREC_BF16)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(sdl.OPT_BF16_FORM, 0)
    orc = oracle.omp(D.astype(np.float64), Y.astype(np.float64), s)
    excused, rounding = check_bf16_codes(D, Y, idx.cpu().numpy(), val.cpu().numpy(), nnz.cpu().numpy(),
                                         r2.cpu().numpy(), orc, max_excused=CAPS[(m, K)], h16=True)
    # near-tie picks cost little: mean residual energy within 5 % of the oracle's
    # (measured 2.7 % at m=30, K=60 where ties are most frequent)
    assert r2.cpu().numpy().astype(np.float64).mean() <= 1.05 * orc["resid2"].mean() + 1e-9
    print(f"form {form} m={m} K={K}: {excused} of {n} supports differ at near-ties, {rounding} more at "
          f"rounding-level steps")


def test_bf16_gram_and_correlation_exact_on_bf16_representable_inputs():
    """With inputs that BF16 represents exactly (multiples of 1/8 in [-1, 1]),
    the tensor-core products are exact: alpha0 = D^T y and the split Gram carry
    no BF16 rounding at all, so the BF16 path must meet the FP32 bar against the
    FP64 oracle (supports equal except at FP32 near-ties, coefficients within
    1e-4).  This holds for the Batch-OMP form (alpha0 = D^T y and G feed every
    step); the residual form rounds each step's residual to BF16.  The atoms
    are not unit norm here; the FP32 gap rule is scaled by the largest atom
    norm."""
    rng = np.random.default_rng(410)
    m, K, n, s = 64, 256, 300, 4
    D = (rng.integers(-8, 9, size=(K, m)) / 8.0).astype(np.float32)
    Y = (rng.integers(-8, 9, size=(n, m)) / 8.0).astype(np.float32)
    ctx = sdl.context(0)
    # the Batch-OMP form with the FP32 Gram throughout: alpha0 and G exact on
    # these inputs (form 3's half-precision copy of G would not be: |G| reaches 64)
    ctx.set_option(sdl.OPT_BF16_FORM, 1)
    try:
        idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp(_t(D), _t(Y), s, prec=sdl.PREC_BF16))
    finally:
        ctx.set_option(sdl.OPT_BF16_FORM, 0)
    D64, Y64 = D.astype(np.float64), Y.astype(np.float64)
    orc = oracle.omp(D64, Y64, s)
    dmax = np.linalg.norm(D64, axis=1).max()
    st = compare_codes(D64, Y64, idx, val, nnz, r2, orc, fp32_gap_tol(m, np.linalg.norm(Y64, axis=1) * dmax), 1e-4,
                       max_excused=0.01)
    print(f"BF16 on BF16-exact inputs: {st['same']} of {n} supports equal the oracle's, {st['excused']} near-ties")


def test_bf16_batched_uneven_subsets():
    rng = np.random.default_rng(411)
    m, K, s = 64, 256, 6
    sizes = [517, 0, 1, 2000, 130]
    L = len(sizes)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(L)]).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Y = rng.standard_normal((offsets[-1], m)).astype(np.float32)
    idx, val, nnz, r2 = sdl.omp_batched(_t(Ds), _t(Y), offsets, s, prec=sdl.PREC_BF16)
    idx, val, nnz, r2 = (t.cpu().numpy() for t in (idx, val, nnz, r2))
    for t in range(L):
        a, b = offsets[t], offsets[t + 1]
        if a == b:
            continue
        orc = oracle.omp(Ds[t].astype(np.float64), Y[a:b].astype(np.float64), s)
        # the signals are Gaussian noise, not sparse: measured at most 4.6 % per subset
        ex, ro = check_bf16_codes(Ds[t], Y[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc, max_excused=0.08)
        print(f"batched subset {t} ({b - a} signals): {ex} differ at near-ties, {ro} at rounding-level steps")


def test_bf16_local_training_per_iteration():
    """One training iteration from a shared dictionary: the BF16 coding pass's
    codes under the BF16 rule, its RMSE within 1e-3 of the oracle's over the
    signals whose codes agree and equal to that of its own codes, and the
    updated atoms equal to the oracle's MOD of the GPU's own codes within the
    FP32 atom tolerance 2e-5."""
    p = si.split_merge_problem("t", 64, 256, 6, 2, 3, 256, [2000, 1500, 2500], 4, 4, 0.01,
                               np.random.default_rng(412))
    Yp = p.Y[p.perm]
    Dl = np.stack([Yp[q] / np.linalg.norm(Yp[q], axis=1, keepdims=True) for q in p.picks]).astype(np.float32)
    Dg, Ypg = _t(Dl.copy()), _t(Yp)
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp_batched(Dg, Ypg, p.offsets, p.s1, prec=sdl.PREC_BF16))
    _, rmse = sdl.local_train(Ypg, p.offsets, Dg, p.s1, 1, prec=sdl.PREC_BF16)
    after, rmse = Dg.cpu().numpy(), rmse.cpu().numpy()[:, 0]
    for t in range(p.L):
        a, b = p.offsets[t], p.offsets[t + 1]
        orc = oracle.omp(Dl[t].astype(np.float64), Yp[a:b].astype(np.float64), p.s1)
        check_bf16_codes(Dl[t], Yp[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc)
        check_rmse(r2[a:b], orc, idx[a:b], nnz[a:b], p.m, rmse[t])
        Dm, *_ = oracle.mod(Yp[a:b].astype(np.float64), idx[a:b], val[a:b].astype(np.float64),
                            Dl[t].astype(np.float64), True)
        np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5, err_msg=f"subset {t}")


def test_bf16_bounded_waits_run_out_and_context_stays_usable():
    """The loader role of the persistent BF16 correlation kernel leaves before
    its first copy (SDL_OPT_WAIT_TEST), so the MMA issuer's first wait for a
    dictionary slab can never complete: with a short limit every role gives
    up, the call returns SDL_ETIMEOUT, and the next call on the same context
    meets the BF16 bar against the oracle (the signals hold 4 atoms and are
    coded with s = 4: a fifth pick would rank noise correlations that tie
    within the BF16 bound on several percent of them)."""
    ctx = sdl.context(0)
    D, Y = _problem(413, 64, 256, 700, 4, 0.02)
    ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 12)
    ctx.set_option(sdl.OPT_WAIT_TEST, 1)
    try:
        with pytest.raises(sdl.SdlError) as err:
            sdl.omp(_t(D), _t(Y), 4, prec=sdl.PREC_BF16)
            torch.cuda.synchronize()
        assert err.value.status == 3, err.value   # SDL_ETIMEOUT
    finally:
        ctx.set_option(sdl.OPT_WAIT_TEST, 0)
        ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 24)
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp(_t(D), _t(Y), 4, prec=sdl.PREC_BF16))
    orc = oracle.omp(D.astype(np.float64), Y.astype(np.float64), 4)
    check_bf16_codes(D, Y, idx, val, nnz, r2, orc, max_excused=0.04)


@pytest.mark.parametrize("m,K,sizes", [(100, 700, [129, 1, 300]), (192, 1000, [257, 3]), (17, 33, [640, 5])])
def test_bf16_correlation_passes_and_ragged_edges(m, K, sizes):
    """Shapes that exercise every edge of the persistent correlation kernel:
    several 256-atom passes per tile with a partial last pass (K = 700, 1000,
    33), signal lengths that are not multiples of 4 or 64 (scalar loads, a
    partial last 64-entry block), K not a multiple of 4 (scalar stores), and
    tiles with 1-129 valid rows over uneven subsets; codes under the BF16 rule
    against the oracle, subset by subset."""
    rng = np.random.default_rng(414 + m)
    s = 4
    L = len(sizes)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(L)]).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Y = np.concatenate([si.sparse_signals(rng, Ds[t].astype(np.float64), n, s, 0.01, dtype=np.float32)[0]
                        for t, n in enumerate(sizes)])
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp_batched(_t(Ds), _t(Y), offsets, s, prec=sdl.PREC_BF16))
    for t in range(L):
        a, b = offsets[t], offsets[t + 1]
        orc = oracle.omp(Ds[t].astype(np.float64), Y[a:b].astype(np.float64), s)
        ex, ro = check_bf16_codes(Ds[t], Y[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc, max_excused=0.05)
        print(f"m={m} K={K} subset {t} ({b - a} signals): {ex} differ at near-ties, {ro} at rounding-level steps")
