"""Single-product TF32 tensor-core path (SDL_PREC_TF32: correlations from one
kind::tf32 product, the Gram from the two-term TF32 split, FP32 correction on
the support) against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic, tests/_parity.py: tf32_unit): each
operand is rounded to nearest with 11 significant bits (u = 2^-11), products
are exact and accumulate in FP32, so alpha0_j = d_j^T y is off by at most
e sum_i |d_ji y_i|, e = 2u + u^2 + gamma_m (unit 2^-23 for the tensor cores'
sums).  That error reaches the running correlations the selection compares as
delta_j - w_j^T delta_S, as on the BF16 path, so the BF16 rule of
check_bf16_codes applies with e in place of the BF16 unit: a support may differ
from the oracle's only at a step where the oracle's top-two gap and the GPU
atom's lag are both below 1.25 (E_o + E_g), and each test caps the share of
signals that differ there.  The Gram is FP32-accurate (about 3 2^-22), so the
correction step makes the coefficients the exact least-squares fit on the
GPU's support within 2e-2 (checked) and in practice far closer."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import check_bf16_codes, check_rmse, compare_codes, fp32_gap_tol, tf32_unit

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TF32 = sdl.PREC_TF32
# Share of signals allowed to differ at near-ties that are not at rounding
# level: the BF16 caps, whose bound is four times wider (TF32 keeps 2 more bits).
CAPS = {(64, 256): 0.04, (64, 128): 0.02, (144, 512): 0.40, (30, 60): 0.04, (256, 1024): 0.65}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _problem(seed, m, K, n, s, sigma):
    rng = np.random.default_rng(seed)
    D0 = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    Y, _, _ = si.sparse_signals(rng, D0.astype(np.float64), n, s, sigma, dtype=np.float32)
    return D0, Y


@pytest.mark.parametrize("m,K,n,s", [(64, 256, 4133, 6), (64, 128, 700, 5), (144, 512, 1500, 10),
                                     (30, 60, 333, 6), (256, 1024, 300, 16)])
def test_tf32_omp_matches_oracle(m, K, n, s):
    D, Y = _problem(450 + m + K, m, K, n, min(s, 6), 0.01)
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp(_t(D), _t(Y), s, prec=TF32))
    orc = oracle.omp(D.astype(np.float64), Y.astype(np.float64), s)
    excused, rounding = check_bf16_codes(D, Y, idx, val, nnz, r2, orc, max_excused=CAPS[(m, K)],
                                         unit=tf32_unit(m))
    assert r2.astype(np.float64).mean() <= 1.05 * orc["resid2"].mean() + 1e-9
    print(f"TF32 m={m} K={K}: {excused} of {n} supports differ at near-ties, {rounding} more at rounding-level steps")


def test_tf32_correlation_exact_on_tf32_representable_inputs():
    """Inputs that TF32 represents exactly (multiples of 1/8 in [-1, 1]) make
    the single product exact, so the TF32 path must meet the FP32 bar against
    the FP64 oracle (the FP32 gap rule scaled by the largest atom norm,
    coefficients within 1e-4)."""
    rng = np.random.default_rng(451)
    m, K, n, s = 64, 256, 300, 4
    D = (rng.integers(-8, 9, size=(K, m)) / 8.0).astype(np.float32)
    Y = (rng.integers(-8, 9, size=(n, m)) / 8.0).astype(np.float32)
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp(_t(D), _t(Y), s, prec=TF32))
    D64, Y64 = D.astype(np.float64), Y.astype(np.float64)
    orc = oracle.omp(D64, Y64, s)
    dmax = np.linalg.norm(D64, axis=1).max()
    st = compare_codes(D64, Y64, idx, val, nnz, r2, orc, fp32_gap_tol(m, np.linalg.norm(Y64, axis=1) * dmax), 1e-4,
                       max_excused=0.01)
    print(f"TF32 on TF32-exact inputs: {st['same']} of {n} supports equal the oracle's, {st['excused']} near-ties")


@pytest.mark.parametrize("m,K,sizes", [(64, 256, [517, 0, 1, 2000, 130]), (100, 700, [129, 1, 300]),
                                       (17, 33, [640, 5])])
def test_tf32_batched_uneven_subsets(m, K, sizes):
    """Uneven subsets (empty, one signal, ragged tiles), K with a partial
    256-atom pass, m not a multiple of 4 or 32: subset by subset against the
    oracle under the TF32 rule."""
    rng = np.random.default_rng(452 + m)
    s = 4
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Y = np.concatenate([si.sparse_signals(rng, Ds[t].astype(np.float64), n, s, 0.01, dtype=np.float32)[0]
                        for t, n in enumerate(sizes)])
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp_batched(_t(Ds), _t(Y), offsets, s, prec=TF32))
    for t in range(len(sizes)):
        a, b = offsets[t], offsets[t + 1]
        if a == b:
            continue
        orc = oracle.omp(Ds[t].astype(np.float64), Y[a:b].astype(np.float64), s)
        ex, ro = check_bf16_codes(Ds[t], Y[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc, max_excused=0.05,
                                  unit=tf32_unit(m))
        print(f"m={m} K={K} subset {t} ({b - a} signals): {ex} differ at near-ties, {ro} at rounding-level steps")


def test_tf32_local_training_per_iteration():
    """One training iteration from a shared start: the TF32 coding pass's codes
    under the TF32 rule, its RMSE within 1e-3 of the oracle's over the signals
    whose codes agree, and the updated atoms equal to the oracle's MOD of the
    GPU's own codes within the FP32 atom tolerance 2e-5."""
    p = si.split_merge_problem("t", 64, 256, 6, 2, 3, 256, [2000, 1500, 2500], 4, 4, 0.01,
                               np.random.default_rng(453))
    Yp = p.Y[p.perm]
    Dl = np.stack([Yp[q] / np.linalg.norm(Yp[q], axis=1, keepdims=True) for q in p.picks]).astype(np.float32)
    Dg, Ypg = _t(Dl.copy()), _t(Yp)
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp_batched(Dg, Ypg, p.offsets, p.s1, prec=TF32))
    _, rmse = sdl.local_train(Ypg, p.offsets, Dg, p.s1, 1, prec=TF32)
    after, rmse = Dg.cpu().numpy(), rmse.cpu().numpy()[:, 0]
    for t in range(p.L):
        a, b = p.offsets[t], p.offsets[t + 1]
        orc = oracle.omp(Dl[t].astype(np.float64), Yp[a:b].astype(np.float64), p.s1)
        check_bf16_codes(Dl[t], Yp[a:b], idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc, unit=tf32_unit(p.m))
        check_rmse(r2[a:b], orc, idx[a:b], nnz[a:b], p.m, rmse[t])
        Dm, *_ = oracle.mod(Yp[a:b].astype(np.float64), idx[a:b], val[a:b].astype(np.float64),
                            Dl[t].astype(np.float64), True)
        np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5, err_msg=f"subset {t}")


def test_tf32_bounded_waits_run_out_and_context_stays_usable():
    """With the loader roles of the TF32 kernels leaving before their first copy
    (SDL_OPT_WAIT_TEST) and a short wait limit, the call returns SDL_ETIMEOUT;
    the next call on the same context meets the TF32 rule."""
    ctx = sdl.context(0)
    D, Y = _problem(454, 64, 256, 700, 4, 0.02)
    ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 12)
    ctx.set_option(sdl.OPT_WAIT_TEST, 1)
    try:
        with pytest.raises(sdl.SdlError) as err:
            sdl.omp(_t(D), _t(Y), 4, prec=TF32)
            torch.cuda.synchronize()
        assert err.value.status == 3, err.value   # SDL_ETIMEOUT
    finally:
        ctx.set_option(sdl.OPT_WAIT_TEST, 0)
        ctx.set_option(sdl.OPT_WAIT_LIMIT, 1 << 24)
    idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp(_t(D), _t(Y), 4, prec=TF32))
    orc = oracle.omp(D.astype(np.float64), Y.astype(np.float64), 4)
    check_bf16_codes(D, Y, idx, val, nnz, r2, orc, max_excused=0.04, unit=tf32_unit(64))
