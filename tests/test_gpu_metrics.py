"""The training metrics through the C ABI against the oracle: ||Y - D X||_F^2
and ||Y||_F^2 of ELL codes (Table 1's MSE_train is 20 log10 of the square root
of their ratio) and the atom recovery count of Sec. 3.1.

The oracle forms both energies in FP64.  On FP64 data the GPU does too, so the
sums agree to summation order (1e-12 relative).  On FP32 data the GPU keeps
each residual entry and both sums in compensated FP32 (about 48 significant
bits), so they agree with the oracle's FP64 sums of the same FP32 values to
1e-9 relative, far inside what the reported dB figure resolves."""
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


@pytest.mark.parametrize("dtype,rtol", [(np.float32, 1e-9), (np.float64, 1e-12)])
@pytest.mark.parametrize("m,K,n,s", [(64, 256, 20000, 6), (37, 100, 3001, 4), (256, 512, 2000, 16)])
def test_residual_energies_match_oracle(dtype, rtol, m, K, n, s):
    rng = np.random.default_rng(700 + m + s)
    D = si.unit_gaussian_atoms(rng, m, K).astype(dtype)
    Y = rng.standard_normal((n, m)).astype(dtype)
    idx = np.stack([rng.choice(K, s, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, s)).astype(dtype) * 0.3
    idx[::5, s // 2:] = -1                  # ragged codes
    val[::5, s // 2:] = 0
    got = sdl.residual(_t(Y), _t(D), _t(idx), _t(val)).cpu().numpy()
    r2, y2 = oracle.residual(Y.astype(np.float64), D.astype(np.float64), idx, val.astype(np.float64))
    np.testing.assert_allclose(got, [r2, y2], rtol=rtol, atol=0)


def test_residual_of_exact_codes_is_zero_to_rounding():
    """Signals built exactly from their codes: the FP32 residual energy is at
    the rounding level of the data, not of an FP32 sum."""
    rng = np.random.default_rng(710)
    m, K, n, s = 64, 128, 4000, 5
    D = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    idx = np.stack([rng.choice(K, s, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, s)).astype(np.float32)
    Y = np.einsum("nsm,ns->nm", D[idx].astype(np.float64), val.astype(np.float64)).astype(np.float32)
    got = sdl.residual(_t(Y), _t(D), _t(idx), _t(val)).cpu().numpy()
    r2, y2 = oracle.residual(Y.astype(np.float64), D.astype(np.float64), idx, val.astype(np.float64))
    # the residual is the FP32 rounding of Y alone (r2 ~ 1e-8 of y2); an FP32
    # sum of FP32 products would miss it by ~1e-13 of y2
    assert abs(got[0] - r2) <= 1e-6 * r2 + 1e-15 * y2, (got[0], r2, y2)
    np.testing.assert_allclose(got[1], y2, rtol=1e-9)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_recovery_count_matches_oracle(dtype):
    rng = np.random.default_rng(720)
    m, K = 30, 60
    D0 = si.unit_gaussian_atoms(rng, m, K)
    noise = np.where(np.arange(K)[:, None] % 2 == 0, 0.02, 0.2)   # half recovered, half not
    D = D0 + noise * rng.standard_normal(D0.shape)
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    assert np.abs(np.abs(D0 @ D.T).max(axis=1) - 0.98).min() > 1e-3   # no count decided by rounding
    got = int(sdl.recovery(_t(D0.astype(dtype)), _t(D.astype(dtype))).cpu()[0])
    want = oracle.recovery(D0, D)
    assert 0 < want < K and got == want
