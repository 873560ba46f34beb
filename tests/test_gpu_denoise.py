"""Denoising (Sec. 3.2.2) through the C ABI against the oracle: patch
extraction (bit-exact), overlap averaging of given codes (FP64 to 1e-12,
FP32 to 2e-5 on [0, 1] images: at most p^2 s FP32 products per pixel), and the
whole pipeline with error-constrained OMP.  In the pipeline a patch's code may
differ from the oracle's only at a near-tie (the FP32 OMP rule), so the
denoised images are compared through their PSNR (within 0.01 dB) and their mean
absolute difference; at full size (a 512 x 512 image, 255,025 patches) sampled
codes are checked under the FP32 rule and the average of the GPU's own codes
against the oracle's average of the same codes."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _psnr(a, clean):
    return 10 * np.log10(1.0 / np.mean((a - clean) ** 2))


@pytest.mark.parametrize("H,W,p", [(37, 29, 8), (16, 16, 16), (9, 11, 1), (64, 48, 5)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_extract_patches_bit_exact(H, W, p, dtype):
    img = np.random.default_rng(H * W + p).standard_normal((H, W)).astype(dtype)
    got = sdl.extract_patches(_t(img), p).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.extract_patches(img, p).astype(dtype))


@pytest.mark.parametrize("dtype,atol", [(np.float64, 1e-12), (np.float32, 2e-5)])
def test_patch_average_of_given_codes(dtype, atol):
    rng = np.random.default_rng(31)
    H, W, p, K, s = 41, 35, 8, 128, 6
    D = si.overcomplete_dct(p, 8, 16)
    n = (H - p + 1) * (W - p + 1)
    idx = np.stack([rng.choice(K, s, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.uniform(-0.3, 0.3, (n, s))
    idx[::3, 4:] = -1                       # ragged codes
    val[::3, 4:] = 0
    want = oracle.patch_average(D, idx, val, H, W, p)
    got = sdl.patch_average(_t(D.astype(dtype)), _t(idx), _t(val.astype(dtype)), H, W, p).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=atol)


def test_denoising_pipeline_matches_oracle():
    rng = np.random.default_rng(32)
    clean = si.synthetic_image(rng, size=72, bumps=8, edges=3, sigma=0.0)
    sigma = 20 / 255
    noisy = clean + sigma * rng.standard_normal(clean.shape)
    p, eps = 8, 8.5 * sigma
    D = si.overcomplete_dct(p, 16, 16)
    den, (idx, val, nnz) = sdl.denoise(_t(noisy.astype(np.float32)), _t(D.astype(np.float32)), p, eps)
    den = den.cpu().numpy().astype(np.float64)
    P = oracle.extract_patches(noisy, p)
    o = oracle.omp(D, P, 32, eps=eps)
    oden = oracle.patch_average(D, o["idx"], o["val"], *clean.shape, p)
    assert abs(_psnr(den, clean) - _psnr(oden, clean)) < 0.01, (_psnr(den, clean), _psnr(oden, clean))
    assert np.abs(den - oden).mean() < 1e-4
    assert _psnr(den, clean) > _psnr(noisy, clean) + 6


def test_denoising_full_size_image_sampled():
    rng = np.random.default_rng(33)
    clean = si.synthetic_image(rng, size=512, sigma=0.0)
    sigma = 20 / 255
    noisy = (clean + sigma * rng.standard_normal(clean.shape)).astype(np.float32)
    p, eps = 8, 8.5 * sigma
    D = si.overcomplete_dct(p, 16, 16).astype(np.float32)
    den, (idx, val, nnz) = sdl.denoise(_t(noisy), _t(D), p, eps)
    den, idx, val, nnz = (x.cpu().numpy() for x in (den, idx, val, nnz))
    P = oracle.extract_patches(noisy.astype(np.float64), p)
    pick = rng.choice(len(P), 3000, replace=False)
    o = oracle.omp(D.astype(np.float64), P[pick], 32, eps=eps)
    Pg = P[pick]
    r2 = np.array([np.sum((Pg[i] - D[idx[q][:nnz[q]]].T.astype(np.float64) @ val[q][:nnz[q]]) ** 2)
                   for i, q in enumerate(pick)])
    compare_codes(D.astype(np.float64), Pg, idx[pick], val[pick], nnz[pick], r2, o,
                  fp32_gap_tol(p * p, np.linalg.norm(Pg, axis=1)), 1e-4, eps=eps)
    oden = oracle.patch_average(D.astype(np.float64), idx, val.astype(np.float64), 512, 512, p)
    np.testing.assert_allclose(den, oden, rtol=0, atol=2e-5)
    assert _psnr(den.astype(np.float64), clean) > _psnr(noisy.astype(np.float64), clean) + 6
