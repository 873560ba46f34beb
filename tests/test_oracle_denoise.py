"""Pins of the oracle's image-denoising pieces (Sec. 3.2.2: error-constrained
coding of every overlapping patch, estimates averaged over the patches covering
each pixel) against facts outside the oracle."""
import numpy as np

import oracle
import sdl_inputs as si


def test_extraction_equals_sliding_windows():
    rng = np.random.default_rng(1)
    img = rng.standard_normal((11, 13))
    for p in (1, 3, 8):
        want = np.lib.stride_tricks.sliding_window_view(img, (p, p)).reshape(-1, p * p)
        np.testing.assert_array_equal(oracle.extract_patches(img, p), want)


def test_exact_patches_average_back_to_the_image():
    """With the identity dictionary and each patch's own pixels as its code,
    every estimate is exact, so every pixel's mean is the pixel."""
    rng = np.random.default_rng(2)
    H, W, p = 9, 7, 3
    img = rng.standard_normal((H, W))
    P = oracle.extract_patches(img, p)
    m = p * p
    idx = np.tile(np.arange(m, dtype=np.int32), (len(P), 1))
    np.testing.assert_allclose(oracle.patch_average(np.eye(m), idx, P, H, W, p), img, rtol=0, atol=1e-14)


def test_average_of_patch_constants_is_the_mean_over_covering_patches():
    """Patch i estimated as the constant i: pixel (y, x) gets the mean of
    r (W-p+1) + c over the covering patches r in [max(0, y-p+1), min(y, H-p)],
    c likewise, i.e. mean(r) (W-p+1) + mean(c)."""
    H, W, p = 8, 10, 3
    nr, nc, m = H - p + 1, W - p + 1, p * p
    D = np.full((1, m), 1.0 / np.sqrt(m))
    idx = np.zeros((nr * nc, 1), np.int32)
    val = (np.arange(nr * nc, dtype=np.float64) * np.sqrt(m))[:, None]
    got = oracle.patch_average(D, idx, val, H, W, p)
    for y in range(H):
        for x in range(W):
            rs = np.arange(max(0, y - p + 1), min(y, nr - 1) + 1)
            cs = np.arange(max(0, x - p + 1), min(x, nc - 1) + 1)
            assert abs(got[y, x] - (rs.mean() * nc + cs.mean())) < 1e-11


def test_error_constrained_coding_with_a_dct_dictionary_denoises():
    """A smooth synthetic image with noise sigma: coding every 8x8 patch with
    the overcomplete DCT at eps = 8.5 sigma (the paper's threshold) and
    averaging raises the PSNR well above the noisy image's."""
    rng = np.random.default_rng(3)
    clean = si.synthetic_image(rng, size=48, bumps=6, edges=2, sigma=0.0)
    sigma = 20 / 255
    noisy = clean + sigma * rng.standard_normal(clean.shape)
    p = 8
    D = si.overcomplete_dct(p, 16, 16)
    P = oracle.extract_patches(noisy, p)
    codes = oracle.omp(D, P, 32, eps=8.5 * sigma)
    den = oracle.patch_average(D, codes["idx"], codes["val"], *clean.shape, p)
    psnr = lambda a: 10 * np.log10(1.0 / np.mean((a - clean) ** 2))
    assert psnr(den) > psnr(noisy) + 6, (psnr(noisy), psnr(den))
