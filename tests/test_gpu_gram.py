"""Gram matrices G_t = D_t D_t^T through the C ABI (sdl_gram) against the FP64
product of the same data.

FP64: FMA chains, within 1e-13.  FP32: an m-term FP32 dot product of unit
atoms is within gamma_m = m 2^-24 / (1 - m 2^-24) of exact.  BF16 (tensor
cores): d = hi + lo + r with hi = bf16(d), lo = bf16(d - hi), |lo| <= 2^-9 |d|,
|r| <= 2^-18 |d| (two roundings to 8-bit significands), so hi hi^T + hi lo^T +
lo hi^T misses each product d_i d_j by the dropped terms lo lo and those with
r, about 3 2^-18 |d_i||d_j|, summed over the m entries: at most 3 2^-18 for
unit atoms (Cauchy-Schwarz), plus the FP32 accumulation's gamma_m.  The test
allows 4 2^-16 + gamma_m, room for an accumulation order the tensor cores do
not document.  A single BF16 product (the split's hi hi^T alone) would be
off by about 2^-8: the bound fails for it, which the last test checks with
numpy on the host.  F32X3 and TF32 (the TF32 precision takes its Gram from the
same split): the two-term TF32 split, within 3 2^-22 per product plus the
FP32 accumulation (tests/_parity.py: x3_unit), doubled."""
import numpy as np
import pytest
import torch

import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import x3_unit

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _gamma(m):
    u = 2.0 ** -24
    return m * u / (1 - m * u)


SHAPES = [(64, 256, 3), (144, 512, 2), (30, 60, 4), (256, 1024, 1), (8, 16, 5), (37, 130, 2)]


@pytest.mark.parametrize("m,K,L", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16", "f32x3", "tf32"])
def test_gram_matches_fp64_product(m, K, L, prec):
    rng = np.random.default_rng(800 + m + K + L)
    D = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(L)])
    if prec == "f64":
        Dd, tol, p = D, 1e-13, sdl.PREC_F64
    else:
        D = D.astype(np.float32)
        Dd = D
        # F32X3 and TF32 share the two-term TF32 split Gram: 3 2^-22 per product
        # plus the accumulation (x3_unit), doubled for an undocumented order
        tol = {"f32": _gamma(m), "bf16": 4 * 2.0 ** -16 + _gamma(m)}.get(prec, 2 * x3_unit(m))
        p = {"f32": sdl.PREC_F32, "bf16": sdl.PREC_BF16, "f32x3": sdl.PREC_F32X3, "tf32": sdl.PREC_TF32}[prec]
    G = sdl.gram(_t(Dd), prec=p).cpu().numpy().astype(np.float64)
    D64 = D.astype(np.float64)
    want = np.einsum("lkm,ljm->lkj", D64, D64)
    np.testing.assert_allclose(G, want, rtol=0, atol=tol)


def test_bf16_split_is_needed_for_the_bound():
    """The hi hi^T term alone (one BF16 product) breaks the bound above, so the
    split's two correction terms are what the test measures."""
    rng = np.random.default_rng(810)
    m, K = 144, 512
    D = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    hi = torch.from_numpy(D).to(torch.bfloat16).to(torch.float64).numpy()
    err = np.abs(hi @ hi.T - D.astype(np.float64) @ D.astype(np.float64).T).max()
    assert err > 4 * 2.0 ** -16 + _gamma(m)
