"""The two FP32 OMP forms (SDL_OPT_OMP_FORM): the fused kernel with the
correlation tile in shared memory, and the correlation GEMM into a scratch
followed by the selection kernel.  Both compute every correlation as the same
sequence of FP32 FMAs over the signal entries and then run the same selection
code, so their codes must be identical bit for bit; the two-kernel form is
also checked against the oracle under the FP32 rule."""
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


def _run(form, Ds, Y, off, s, eps):
    ctx = sdl.context(0)
    ctx.set_option(sdl.OPT_OMP_FORM, form)
    try:
        out = sdl.omp_batched(_t(Ds), _t(Y), off, s, eps=eps)
    finally:
        ctx.set_option(sdl.OPT_OMP_FORM, 0)
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("m,K,s,eps", [(64, 256, 6, 0.0), (20, 100, 5, 0.0), (144, 512, 10, 0.0),
                                       (256, 512, 8, 0.0), (64, 256, 32, 0.3), (8, 16, 3, 0.0),
                                       (256, 1024, 16, 0.0), (37, 130, 4, 0.0)])
def test_forms_agree_bit_for_bit(m, K, s, eps):
    rng = np.random.default_rng(600 + m + K + s)
    sizes = [517, 0, 1, 2000, 130]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    Y = rng.standard_normal((int(off[-1]), m)).astype(np.float32)
    fused = _run(1, Ds, Y, off, s, eps)
    split = _run(2, Ds, Y, off, s, eps)
    for a, b in zip(fused, split):
        np.testing.assert_array_equal(a, b)


def test_two_kernel_form_matches_oracle():
    rng = np.random.default_rng(610)
    m, K, s = 144, 512, 10
    sizes = [300, 129, 1]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    D0 = si.unit_gaussian_atoms(rng, m, K)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    Y, _, _ = si.sparse_signals(rng, D0, int(off[-1]), s, 0.02, dtype=np.float32)
    idx, val, nnz, r2 = _run(2, Ds, Y, off, s, 0.0)
    for t in range(len(sizes)):
        a, b = off[t], off[t + 1]
        D64, Y64 = Ds[t].astype(np.float64), Y[a:b].astype(np.float64)
        orc = oracle.omp(D64, Y64, s)
        compare_codes(D64, Y64, idx[a:b], val[a:b], nnz[a:b], r2[a:b], orc,
                      fp32_gap_tol(m, np.linalg.norm(Y64, axis=1)), 1e-4)
