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


@pytest.mark.parametrize("prec", [sdl.PREC_F32, sdl.PREC_BF16, sdl.PREC_F32X3])
@pytest.mark.parametrize("m,K,s", [(64, 256, 6), (37, 130, 4), (256, 1024, 16)])
def test_selection_shapes_agree_bit_for_bit(prec, m, K, s):
    """The autotuner's knobs of the selection launch (SDL_OPT_SEL_SPW: 1, 2 or
    4 signals per warp; SDL_OPT_SEL_GCACHE: the support's Gram columns cached
    in shared memory or none) change which warp codes a signal and where the
    columns are read from, not the arithmetic: every shape gives the same
    codes bit for bit, over uneven subsets with ragged tiles, in each
    precision of the two-kernel passes; the default shape is checked against
    the oracle by the other tests."""
    rng = np.random.default_rng(620 + m + K)
    sizes = [517, 0, 1, 300, 130]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    Y = rng.standard_normal((int(off[-1]), m)).astype(np.float32)
    ctx = sdl.context(0)
    outs = {}
    try:
        for spw in (4, 2, 1):
            for gc in (1, 2):
                ctx.set_option(sdl.OPT_SEL_SPW, spw)
                ctx.set_option(sdl.OPT_SEL_GCACHE, gc)
                outs[(spw, gc)] = [o.cpu().numpy() for o in sdl.omp_batched(_t(Ds), _t(Y), off, s, prec=prec)]
    finally:
        ctx.set_option(sdl.OPT_SEL_SPW, 0)
        ctx.set_option(sdl.OPT_SEL_GCACHE, 0)
    ref = outs[(4, 1)]
    for k, out in outs.items():
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b, err_msg=f"shape {k}")


def test_autotuned_selection_matches_fixed_shape():
    """A call large enough to be tuned (at least two 128-signal tiles per SM)
    gives the codes of the fixed default shape bit for bit, first call (which
    times every shape) and second (the cached choice) alike."""
    rng = np.random.default_rng(630)
    m, K, s = 64, 256, 6
    n = 128 * 2 * 160
    D = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    Y, _, _ = si.sparse_signals(rng, D.astype(np.float64), n, s, 0.02, dtype=np.float32)
    ctx = sdl.context(0)
    ctx.set_option(sdl.OPT_AUTOTUNE, 0)   # forget earlier choices
    ctx.set_option(sdl.OPT_SEL_SPW, 4)
    ctx.set_option(sdl.OPT_SEL_GCACHE, 1)
    try:
        fixed = [o.cpu().numpy() for o in sdl.omp(_t(D), _t(Y), s, prec=sdl.PREC_BF16)]
    finally:
        ctx.set_option(sdl.OPT_SEL_SPW, 0)
        ctx.set_option(sdl.OPT_SEL_GCACHE, 0)
        ctx.set_option(sdl.OPT_AUTOTUNE, 1)
    for _ in range(2):
        tuned = [o.cpu().numpy() for o in sdl.omp(_t(D), _t(Y), s, prec=sdl.PREC_BF16)]
        for a, b in zip(fixed, tuned):
            np.testing.assert_array_equal(a, b)
