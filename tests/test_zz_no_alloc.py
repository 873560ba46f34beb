"""The allocation-free OMP entry point, sdl_omp_noalloc, against sdl_omp.

sdl_omp_noalloc serves callers that cannot call cudaMalloc where they code
signals (device memory owned entirely by another allocator, or loops that must
not take an allocation's implicit synchronisation).  It keeps its scratch in a
fixed array inside the library instead of a context workspace.  This file is
collected last so that a run stopping at the first failure has already run
every other test.

Each check calls the entry point through the C ABI (ctypes, raw device
pointers) and compares its codes with sdl_omp's on the same inputs, using the
tolerances of the OMP parity tests: identical supports and nnz, coefficients
within 1e-4 relative, residual energies within 1e-4 relative.  Two calls of
different shapes run back to back, so stale scratch from the first would show
up in the second.  At the array's size limit (K = 512, m = 256) the codes are
compared bit for bit with sdl_omp's fused FP32 form (the same kernels) and,
once, with the FP64 oracle under the FP32 parity rule.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SDL_ERANGE = 6


def _inputs(seed, m, K, n, s):
    rng = np.random.default_rng(seed)
    D = si.unit_gaussian_atoms(rng, m, K).astype(np.float32)
    Y, _, _ = si.sparse_signals(rng, D.astype(np.float64), n, s, 0.01, dtype=np.float32)
    return torch.from_numpy(D).to(DEV), torch.from_numpy(Y).to(DEV)


def _noalloc(D, Y, s, eps=0.0):
    K, m = D.shape
    n = Y.shape[0]
    idx = torch.full((n, s), -7, dtype=torch.int32, device=DEV)
    val = torch.full((n, s), 7.0, dtype=torch.float32, device=DEV)
    nnz = torch.full((n,), -7, dtype=torch.int32, device=DEV)
    r2 = torch.full((n,), -7.0, dtype=torch.float32, device=DEV)
    stream = torch.cuda.current_stream().cuda_stream
    rc = sdl.lib().sdl_omp_noalloc(stream, D.data_ptr(), m, K, Y.data_ptr(), n, s, float(eps),
                                   idx.data_ptr(), val.data_ptr(), nnz.data_ptr(), r2.data_ptr())
    torch.cuda.synchronize()
    return rc, idx, val, nnz, r2


def _same_codes(got, ref):
    gi, gv, gn, gr = (t.cpu().numpy() for t in got)
    ri, rv, rn, rr = (t.cpu().numpy() for t in ref)
    assert (gi == ri).all() and (gn == rn).all()
    scale = np.maximum(np.abs(rv), 1e-2 * np.abs(rv).max(axis=1, keepdims=True) + 1e-30)
    assert (np.abs(gv - rv) / scale).max() <= 1e-4
    assert (np.abs(gr - rr) / np.maximum(np.abs(rr), 1e-12)).max() <= 1e-4


def test_noalloc_matches_sdl_omp_on_two_calls_in_a_row():
    D1, Y1 = _inputs(300, 64, 256, 5017, 6)
    D2, Y2 = _inputs(301, 30, 60, 333, 4)
    first = _noalloc(D1, Y1, 6)
    second = _noalloc(D2, Y2, 4, eps=0.05)
    assert first[0] == 0 and second[0] == 0
    _same_codes(first[1:], sdl.omp(D1, Y1, 6))
    _same_codes(second[1:], sdl.omp(D2, Y2, 4, eps=0.05))


@pytest.mark.parametrize("s", [16, 32])
def test_noalloc_at_its_size_limit(s):
    """K = 512 and m = 256 fill the Gram part of the array exactly; n = 1,000
    leaves a ragged last tile of 8 signals.  A smaller call first leaves other
    contents in the array."""
    Ds, Ys = _inputs(303, 40, 100, 77, 3)
    assert _noalloc(Ds, Ys, 3)[0] == 0
    D, Y = _inputs(304 + s, 256, 512, 1000, 12)
    rc, *got = _noalloc(D, Y, s)
    assert rc == 0
    ctx = sdl.context(0)
    ctx.set_option(sdl.OPT_OMP_FORM, 1)
    try:
        fused = sdl.omp(D, Y, s)
    finally:
        ctx.set_option(sdl.OPT_OMP_FORM, 0)
    for a, b in zip(got, fused):
        assert torch.equal(a, b)
    _same_codes(got, sdl.omp(D, Y, s))
    gi, gv, gn, gr = (t.cpu().numpy() for t in got)
    D64, Y64 = D.cpu().numpy().astype(np.float64), Y.cpu().numpy().astype(np.float64)
    orc = oracle.omp(D64, Y64, s)
    # picks past the signals' 12-atom supports code the noise, whose largest
    # correlations lie close together: more near-ties than the default cap allows
    st = compare_codes(D64, Y64, gi, gv, gn, gr, orc, fp32_gap_tol(256, np.linalg.norm(Y64, axis=1)), 1e-4,
                       max_excused=0.05)
    print(f"noalloc K=512 m=256 s={s}: {st['same']} of 1000 codes equal the oracle's, {st['excused']} near-ties")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    D, Y = _inputs(302, 16, 513, 40, 3)
    rc, idx, val, nnz, r2 = _noalloc(D, Y, 3)
    assert rc == SDL_ERANGE
    assert (idx.cpu() == -7).all() and (nnz.cpu() == -7).all()     # nothing launched
