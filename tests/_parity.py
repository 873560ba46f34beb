"""Element-by-element comparison of GPU OMP codes with the oracle's.

Greedy OMP is discontinuous in its inputs: where two atoms tie for the largest
|d_j^T r| (to within rounding) either choice is a correct execution of the
definition.  So a signal's support must equal the oracle's unless, at the
first step where they differ, the oracle's top-two gap is below `gap_tol`;
such a signal is then checked for validity on its own support (coefficients
are the least-squares fit, the reported residual is that fit's residual).
"""
from __future__ import annotations

import numpy as np


def fp32_gap_tol(m: int, ynorm: np.ndarray) -> np.ndarray:
    """Rounding bound for a correlation computed in FP32: the forward error of an
    m-term dot product of unit-norm d_j with y is at most gamma_m ||y||,
    gamma_m = m u / (1 - m u), u = 2^-24; two correlations must move for their
    order to flip, so ties closer than 2 gamma_m ||y|| are undecidable in FP32."""
    u = 2.0 ** -24
    gm = m * u / (1 - m * u)
    return np.maximum(1e-6, 2 * gm * ynorm)


def compare_codes(D, Y, gpu_idx, gpu_val, gpu_nnz, gpu_r2, orc, gap_tol, coef_rtol, r2_rtol=None, eps=None):
    """Returns a dict of counts; raises AssertionError on a real mismatch.

    D (K, m) and Y (n, m) are float64 numpy arrays of the inputs both sides saw.
    gap_tol: scalar or per-signal array.  eps: the error-constrained stop, if
    any; a code that agrees with the oracle's on their common prefix but stops
    at another length is then a near-tie on the stop itself when the prefix's
    least-squares residual norm is eps to within 1e-4 eps."""
    n, s = gpu_idx.shape
    gap_tol = np.broadcast_to(np.asarray(gap_tol, dtype=np.float64), (n,))
    r2_rtol = coef_rtol if r2_rtol is None else r2_rtol
    same = (gpu_idx == orc["idx"]).all(axis=1) & (gpu_nnz == orc["nnz"])
    stats = dict(n=n, same=int(same.sum()), excused=0)
    # identical supports: coefficients and residual energies
    if same.any():
        xo, xg = orc["val"][same], gpu_val[same].astype(np.float64)
        scale = np.maximum(np.abs(xo), 1e-2 * np.abs(xo).max(axis=1, keepdims=True))
        scale = np.where(scale > 0, scale, 1.0)
        rel = np.abs(xg - xo) / scale
        worst = np.unravel_index(np.argmax(rel), rel.shape)
        assert rel.max() <= coef_rtol, (
            f"coefficient rel err {rel.max():.3e} > {coef_rtol} at {worst}: gpu {xg[worst]} orc {xo[worst]}")
        ro, rg = orc["resid2"][same], gpu_r2[same].astype(np.float64)
        yn2 = (Y[same] ** 2).sum(axis=1)
        err = np.abs(rg - ro) / np.maximum(ro, 1e-6 * yn2 + 1e-300)
        assert err.max() <= max(r2_rtol, 1e-4) * 10, f"resid2 rel err {err.max():.3e}"
        stats["coef_rel_max"] = float(rel.max())
    # differing supports: must be a near-tie in the oracle, and valid on its own
    for i in np.nonzero(~same)[0]:
        gi, oi = gpu_idx[i], orc["idx"][i]
        kmin = int(min(gpu_nnz[i], orc["nnz"][i]))
        if eps is not None and gpu_nnz[i] != orc["nnz"][i] and (gi[:kmin] == oi[:kmin]).all():
            S = gi[:kmin]
            if len(S):
                x, *_ = np.linalg.lstsq(D[S].T, Y[i], rcond=None)
                rk = np.linalg.norm(Y[i] - D[S].T @ x)
            else:
                rk = np.linalg.norm(Y[i])
            assert abs(rk - eps) <= 1e-4 * eps, (
                f"signal {i}: stops at {gpu_nnz[i]} (oracle {orc['nnz'][i]}) with ||r|| {rk:.8e} vs eps {eps:.8e}")
            stats["excused"] += 1
            continue
        k = int(np.argmax(gi != oi)) if (gi != oi).any() else kmin
        g = orc["gap"][i][k] if k < s else np.inf
        assert g < gap_tol[i], (
            f"signal {i}: support differs at step {k} (gpu {gi.tolist()} orc {oi.tolist()}) "
            f"but the oracle gap there is {g:.3e} >= {gap_tol[i]:.3e}")
        S = gi[: gpu_nnz[i]]
        assert len(set(S.tolist())) == len(S) and (gi[gpu_nnz[i]:] == -1).all()
        if len(S):
            x, *_ = np.linalg.lstsq(D[S].T, Y[i], rcond=None)
            xg = gpu_val[i][: len(S)].astype(np.float64)
            assert np.abs(xg - x).max() <= 10 * coef_rtol * max(1.0, np.abs(x).max()), (i, xg, x)
        stats["excused"] += 1
    return stats


def check_bf16_codes(D, Y, idx, val, nnz, r2, orc, coef_rtol=2e-2):
    D64, Y64 = D.astype(np.float64), Y.astype(np.float64)
    n, s = idx.shape
    tol = 2 * 2.0 ** -8 * (np.linalg.norm(Y64, axis=1) + 2 * np.abs(orc["val"]).sum(axis=1))
    excused = 0
    for i in range(n):
        k = int(nnz[i])
        S = idx[i, :k]
        assert len(set(S.tolist())) == k and (idx[i, k:] == -1).all()
        if k:
            x, *_ = np.linalg.lstsq(D64[S].T, Y64[i], rcond=None)
            scale = max(np.abs(x).max(), 1e-12)
            assert np.abs(val[i, :k] - x).max() <= coef_rtol * scale, (i, val[i, :k], x)
            res = Y64[i] - D64[S].T @ x
            assert abs(r2[i] - res @ res) <= 1e-3 * (Y64[i] @ Y64[i]) + 1e-6
        if not ((idx[i] == orc["idx"][i]).all() and nnz[i] == orc["nnz"][i]):
            diff = np.nonzero(idx[i] != orc["idx"][i])[0]
            step = int(diff[0]) if len(diff) else min(int(nnz[i]), int(orc["nnz"][i]))
            g = orc["gap"][i][step] if step < s else np.inf
            assert g < tol[i], (i, step, g, tol[i], idx[i], orc["idx"][i])
            excused += 1
    return excused
