"""Element-by-element comparison of GPU OMP codes with the oracle's.

Greedy OMP is discontinuous in its inputs: where two atoms tie for the largest
|d_j^T r| (to within rounding) either choice is a correct execution of the
definition.  So a signal's support must equal the oracle's unless, at the
first step k where they differ, both hold:
  (a) the oracle's top-two gap there is below the path's rounding bound;
  (b) the GPU's atom g was near-maximal under the oracle's residual r_k (the
      least-squares residual of y on the common prefix, recomputed here in
      FP64): max_j |d_j^T r_k| - |d_g^T r_k| is within that bound too.
Such a signal is then checked for validity on its own support (coefficients
are the least-squares fit, the reported residual is that fit's residual), and
a test caps how many signals may be excused this way.  Differences at a
rounding-level step, where even the oracle's largest correlation is within the
bound (the prefix already fits y to rounding, as when a signal is itself an
atom of the dictionary, or what is left is noise below the path's
resolution), are counted apart and not capped: there every atom is a correct
choice at that precision.

Rounding bounds.  A correlation the GPU forms at step k is
alpha0_j - g_j^T G_SS^-1 alpha0_S (Batch-OMP, Sec. 1 greedy choice): with
alpha0 = D^T y off by delta, the compared value is off by
delta_j - w_j^T delta_S, w_j = G_SS^-1 D_S^T d_j the coefficients of d_j on the
prefix atoms.  |delta_j| <= e sum_i |d_ji y_i| with e = gamma_m for FP32
products (u = 2^-24), e = 2u_b + u_b^2 + gamma_m for BF16 operands
(round to nearest, u_b = 2^-9, exact products, FP32 accumulation), and
e = 3 2^-22 + gamma_m(2^-23) for the two-term TF32 split (x = hi + lo, three
products, FP32 accumulation whose rounding the tensor cores do not document:
one unit 2^-23 per addition instead of half).
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
UB16 = 2.0 ** -9


def gamma(m: int, u: float = U32) -> float:
    return m * u / (1 - m * u)


def fp32_gap_tol(m: int, ynorm: np.ndarray) -> np.ndarray:
    """Rounding bound for a correlation computed in FP32: the forward error of an
    m-term dot product of unit-norm d_j with y is at most gamma_m ||y||,
    gamma_m = m u / (1 - m u), u = 2^-24; two correlations must move for their
    order to flip, so ties closer than 2 gamma_m ||y|| are undecidable in FP32."""
    return np.maximum(1e-6, 2 * gamma(m) * ynorm)


def x3_unit(m: int) -> float:
    """Relative error bound of a correlation from the two-term TF32 split: each
    operand is hi + lo to within 2^-22 (hi = tf32(x) keeps 11 significant bits,
    lo = tf32(x - hi) 11 more), the dropped lo lo term is below 2^-22 of the
    product, so each of the m products is within 3 2^-22 of x_i z_i; the FP32
    accumulation adds gamma_m with a unit of 2^-23."""
    return 3 * 2.0 ** -22 + gamma(m, 2.0 ** -23)


def x3_gap_tol(m: int, ynorm: np.ndarray) -> np.ndarray:
    """The FP32 gap rule with the TF32-split bound: ties closer than
    2 e ||y|| (e = x3_unit(m)) are undecidable on that path."""
    return np.maximum(1e-6, 2 * x3_unit(m) * ynorm)


def tf32_unit(m: int) -> float:
    """Relative error bound of one TF32-operand correlation term sum: each
    operand rounded to nearest with 11 significant bits (unit 2^-11), the
    product of the two exact, the FP32 accumulation of the tensor cores with a
    unit of 2^-23 per addition (their rounding of the sum is not documented)."""
    u = 2.0 ** -11
    return 2 * u + u * u + gamma(m, 2.0 ** -23) * (1 + 2 * u)


def bf16_unit(m: int) -> float:
    """Relative error bound of one BF16-operand correlation term sum."""
    return 2 * UB16 + UB16 ** 2 + gamma(m) * (1 + 2 * UB16)


def step_correlations(D, y, S):
    """|d_j^T r| of every atom, r the FP64 least-squares residual of y on the
    atoms S (selected atoms masked to -inf), the coefficients W (|S| x K) of
    every atom on D_S, and r."""
    if len(S):
        B = D[S].T
        x, *_ = np.linalg.lstsq(B, y, rcond=None)
        r = y - B @ x
        W, *_ = np.linalg.lstsq(B, D.T, rcond=None)
    else:
        r, W = y, np.zeros((0, D.shape[0]))
    c = np.abs(D @ r)
    c[list(S)] = -np.inf
    return c, W, r


U16 = 2.0 ** -11


def corr_error_bound(D, y, S, W, e, r=None, h16=False):
    """Per-atom bound on the error of the correlation the GPU compares at a
    step with prefix S.  Running correlations (Batch-OMP): e (a_j + |w_j|^T a_S),
    a_j = sum_i |d_ji y_i|; with h16 the running update reads a half-precision
    copy of G (round to nearest, u = 2^-11 per entry), which adds
    u sum_p |G_jp x_p|, x the prefix's coefficients.  Recomputed from the
    residual (r given): e b_j, b_j = sum_i |d_ji r_i|."""
    if r is not None:
        return e * (np.abs(D) @ np.abs(r))
    a = np.abs(D) @ np.abs(y)
    E = e * (a + (np.abs(W).T @ a[list(S)] if len(S) else 0.0))
    if h16 and len(S):
        x, *_ = np.linalg.lstsq(D[list(S)].T, y, rcond=None)
        E = E + U16 * (np.abs(D @ D[list(S)].T) @ np.abs(x))
    return E


def _first_difference(gi, gn, oi, on):
    k = int(np.argmax(gi != oi)) if (gi != oi).any() else int(min(gn, on))
    g = int(gi[k]) if k < len(gi) and k < gn else -1
    o = int(oi[k]) if k < len(oi) and k < on else -1
    return k, g, o


def _near_tie(D, y, gi, gn, oi, on, orc_gap_k, tol_a, tol_b, e, residual=False, h16=False):
    """Checks (a) with tolerance tol_a(E, o, g) and (b) with tol_b(E, o, g) at
    the first differing step (E: the per-atom bound there, of the residual form
    when `residual`); returns whether that step is at rounding level (the
    largest correlation within tol_b)."""
    k, g, o = _first_difference(gi, gn, oi, on)
    S = [int(v) for v in gi[:k]]
    c, W, r = step_correlations(D, y, S)
    E = corr_error_bound(D, y, S, W, e, r if residual else None, h16=h16 and not residual)
    if o >= 0 and g >= 0:
        assert orc_gap_k < tol_a(E, o, g), (
            f"support differs at step {k} (gpu {gi.tolist()} orc {oi.tolist()}) but the oracle gap there is "
            f"{orc_gap_k:.3e} >= {tol_a(E, o, g):.3e}")
        lag = c[o] - c[g]
        assert lag <= tol_b(E, o, g), (
            f"step {k}: the GPU's atom {g} trails the oracle's {o} by {lag:.3e} under the oracle's residual, "
            f"beyond the rounding bound {tol_b(E, o, g):.3e} (gpu {gi.tolist()} orc {oi.tolist()})")
        return bool(c[o] <= tol_b(E, o, o))
    else:
        # one side stopped where the other went on: the atom it went on with
        # must have a correlation within rounding of zero, or (the GPU having
        # stopped) the prefix fits y to FP32 rounding, or that atom is
        # dependent on the support to within the FP32 pivot rule
        # (squared distance to span(D_S) at most 1e-6 of its squared norm; the
        # FP64 oracle's rule is 1e-10), checked here with a 4x margin
        j = o if o >= 0 else g
        assert j >= 0
        if c[j] <= tol_b(E, j, j):
            return True
        # the prefix already fits y to FP32 rounding: the path's own residual
        # may be exactly zero, which leaves no atom with |d^T r| > 0
        if o >= 0 and np.linalg.norm(r) <= 2 * gamma(len(y)) * np.linalg.norm(y):
            return True
        if o >= 0 and len(S):
            dj = D[j]
            resid = dj - D[S].T @ W[:, j]
            assert resid @ resid <= 4e-6 * (dj @ dj), (
                f"step {k}: the GPU stops (gpu {gi.tolist()} orc {oi.tolist()}) while atom {j} still has "
                f"|d^T r| = {c[j]:.3e} and relative pivot {resid @ resid / (dj @ dj):.3e}")
            return True
        raise AssertionError(f"step {k}: one side stops (gpu {gi.tolist()} orc {oi.tolist()}) while atom {j} still "
                             f"has |d^T r| = {c[j]:.3e}")


def compare_codes(D, Y, gpu_idx, gpu_val, gpu_nnz, gpu_r2, orc, gap_tol, coef_rtol, r2_rtol=None, eps=None,
                  max_excused=0.002, e=None):
    """Returns a dict of counts; raises AssertionError on a real mismatch.

    D (K, m) and Y (n, m) are float64 numpy arrays of the inputs both sides saw.
    gap_tol: scalar or per-signal array (the FP32 rule of fp32_gap_tol, or the
    stated 1e-6 on FP64).  eps: the error-constrained stop, if any; a code that
    agrees with the oracle's on their common prefix but stops at another length
    is then a near-tie on the stop itself when the prefix's least-squares
    residual norm is eps to within 1e-4 eps.  At most max_excused of the
    signals may be excused near-ties (stop near-ties and rounding-level steps
    are counted apart, as excused_eps and excused_rounding).  e: the relative
    bound of one correlation on the path (gamma_m for FP32 products, the
    default; x3_unit for the TF32 split)."""
    n, s = gpu_idx.shape
    m = D.shape[1]
    gap_tol = np.broadcast_to(np.asarray(gap_tol, dtype=np.float64), (n,))
    r2_rtol = coef_rtol if r2_rtol is None else r2_rtol
    same = (gpu_idx == orc["idx"]).all(axis=1) & (gpu_nnz == orc["nnz"])
    stats = dict(n=n, same=int(same.sum()), excused=0, excused_eps=0, excused_rounding=0)
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
    # differing supports: a near-tie in the oracle at which the GPU's atom was
    # near-maximal, and a valid code on its own support
    e32 = gamma(m) if e is None else e
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
            stats["excused_eps"] += 1
            continue
        k, _, _ = _first_difference(gi, gpu_nnz[i], oi, orc["nnz"][i])
        gk = orc["gap"][i][k] if k < s else np.inf
        # (a) with the gap rule as given; (b) with it widened by the
        # running-correlation term where that is larger
        t = gap_tol[i]
        rounding = _near_tie(D, Y[i], gi, int(gpu_nnz[i]), oi, int(orc["nnz"][i]), gk, lambda E, o, g: t,
                             lambda E, o, g: 2.0 * max(t, E[o] + E[g]), e32)
        S = gi[: gpu_nnz[i]]
        assert len(set(S.tolist())) == len(S) and (gi[gpu_nnz[i]:] == -1).all()
        if len(S):
            x, *_ = np.linalg.lstsq(D[S].T, Y[i], rcond=None)
            xg = gpu_val[i][: len(S)].astype(np.float64)
            assert np.abs(xg - x).max() <= 10 * coef_rtol * max(1.0, np.abs(x).max()), (i, xg, x)
        stats["excused_rounding" if rounding else "excused"] += 1
    assert stats["excused"] + stats["excused_eps"] <= max(2, max_excused * n), (
        f"{stats['excused']} + {stats['excused_eps']} (stop) of {n} signals differ at near-ties, above the cap "
        f"{max_excused:.2%} ({stats['excused_rounding']} more at rounding-level steps)")
    return stats


def check_bf16_codes(D, Y, idx, val, nnz, r2, orc, coef_rtol=2e-2, max_excused=0.05, residual=False, eps=None,
                     h16=False, unit=None):
    """BF16-operand correlations (tcgen05) with FP32 refits: every code is valid
    on its own support (exact least squares within coef_rtol, the reported
    residual that fit's); a support may differ from the oracle's only at a step
    where the oracle's top-two gap and the GPU atom's lag are both within
    1.25 (E_o + E_g), the BF16 bound of the module docstring (the factor covers
    the FP32 Gram and solve, about 2^-16 against 2^-8); at most max_excused of
    the signals may differ at steps that are not at rounding level.
    residual: the path recomputed D^T r from the BF16-rounded residual at every
    step, so E is the residual form's bound e sum_i |d_ji r_i| (tighter as the
    residual shrinks).  h16: the Batch-OMP form's running update read a
    half-precision copy of the Gram (form 3), whose rounding adds
    2^-11 sum_p |G_jp x_p| to E.  eps: the error-constrained stop; a code that agrees
    with the oracle's on their common prefix but stops at another length is a
    near-tie on the stop itself when the prefix's least-squares residual norm
    is eps to within 1e-4 eps (counted with the rounding-level ones).  unit:
    the per-term bound e in place of the BF16 one (tf32_unit for one TF32
    product).  Returns (signals that differ there, signals that differ at
    rounding-level steps or at the stop)."""
    D64, Y64 = D.astype(np.float64), Y.astype(np.float64)
    n, s = idx.shape
    e16 = bf16_unit(D.shape[1]) if unit is None else unit
    excused = rounding = 0
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
            kmin = min(k, int(orc["nnz"][i]))
            if eps is not None and k != orc["nnz"][i] and (idx[i, :kmin] == orc["idx"][i, :kmin]).all():
                P = idx[i, :kmin]
                if kmin:
                    xp, *_ = np.linalg.lstsq(D64[P].T, Y64[i], rcond=None)
                    rk = np.linalg.norm(Y64[i] - D64[P].T @ xp)
                else:
                    rk = np.linalg.norm(Y64[i])
                assert abs(rk - eps) <= 1e-4 * eps, (i, k, orc["nnz"][i], rk, eps)
                rounding += 1
                continue
            kk, _, _ = _first_difference(idx[i], k, orc["idx"][i], int(orc["nnz"][i]))
            gk = orc["gap"][i][kk] if kk < s else np.inf
            tol = lambda E, o, g: 1.25 * (E[o] + E[g])  # noqa: E731
            if _near_tie(D64, Y64[i], idx[i], k, orc["idx"][i], int(orc["nnz"][i]), gk, tol, tol, e16, residual,
                         h16):
                rounding += 1
            else:
                excused += 1
    assert excused <= max(2, max_excused * n), (
        f"{excused} of {n} supports differ at near-ties, above the cap {max_excused:.2%} "
        f"({rounding} more at rounding-level steps)")
    return excused, rounding


def check_rmse(r2_gpu, orc, idx, nnz, m, rmse_gpu=None, rtol=1e-3):
    """The coding pass's RMSE against the oracle's, signal by signal.  A signal
    whose support differs from the oracle's at a validated near-tie (checked by
    compare_codes / check_bf16_codes) may legitimately end at another residual:
    greedy OMP from another first pick follows another path.  So the RMSE over
    the signals whose codes equal the oracle's must be within rtol of the
    oracle's over the same signals, and the RMSE the GPU reports (rmse_gpu, if
    given) must be that of its own residual energies r2_gpu.  Returns the
    relative RMSE difference over all signals (for the printout)."""
    r2g = np.asarray(r2_gpu, dtype=np.float64)
    r2o = np.asarray(orc["resid2"], dtype=np.float64)
    n = len(r2g)
    same = (idx == orc["idx"]).all(axis=1) & (nnz == orc["nnz"])
    if same.any():
        a, b = np.sqrt(r2g[same].sum() / (m * same.sum())), np.sqrt(r2o[same].sum() / (m * same.sum()))
        assert abs(a - b) <= rtol * b, (a, b, int(same.sum()), n)
    full_g, full_o = np.sqrt(r2g.sum() / (m * n)), np.sqrt(r2o.sum() / (m * n))
    if rmse_gpu is not None:
        assert abs(rmse_gpu - full_g) <= 1e-5 * full_g + 1e-12, (rmse_gpu, full_g)
    return (full_g - full_o) / full_o
