"""Plain FP64 CPU oracle for split-and-merge dictionary learning.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline legs are the only callers.  The CUDA library never imports, links
or calls anything here, and nothing here imports the CUDA library.

The arithmetic lives in ``sdl_oracle.c`` (plain loops in double precision,
each routine citing the definition it writes out); this module only compiles
it with gcc and marshals numpy arrays through ctypes.  Arrays use the paper's
column-major convention with one signal / one atom contiguous, i.e. numpy
shape ``(N, m)`` for Y and ``(K, m)`` for D.

Readings of the paper fixed here (Sec. 1, 2, 3.1, Algorithm 1):
  * OMP: greedy atom with the largest |d_j^T r|, lowest index on ties,
    least squares on the support, stop at s atoms or ||r|| <= eps.
  * MOD: D = Y X^T (X X^T)^{-1} over the used atoms, unused atoms kept,
    columns renormalised.
  * Atom replacement (not in the paper; off unless min_use > 0): after the MOD
    update, atoms used by fewer than min_use signals become the worst-coded
    training signals, normalised.  Parity unpinned against the paper, which has
    no such step: its pins are hand-worked cases and the definition above.
  * Dictionary-conditioned proposer input (not in the paper): |D_t^T y| of each
    signal against its own subset's dictionary, the magnitudes OMP's first
    greedy step ranks.
  * Proposer training (not in the paper): binary cross-entropy of the MLP's
    logits against support labels, minimised by Adam (Kingma & Ba 2015,
    Algorithm 1: bias-corrected moment estimates, beta1 0.9, beta2 0.999).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile sdl_oracle.c into liborc.so next to it (gcc, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                          os.path.getmtime(os.path.join(_HERE, "sdl_oracle.h"))))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.orc_omp.argtypes = [_dp, i32, i32, _dp, i64, i32, dbl, _ip, _dp, _ip, _dp, _dp, i32]
            lib.orc_mod.argtypes = [_dp, i32, i64, _ip, _dp, i32, _dp, i32, i32, _dp, _ip,
                                    ctypes.POINTER(ctypes.c_int)]
            lib.orc_train.argtypes = [_dp, i32, i64, _dp, i32, i32, dbl, i32, i32, _dp, _dp, _ip,
                                      _dp, _ip, i32]
            lib.orc_split.argtypes = [_dp, i32, i64, _lp, _dp]
            lib.orc_local_train.argtypes = [_dp, i32, _lp, i32, _dp, i32, i32, dbl, i32, i32, _dp,
                                            _dp, i32]
            lib.orc_merge.argtypes = [_dp, _dp, i32, i32, i32, _ip, i32, i32, dbl, i32, i32, _dp,
                                      _dp, _dp, i32]
            lib.orc_replace_atoms.argtypes = [_dp, i32, i64, _ip, _dp, i32, _dp, i32, _ip,
                                              ctypes.POINTER(ctypes.c_int)]
            lib.orc_residual.argtypes = [_dp, i32, i64, _dp, i32, _ip, _dp, i32, _dp, _dp]
            lib.orc_recovery.argtypes = [_dp, i32, _dp, i32, i32, dbl, ctypes.POINTER(ctypes.c_int)]
            lib.orc_mlp_forward.argtypes = [_dp, i32, i32, i32, i32, _dp, i64, _dp]
            lib.orc_adam_step.argtypes = [_dp, _dp, _dp, _dp, i64, i32, dbl, dbl, dbl, dbl]
            lib.orc_mlp_loss_grad.argtypes = [_dp, i32, i32, i32, i32, _dp, _ip, i32, i64, _dp, _dp]
            lib.orc_extract_patches.argtypes = [_dp, i32, i32, i32, _dp]
            lib.orc_patch_average.argtypes = [_dp, i32, _ip, _dp, i32, i32, i32, i32, _dp]
            lib.orc_corr_features.argtypes = [_dp, i32, i32, _dp, _lp, i32, _dp]
            for f in ("orc_omp", "orc_mod", "orc_train", "orc_split", "orc_local_train",
                      "orc_merge", "orc_residual", "orc_recovery", "orc_mlp_forward",
                      "orc_mlp_loss_grad", "orc_extract_patches", "orc_patch_average",
                      "orc_replace_atoms", "orc_corr_features"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def _l(a):
    return a.ctypes.data_as(_lp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc == 1:
        raise OracleError(f"{what}: invalid argument")
    if rc not in (0, 2):
        raise OracleError(f"{what}: status {rc}")


def omp(D, Y, s, eps=0.0, nthreads=None):
    """OMP of every row of Y (shape (n, m)) against D (shape (K, m)).

    Returns dict(idx (n,s) int32, val (n,s) f64, nnz (n,), resid2 (n,), gap (n,s))."""
    lib = _load()
    D = _f64(D)
    K, m = D.shape
    Y = _f64(Y).reshape(-1, m)
    n = Y.shape[0]
    idx = np.empty((n, s), np.int32)
    val = np.empty((n, s), np.float64)
    nnz = np.empty((n,), np.int32)
    r2 = np.empty((n,), np.float64)
    gap = np.empty((n, s), np.float64)
    rc = lib.orc_omp(_d(D), m, K, _d(Y), n, s, float(eps), _i(idx), _d(val), _i(nnz), _d(r2),
                     _d(gap), nthreads or default_threads())
    _check(rc, "orc_omp")
    return dict(idx=idx, val=val, nnz=nnz, resid2=r2, gap=gap)


def mod(Y, idx, val, Dprev, normalise=True):
    """MOD update; returns (D (K,m), usage (K,), ridge_used, status)."""
    lib = _load()
    Y, Dprev = _f64(Y), _f64(Dprev)
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f64(val)
    n, m = Y.shape
    K = Dprev.shape[0]
    s = idx.shape[1]
    Dout = np.empty_like(Dprev)
    usage = np.empty((K,), np.int32)
    ridge = ctypes.c_int(0)
    rc = lib.orc_mod(_d(Y), m, n, _i(idx), _d(val), s, _d(Dprev), K, int(bool(normalise)),
                     _d(Dout), _i(usage), ctypes.byref(ridge))
    _check(rc, "orc_mod")
    return Dout, usage, bool(ridge.value), rc


def replace_atoms(Y, usage, resid2, min_use, D):
    """Atom replacement (not in the paper): atoms used by fewer than min_use
    signals become the worst-coded signals, normalised.  Returns (D (K,m), rep (K,), count)."""
    lib = _load()
    Y = _f64(Y)
    n, m = Y.shape
    D = _f64(D).copy()
    K = D.shape[0]
    usage = np.ascontiguousarray(usage, np.int32)
    resid2 = _f64(resid2)
    rep = np.empty((K,), np.int32)
    cnt = ctypes.c_int(0)
    _check(lib.orc_replace_atoms(_d(Y), m, n, _i(usage), _d(resid2), int(min_use), _d(D), K, _i(rep),
                                 ctypes.byref(cnt)), "orc_replace_atoms")
    return D, rep, cnt.value


def train(Y, D0, s, iters, eps=0.0, nthreads=None, min_use=0):
    """Standard alternating OMP/MOD training (min_use > 0: atom replacement after
    every MOD update); returns dict(D, rmse, xfro, idx, val, nnz, status)."""
    lib = _load()
    Y = _f64(Y)
    D = _f64(D0).copy()
    n, m = Y.shape
    K = D.shape[0]
    rmse = np.empty((iters,), np.float64)
    xf = ctypes.c_double(0.0)
    idx = np.empty((n, s), np.int32)
    val = np.empty((n, s), np.float64)
    nnz = np.empty((n,), np.int32)
    rc = lib.orc_train(_d(Y), m, n, _d(D), K, s, float(eps), iters, int(min_use), _d(rmse),
                       ctypes.cast(ctypes.byref(xf), _dp), _i(idx), _d(val), _i(nnz),
                       nthreads or default_threads())
    _check(rc, "orc_train")
    return dict(D=D, rmse=rmse, xfro=xf.value, idx=idx, val=val, nnz=nnz, status=rc)


def split(Y, perm):
    lib = _load()
    Y = _f64(Y)
    perm = np.ascontiguousarray(perm, np.int64)
    N, m = Y.shape
    out = np.empty_like(Y)
    _check(lib.orc_split(_d(Y), m, N, _l(perm), _d(out)), "orc_split")
    return out


def local_train(Y, offsets, Dloc0, s1, iters, eps=0.0, nthreads=None, min_use=0):
    """Algorithm 1 step 2 over every subset; returns dict(D (L,K1,m), xfro (L,), rmse (L,iters))."""
    lib = _load()
    Y = _f64(Y)
    offsets = np.ascontiguousarray(offsets, np.int64)
    D = _f64(Dloc0).copy()
    L, K1, m = D.shape
    xfro = np.empty((L,), np.float64)
    rmse = np.empty((L, iters), np.float64)
    rc = lib.orc_local_train(_d(Y), m, _l(offsets), L, _d(D), K1, s1, float(eps), iters,
                             int(min_use), _d(xfro), _d(rmse), nthreads or default_threads())
    _check(rc, "orc_local_train")
    return dict(D=D, xfro=xfro, rmse=rmse, status=rc)


def merge(Dloc, xfro, pick, K, s2, iters, eps=0.0, nthreads=None, min_use=0):
    """Algorithm 1 step 3; returns dict(D (K,m), rmse (iters,), Ytilde (K1 L, m))."""
    lib = _load()
    Dloc = _f64(Dloc)
    L, K1, m = Dloc.shape
    xfro = _f64(xfro)
    pick = np.ascontiguousarray(pick, np.int32)
    D = np.empty((K, m), np.float64)
    rmse = np.empty((iters,), np.float64)
    Yt = np.empty((K1 * L, m), np.float64)
    rc = lib.orc_merge(_d(Dloc), _d(xfro), m, K1, L, _i(pick), K, s2, float(eps), iters,
                       int(min_use), _d(D),
                       _d(rmse), _d(Yt), nthreads or default_threads())
    _check(rc, "orc_merge")
    return dict(D=D, rmse=rmse, Ytilde=Yt, status=rc)


def residual(Y, D, idx, val):
    """Returns (||Y - D X||_F^2, ||Y||_F^2)."""
    lib = _load()
    Y, D = _f64(Y), _f64(D)
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f64(val)
    n, m = Y.shape
    r2, y2 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.orc_residual(_d(Y), m, n, _d(D), D.shape[0], _i(idx), _d(val), idx.shape[1],
                            ctypes.cast(ctypes.byref(r2), _dp), ctypes.cast(ctypes.byref(y2), _dp)),
           "orc_residual")
    return r2.value, y2.value


def recovery(D0, D, thresh=0.98):
    """Number of atoms of D0 recovered by D (Sec. 3.1 criterion)."""
    lib = _load()
    D0, D = _f64(D0), _f64(D)
    c = ctypes.c_int(0)
    _check(lib.orc_recovery(_d(D0), D0.shape[0], _d(D), D.shape[0], D.shape[1], float(thresh),
                            ctypes.byref(c)), "orc_recovery")
    return c.value


def corr_features(D, offsets, Y):
    """|d_(t,j)^T y_i| of every row i of Y against the dictionary D[t] (D: (L, K, m))
    of its subset (rows offsets[t] .. offsets[t+1]-1): shape (n, K)."""
    lib = _load()
    D, Y = _f64(D), _f64(Y)
    L, K, m = D.shape
    off = np.ascontiguousarray(offsets, np.int64)
    F = np.empty((Y.shape[0], K))
    _check(lib.orc_corr_features(_d(D), m, K, _d(Y), _l(off), L, _d(F)), "orc_corr_features")
    return F


def mlp_sizes(m, h1, h2, K):
    """Offsets of W1, b1, W2, b2, W3, b3 in the packed proposer parameters."""
    sizes = [h1 * m, h1, h2 * h1, h2, K * h2, K]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    return offs


def mlp_forward(params, m, h1, h2, K, Y):
    """Logits z (B, K) of the proposer MLP."""
    lib = _load()
    params, Y = _f64(params), _f64(Y).reshape(-1, m)
    Z = np.empty((Y.shape[0], K))
    _check(lib.orc_mlp_forward(_d(params), m, h1, h2, K, _d(Y), Y.shape[0], _d(Z)), "orc_mlp_forward")
    return Z


def mlp_loss_grad(params, m, h1, h2, K, Y, idx, with_grad=True):
    """(loss, grad) of the proposer's binary cross-entropy on support labels."""
    lib = _load()
    params, Y = _f64(params), _f64(Y).reshape(-1, m)
    idx = np.ascontiguousarray(idx, np.int32)
    loss = ctypes.c_double(0.0)
    grad = np.empty_like(params) if with_grad else None
    _check(lib.orc_mlp_loss_grad(_d(params), m, h1, h2, K, _d(Y), _i(idx), idx.shape[1], Y.shape[0],
                                 ctypes.cast(ctypes.byref(loss), _dp), _d(grad)), "orc_mlp_loss_grad")
    return loss.value, grad


def adam_step(theta, g, m, v, t, alpha, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1); returns new (theta, m, v)."""
    lib = _load()
    theta, g = _f64(theta).copy(), _f64(g)
    m, v = _f64(m).copy(), _f64(v).copy()
    n = theta.size
    assert g.size == n and m.size == n and v.size == n
    _check(lib.orc_adam_step(_d(theta), _d(g), _d(m), _d(v), n, int(t), float(alpha), float(beta1), float(beta2),
                             float(eps)), "orc_adam_step")
    return theta, m, v


def extract_patches(img, p):
    """Every p x p patch of img (H, W), row-major: shape ((H-p+1)(W-p+1), p*p)."""
    lib = _load()
    img = _f64(img)
    H, W = img.shape
    out = np.empty(((H - p + 1) * (W - p + 1), p * p))
    _check(lib.orc_extract_patches(_d(img), H, W, p, _d(out)), "orc_extract_patches")
    return out


def patch_average(D, idx, val, H, W, p):
    """Denoised image (H, W): per pixel, the mean of D x over the patches covering it."""
    lib = _load()
    D = _f64(D)
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f64(val)
    out = np.empty((H, W))
    _check(lib.orc_patch_average(_d(D), D.shape[0], _i(idx), _d(val), idx.shape[1], H, W, p, _d(out)),
           "orc_patch_average")
    return out
