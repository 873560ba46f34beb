"""GB300 (sm_103a) split-and-merge dictionary learning: Python binding.

The arithmetic lives in ``libsdl_gb300.so`` (hand-written CUDA kernels behind
the C ABI of ``include/sdl.h``).  This module only marshals arguments: it
loads the library with ctypes, exposes each C entry point under its own name
(``sdl_omp``, ``sdl_mod_update``, ``sdl_local_train``, ``sdl_merge``, ...) and
adds small helpers that take torch CUDA tensors, allocate outputs with torch
and pass ``data_ptr()`` plus the current CUDA stream.  There is no CPU
fallback: if the library or a GPU is missing, calls raise.

Layout (Sec. 2 notation): Y in R^{m x N} is a tensor of shape (N, m); D in
R^{m x K} is shape (K, m); codes are ELL tensors idx (N, s) int32, val (N, s).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import _build

__all__ = [
    "PREC_F64", "PREC_F32", "PREC_BF16", "PREC_F32X3", "PREC_TF32", "SdlError", "lib", "library_path", "declared_symbols",
    "Context", "context", "omp", "omp_batched", "mod_update", "mod_update_batched", "split",
    "init_dict", "local_train", "merge", "residual", "recovery", "Proposer",
]

PREC_F64, PREC_F32, PREC_BF16, PREC_F32X3, PREC_TF32 = 0, 1, 2, 3, 4
_STATUS = {0: "SDL_OK", 1: "SDL_EINVAL", 2: "SDL_ENOTPD", 3: "SDL_ETIMEOUT", 4: "SDL_ECUDA",
           5: "SDL_ENOMEM", 6: "SDL_ERANGE"}

_lock = threading.Lock()
_lib = None


class SdlError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def declared_symbols() -> list[str]:
    """Function names declared in include/sdl.h."""
    with open(os.path.join(_build.INCLUDE, "sdl.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(sdl_[a-z0-9_]+)\s*\(", text)))


_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "sdl_create": (_i32, [ctypes.POINTER(_vp), _i32, _vp]),
    "sdl_destroy": (_i32, [_vp]),
    "sdl_set_stream": (_i32, [_vp, _vp]),
    "sdl_last_error": (ctypes.c_char_p, [_vp]),
    "sdl_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "sdl_omp": (_i32, [_vp, _i32, _vp, _i32, _i32, _vp, _i64, _i32, _dbl, _vp, _vp, _vp, _vp]),
    "sdl_omp_batched": (_i32, [_vp, _i32, _vp, _i32, _i32, _vp, _vp, _i32, _i32, _dbl, _vp, _vp, _vp,
                               _vp]),
    "sdl_mod_update": (_i32, [_vp, _i32, _vp, _i32, _i64, _vp, _vp, _i32, _vp, _i32, _vp]),
    "sdl_mod_update_batched": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _vp, _vp, _i32, _vp, _i32, _vp]),
    "sdl_replace_atoms": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _vp, _vp, _i32, _vp, _i32, _vp]),
    "sdl_split": (_i32, [_vp, _i32, _vp, _i32, _i64, _vp, _vp]),
    "sdl_init_dict": (_i32, [_vp, _i32, _vp, _i32, _i64, _vp, _vp, _i64, _vp]),
    "sdl_local_train": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _i32, _i32, _dbl, _i32, _vp, _vp, _vp]),
    "sdl_merge": (_i32, [_vp, _i32, _vp, _vp, _i32, _i32, _i32, _vp, _i32, _i32, _dbl, _i32, _vp, _vp]),
    "sdl_residual": (_i32, [_vp, _i32, _vp, _i32, _i64, _vp, _i32, _vp, _vp, _i32, _vp]),
    "sdl_recovery": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _i32, _dbl, _vp]),
    "sdl_gram": (_i32, [_vp, _i32, _vp, _i32, _i32, _i32, _vp]),
    "sdl_profile_enable": (_i32, [_vp, _i32]),
    "sdl_profile_reset": (_i32, [_vp]),
    "sdl_profile_count": (_i32, [_vp]),
    "sdl_profile_entry": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_i64),
                                 ctypes.POINTER(_i64), ctypes.POINTER(_dbl)]),
    "sdl_launch_count": (_i64, [_vp]),
    "sdl_omp_noalloc": (_i32, [_vp, _vp, _i32, _i32, _vp, _i64, _i32, _dbl, _vp, _vp, _vp, _vp]),
    "sdl_extract_patches": (_i32, [_vp, _i32, _vp, _i32, _i32, _i32, _vp]),
    "sdl_patch_average": (_i32, [_vp, _i32, _vp, _i32, _vp, _vp, _i32, _i32, _i32, _i32, _vp]),
    "sdl_sq_error": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp]),
    "sdl_set_option": (_i32, [_vp, _i32, _i64]),
    "sdl_proposer_create": (_i32, [_vp, _i32, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "sdl_proposer_destroy": (_i32, [_vp]),
    "sdl_proposer_get_params": (_i32, [_vp, _vp, _vp]),
    "sdl_proposer_loss_grad": (_i32, [_vp, _vp, _vp, _vp, _i32, _i64, _vp, _vp]),
    "sdl_proposer_train_step": (_i32, [_vp, _vp, _vp, _vp, _i32, _i64, ctypes.c_float, _vp]),
    "sdl_proposer_scores": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "sdl_omp_proposed": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _i64, _i32, _i32, _dbl, _vp, _vp, _vp, _vp,
                                ctypes.POINTER(_i64)]),
    "sdl_corr_features": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _i32, _vp]),
    "sdl_omp_proposed_batched": (_i32, [_vp, _vp, _i32, _vp, _i32, _i32, _vp, _vp, _i32, _i32, _i32, _dbl, _vp, _vp,
                                        _vp, _vp, ctypes.POINTER(_i64)]),
}
FEATURES_SIGNAL, FEATURES_CORR = 0, 1
OPT_MOD_SOLVE, OPT_CLUSTER, OPT_MOD_TILE, OPT_AUTOTUNE, OPT_GRAPH, OPT_SM_BLOCKS, OPT_REPLACE = 1, 2, 3, 4, 5, 6, 7
OPT_OMP_FORM = 8
OPT_BF16_FORM = 9
OPT_WAIT_LIMIT, OPT_WAIT_TEST = 10, 11
OPT_MOD_MIXED, OPT_MOD_CHECK_TOL, OPT_A0_CHUNK_MB = 12, 13, 14
OPT_SEL_SPW, OPT_SEL_GCACHE = 15, 16


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _call(name: str, ctx_handle, *args):
    rc = getattr(lib(), name)(ctx_handle, *args)
    if rc != 0:
        msg = lib().sdl_last_error(ctx_handle)
        raise SdlError(rc, name, msg.decode() if msg else "")


# ------------------------------------------------------------------ contexts --
class Context:
    """An ``sdl_ctx`` bound to one device; each call enqueues on torch's current stream."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1403_4781_gb300 needs a CUDA device (no CPU fallback)")
        self.device = device
        h = _vp()
        stream = torch.cuda.current_stream(device).cuda_stream
        rc = lib().sdl_create(ctypes.byref(h), device, stream)
        if rc != 0:
            raise SdlError(rc, "sdl_create", "cannot create a context")
        self.handle = h

    def bind_stream(self):
        import torch
        lib().sdl_set_stream(self.handle, torch.cuda.current_stream(self.device).cuda_stream)
        return self.handle

    def profile(self, on: bool = True):
        lib().sdl_profile_enable(self.handle, int(bool(on)))

    def profile_reset(self):
        lib().sdl_profile_reset(self.handle)

    def profile_read(self) -> dict:
        """{kernel name: (kernels launched, launcher calls, total ms)}; synchronises."""
        out = {}
        for i in range(lib().sdl_profile_count(self.handle)):
            name, nl, nc, ms = ctypes.c_char_p(), _i64(), _i64(), _dbl()
            _call("sdl_profile_entry", self.handle, i, ctypes.byref(name), ctypes.byref(nl),
                  ctypes.byref(nc), ctypes.byref(ms))
            out[name.value.decode()] = (int(nl.value), int(nc.value), float(ms.value))
        return out

    def set_option(self, option: int, value: int):
        _call("sdl_set_option", self.handle, option, value)

    def launch_count(self) -> int:
        return int(lib().sdl_launch_count(self.handle))

    def workspace_bytes(self) -> int:
        return int(lib().sdl_workspace_bytes(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().sdl_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts: dict[int, Context] = {}


def context(device: int | None = None) -> Context:
    import torch
    dev = torch.cuda.current_device() if device is None else device
    if dev not in _contexts:
        _contexts[dev] = Context(dev)
    return _contexts[dev]


# ------------------------------------------------------------ marshalling ----
def _prec_of(t, prec):
    import torch
    if prec is None:
        return PREC_F64 if t.dtype == torch.float64 else PREC_F32
    return prec


def _dtype_of(prec):
    import torch
    return torch.float64 if prec == PREC_F64 else torch.float32


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr()


def _offsets_host(offsets):
    import numpy as np
    o = np.ascontiguousarray(np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets,
                                        dtype=np.int64))
    return o, o.ctypes.data_as(_vp)


def omp(D, Y, s, eps=0.0, prec=None, with_resid=True):
    """OMP (Sec. 1, 3.2.2) of every row of Y (n, m) against D (K, m).
    Returns (idx (n,s) int32, val (n,s), nnz (n,) int32, resid2 (n,) or None)."""
    import torch
    prec = _prec_of(D, prec)
    K, m = D.shape
    n = Y.shape[0]
    dev = D.device
    idx = torch.empty((n, s), dtype=torch.int32, device=dev)
    val = torch.empty((n, s), dtype=_dtype_of(prec), device=dev)
    nnz = torch.empty((n,), dtype=torch.int32, device=dev)
    r2 = torch.empty((n,), dtype=_dtype_of(prec), device=dev) if with_resid else None
    ctx = context(dev.index)
    _call("sdl_omp", ctx.bind_stream(), prec, _ptr(D), m, K, _ptr(Y), n, s, float(eps), _ptr(idx),
          _ptr(val), _ptr(nnz), _ptr(r2))
    return idx, val, nnz, r2


def omp_batched(D, Y, offsets, s, eps=0.0, prec=None, with_resid=True):
    """Batched OMP: rows offsets[t]..offsets[t+1] of Y coded against D[t] (D: (L, K, m))."""
    import torch
    prec = _prec_of(D, prec)
    L, K, m = D.shape
    n = Y.shape[0]
    dev = D.device
    oh, op = _offsets_host(offsets)
    assert len(oh) == L + 1 and oh[-1] == n
    idx = torch.empty((n, s), dtype=torch.int32, device=dev)
    val = torch.empty((n, s), dtype=_dtype_of(prec), device=dev)
    nnz = torch.empty((n,), dtype=torch.int32, device=dev)
    r2 = torch.empty((n,), dtype=_dtype_of(prec), device=dev) if with_resid else None
    ctx = context(dev.index)
    _call("sdl_omp_batched", ctx.bind_stream(), prec, _ptr(D), m, K, _ptr(Y), op, L, s, float(eps),
          _ptr(idx), _ptr(val), _ptr(nnz), _ptr(r2))
    return idx, val, nnz, r2


def mod_update(Y, idx, val, D, prec=None):
    """MOD update (Sec. 1) in place on D (K, m); returns usage (K,) int32."""
    import torch
    prec = _prec_of(D, prec)
    K, m = D.shape
    n, s = idx.shape
    usage = torch.empty((K,), dtype=torch.int32, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_mod_update", ctx.bind_stream(), prec, _ptr(Y), m, n, _ptr(idx), _ptr(val), s, _ptr(D), K,
          _ptr(usage))
    return usage


def mod_update_batched(Y, offsets, idx, val, D, prec=None):
    """Batched MOD in place on D (L, K, m); returns usage (L, K) int32."""
    import torch
    prec = _prec_of(D, prec)
    L, K, m = D.shape
    s = idx.shape[1]
    oh, op = _offsets_host(offsets)
    usage = torch.empty((L, K), dtype=torch.int32, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_mod_update_batched", ctx.bind_stream(), prec, _ptr(Y), m, op, L, _ptr(idx), _ptr(val), s,
          _ptr(D), K, _ptr(usage))
    return usage


def replace_atoms(Y, offsets, usage, resid2, min_use, D, prec=None):
    """Atom replacement in place on D (L, K, m): per subset, atoms used by fewer
    than min_use signals become the worst-coded signals (largest resid2),
    normalised.  Returns rep (L, K) int32: the signal row per replaced atom, else -1."""
    import torch
    prec = _prec_of(D, prec)
    L, K, m = D.shape
    oh, op = _offsets_host(offsets)
    rep = torch.empty((L, K), dtype=torch.int32, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_replace_atoms", ctx.bind_stream(), prec, _ptr(Y), m, op, L, _ptr(usage), _ptr(resid2),
          int(min_use), _ptr(D), K, _ptr(rep))
    return rep


def split(Y, perm, prec=None, out=None):
    """Algorithm 1 step 1: returns Y[perm] computed by the gather kernel (into
    `out` when given)."""
    import torch
    prec = _prec_of(Y, prec)
    N, m = Y.shape
    out = torch.empty_like(Y) if out is None else out
    ctx = context(Y.device.index)
    _call("sdl_split", ctx.bind_stream(), prec, _ptr(Y), m, N, _ptr(perm), _ptr(out))
    return out


def init_dict(Y, pick, fill=None, prec=None, out=None):
    """Unit-normalised Y[pick] (fill[c] where pick[c] < 0); pick int64 (count,);
    written into `out` (count, m) when given."""
    import torch
    prec = _prec_of(Y, prec)
    nY, m = Y.shape
    count = pick.numel()
    out = torch.empty((count, m), dtype=Y.dtype, device=Y.device) if out is None else out
    ctx = context(Y.device.index)
    _call("sdl_init_dict", ctx.bind_stream(), prec, _ptr(Y), m, nY, _ptr(pick), _ptr(fill), count, _ptr(out))
    return out


def local_train(Y, offsets, D_local, s1, iters, eps=0.0, prec=None, with_rmse=True, xfro=None):
    """Algorithm 1 step 2 in place on D_local (L, K1, m).
    Returns (xfro (L,) f64 -- the buffer given, if any -- , rmse (L, iters) f64 or None)."""
    import torch
    prec = _prec_of(D_local, prec)
    L, K1, m = D_local.shape
    oh, op = _offsets_host(offsets)
    if xfro is None:
        xfro = torch.empty((L,), dtype=torch.float64, device=D_local.device)
    rmse = torch.empty((L, iters), dtype=torch.float64, device=D_local.device) if with_rmse else None
    ctx = context(D_local.device.index)
    _call("sdl_local_train", ctx.bind_stream(), prec, _ptr(Y), m, op, L, K1, s1, float(eps), iters,
          _ptr(D_local), _ptr(xfro), _ptr(rmse))
    return xfro, rmse


def merge(D_local, xfro, pick, K, s2, iters, eps=0.0, prec=None, with_rmse=True, D_init=None, out=None):
    """Algorithm 1 step 3.  pick (K,) int32 selects the initial stacked columns;
    pick=None starts from D_init (K, m) instead.  The merged dictionary goes to
    `out` (K, m) when given.  Returns (D (K, m), rmse (iters,) f64 or None)."""
    import torch
    prec = _prec_of(D_local, prec)
    L, K1, m = D_local.shape
    D = torch.empty((K, m), dtype=D_local.dtype, device=D_local.device) if out is None else out
    if pick is None:
        if D_init is None or tuple(D_init.shape) != (K, m):
            raise ValueError("pick=None needs D_init of shape (K, m)")
        D.copy_(D_init)
    rmse = torch.empty((iters,), dtype=torch.float64, device=D_local.device) if with_rmse else None
    ctx = context(D_local.device.index)
    _call("sdl_merge", ctx.bind_stream(), prec, _ptr(D_local), _ptr(xfro), m, K1, L, _ptr(pick), K, s2,
          float(eps), iters, _ptr(D), _ptr(rmse))
    return D, rmse


def residual(Y, D, idx, val, prec=None):
    """(||Y - D X||_F^2, ||Y||_F^2) as a device float64 tensor of 2 entries."""
    import torch
    prec = _prec_of(D, prec)
    n, m = Y.shape
    K = D.shape[0]
    s = idx.shape[1]
    out = torch.empty((2,), dtype=torch.float64, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_residual", ctx.bind_stream(), prec, _ptr(Y), m, n, _ptr(D), K, _ptr(idx), _ptr(val), s,
          _ptr(out))
    return out


def extract_patches(img, p, prec=None):
    """Every p x p patch of img (H, W), row-major: ((H-p+1)(W-p+1), p*p)."""
    import torch
    prec = _prec_of(img, prec)
    H, W = img.shape
    out = torch.empty(((H - p + 1) * (W - p + 1), p * p), dtype=img.dtype, device=img.device)
    ctx = context(img.device.index)
    _call("sdl_extract_patches", ctx.bind_stream(), prec, _ptr(img), H, W, p, _ptr(out))
    return out


def patch_average(D, idx, val, H, W, p, prec=None):
    """Per pixel, the mean of the estimates D x of the patches covering it: (H, W)."""
    import torch
    prec = _prec_of(D, prec)
    out = torch.empty((H, W), dtype=D.dtype, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_patch_average", ctx.bind_stream(), prec, _ptr(D), D.shape[0], _ptr(idx), _ptr(val), idx.shape[1], H,
          W, p, _ptr(out))
    return out


def sq_error(a, b, prec=None):
    """(sum (a - b)^2, sum b^2) as a device float64 tensor of 2 entries."""
    import torch
    prec = _prec_of(a, prec)
    out = torch.empty((2,), dtype=torch.float64, device=a.device)
    ctx = context(a.device.index)
    _call("sdl_sq_error", ctx.bind_stream(), prec, _ptr(a), _ptr(b), a.numel(), _ptr(out))
    return out


def denoise(noisy, D, p, eps, s_max=32, prec=None):
    """Sec. 3.2.2 denoising of noisy (H, W) with dictionary D (K, p*p): every
    overlapping patch coded by OMP until ||r|| <= eps (at most s_max atoms),
    estimates averaged per pixel.  Returns (denoised (H, W), codes (idx, val, nnz))."""
    H, W = noisy.shape
    P = extract_patches(noisy, p, prec=prec)
    idx, val, nnz, _ = omp(D, P, s_max, eps=eps, prec=prec, with_resid=False)
    return patch_average(D, idx, val, H, W, p, prec=None if prec == PREC_BF16 else prec), (idx, val, nnz)


def corr_features(D, Y, offsets):
    """|D_t^T y| of every row of Y against its subset's dictionary (D: (L, K, m),
    FP32), shape (n, K): the input of a dictionary-conditioned proposer."""
    import torch
    L, K, m = D.shape
    n = Y.shape[0]
    oh, op = _offsets_host(offsets)
    assert len(oh) == L + 1 and oh[-1] == n
    F = torch.empty((n, K), dtype=torch.float32, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_corr_features", ctx.bind_stream(), _ptr(D), m, K, _ptr(Y), op, L, _ptr(F))
    return F


def gram(D, prec=None):
    """Gram matrices of D (L, K, m) or (K, m): D_t D_t^T, shape (L, K, K) or (K, K)."""
    import torch
    prec = _prec_of(D, prec)
    Db = D if D.dim() == 3 else D[None]
    L, K, m = Db.shape
    G = torch.empty((L, K, K), dtype=torch.float64 if prec == PREC_F64 else torch.float32, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_gram", ctx.bind_stream(), prec, _ptr(Db), m, K, L, _ptr(G))
    return G if D.dim() == 3 else G[0]


def recovery(D0, D, thresh=0.98, prec=None):
    """Number of atoms of D0 recovered by D (Sec. 3.1), as a device int32 tensor."""
    import torch
    prec = _prec_of(D, prec)
    K0, m = D0.shape
    K = D.shape[0]
    out = torch.empty((1,), dtype=torch.int32, device=D.device)
    ctx = context(D.device.index)
    _call("sdl_recovery", ctx.bind_stream(), prec, _ptr(D0), K0, _ptr(D), K, m, float(thresh), _ptr(out))
    return out


class Proposer:
    """The learned support proposer (MLP m -> h1 -> h2 -> K) living on one device."""

    def __init__(self, params, m, h1, h2, K, ctx=None):
        import torch
        self.ctx = ctx or context(params.device.index)
        self.m, self.h1, self.h2, self.K = m, h1, h2, K
        self.nparams = params.numel()
        h = _vp()
        _call("sdl_proposer_create", self.ctx.bind_stream(), m, h1, h2, K, _ptr(params.contiguous()),
              ctypes.byref(h))
        self.handle = h
        self.device = params.device

    def params(self):
        import torch
        out = torch.empty((self.nparams,), dtype=torch.float32, device=self.device)
        _call("sdl_proposer_get_params", self.ctx.bind_stream(), self.handle, _ptr(out))
        return out

    def loss_grad(self, Y, idx):
        import torch
        B, s = idx.shape
        loss = torch.empty((4,), dtype=torch.float32, device=self.device)
        grad = torch.empty((self.nparams,), dtype=torch.float32, device=self.device)
        _call("sdl_proposer_loss_grad", self.ctx.bind_stream(), self.handle, _ptr(Y), _ptr(idx), s, B,
              _ptr(loss), _ptr(grad))
        return loss[0], grad

    def train_step(self, Y, idx, lr, loss=None):
        B, s = idx.shape
        _call("sdl_proposer_train_step", self.ctx.bind_stream(), self.handle, _ptr(Y), _ptr(idx), s, B,
              float(lr), _ptr(loss))

    def scores(self, Y):
        import torch
        n = Y.shape[0]
        Z = torch.empty((n, self.K), dtype=torch.float32, device=self.device)
        _call("sdl_proposer_scores", self.ctx.bind_stream(), self.handle, _ptr(Y), n, _ptr(Z))
        return Z

    def omp(self, D, Y, s, ncand, eps_fb, with_resid=True):
        """Proposer-assisted OMP; returns (idx, val, nnz, resid2, n_fallback)."""
        import torch
        K, m = D.shape
        n = Y.shape[0]
        idx = torch.empty((n, s), dtype=torch.int32, device=self.device)
        val = torch.empty((n, s), dtype=torch.float32, device=self.device)
        nnz = torch.empty((n,), dtype=torch.int32, device=self.device)
        r2 = torch.empty((n,), dtype=torch.float32, device=self.device) if with_resid else None
        nf = ctypes.c_int64(0)
        _call("sdl_omp_proposed", self.ctx.bind_stream(), self.handle, _ptr(D), m, K, _ptr(Y), n, s, ncand,
              float(eps_fb), _ptr(idx), _ptr(val), _ptr(nnz), _ptr(r2), ctypes.byref(nf))
        return idx, val, nnz, r2, int(nf.value)

    def omp_batched(self, D, Y, offsets, s, ncand, eps_fb, features=FEATURES_CORR, with_resid=True):
        """Proposer-assisted OMP over subsets (D: (L, K, m)), the network reading
        |D_t^T y| (FEATURES_CORR) or y (FEATURES_SIGNAL); returns (idx, val, nnz,
        resid2, n_fallback)."""
        import torch
        L, K, m = D.shape
        n = Y.shape[0]
        oh, op = _offsets_host(offsets)
        assert len(oh) == L + 1 and oh[-1] == n
        idx = torch.empty((n, s), dtype=torch.int32, device=self.device)
        val = torch.empty((n, s), dtype=torch.float32, device=self.device)
        nnz = torch.empty((n,), dtype=torch.int32, device=self.device)
        r2 = torch.empty((n,), dtype=torch.float32, device=self.device) if with_resid else None
        nf = ctypes.c_int64(0)
        _call("sdl_omp_proposed_batched", self.ctx.bind_stream(), self.handle, features, _ptr(D), m, K, _ptr(Y), op,
              L, s, ncand, float(eps_fb), _ptr(idx), _ptr(val), _ptr(nnz), _ptr(r2), ctypes.byref(nf))
        return idx, val, nnz, r2, int(nf.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().sdl_proposer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
