"""Seeded synthetic inputs for split-and-merge dictionary learning.

This module only draws random data; it holds none of the method's arithmetic
(no sparse coding, no dictionary update).  Both the CUDA path's tests/bench and
the CPU oracle consume what it returns, so every random choice the method makes
(the random partition of Algorithm 1 step 1, the initial atoms) is drawn here and
passed in as an input.

Layout: a signal matrix Y in R^{m x N} is returned as a numpy array of shape
(N, m) (one signal contiguous), a dictionary D in R^{m x K} as shape (K, m).

Data model (Def. 1, Sec. 3.1): ground-truth atoms are i.i.d. N(0,1) columns
scaled to unit length; each signal combines s atoms on a uniformly random
support with N(0,1) coefficients, plus i.i.d. N(0, sigma^2) noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(config: int, trial: int = 0) -> np.random.Generator:
    """Seed convention: 1000 + config for trial 0, 1000 + 100 config + t otherwise."""
    seed = 1000 + config if trial == 0 else 1000 + 100 * config + trial
    return np.random.default_rng(seed)


def unit_gaussian_atoms(rng: np.random.Generator, m: int, K: int, dtype=np.float64) -> np.ndarray:
    """K atoms in R^m, i.i.d. N(0,1) entries, each scaled to unit Euclidean length."""
    D = rng.standard_normal((K, m))
    D /= np.sqrt((D * D).sum(axis=1, keepdims=True))
    return D.astype(dtype)


def sparse_signals(rng: np.random.Generator, D0: np.ndarray, N: int, s: int, sigma: float,
                   dtype=np.float64):
    """N signals y = D0 x + n with s-sparse x (uniform random support, N(0,1) values).

    Returns (Y (N, m), support (N, s) int64, coeffs (N, s))."""
    K, m = D0.shape
    support = np.empty((N, s), dtype=np.int64)
    coeffs = np.empty((N, s))
    Y = np.empty((N, m), dtype=dtype)
    chunk = max(1, min(N, 2**22 // max(K, s * m)))
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        keys = rng.random((b - a, K))
        sup = np.argpartition(keys, s - 1, axis=1)[:, :s] if s < K else np.tile(np.arange(K), (b - a, 1))
        c = rng.standard_normal((b - a, s))
        y = np.einsum("nk,nkm->nm", c, D0[sup])
        if sigma > 0:
            y += sigma * rng.standard_normal((b - a, m))
        support[a:b], coeffs[a:b], Y[a:b] = sup, c, y
    return Y, support, coeffs


def random_partition(rng: np.random.Generator, sizes) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 1 step 1's random split: a permutation of range(sum(sizes)) and the
    CSR offsets [L+1] of the consecutive subsets it defines."""
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    perm = rng.permutation(int(offsets[-1])).astype(np.int64)
    return perm, offsets


def uneven_sizes(rng: np.random.Generator, L: int, lo: int, hi: int) -> np.ndarray:
    """L subset sizes uniform on the integers [lo, hi]."""
    return rng.integers(lo, hi + 1, size=L).astype(np.int64)


def init_picks(rng: np.random.Generator, offsets: np.ndarray, K1: int) -> np.ndarray:
    """For every subset, K1 distinct signal indices (global, after the split) drawn
    uniformly from that subset; where the subset has fewer than K1 signals the
    remaining entries are -1 (filled by fresh Gaussian atoms, see init_fill)."""
    L = len(offsets) - 1
    picks = np.full((L, K1), -1, dtype=np.int64)
    for t in range(L):
        n = int(offsets[t + 1] - offsets[t])
        k = min(n, K1)
        picks[t, :k] = offsets[t] + rng.choice(n, size=k, replace=False)
    return picks


def init_fill(rng: np.random.Generator, L: int, K1: int, m: int) -> np.ndarray:
    """Gaussian columns used for initial atoms where a subset is smaller than K1."""
    return rng.standard_normal((L, K1, m))


def merge_pick(rng: np.random.Generator, n_stacked: int, K: int) -> np.ndarray:
    """K distinct columns of the stacked local dictionaries that seed the merge."""
    return rng.choice(n_stacked, size=K, replace=False).astype(np.int32)


@dataclass
class SplitMergeProblem:
    """One synthetic split-and-merge workload with every random choice drawn."""
    name: str
    m: int
    K: int
    s: int
    s1: int
    s2: int
    K1: int
    iters_local: int
    iters_merge: int
    sigma: float
    D0: np.ndarray
    Y: np.ndarray                # (N, m), original order
    perm: np.ndarray             # (N,)
    offsets: np.ndarray          # (L+1,)
    picks: np.ndarray            # (L, K1) global indices into the permuted Y, -1 = fill
    fill: np.ndarray             # (L, K1, m)
    mpick: np.ndarray            # (K,) merge init columns
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.Y.shape[0]

    @property
    def L(self) -> int:
        return len(self.offsets) - 1


def split_merge_problem(name, m, K, s, s1, s2, K1, sizes, iters_local, iters_merge, sigma,
                        rng, dtype=np.float32) -> SplitMergeProblem:
    D0 = unit_gaussian_atoms(rng, m, K)
    sizes = np.asarray(sizes, dtype=np.int64)
    N = int(sizes.sum())
    Y, _, _ = sparse_signals(rng, D0, N, s, sigma, dtype=dtype)
    perm, offsets = random_partition(rng, sizes)
    picks = init_picks(rng, offsets, K1)
    fill = init_fill(rng, len(sizes), K1, m).astype(dtype)
    mpick = merge_pick(rng, K1 * len(sizes), K)
    return SplitMergeProblem(name, m, K, s, s1, s2, K1, iters_local, iters_merge, sigma,
                             D0.astype(dtype), Y, perm, offsets, picks, fill, mpick)


def config1(scale: float = 1.0, iters_local: int = 20, iters_merge: int = 20) -> SplitMergeProblem:
    """Split-and-merge FP32 workload: m=64, K=256, s=6 (s1=2, s2=3), L=100 subsets of
    2,000 signals (N=200,000), K1=256, noise sigma=0.01.  `scale` < 1 shrinks L."""
    L = max(1, int(round(100 * scale)))
    return split_merge_problem("splitmerge_m64_K256_N200k", 64, 256, 6, 2, 3, 256,
                               [2000] * L, iters_local, iters_merge, 0.01, rng_for(1))


def config0():
    """Plain standard MOD/OMP in FP64: m=64, K=128, s=5, N=10,000, noise 0.01,
    initial atoms = 128 random training signals, 10 iterations."""
    rng = rng_for(0)
    D0 = unit_gaussian_atoms(rng, 64, 128)
    Y, _, _ = sparse_signals(rng, D0, 10_000, 5, 0.01)
    pick = rng.choice(10_000, size=128, replace=False)
    return dict(D0=D0, Y=Y, pick=pick, s=5, iters=10)


def e1_problem(trial: int = 0):
    """Sec. 3.1 synthetic experiment: D 30x60, N=40,000 noiseless 6-sparse signals;
    split L=40 x 1,000, K1=50, s1=3, s2=2; standard init = first 60 signals."""
    rng = np.random.default_rng(5000 + trial)
    D0 = unit_gaussian_atoms(rng, 30, 60)
    Y, _, _ = sparse_signals(rng, D0, 40_000, 6, 0.0)
    perm, offsets = random_partition(rng, [1000] * 40)
    picks = init_picks(rng, offsets, 50)
    mpick = merge_pick(rng, 50 * 40, 60)
    return dict(D0=D0, Y=Y, perm=perm, offsets=offsets, picks=picks, mpick=mpick)


def mlp_init(rng: np.random.Generator, m: int, h1: int, h2: int, K: int, s: int) -> np.ndarray:
    """Packed initial proposer parameters (W1, b1, W2, b2, W3, b3): He-scaled
    Gaussian weights, zero hidden biases, output bias at the label prior log(s/(K-s))."""
    parts = [rng.standard_normal(h1 * m) * np.sqrt(2.0 / m), np.zeros(h1),
             rng.standard_normal(h2 * h1) * np.sqrt(2.0 / h1), np.zeros(h2),
             rng.standard_normal(K * h2) * np.sqrt(1.0 / h2), np.full(K, np.log(s / (K - s)))]
    return np.concatenate(parts).astype(np.float32)


def config3(n_train: int = 1_000_000, n_eval: int = 1_000_000):
    """Learned-proposer workload: D0 64x256 unit atoms, s=6, noise 0.01; training
    and evaluation signals drawn independently from the same model."""
    rng = rng_for(3)
    D0 = unit_gaussian_atoms(rng, 64, 256).astype(np.float32)
    Ytr, _, _ = sparse_signals(rng, D0.astype(np.float64), n_train, 6, 0.01, dtype=np.float32)
    Yev, _, _ = sparse_signals(rng, D0.astype(np.float64), n_eval, 6, 0.01, dtype=np.float32)
    params = mlp_init(rng, 64, 512, 512, 256, 6)
    return dict(D0=D0, Ytr=Ytr, Yev=Yev, params=params, m=64, h1=512, h2=512, K=256, s=6)


def config2(shape: str = "A", L: int = 512, iters: int = 20) -> SplitMergeProblem:
    """Uneven batched local-training workload: L subsets with sizes uniform on
    the integers [500, 8000], one ground-truth dictionary per shape, noise 0.02.
    Shape A: m=64, K=256, s=6; shape B: m=144, K=512, s=10.  Each subset is
    trained with K atoms and sparsity s; its initial atoms are K distinct
    signals of the subset, Gaussian fill columns where it has fewer."""
    if shape not in ("A", "B"):
        raise ValueError("shape is 'A' or 'B'")
    rng = rng_for(2, trial=0 if shape == "A" else 1)
    m, K, s = (64, 256, 6) if shape == "A" else (144, 512, 10)
    sizes = uneven_sizes(rng, L, 500, 8000)
    return split_merge_problem(f"uneven_{shape}_m{m}_K{K}", m, K, s, s, 1, K, sizes, iters, 0, 0.02, rng)


def synthetic_image(rng: np.random.Generator, size: int = 512, bumps: int = 32, edges: int = 8,
                    sigma: float = 0.1) -> np.ndarray:
    """A piecewise-smooth random field: the sum of `bumps` 2-D Gaussian bumps
    (centres uniform over the image, widths uniform on [8, 64] pixels,
    amplitudes uniform on [-1, 1]) and `edges` straight edges (a step uniform on
    [-0.5, 0.5] on one side of a line through a uniform point at a uniform
    angle), min-max scaled to [0, 1], plus N(0, sigma^2) noise (not clipped)."""
    g = np.arange(size, dtype=np.float64)
    img = np.zeros((size, size))
    for _ in range(bumps):
        cy, cx = rng.uniform(0, size, 2)
        w = rng.uniform(8, 64)
        a = rng.uniform(-1, 1)
        img += a * np.outer(np.exp(-0.5 * ((g - cy) / w) ** 2), np.exp(-0.5 * ((g - cx) / w) ** 2))
    for _ in range(edges):
        py, px = rng.uniform(0, size, 2)
        th = rng.uniform(0, np.pi)
        step = rng.uniform(-0.5, 0.5)
        side = (np.cos(th) * (g[:, None] - py) + np.sin(th) * (g[None, :] - px)) > 0
        img += step * side
    lo, hi = img.min(), img.max()
    img = (img - lo) / (hi - lo) if hi > lo else np.zeros_like(img)
    return img + sigma * rng.standard_normal(img.shape)


def random_patches(rng: np.random.Generator, img: np.ndarray, count: int, p: int = 16) -> np.ndarray:
    """`count` p x p patches at uniform positions, each flattened row-major."""
    H, W = img.shape
    ys = rng.integers(0, H - p + 1, size=count)
    xs = rng.integers(0, W - p + 1, size=count)
    win = np.lib.stride_tricks.sliding_window_view(img, (p, p))
    return win[ys, xs].reshape(count, p * p)


def overcomplete_dct(p: int, qa: int, qb: int) -> np.ndarray:
    """Separable overcomplete DCT dictionary for p x p patches with qa x qb
    atoms, returned [qa qb][p p]: atom (a, b) is the outer product of 1-D
    cosines cos(pi i a / qa) and cos(pi j b / qb) (i, j = 0..p-1), each 1-D
    frame with its non-constant columns made zero-mean, every atom scaled to
    unit norm."""
    def frame(q):
        i = np.arange(p)[:, None]
        F = np.cos(np.pi * i * np.arange(q)[None, :] / q)
        F[:, 1:] -= F[:, 1:].mean(axis=0, keepdims=True)
        return F / np.linalg.norm(F, axis=0, keepdims=True)
    Fa, Fb = frame(qa), frame(qb)
    D = np.einsum("ia,jb->abij", Fa, Fb).reshape(qa * qb, p * p)
    return D / np.linalg.norm(D, axis=1, keepdims=True)


def config4(n_images: int = 256, per_image: int = 16384, L: int = 256, iters_local: int = 20,
            iters_merge: int = 20) -> SplitMergeProblem:
    """Large image-patch split-and-merge workload: 16 x 16 patches (m = 256,
    FP32) of synthetic images, split at random into L equal subsets; local
    K1 = 512 atoms with s1 = 4, merge to K = 1024 atoms with s2 = 4, final
    sparsity 16.  Both the local and the merge dictionaries start from an
    overcomplete DCT (256 x 512 and 256 x 1024), as the paper's image experiment
    does; `extra` holds those initial dictionaries and the final sparsity.
    Smaller n_images / per_image / L give the same recipe at a smaller size."""
    rng = rng_for(4)
    N = n_images * per_image
    Y = np.empty((N, 256), dtype=np.float32)
    for q in range(n_images):
        img = synthetic_image(rng)
        Y[q * per_image:(q + 1) * per_image] = random_patches(rng, img, per_image)
    sizes = np.full(L, N // L, dtype=np.int64)
    sizes[: N % L] += 1
    perm, offsets = random_partition(rng, sizes)
    K1, K = 512, 1024
    D_loc0 = overcomplete_dct(16, 16, 32).astype(np.float32)
    D_mer0 = overcomplete_dct(16, 32, 32).astype(np.float32)
    prob = SplitMergeProblem("patches_m256_K1024", 256, K, 16, 4, 4, K1, iters_local, iters_merge, 0.1,
                             D_mer0, Y, perm, offsets, np.full((L, K1), -1, np.int64),
                             np.broadcast_to(D_loc0, (L, K1, 256)).copy(), np.zeros(K, np.int32),
                             extra={"D_local0": D_loc0, "D_merge0": D_mer0, "s_final": 16})
    return prob
