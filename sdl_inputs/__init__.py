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
