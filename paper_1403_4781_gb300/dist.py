"""Algorithm 1 across ranks (one process per GPU): the host logic of the sharded
split-and-merge.

Step 2 of Algorithm 1 trains every subset independently, so the subsets are
dealt to the ranks and trained with no communication; step 3 needs every local
dictionary and its scale ||X^(t)||_F, which is the one exchange: an all-gather
of the stacked local dictionaries and scales, after which every rank holds the
same [L][K1][m] stack in subset order and can run the merge.

Nothing here touches a kernel: the local trainer is passed in (the library's
batched `local_train` on a GPU rank), and the collectives are torch.distributed
calls on whatever backend the process group was created with.
"""
from __future__ import annotations

import numpy as np


def assign_subsets(sizes, world: int) -> list[list[int]]:
    """Deal subsets to `world` ranks, largest first, each to the rank with the
    least work so far (ties: lowest rank), work = subset size.  Deterministic;
    every rank computes the same assignment.  Each rank's list is in ascending
    subset order."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = np.zeros(world, dtype=np.int64)
    owned: list[list[int]] = [[] for _ in range(world)]
    for t in sorted(range(len(sizes)), key=lambda q: (-int(sizes[q]), q)):
        r = int(np.argmin(load))          # first minimum = lowest rank on ties
        owned[r].append(t)
        load[r] += int(sizes[t])
    return [sorted(o) for o in owned]


def local_batch(Yp, offsets, subsets):
    """The rows of the permuted signals belonging to `subsets` (consecutive in
    the order given) and their offsets [len(subsets)+1]."""
    offsets = np.asarray(offsets, dtype=np.int64)
    parts = [(int(offsets[t]), int(offsets[t + 1])) for t in subsets]
    sizes = np.array([b - a for a, b in parts], dtype=np.int64)
    loc_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return parts, loc_off


def gather_local(D_mine, xfro_mine, subsets_by_rank, rank: int, L: int):
    """All-gather the local dictionaries and scales of every rank into the full
    [L][K1][m] stack and [L] scales in subset order.

    D_mine: tensor [len(subsets_by_rank[rank])][K1][m]; xfro_mine: [same] (f64).
    Every rank's block is padded to the largest rank's count so one all_gather
    of equal shapes moves them."""
    import torch
    import torch.distributed as dist

    world = len(subsets_by_rank)
    K1, m = D_mine.shape[1], D_mine.shape[2]
    if world == 1:   # a single rank holds every subset already, in order
        return D_mine.reshape(L, K1, m), xfro_mine.to(torch.float64)
    n_max = max(len(s) for s in subsets_by_rank)
    pad_D = torch.zeros((n_max, K1, m), dtype=D_mine.dtype, device=D_mine.device)
    pad_x = torch.zeros((n_max,), dtype=torch.float64, device=D_mine.device)
    n = len(subsets_by_rank[rank])
    pad_D[:n] = D_mine
    pad_x[:n] = xfro_mine.to(torch.float64)
    all_D = [torch.empty_like(pad_D) for _ in range(world)]
    all_x = [torch.empty_like(pad_x) for _ in range(world)]
    dist.all_gather(all_D, pad_D)
    dist.all_gather(all_x, pad_x)
    D = torch.empty((L, K1, m), dtype=D_mine.dtype, device=D_mine.device)
    xfro = torch.empty((L,), dtype=torch.float64, device=D_mine.device)
    for r, subs in enumerate(subsets_by_rank):
        for q, t in enumerate(subs):
            D[t] = all_D[r][q]
            xfro[t] = all_x[r][q]
    return D, xfro


def sharded_local_phase(Yp, offsets, D_init, rank: int, world: int, train):
    """Step 2 of Algorithm 1 on this rank's subsets, then the exchange.

    Yp: permuted signals [N][m]; offsets: host [L+1]; D_init: [L][K1][m] initial
    atoms of every subset (only this rank's are used); train(Y_batch,
    offsets_batch, D_batch) trains D_batch in place and returns ||X||_F per
    subset.  Returns the full trained stack [L][K1][m] and scales [L], identical
    on every rank."""
    import torch

    offsets = np.asarray(offsets, dtype=np.int64)
    L = len(offsets) - 1
    subsets_by_rank = assign_subsets(np.diff(offsets), world)
    mine = subsets_by_rank[rank]
    parts, loc_off = local_batch(Yp, offsets, mine)
    if mine:
        Yb = torch.cat([Yp[a:b] for a, b in parts])
        Db = D_init[mine].clone()
        xb = train(Yb, loc_off, Db)
    else:
        Db = D_init[:0].clone()
        xb = torch.zeros((0,), dtype=torch.float64, device=D_init.device)
    return gather_local(Db, xb, subsets_by_rank, rank, L)
