"""Multi-rank host logic on CPU (world size 2, gloo, 127.0.0.1): the sharded
Algorithm 1 and the bench's whole-job timing.

The sharded local phase deals subsets to ranks by size, trains each rank's
subsets independently (here with the oracle's local training on CPU), and
all-gathers the local dictionaries and scales; the stack every rank ends with
must equal the single-process oracle's local phase, and the merge run on it
must equal the single-process oracle's split-and-merge.  The bench reduces the
per-rank timed totals with a max over ranks and reports the whole job's
throughput from it.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
import sdl_inputs as si
from paper_1403_4781_gb300 import dist as sdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    sizes = [300, 120, 410, 77, 256, 190, 333]
    return si.split_merge_problem("t", 12, 20, 4, 2, 2, 20, sizes, 4, 3, 0.02, np.random.default_rng(600),
                                  dtype=np.float64)


def _init_stack(p):
    Yp = p.Y[p.perm]
    return Yp, np.stack([Yp[q] / np.linalg.norm(Yp[q], axis=1, keepdims=True) for q in p.picks])


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        Yp, Dinit = _init_stack(p)

        def train(Yb, off_b, Db):   # the oracle's local training stands in for the GPU's
            out = oracle.local_train(Yb.numpy(), off_b, Db.numpy(), p.s1, p.iters_local, nthreads=1)
            Db.copy_(torch.from_numpy(out["D"]))
            return torch.from_numpy(out["xfro"])

        D, xfro = sdist.sharded_local_phase(torch.from_numpy(Yp), p.offsets, torch.from_numpy(Dinit),
                                            rank, world, train)
        mer = oracle.merge(D.numpy(), xfro.numpy(), p.mpick, p.K, p.s2, p.iters_merge, nthreads=1)
        import bench
        t_max = bench.max_over_ranks([12.5, 30.0][rank], world, "cpu")
        rate = bench.whole_job_rate(1000, world, 5, t_max)
        q.put((rank, D.numpy(), xfro.numpy(), mer["D"], t_max, rate))
    finally:
        dist.destroy_process_group()


def test_assignment_balances_by_size_and_covers_every_subset():
    sizes = [300, 120, 410, 77, 256, 190, 333]
    a = sdist.assign_subsets(sizes, 2)
    assert sorted(a[0] + a[1]) == list(range(len(sizes)))
    loads = [sum(sizes[t] for t in r) for r in a]
    assert abs(loads[0] - loads[1]) <= max(sizes)
    assert sdist.assign_subsets(sizes, 1) == [list(range(len(sizes)))]
    assert sdist.assign_subsets([5, 5], 3) == [[0], [1], []]


def test_sharded_split_and_merge_equals_single_process_gloo_world2():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in procs:
        r, D, xfro, Dm, t_max, rate = q.get(timeout=180)
        res[r] = (D, xfro, Dm, t_max, rate)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = _problem()
    Yp, Dinit = _init_stack(p)
    loc = oracle.local_train(Yp, p.offsets, Dinit, p.s1, p.iters_local, nthreads=1)
    mer = oracle.merge(loc["D"], loc["xfro"], p.mpick, p.K, p.s2, p.iters_merge, nthreads=1)
    for r in (0, 1):
        D, xfro, Dm, t_max, rate = res[r]
        np.testing.assert_allclose(D, loc["D"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(xfro, loc["xfro"], rtol=1e-12)
        np.testing.assert_allclose(Dm, mer["D"], rtol=0, atol=1e-12)
        assert t_max == 30.0
        assert rate == pytest.approx(2 * 1000 * 5 / 0.030)


@pytest.mark.gpu
def test_sharded_local_phase_single_gpu_rank_uses_the_batched_trainer():
    """World size 1 on one GPU: the sharded local phase with the library's
    batched local training equals calling that training directly."""
    import torch

    import paper_1403_4781_gb300 as sdl
    p = _problem()
    Yp, Dinit = _init_stack(p)
    Yg = torch.from_numpy(Yp.astype(np.float32)).cuda()
    Dg = torch.from_numpy(Dinit.astype(np.float32)).cuda()

    def train(Yb, off_b, Db):
        xf, _ = sdl.local_train(Yb, off_b, Db, p.s1, p.iters_local, with_rmse=False)
        return xf

    D, xfro = sdist.sharded_local_phase(Yg, p.offsets, Dg, 0, 1, train)
    Dd = Dg.clone()
    xd, _ = sdl.local_train(Yg, p.offsets, Dd, p.s1, p.iters_local, with_rmse=False)
    np.testing.assert_allclose(D.cpu().numpy(), Dd.cpu().numpy(), rtol=0, atol=1e-5)
    np.testing.assert_allclose(xfro.cpu().numpy(), xd.cpu().numpy(), rtol=1e-5)
