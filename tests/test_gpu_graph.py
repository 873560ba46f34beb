"""Training loops replayed as CUDA graphs (SDL_OPT_GRAPH) give the eager
results: the first call with a given set of buffers runs eagerly, a later one
captures the iterations, later ones relaunch the graph.  FP64 results agree to
1e-9 (the accumulation visits each atom's signals in an order set by atomics,
so runs agree to rounding level); the launch count of a replay equals an eager
call's."""
import numpy as np
import pytest
import torch

import paper_1403_4781_gb300 as sdl
import sdl_inputs as si

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture
def ctx():
    c = sdl.context(0)
    yield c
    c.set_option(sdl.OPT_GRAPH, 0)


@pytest.mark.parametrize("dtype,atol", [(np.float64, 1e-9), (np.float32, 2e-5)])
def test_graph_replay_matches_eager(ctx, dtype, atol):
    iters = 5 if dtype == np.float64 else 2
    p = si.split_merge_problem("g", 32, 64, 4, 2, 2, 64, [700, 1300, 450, 900], iters, iters, 0.02,
                               np.random.default_rng(900), dtype=dtype)
    Yp = _t(p.Y[p.perm])
    D0 = sdl.init_dict(Yp, _t(p.picks.reshape(-1)), _t(p.fill.reshape(-1, p.m).astype(dtype))).reshape(p.L, p.K1, p.m)
    D = D0.clone()
    ctx.set_option(sdl.OPT_GRAPH, 0)
    sdl.local_train(Yp, p.offsets, D, p.s1, iters)   # warm-up: the autotuner's launches happen here
    D.copy_(D0)
    n0 = ctx.launch_count()
    xe, re = sdl.local_train(Yp, p.offsets, D, p.s1, iters)
    eager_launches = ctx.launch_count() - n0
    De = D.clone()
    ctx.set_option(sdl.OPT_GRAPH, 1)
    for call in range(4):           # eager, eager (after tuning), capture + launch, replay
        D.copy_(D0)
        n0 = ctx.launch_count()
        xg, rg = sdl.local_train(Yp, p.offsets, D, p.s1, iters)
        torch.cuda.synchronize()
        assert ctx.launch_count() - n0 == eager_launches, call
        np.testing.assert_allclose(D.cpu().numpy(), De.cpu().numpy(), rtol=0, atol=atol, err_msg=f"call {call}")
        np.testing.assert_allclose(rg.cpu().numpy(), re.cpu().numpy(), rtol=1e-6 if dtype == np.float32 else 1e-12)
        np.testing.assert_allclose(xg.cpu().numpy(), xe.cpu().numpy(), rtol=1e-6 if dtype == np.float32 else 1e-12)
    ctx.set_option(sdl.OPT_GRAPH, 0)   # drops the cache
    D.copy_(D0)
    sdl.local_train(Yp, p.offsets, D, p.s1, iters)
    np.testing.assert_allclose(D.cpu().numpy(), De.cpu().numpy(), rtol=0, atol=atol)
