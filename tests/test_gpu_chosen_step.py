"""The bench's chosen form, step by step, against the oracle: the split-and-merge
FP32 workload at full size (N=200,000, m=64, L=100 x 2,000, K1=256, s1=2; merge
of the 25,600 scaled local atoms to K=256 with s2=3; final coding at s=6), with
BF16 tensor-core correlations and Gram, FP32 refits and the training loops
replayed as CUDA graphs, in the launch configuration bench.py times.

Each training iteration starts the GPU and the oracle from the same dictionary
(the GPU's current one), and runs through the same library calls as the bench
with graph replay on: the first call of a shape runs eagerly and tunes the MOD
solve, the second runs eagerly again, the third is captured and every later
one is a replay.  Per iteration, on sampled subsets (all of the merge):
  * the coding pass (the batched BF16 OMP the training runs) meets the BF16
    parity rule against the oracle's OMP on the same dictionary, with the
    excused share capped;
  * its RMSE is within the stated 1e-3 (relative) of the oracle's over the
    signals whose codes agree (a near-tie pick may lead greedy OMP elsewhere);
  * the updated atoms equal the oracle's MOD of the GPU's own codes within the
    FP32 atom tolerance 2e-5 (unit atoms; FP64 normal equations, FP32 output).
Then the final coding of every signal against the merged dictionary is
checked the same way on 2,000 sampled signals, and the residual the bench
reports against numpy.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import check_bf16_codes, check_rmse

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ITERS = 5          # 0, 1 eager; 2 captured; 3, 4 replayed
CAP = 0.04         # share of sampled codes allowed to differ at BF16 near-ties not at rounding
                   # level, per check (measured at most 2.05 %)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_chosen_step_bf16_graph_replay_teacher_forced():
    p = si.config1()
    ctx = sdl.context(0)
    ctx.set_option(sdl.OPT_GRAPH, 1)
    rng = np.random.default_rng(960)
    try:
        Yp = sdl.split(_t(p.Y), _t(p.perm), out=torch.empty((p.N, p.m), dtype=torch.float32, device=DEV))
        Dl = sdl.init_dict(Yp, _t(p.picks.reshape(-1)),
                           out=torch.empty((p.L * p.K1, p.m), dtype=torch.float32, device=DEV)).view(p.L, p.K1, p.m)
        xfro_buf = torch.empty((p.L,), dtype=torch.float64, device=DEV)
        Ypn = Yp.cpu().numpy().astype(np.float64)
        sample = [0, 37, 99]
        excused = rounding = coded = 0
        for it in range(ITERS):
            before = Dl.cpu().numpy()
            idx, val, nnz, r2 = (x.cpu().numpy() for x in
                                 sdl.omp_batched(Dl, Yp, p.offsets, p.s1, prec=sdl.PREC_BF16))
            sdl.local_train(Yp, p.offsets, Dl, p.s1, 1, prec=sdl.PREC_BF16, with_rmse=False, xfro=xfro_buf)
            after = Dl.cpu().numpy()
            for t in sample:
                a, b = p.offsets[t], p.offsets[t + 1]
                Dt = before[t].astype(np.float64)
                orc = oracle.omp(Dt, Ypn[a:b], p.s1)
                ex, ro = check_bf16_codes(before[t], Ypn[a:b].astype(np.float32), idx[a:b], val[a:b], nnz[a:b],
                                          r2[a:b], orc, max_excused=CAP)
                excused, rounding = excused + ex, rounding + ro
                print(f"{ex} differ, {ro} at rounding level")
                coded += b - a
                check_rmse(r2[a:b], orc, idx[a:b], nnz[a:b], p.m)
                Dm, *_ = oracle.mod(Ypn[a:b], idx[a:b], val[a:b].astype(np.float64), Dt, True)
                np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5, err_msg=f"local it {it} subset {t}")
        # the last local coding pass gives each subset's ||X^(t)||_F (Algorithm 1 step 3)
        xf = xfro_buf.cpu().numpy()
        xf_np = np.sqrt(np.add.reduceat((val.astype(np.float64) ** 2).sum(axis=1), p.offsets[:-1]))
        np.testing.assert_allclose(xf, xf_np, rtol=1e-6)
        # merge: the scaled stack of the GPU's local atoms, as both sides form it
        Yt = (after.astype(np.float64) * xf[:, None, None]).reshape(-1, p.m).astype(np.float32)
        Ytg, Yt64 = _t(Yt), Yt.astype(np.float64)
        Dbuf = torch.empty((p.K, p.m), dtype=torch.float32, device=DEV)
        D = Yt64[p.mpick] / np.linalg.norm(Yt64[p.mpick], axis=1, keepdims=True)
        for it in range(ITERS):
            Dg = _t(D.astype(np.float32))
            idx, val, nnz, r2 = (x.cpu().numpy() for x in sdl.omp(Dg, Ytg, p.s2, prec=sdl.PREC_BF16))
            # one merge iteration (stack, then a training iteration on it) from
            # the current dictionary; the picked initial columns are numpy's here
            Dbuf.copy_(Dg)
            sdl.merge(Dl, xfro_buf, None, p.K, p.s2, 1, prec=sdl.PREC_BF16, with_rmse=False, D_init=Dbuf, out=Dbuf)
            Dn = Dbuf.cpu().numpy()
            pick = np.sort(rng.choice(len(Yt), 2000, replace=False))
            orc = oracle.omp(D, Yt64[pick], p.s2)
            ex, ro = check_bf16_codes(D.astype(np.float32), Yt[pick], idx[pick], val[pick], nnz[pick], r2[pick],
                                      orc, max_excused=CAP)
            excused, rounding = excused + ex, rounding + ro
            print(f"{ex} differ, {ro} at rounding level")
            coded += len(pick)
            check_rmse(r2, oracle.omp(D, Yt64, p.s2), idx, nnz, p.m)
            Dm, *_ = oracle.mod(Yt64, idx, val.astype(np.float64), D, True)
            np.testing.assert_allclose(Dn, Dm, rtol=0, atol=2e-5, err_msg=f"merge it {it}")
            D = Dn.astype(np.float64)
        # final coding of every signal with the merged dictionary, and the residual
        Yg = _t(p.Y)
        idx, val, nnz, r2 = sdl.omp(Dbuf, Yg, p.s, prec=sdl.PREC_BF16)
        res = sdl.residual(Yg, Dbuf, idx, val).cpu().numpy()
        idx, val, nnz, r2 = (x.cpu().numpy() for x in (idx, val, nnz, r2))
        pick = np.sort(rng.choice(p.N, 2000, replace=False))
        Y64 = p.Y.astype(np.float64)
        orc = oracle.omp(D, Y64[pick], p.s)
        ex, ro = check_bf16_codes(D.astype(np.float32), p.Y[pick], idx[pick], val[pick], nnz[pick], r2[pick], orc,
                                  max_excused=CAP)
        excused, rounding = excused + ex, rounding + ro
        print(f"{ex} differ, {ro} at rounding level")
        coded += len(pick)
        rec = np.einsum("ns,nsm->nm", np.where(idx >= 0, val, 0).astype(np.float64), D[np.maximum(idx, 0)])
        r2_np = ((Y64 - rec) ** 2).sum()
        assert abs(res[0] - r2_np) <= 1e-5 * r2_np and abs(res[1] - (Y64 ** 2).sum()) <= 1e-9 * res[1]
        print(f"chosen step: {excused} of {coded} sampled BF16 codes differ at near-ties "
              f"({excused / coded:.3%}, cap {CAP:.0%} per check), {rounding} more at rounding-level steps")
    finally:
        ctx.set_option(sdl.OPT_GRAPH, 0)
