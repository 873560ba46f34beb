"""The uneven batched BF16 workload at full size: 512 subsets with sizes uniform
on [500, 8000], shapes m=64/K=256/s=6 and m=144/K=512/s=10, noise 0.02, all
subsets of a shape trained in one batched launch per kernel with BF16
tensor-core correlations and Gram and FP32 refits.

Sampled subsets (the smallest, the largest and two seeded others) are compared
with the oracle iteration by iteration, each iteration starting the GPU and the
oracle from the same dictionary (the GPU's):
  * the iteration's codes (the same batched BF16 OMP the training runs) meet the
    BF16 parity rule against the oracle's OMP: supports equal except at
    near-ties, coefficients the exact least squares on the GPU's support;
  * the iteration's coding RMSE is within 1e-3 of the oracle's over the
    signals whose codes agree, and the reported RMSE is that of the GPU's own
    codes (a near-tie pick may lead greedy OMP to another final residual);
  * the updated atoms equal the oracle's MOD of the GPU's own codes within the
    FP32 atom tolerance 2e-5.
Free-running BF16 and FP64 trajectories separate through near-tie support
flips, which the BF16 rule allows, so only teacher-forced iterations are
compared.
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
ITERS = 4
# share of a subset's signals allowed to differ at near-ties not at rounding
# level, per iteration (measured at most 7.4 % on shape A and 15.5 % on shape
# B, both on their smallest subsets)
CAP = {"A": 0.12, "B": 0.25}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("shape", ["A", "B"])
def test_uneven_bf16_training_full_size_sampled_subsets(shape):
    p = si.config2(shape, iters=ITERS)
    sizes = np.diff(p.offsets)
    rng = np.random.default_rng(700)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *map(int, rng.choice(p.L, 2, replace=False))})
    Yg = sdl.split(_t(p.Y), _t(p.perm))
    Dg = sdl.init_dict(Yg, _t(p.picks.reshape(-1)), _t(p.fill.reshape(-1, p.m))).reshape(p.L, p.K1, p.m)
    Yp = Yg.cpu().numpy().astype(np.float64)
    worst, excused, rounding, coded = 0.0, 0, 0, 0
    for it in range(ITERS):
        before = Dg.cpu().numpy()
        idx, val, nnz, r2 = (x.cpu().numpy() for x in
                             sdl.omp_batched(Dg, Yg, p.offsets, p.s1, prec=sdl.PREC_BF16))
        _, rmse = sdl.local_train(Yg, p.offsets, Dg, p.s1, 1, prec=sdl.PREC_BF16)
        rmse = rmse.cpu().numpy()[:, 0]
        after = Dg.cpu().numpy()
        assert np.isfinite(rmse).all() and np.isfinite(after).all()
        for t in sample:
            a, b = p.offsets[t], p.offsets[t + 1]
            Dt = before[t].astype(np.float64)
            orc = oracle.omp(Dt, Yp[a:b], p.s1)
            ex, ro = check_bf16_codes(before[t], Yp[a:b].astype(np.float32), idx[a:b], val[a:b], nnz[a:b],
                                      r2[a:b], orc, max_excused=CAP[shape])
            excused, rounding = excused + ex, rounding + ro
            print(f"shape {shape} it {it} subset {t} ({b - a} signals): {ex} differ, {ro} at rounding level")
            coded += b - a
            rel = abs(check_rmse(r2[a:b], orc, idx[a:b], nnz[a:b], p.m, rmse[t]))
            worst = max(worst, rel)
            Dm, *_ = oracle.mod(Yp[a:b], idx[a:b], val[a:b].astype(np.float64), Dt, True)
            np.testing.assert_allclose(after[t], Dm, rtol=0, atol=2e-5, err_msg=f"{shape} it {it} subset {t}")
    print(f"shape {shape}: sampled subsets {sample} (sizes {sizes[sample].tolist()}), "
          f"worst per-iteration RMSE difference (near-tie paths included) {worst:.2e}, {excused} of {coded} codes differ at near-ties, "
          f"{rounding} more at rounding-level steps")
