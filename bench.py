#!/usr/bin/env python
"""Benchmark: split-and-merge dictionary learning (Algorithm 1) on one GB300.

Default line: the large image-patch workload (Sec. 3.2.1's patch training at
scale, on synthetic images): 4,194,304 16x16 patches (m=256, FP32) of 256
synthetic 512x512 piecewise-smooth images with noise 0.1, split at random into
L=256 subsets of 16,384; local K1=512 atoms, s1=4, 20 MOD/OMP iterations of
all subsets in one batched launch per kernel; merge of the 131,072 scaled local
atoms to K=1024 with s2=4 over 20 iterations; final OMP coding of every patch
with s=16 and the MSE of Table 1.  Both phases start from an overcomplete DCT.
One step = split gather -> initial atoms -> local training -> scaled stack +
merge training -> final coding -> residual.

The chosen form (batched launches, training loops replayed as CUDA graphs,
autotuned MOD solve: a checked FP32 solve with FP64 re-solves where the check
fails, BF16 tensor-core correlations and Gram with an FP32 correction step) is
timed against the plain form (the same algorithm with one launch
sequence per subset, FP32 CUDA-core correlations, no graphs), both to the
RMSE they reach.  The split-and-merge FP32 workload of 200,000 signals
(m=64, K=256, L=100 x 2,000) is measured in the same run as an extra key, and
is the main line with ``--workload splitmerge``.

metric: OMP-coded signals per second (local + merge + final codings per step
divided by the step time); the train-to-RMSE time and the RMSE reached are
reported beside it.  `--impl reference` times the CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sdl_inputs as si  # noqa: E402

METRIC = "OMP signals/sec and train-to-RMSE time, chosen vs plain form on 1 GB300"
UNIT = "signals/s"
WORKLOADS = {
    "patches": "patches_m256_N4194304_L256x16384_K1_512_K1024_s4x4_s16_iters20+20",
    "splitmerge": "splitmerge_fp32_m64_K256_s6_N200000_L100x2000_iters20+20",
}

# Nominal FP64 rate of the part (recipe table: 1.25 TFLOP/s); with 152 SMs at the
# 2,070 MHz maximum clock this is 2 DFMA per clock per SM (152*2*2*2.07e9 = 1.259e12).
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9
# FP32 CUDA-core rate: 152 SMs x 128 FFMA/clock x 2 flops x 2.07 GHz.
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9
# DRAM bytes (read + write) per launch of a kernel family, each from one ncu
# capture named beside it; a family with no capture of its current code has none.
TRAFFIC = {
    ("patches", "mod_solve_fp64"): (17.835e9, "ncu capture, profiles/mod_tiled_fp64_patches_local_L256_K512.md"),
    ("splitmerge", "mod_solve_fp64"): (53.3e6, "ncu capture, profiles/mod_tiled_fp64_splitmerge_local_L100_K256.md"),
}

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------ clocks ------
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    mhz.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(mhz)) if mhz else None, "sm_max_mhz": mx,
                "samples": len(mhz), "reasons": sorted(reasons)}


# ------------------------------------------------------------ workload ------
# Relative tolerance of "reaches the plain form's RMSE": the run-to-run spread of
# the final RMSE among forms of the same algorithm that differ only in rounding.
RMSE_TOL = 5e-3


def counts(p):
    """OMP-coded signals per step: local passes, merge passes, final coding."""
    local = p.iters_local * p.N
    merge = p.iters_merge * p.K1 * p.L
    return local + merge + p.N


def algorithmic_work(p):
    """Per-step algorithmic flops of each kernel family (unit figures x units)."""
    m, K, K1, L = p.m, p.K, p.K1, p.L
    nm = p.K1 * p.L
    def omp_flops(K_, s_):          # 2mK (alpha0) + K s (s+1) (Batch-OMP updates)
        return 2 * m * K_ + K_ * s_ * (s_ + 1)
    return {
        # FP64 MOD solve per system: Cholesky K^3/3 + forward and back substitution
        # of m right-hand sides 2 K^2 m
        "mod_solve_fp64": ("alu", p.iters_local * L * (K1 ** 3 / 3 + 2 * K1 ** 2 * m)),
        "mod_solve_fp64_single": ("alu", p.iters_merge * (K ** 3 / 3 + 2 * K ** 2 * m)),
        # the checked FP32 pass of the same solve (FP32 data)
        "mod_solve_fp32": ("alu", p.iters_local * L * (K1 ** 3 / 3 + 2 * K1 ** 2 * m)),
        "mod_solve_fp32_single": ("alu", p.iters_merge * (K ** 3 / 3 + 2 * K ** 2 * m)),
        "chol_fp64": ("alu", p.iters_local * L * K1 ** 3 / 3 + p.iters_merge * K ** 3 / 3),
        "solve_fp64": ("alu", p.iters_local * L * 2 * K1 ** 2 * m + p.iters_merge * 2 * K ** 2 * m),
        "omp": ("alu", p.iters_local * p.N * omp_flops(K1, p.s1) + p.iters_merge * nm * omp_flops(K, p.s2)
                + p.N * omp_flops(K, p.s)),
        "omp_split": ("alu", p.iters_local * p.N * omp_flops(K1, p.s1) + p.iters_merge * nm * omp_flops(K, p.s2)
                      + p.N * omp_flops(K, p.s)),
        "omp_tc": ("alu", p.iters_local * p.N * omp_flops(K1, p.s1) + p.iters_merge * nm * omp_flops(K, p.s2)
                   + p.N * omp_flops(K, p.s)),
        "omp_x3": ("alu", p.iters_local * p.N * omp_flops(K1, p.s1) + p.iters_merge * nm * omp_flops(K, p.s2)
                   + p.N * omp_flops(K, p.s)),
        "omp_tf32": ("alu", p.iters_local * p.N * omp_flops(K1, p.s1) + p.iters_merge * nm * omp_flops(K, p.s2)
                     + p.N * omp_flops(K, p.s)),
        # residual form: D^T r of every step on the tensor cores (2 m K s per signal)
        "omp_rtc": ("tensor", 2 * m * (p.iters_local * p.N * K1 * p.s1 + p.iters_merge * nm * K * p.s2 + p.N * K * p.s)),
        "gram": ("alu", p.iters_local * L * 2 * K1 * K1 * m + p.iters_merge * 2 * K * K * m),
    }


def max_over_ranks(v: float, world: int, device) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, world: int, steps: int, max_total_ms: float) -> float:
    """Units all ranks processed over `steps` steps per second of the slowest
    rank's timed total."""
    return world * units_per_rank_step * steps / (max_total_ms / 1e3)


def _timed_steps(step, inputs, steps, flush, stream, clk=None):
    """Run `steps` steps with the L2 flushed before each; CUDA events on `stream`
    around each step.  Returns (per-step ms list, last outputs)."""
    import torch
    ms, out = [], None
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = step(*inputs)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, out


def make_workload(name):
    """The problem of a bench workload and its per-step inputs as host arrays:
    (Y, perm, picks, fill, mpick, D_merge0), None where the workload has none."""
    if name == "patches":
        p = si.config4()
        host = (p.Y, p.perm, p.picks.reshape(-1), p.fill.reshape(-1, p.m), None, p.extra["D_merge0"])
    else:
        p = si.config1()
        host = (p.Y, p.perm, p.picks.reshape(-1), None, p.mpick, None)
    return p, host


def workload_config(p, name, world=1):
    """The `config` object of the JSON line: the same in both arms."""
    return {"workload": WORKLOADS[name], "m": p.m, "N": p.N, "L": p.L, "n": int(p.N // p.L), "K1": p.K1,
            "K": p.K, "s1": p.s1, "s2": p.s2, "s_final": p.s, "iters_local": p.iters_local,
            "iters_merge": p.iters_merge,
            "init": ("overcomplete DCT (256x512 local, 256x1024 merge)" if name == "patches"
                     else "random distinct signals of each subset (local), random stacked columns (merge)"),
            "l2": "flushed between timed steps (512 MB write); the inputs are also larger than L2",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


class Forms:
    """The chosen, FP32 and plain forms of one workload's step on one device.
    Every step reuses the same output buffers, so repeated steps present the
    same pointers to the library (its cached training-loop graphs apply)."""

    def __init__(self, sdl, p, dev):
        import torch
        self.sdl, self.p, self.dev = sdl, p, dev
        self.Yp = torch.empty((p.N, p.m), dtype=torch.float32, device=dev)
        self.Dl = torch.empty((p.L * p.K1, p.m), dtype=torch.float32, device=dev)
        self.xfro = torch.empty((p.L,), dtype=torch.float64, device=dev)
        self.D = torch.empty((p.K, p.m), dtype=torch.float32, device=dev)

    def step(self, inp, prec, s1=None):
        """Every subset of a phase in one batched launch per kernel, launch
        shapes chosen by the library's autotuner; coding passes in `prec`.
        Returns (D, (||Y - D X||^2, ||Y||^2), final idx, final val)."""
        sdl, p = self.sdl, self.p
        Y, perm, picks, fill, mpick, Dm0 = inp
        Yp = sdl.split(Y, perm, out=self.Yp)
        Dl = sdl.init_dict(Yp, picks, fill, out=self.Dl).view(p.L, p.K1, p.m)
        xfro, _ = sdl.local_train(Yp, p.offsets, Dl, s1 or p.s1, p.iters_local, prec=prec, with_rmse=False,
                                  xfro=self.xfro)
        D, _ = sdl.merge(Dl, xfro, mpick, p.K, p.s2, p.iters_merge, prec=prec, with_rmse=False, D_init=Dm0,
                         out=self.D)
        idx, val, nnz, _ = sdl.omp(D, Y, p.s, prec=prec, with_resid=False)
        return D, sdl.residual(Y, D, idx, val), idx, val

    def plain(self, inp, subsets=None, iters=None):
        """Plain form: the same algorithm with one launch sequence per subset
        (FP32 CUDA-core OMP, no graph capture).  `subsets`/`iters` < the
        workload's run a warm-up of those launch shapes only."""
        import torch
        sdl, p = self.sdl, self.p
        Y, perm, picks, fill, mpick, Dm0 = inp
        Yp = sdl.split(Y, perm)
        Dl = sdl.init_dict(Yp, picks, fill).view(p.L, p.K1, p.m)
        xfro = torch.empty((p.L,), dtype=torch.float64, device=self.dev)
        for t in range(p.L if subsets is None else subsets):
            a, b = int(p.offsets[t]), int(p.offsets[t + 1])
            xf, _ = sdl.local_train(Yp[a:b], [0, b - a], Dl[t:t + 1], p.s1, iters or p.iters_local,
                                    prec=sdl.PREC_F32, with_rmse=False)
            xfro[t:t + 1] = xf
        if subsets is not None:
            return None
        D, _ = sdl.merge(Dl, xfro, mpick, p.K, p.s2, p.iters_merge, prec=sdl.PREC_F32, with_rmse=False,
                         D_init=Dm0)
        idx, val, nnz, _ = sdl.omp(D, Y, p.s, prec=sdl.PREC_F32, with_resid=False)
        return D, sdl.residual(Y, D, idx, val), idx, val


def precision_error(p, Y_np, D, idx, val, n_sample, seed=11):
    """Error of a coding pass against the FP64 oracle on sampled signals: the
    oracle codes the same signals against the same (GPU-trained) dictionary.
    Reports the fraction of supports that differ, the largest coefficient error
    relative to the signal's largest coefficient where supports agree, and the
    sample's RMSE from the GPU's codes next to the oracle's."""
    import oracle
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(Y_np), n_sample, replace=False))
    D64 = D.cpu().numpy().astype(np.float64)
    Ys = Y_np[pick].astype(np.float64)
    import torch
    sel = torch.from_numpy(pick).to(idx.device)
    gi = idx[sel].cpu().numpy()
    gv = val[sel].cpu().numpy().astype(np.float64)
    o = oracle.omp(D64, Ys, p.s)
    same = (gi == o["idx"]).all(axis=1)
    scale = np.maximum(np.abs(o["val"]).max(axis=1, keepdims=True), 1e-300)
    cerr = (np.abs(gv - o["val"]) / scale)[same]

    def rmse(ix, vx):
        xs = np.where(ix >= 0, vx, 0.0)
        rec = np.einsum("ns,nsm->nm", xs, D64[np.maximum(ix, 0)])
        return float(np.sqrt(((Ys - rec) ** 2).sum() / Ys.size))
    rg, ro = rmse(gi, gv), rmse(o["idx"], o["val"])
    return {"signals": int(n_sample), "support_disagreement": float(1 - same.mean()),
            "max_coef_rel_err_same_support": float(cerr.max()) if cerr.size else None,
            "rmse_gpu": rg, "rmse_oracle": ro, "rmse_rel_delta": (rg - ro) / ro}


def run_main(args, rank, world, local_rank, name, extra_key=False):
    """The main line of workload `name` (or, with extra_key, the dictionary
    that goes under an extra key of another workload's line)."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", local_rank)
    p, host = make_workload(name)
    host_t = tuple(None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in host)
    inputs = tuple(None if a is None else a.to(dev) for a in host_t)
    torch.cuda.synchronize()
    ctx = sdl.context(local_rank)
    stream = torch.cuda.current_stream(dev)
    forms = Forms(sdl, p, dev)
    steps, warmup = (args.steps, args.warmup) if not extra_key else (max(3, min(args.steps, 10)), 3)
    n_sig = counts(p)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    precs = {"f32x3": sdl.PREC_F32X3, "bf16": sdl.PREC_BF16, "fp32": sdl.PREC_F32, "tf32": sdl.PREC_TF32}
    chosen = args.chosen_prec

    def step(*inp):
        return forms.step(inp, precs[chosen])

    # ---- chosen form, device-resident timed region: training loops replayed as
    # CUDA graphs (the first warm-up step runs eagerly and tunes, the next
    # captures), no instrumentation inside
    ctx.set_option(sdl.OPT_GRAPH, 1)
    for _ in range(max(warmup, 3)):
        step(*inputs)
    launches0 = ctx.launch_count()
    barrier()
    with ClockSampler(local_rank) as clk:
        ms, (D, out2, fidx, fval) = _timed_steps(step, inputs, steps, flush, stream)
    barrier()
    launches = ctx.launch_count() - launches0
    clocks = clk.summary()
    total_ms = max_over_ranks(float(sum(ms)), world, dev)
    r2, y2 = out2.cpu().tolist()
    value = whole_job_rate(n_sig, world, steps, total_ms)
    rmse = float(np.sqrt(r2 / (p.m * p.N)))
    perr = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        perr = {chosen: precision_error(p, host[0], D, fidx, fval, args.error_sample)}
    del fidx, fval

    # ---- the same form with the other coding precisions (graphs as above)
    labels = {"fp32": "FP32 CUDA-core correlations and Gram",
              "bf16": "BF16 tensor-core correlations and Gram (two-term split) with an FP32 correction step",
              "f32x3": "FP32-accurate tensor-core correlations and Gram (two-term TF32 split)",
              "tf32": "single-product TF32 tensor-core correlations, the TF32-split Gram, an FP32 correction step"}
    alt_forms = {}
    for alt in [a for a in ("fp32", "bf16", "tf32", "f32x3") if a != chosen]:
        fsteps = min(steps, 3)
        for _ in range(3):
            forms.step(inputs, precs[alt])
        barrier()
        fms, (fD, fout2, gidx, gval) = _timed_steps(lambda *inp: forms.step(inp, precs[alt]), inputs, fsteps,
                                                    flush, stream)
        ftot = max_over_ranks(float(sum(fms)), world, dev)
        fr2, _ = fout2.cpu().tolist()
        if perr is not None:
            perr[alt] = precision_error(p, host[0], fD, gidx, gval, args.error_sample)
        del gidx, gval
        alt_forms[alt + "_form"] = {"value": whole_job_rate(n_sig, world, fsteps, ftot), "unit": UNIT,
                                    "steps": fsteps, "ms_per_step": ftot / fsteps,
                                    "rmse_final": float(np.sqrt(fr2 / (p.m * p.N))),
                                    "form": "the chosen form with " + labels[alt]}

    # ---- the same steps eagerly with CUDA events around every launcher: the
    # per-kernel device times of the roofline and the breakdown (instrumented
    # calls run eagerly; the cached graphs stay for the end-to-end pass)
    psteps = min(steps, 3)
    ctx.profile(True)
    ctx.profile_reset()
    barrier()
    prof_ms, _ = _timed_steps(step, inputs, psteps, flush, stream)
    barrier()
    prof = ctx.profile_read()
    ctx.profile(False)
    prof_total_ms = float(sum(prof_ms))

    # ---- end to end: pinned host inputs -> device, step, result -> host, every step
    D_host = torch.empty((p.K, p.m), dtype=torch.float32).pin_memory()
    out_host = torch.empty((2,), dtype=torch.float64).pin_memory()

    # The inputs are copied into device buffers allocated once (a caller streaming
    # batches would do the same), so every step presents the same pointers and
    # the cached training-loop graphs apply; warm-up as for the device-resident
    # steps.
    dev_in = tuple(None if a is None else torch.empty(a.shape, dtype=a.dtype, device=dev) for a in host_t)

    def step_e2e(*inp_h):
        for b, a in zip(dev_in, inp_h):
            if a is not None:
                b.copy_(a, non_blocking=True)
        Dd, o2, _, _ = step(*dev_in)
        D_host.copy_(Dd, non_blocking=True)
        out_host.copy_(o2, non_blocking=True)
        return Dd, o2

    for _ in range(max(warmup, 3)):
        step_e2e(*host_t)
    barrier()
    e2e_ms, _ = _timed_steps(step_e2e, host_t, steps, flush, stream)
    e2e_total = max_over_ranks(float(sum(e2e_ms)), world, dev)
    h2d = sum(t.numel() * t.element_size() for t in host_t if t is not None)
    d2h = D_host.numel() * 4 + 16

    # ---- plain form (per-subset launch sequences), fewer steps: it is slow by
    # design.  Its warm-up runs one subset for one iteration (the per-subset
    # launch shapes); the merge and final coding shapes are the chosen form's.
    plain = None
    ctx.set_option(sdl.OPT_GRAPH, 0)
    if args.plain_steps > 0:
        forms.plain(inputs, subsets=1, iters=1)
        barrier()
        pms, (_, pout2, _, _) = _timed_steps(lambda *inp: forms.plain(inp), inputs, args.plain_steps, flush,
                                             stream)
        ptot = max_over_ranks(float(sum(pms)), world, dev)
        pr2, _ = pout2.cpu().tolist()
        prmse = float(np.sqrt(pr2 / (p.m * p.N)))
        plain = {"value": whole_job_rate(n_sig, world, args.plain_steps, ptot), "unit": UNIT,
                 "ms_per_step": ptot / args.plain_steps, "steps": args.plain_steps,
                 "train_to_rmse_s": ptot / args.plain_steps / 1e3, "rmse_final": prmse,
                 "form": f"one launch sequence per subset ({p.L} local trainings in turn), FP32 CUDA-core OMP, "
                         "FP64 MOD solve, no proposer, no graph capture",
                 "chosen_speedup": (ptot / args.plain_steps) / (total_ms / steps),
                 "target_rmse": prmse * (1 + RMSE_TOL),
                 "target_rule": f"the plain form's final RMSE x (1 + {RMSE_TOL}): forms that differ only in rounding "
                                "(FP64 or FP32 MOD solve, FP32, FP32-accurate or BF16 coding) end 20 + 20 "
                                "alternating iterations on different local minima, measured up to 0.5 % apart",
                 "chosen_reaches_rmse": bool(rmse <= prmse * (1 + RMSE_TOL)),
                 **{k + "_reaches_rmse": bool(v["rmse_final"] <= prmse * (1 + RMSE_TOL)) for k, v in alt_forms.items()}}

    # ---- roofline of the dominant kernel (device time measured inside the timed region)
    work = algorithmic_work(p)
    name_k, (nl, ncalls, kms) = max(prof.items(), key=lambda kv: kv[1][2])
    roof = None
    if name_k in work:
        kind, flops_step = work[name_k]
        peaks = load_peaks()
        # a kernel timed inside a long step: the sustained BF16 figure
        peak = (FP64_PEAK_FLOPS if "fp64" in name_k else
                peaks.get("bf16_tflops_sustained", 1700.0) * 1e12 if kind == "tensor" else FP32_PEAK_FLOPS)
        achieved = flops_step * psteps / (kms / 1e3)
        tr = TRAFFIC.get((name, name_k))
        roof = {"kernel": name_k, "bound": kind, "achieved": achieved / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tr[0] if tr else None, "traffic_unit": "DRAM bytes per launch",
                "traffic_source": tr[1] if tr else "no ncu capture of this kernel's current code",
                "algorithmic_flops_per_launch": flops_step / max(nl / psteps, 1),
                "peak_source": ("FP64 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived from unit counts and "
                                "the maximum clock; a DFMA probe measured 1.254 TFLOP/s)" if "fp64" in name_k else
                                "measured BF16 dense, sustained (MEASURED_PEAKS.json)" if kind == "tensor" else
                                "FP32 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz"),
                "share_of_step": kms / prof_total_ms, "launches": nl,
                "timed": "instrumented eager pass over %d steps (%.2f ms/step)" % (psteps, prof_total_ms / psteps)}
    kernels = {k: {"ms_per_step": v[2] / psteps, "launches_per_step": v[0] / psteps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])}
    omp_names = ("omp", "omp_split", "gram", "omp_tc", "omp_rtc", "gram_tc", "bf16_image", "omp_x3", "omp_tf32",
                 "gram_x3", "x3_image")
    omp_ms = sum(v[2] for k, v in prof.items() if k in omp_names) / psteps

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32x3": "tf32x3+f32+f64", "bf16": "bf16+f32+f64", "fp32": "f32+f64", "tf32": "tf32+f32+f64"}[chosen],
        "data": ("synthetic images (seeded piecewise-smooth fields + noise 0.1), 16x16 patches"
                 if name == "patches" else "synthetic (seeded; Sec. 3.1 data model)"),
        "config": workload_config(p, name, world),
        "form": "chosen: batched (all subsets of a phase per launch), training loops replayed as CUDA graphs, "
                "autotuned MOD solve (checked FP32 solve, FP64 where the check fails or is faster), " + labels[chosen] + "; no proposer (see proposer_final_coding)",
        "signals_per_step": n_sig,
        "omp_stage": {"signals_per_s": n_sig / (omp_ms / 1e3) if omp_ms > 0 else None, "ms_per_step": omp_ms,
                      "kernels": [k for k in omp_names if k in prof],
                      "note": "coded signals per second of OMP-stage kernel time (instrumented pass); value "
                              "divides by the whole step"},
        "train_to_rmse_s": total_ms / steps / 1e3,
        "rmse_final": rmse,
        "mse_train_db": float(10 * np.log10(r2 / y2)),
        "plain": plain,
        **alt_forms,
        "precision_error": perr,
        "e2e": {"value": whole_job_rate(n_sig, world, steps, e2e_total), "unit": UNIT, "steps": steps,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernels,
        "clocks": clocks,
    }
    if name == "patches" and rank == 0 and world == 1 and not args.no_proposer:
        try:
            res["proposer_final_coding"] = patches_proposer_bench(sdl, dev, p, inputs[0], D, flush, stream)
        except Exception as exc:   # an extra measurement: report it and keep the line
            res["proposer_final_coding"] = {"error": f"{type(exc).__name__}: {str(exc)[:200]}"}
    del inputs, forms, flush
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(p, name, host[0])
        if name == "splitmerge":
            res["oracle_rmse_final"] = res["cpu_baseline"].get("oracle_rmse_final")
    return res


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    res = run_main(args, rank, world, local_rank, args.workload)
    if rank == 0 and world == 1 and args.workload == "patches" and not args.no_extra:
        # the 200,000-signal split-and-merge workload, measured in the same run
        ex = run_main(args, rank, world, local_rank, "splitmerge", extra_key=True)
        res["splitmerge_200k"] = {k: ex.get(k) for k in (
            "config", "value", "unit", "steps", "ms_per_step", "rmse_final", "oracle_rmse_final", "mse_train_db",
            "plain", "fp32_form", "bf16_form", "tf32_form", "f32x3_form", "precision_error", "e2e", "roofline", "omp_stage",
            "cpu_baseline", "clocks")}
    if rank == 0 and world == 1 and not args.no_proposer:
        flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream(dev)
        res["proposer"] = proposer_bench(sdl, dev, flush, stream)
        res["proposer"]["conditioned"] = conditioned_bench(sdl, dev, flush, stream)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def proposer_bench(sdl, dev, flush, stream):
    """Learned support proposer on its own workload (64 -> 512 -> 512 -> 256 MLP,
    D0 64 x 256, s = 6, noise 0.01): labels from plain OMP on the training
    signals, Adam training (timed), then proposer-assisted OMP (top-2s
    candidates, restricted OMP, plain OMP where ||r|| > 8.5 sigma) against plain
    OMP on fresh signals: 2^20 training pairs and 2^20 fresh evaluation
    signals, the workload's 1M / 1M (stated in the output)."""
    import torch
    n_train, n_eval, epochs, B = 1 << 20, 1 << 20, 4, 4096
    c = si.config3(n_train=n_train, n_eval=n_eval)
    D = torch.from_numpy(c["D0"]).to(dev)
    Ytr = torch.from_numpy(c["Ytr"]).to(dev)
    Yev = torch.from_numpy(c["Yev"]).to(dev)
    s, ncand, eps_fb = c["s"], 2 * c["s"], 8.5 * 0.01
    labels, *_ = sdl.omp(D, Ytr, s, with_resid=False)
    prop = sdl.Proposer(torch.from_numpy(c["params"]).to(dev), c["m"], c["h1"], c["h2"], c["K"])
    loss = torch.zeros(4, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    first = None
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for epoch in range(epochs):
        lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * epoch / epochs))
        order = torch.randperm(n_train, device=dev, generator=g)
        Ys, Is = Ytr[order], labels[order]
        for a in range(0, n_train, B):
            prop.train_step(Ys[a:a + B], Is[a:a + B], lr, loss)
            if first is None:
                first = float(loss[0])
    e1.record(stream)
    e1.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    last = float(loss[0])

    def timed(fn):
        fn()
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        out = fn()
        a1.record(stream)
        a1.synchronize()
        return a0.elapsed_time(a1) / 1e3, out

    t_plain, (pi, pv, pn, pr) = timed(lambda: sdl.omp(D, Yev, s))
    t_prop, (qi, qv, qn, qr, nf) = timed(lambda: prop.omp(D, Yev, s, ncand, eps_fb))
    same = (torch.sort(pi, dim=1).values == torch.sort(qi, dim=1).values).all(dim=1).float().mean().item()
    met = (torch.sqrt(qr) <= eps_fb).float().mean().item()
    # one more epoch, after the evaluation, with each training step bracketed
    # by events: the device time of training alone (the timed loop above also
    # holds the gaps while Python issues each step)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(0, n_train, B)]
    for q, a in enumerate(range(0, n_train, B)):
        evs[q][0].record(stream)
        prop.train_step(Ytr[a:a + B], labels[a:a + B], 1e-4, loss)
        evs[q][1].record(stream)
    evs[-1][1].synchronize()
    dev_ms = sum(b.elapsed_time(e) for b, e in evs)
    prop.close()
    return {"train_pairs": n_train, "epochs": epochs, "batch": B, "train_s": train_s,
            "train_samples_per_s": epochs * n_train / train_s,
            "train_device_samples_per_s": n_train / (dev_ms / 1e3), "loss_first": first, "loss_last": last,
            "eval_signals": n_eval, "plain_omp_signals_per_s": n_eval / t_plain,
            "proposed_omp_signals_per_s": n_eval / t_prop, "fallback_rate": nf / n_eval,
            "support_agreement_with_plain": same, "residual_within_eps_fb": met,
            "candidates": ncand, "eps_fb": eps_fb}


def patches_proposer_bench(sdl, dev, p, Y, D, flush, stream):
    """The learned proposer where one dictionary codes many signals: the image-
    patch workload's final coding (the trained 256 x 1024 dictionary, s = 16).
    An MLP 256 -> 512 -> 512 -> 1024 is trained on (patch, plain-OMP support)
    pairs of 2^18 patches for 2 epochs of Adam, its top-32 candidates feed the
    restricted OMP, and a patch falls back to full OMP where its residual norm
    exceeds eps_fb, the 99th percentile of plain OMP's own residual norms on the
    training patches (so that plain OMP meets it on 99 % of them).  Evaluated
    on 2^20 other patches against plain OMP (FP32, the fallback's coder, and
    BF16, the chosen form's); the net effect on the final coding of all N
    patches counts the training, which the proposer needs once per dictionary."""
    import torch
    n_train, n_eval, epochs, B, s = 1 << 18, 1 << 20, 2, 4096, p.s
    rng = np.random.default_rng(41)
    sel = torch.from_numpy(rng.permutation(p.N)[: n_train + n_eval]).to(dev)
    Ytr, Yev = Y[sel[:n_train]].contiguous(), Y[sel[n_train:]].contiguous()
    labels, _, _, r2 = sdl.omp(D, Ytr, s)
    eps_fb = float(torch.quantile(torch.sqrt(r2.double()), 0.99))
    prop = sdl.Proposer(torch.from_numpy(si.mlp_init(rng, p.m, 512, 512, p.K, s)).to(dev), p.m, 512, 512, p.K)
    loss = torch.zeros(4, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    first = None
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for epoch in range(epochs):
        lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * epoch / epochs))
        order = torch.randperm(n_train, device=dev, generator=g)
        Ys, Is = Ytr[order], labels[order]
        for a in range(0, n_train, B):
            prop.train_step(Ys[a:a + B], Is[a:a + B], lr, loss)
            if first is None:
                first = float(loss[0])
    e1.record(stream)
    e1.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3

    def timed(fn):
        fn()
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        out = fn()
        a1.record(stream)
        a1.synchronize()
        return a0.elapsed_time(a1) / 1e3, out

    t_f32, (pi, pv, pn, pr) = timed(lambda: sdl.omp(D, Yev, s))
    t_b16, _ = timed(lambda: sdl.omp(D, Yev, s, prec=sdl.PREC_BF16, with_resid=False))
    t_prop, (qi, qv, qn, qr, nf) = timed(lambda: prop.omp(D, Yev, s, 2 * s, eps_fb))
    scores = prop.scores(Yev[:65536])
    top = torch.topk(scores, 2 * s, dim=1).indices
    recall = (top[:, :, None] == pi[:65536, None, :].long()).any(dim=1).float().mean().item()
    same = (torch.sort(pi, dim=1).values == torch.sort(qi, dim=1).values).all(dim=1).float().mean().item()
    rm_plain = float(torch.sqrt(pr.double().sum() / (p.m * n_eval)))
    rm_prop = float(torch.sqrt(qr.double().sum() / (p.m * n_eval)))
    prop.close()
    scale = p.N / n_eval
    return {"train_pairs": n_train, "epochs": epochs, "batch": B, "train_s": train_s, "loss_first": first,
            "loss_last": float(loss[0]), "eps_fb": eps_fb, "eps_fb_rule": "99th percentile of plain OMP's ||r||",
            "candidates": 2 * s, "eval_signals": n_eval, "top32_recall_of_plain_support": recall,
            "fallback_rate": nf / n_eval, "support_agreement_with_plain": same,
            "rmse_plain": rm_plain, "rmse_proposed": rm_prop,
            "signals_per_s": {"plain_fp32": n_eval / t_f32, "plain_bf16": n_eval / t_b16, "proposed": n_eval / t_prop},
            "final_coding_s": {"plain_bf16": t_b16 * scale, "plain_fp32": t_f32 * scale,
                               "proposed_with_training": train_s + t_prop * scale},
            "pays": bool(train_s + t_prop * scale < t_b16 * scale)}


def conditioned_bench(sdl, dev, flush, stream):
    """Dictionary-conditioned proposer: one network (256 -> 512 -> 512 -> 256)
    reading |D_t^T y| serves L = 64 dictionaries (64 x 256 unit atoms each),
    every subset 8,192 signals sparse over its own dictionary (s = 6, noise
    0.01).  Labels from plain batched OMP, 4 epochs of Adam at batch 4,096.
    Evaluated on 8,192 fresh signals per subset, and on 8 dictionaries the
    network never saw: top-12 recall of the plain-OMP supports against the
    ranking by |D_t^T y| alone (OMP's first step), fallback rate at 8.5 sigma,
    and coded signals per second against plain batched OMP."""
    import torch
    L, n_t, m, K, s, sigma, h, B, epochs = 64, 8192, 64, 256, 6, 0.01, 512, 4096, 4
    rng = np.random.default_rng(31)

    def batch(nd):
        Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in range(nd)])
        Y = np.concatenate([si.sparse_signals(rng, Ds[t], n_t, s, sigma, dtype=np.float32)[0] for t in range(nd)])
        off = np.arange(nd + 1, dtype=np.int64) * n_t
        return torch.from_numpy(Ds.astype(np.float32)).to(dev), torch.from_numpy(Y).to(dev), off, Ds

    Dg, Ytr, off, D64 = batch(L)
    Yev = torch.from_numpy(np.concatenate([si.sparse_signals(rng, D64[t], n_t, s, sigma, dtype=np.float32)[0]
                                           for t in range(L)])).to(dev)
    Du, Yu, offu, _ = batch(8)
    labels, *_ = sdl.omp_batched(Dg, Ytr, off, s, with_resid=False)
    Ftr = sdl.corr_features(Dg, Ytr, off)
    prop = sdl.Proposer(torch.from_numpy(si.mlp_init(rng, K, h, h, K, s)).to(dev), K, h, h, K)
    loss = torch.zeros(4, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(4)
    first = None
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n = Ftr.shape[0]
    for epoch in range(epochs):
        lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * epoch / epochs))
        order = torch.randperm(n, device=dev, generator=g)
        Fs, Ls = Ftr[order], labels[order]
        for a in range(0, n, B):
            prop.train_step(Fs[a:a + B], Ls[a:a + B], lr, loss)
            if first is None:
                first = float(loss[0])
    e1.record(stream)
    e1.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    del Ftr, Ls, Fs

    def recall(D, Y, offs, nc):
        lab, *_ = sdl.omp_batched(D, Y, offs, s, with_resid=False)
        F = sdl.corr_features(D, Y, offs)
        out = []
        for sc in (prop.scores(F), F):
            top = torch.topk(sc, nc, dim=1).indices
            out.append((top[:, :, None] == lab[:, None, :].long()).any(dim=1).float().mean().item())
        return out

    ncand, eps_fb = 2 * s, 8.5 * sigma
    r_net, r_corr = recall(Dg, Yev, off, ncand)
    u_net, u_corr = recall(Du, Yu, offu, ncand)

    def timed(fn):
        fn()
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        out = fn()
        a1.record(stream)
        a1.synchronize()
        return a0.elapsed_time(a1) / 1e3, out

    t_plain, (pi, *_) = timed(lambda: sdl.omp_batched(Dg, Yev, off, s))
    t_prop, (qi, qv, qn, qr, nf) = timed(lambda: prop.omp_batched(Dg, Yev, off, s, ncand, eps_fb))
    same = (torch.sort(pi, dim=1).values == torch.sort(qi, dim=1).values).all(dim=1).float().mean().item()
    # one more pass with the library's per-kernel events: where the time goes
    ctx = sdl.context(dev.index or 0)
    ctx.profile(True)
    ctx.profile_reset()
    prop.omp_batched(Dg, Yev, off, s, ncand, eps_fb)
    prof = ctx.profile_read()
    ctx.profile(False)
    prop.close()
    ne = Yev.shape[0]
    return {"dictionaries": L, "signals_per_dictionary": n_t, "train_pairs": n, "epochs": epochs,
            "train_s": train_s, "loss_first": first, "loss_last": float(loss[0]),
            "recall_at_12": {"network_on_abs_Dty": r_net, "abs_Dty_ranking": r_corr},
            "recall_at_12_unseen_dictionaries": {"network_on_abs_Dty": u_net, "abs_Dty_ranking": u_corr},
            "eval_signals": ne, "plain_batched_omp_signals_per_s": ne / t_plain,
            "proposed_batched_omp_signals_per_s": ne / t_prop, "fallback_rate": nf / ne,
            "support_agreement_with_plain": same, "candidates": ncand, "eps_fb": eps_fb,
            "proposed_pass_kernel_ms": {k: round(v[2], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])}}


def run_proposer(args):
    """The learned-proposer workload (config of 2^20 training and 2^20
    evaluation pairs, m=64, K=256, s=6) alone, printed as its own line."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    res = {"metric": METRIC, "workload": "proposer_m64_K256_s6_train1048576_eval1048576",
           "data": "synthetic (seeded; Sec. 3.1 data model)",
           **proposer_bench(sdl, dev, flush, torch.cuda.current_stream(dev))}
    print(json.dumps(res), flush=True)


def run_conditioned(args):
    """The dictionary-conditioned proposer workload alone, printed as its own line."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    res = {"metric": METRIC, "workload": "conditioned_proposer_L64_m64_K256_s6_n8192",
           "data": "synthetic (seeded; Sec. 3.1 data model, one dictionary per subset)",
           **conditioned_bench(sdl, dev, flush, torch.cuda.current_stream(dev))}
    print(json.dumps(res), flush=True)


def run_uneven(args, shape):
    """The uneven batched local-training workload (512 subsets, sizes on
    [500, 8000]; shape A m=64/K=256/s=6 or B m=144/K=512/s=10): all subsets
    trained for 20 iterations in one batched launch per kernel, BF16 tensor-core
    correlations and Gram (the workload's precision) and the FP32 CUDA-core path
    beside it.  A measurement of a parity workload, printed as its own line."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    p = si.config2(shape)
    Yg = sdl.split(torch.from_numpy(p.Y).to(dev), torch.from_numpy(p.perm).to(dev))
    D0 = sdl.init_dict(Yg, torch.from_numpy(p.picks.reshape(-1)).to(dev),
                       torch.from_numpy(p.fill.reshape(-1, p.m)).to(dev)).reshape(p.L, p.K1, p.m)
    ctx = sdl.context(0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, prec in (("bf16", sdl.PREC_BF16), ("fp32", sdl.PREC_F32)):
        D = D0.clone()
        sdl.local_train(Yg, p.offsets, D, p.s1, 1, prec=prec, with_rmse=False)   # warm-up, autotune
        D = D0.clone()
        flush.zero_()
        ctx.profile(True)
        ctx.profile_reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(stream)
            _, rmse = sdl.local_train(Yg, p.offsets, D, p.s1, p.iters_local, prec=prec)
            e1.record(stream)
            e1.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        ms = e0.elapsed_time(e1)
        r = rmse.cpu().numpy()
        w = (np.diff(p.offsets) * p.m).astype(np.float64)
        out[name] = {"value": p.iters_local * p.N / (ms / 1e3), "unit": UNIT, "ms": ms,
                     "ms_per_iteration": ms / p.iters_local,
                     "rmse_last": float(np.sqrt((r[:, -1] ** 2 * w).sum() / w.sum())),
                     "kernels": {k: round(v[2], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])},
                     "clocks": clk.summary()}
    res = {"metric": METRIC, "workload": p.name, "L": p.L, "N": p.N, "m": p.m, "K": p.K, "s": p.s1,
           "iters": p.iters_local, "sizes": [int(np.diff(p.offsets).min()), int(np.diff(p.offsets).max())],
           "data": "synthetic (seeded; uneven batched workload)", **out}
    print(json.dumps(res), flush=True)


def run_denoise(args):
    """Image denoising as in the paper's image experiment (Sec. 3.2), on
    synthetic images: dictionaries trained on 10^5 clean 8x8 patches, by
    split-and-merge (20 subsets of 5,000, K1=128, s1=4, merged to K=256 with
    s2=2) and by the standard approach (K=256, s=8), both from overcomplete DCT
    dictionaries with 20 (+20) iterations; a new noisy image (sigma = 20/255)
    denoised with each and with the DCT itself (every overlapping patch coded
    to ||r|| <= 8.5 sigma, at most 32 atoms, estimates averaged per pixel).
    Both trainings are repeated with atom replacement (atoms no training patch
    uses become the worst-coded patches after every MOD update).
    A measurement of a widening workload, printed as its own line."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    rng = si.rng_for(5)
    train = np.concatenate([si.random_patches(rng, si.synthetic_image(rng, sigma=0.0), 12_500, 8)
                            for _ in range(8)]).astype(np.float32)
    clean = si.synthetic_image(rng, sigma=0.0)
    sigma = 20 / 255
    noisy = (clean + sigma * rng.standard_normal(clean.shape)).astype(np.float32)
    L, n = 20, 5000
    perm, offsets = si.random_partition(rng, [n] * L)
    D_loc0 = si.overcomplete_dct(8, 8, 16).astype(np.float32)
    D_mer0 = si.overcomplete_dct(8, 16, 16).astype(np.float32)
    Y = torch.from_numpy(train).to(dev)
    Yp = sdl.split(Y, torch.from_numpy(perm).to(dev))
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    def split_merge():
        Dl = torch.from_numpy(np.broadcast_to(D_loc0, (L, 128, 64)).copy()).to(dev)
        xf, _ = sdl.local_train(Yp, offsets, Dl, 4, 20, with_rmse=False)
        D, _ = sdl.merge(Dl, xf, None, 256, 2, 20, with_rmse=False, D_init=torch.from_numpy(D_mer0).to(dev))
        return D

    def standard():
        D = torch.from_numpy(D_mer0.copy()).to(dev)[None]
        sdl.local_train(Y, [0, len(train)], D, 8, 20, with_rmse=False)
        return D[0]

    ctx = sdl.context(0)
    split_merge(), standard()   # warm-up: autotuner, workspace
    t_sm, D_sm = timed(split_merge)
    t_std, D_std = timed(standard)
    # the same trainings with atom replacement after every MOD update (min_use 1)
    ctx.set_option(sdl.OPT_REPLACE, 1)
    try:
        split_merge(), standard()
        t_smr, D_smr = timed(split_merge)
        t_stdr, D_stdr = timed(standard)
        ctx.profile(True)
        ctx.profile_reset()
        split_merge()
        prof = ctx.profile_read()
        ctx.profile(False)
    finally:
        ctx.set_option(sdl.OPT_REPLACE, 0)
    ng = torch.from_numpy(noisy).to(dev)
    cg = torch.from_numpy(clean.astype(np.float32)).to(dev)

    def psnr(img):
        e2 = sdl.sq_error(img, cg).cpu().numpy()[0]
        return float(10 * np.log10(img.numel() / e2))

    def unused_atoms(D, s):
        idx = sdl.omp(D, Y, s, with_resid=False)[0]
        return int(D.shape[0] - torch.unique(idx[idx >= 0]).numel())

    out = {"train_s": {"split_merge": t_sm, "standard": t_std, "split_merge_replace": t_smr,
                       "standard_replace": t_stdr},
           "replace_kernel": {"ms_per_launch": prof["replace"][2] / max(prof["replace"][0], 1),
                              "launches": prof["replace"][0],
                              "share_of_training": prof["replace"][2] / sum(v[2] for v in prof.values())},
           "psnr_noisy": psnr(ng)}
    for name, D, s_tr in (("split_merge", D_sm, 2), ("standard", D_std, 8), ("split_merge_replace", D_smr, 2),
                          ("standard_replace", D_stdr, 8), ("dct", torch.from_numpy(D_mer0).to(dev), 8)):
        sdl.denoise(ng, D, 8, 8.5 * sigma)
        t, (den, (idx, val, nnz)) = timed(lambda: sdl.denoise(ng, D, 8, 8.5 * sigma))
        out[name] = {"psnr": psnr(den), "denoise_s": t, "patches_per_s": idx.shape[0] / t,
                     "mean_atoms": float(nnz.float().mean()), "atoms_unused_on_training_patches": unused_atoms(D, s_tr)}
    res = {"metric": METRIC, "workload": "denoise_synthetic_512x512_sigma20", "train_patches": len(train),
           "data": "synthetic piecewise-smooth images (seeded), pixel values in [0, 1]", **out}
    print(json.dumps(res), flush=True)


def run_coding(args):
    """One OMP coding pass of 2^19 signals (m=256, K=512, s=8, noise 0.02, one
    dictionary) with FP32 CUDA-core correlations, with FP32-accurate
    tensor-core ones (two-term TF32 split), with single-product TF32 ones,
    with BF16 tensor-core ones
    (Batch-OMP selection) and with the BF16 residual form: the shape where the
    correlation GEMM is most of the arithmetic.  Printed as its own line; also
    the small case the tensor-core kernels are profiled on."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    rng = si.rng_for(6)
    m, K, s, n = 256, 512, 8, 1 << 19
    D0 = si.unit_gaussian_atoms(rng, m, K)
    Y, _, _ = si.sparse_signals(rng, D0, n, s, 0.02, dtype=np.float32)
    D = torch.from_numpy(D0.astype(np.float32)).to(dev)
    Yg = torch.from_numpy(Y).to(dev)
    ctx = sdl.context(0)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, prec, form in (("fp32", sdl.PREC_F32, 0), ("f32x3", sdl.PREC_F32X3, 0), ("tf32", sdl.PREC_TF32, 0),
                             ("bf16", sdl.PREC_BF16, 1), ("bf16_residual_form", sdl.PREC_BF16, 2)):
        ctx.set_option(sdl.OPT_BF16_FORM, form)
        sdl.omp(D, Yg, s, prec=prec)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sdl.omp(D, Yg, s, prec=prec)
        e1.record(stream)
        e1.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        ms = e0.elapsed_time(e1)
        out[name] = {"signals_per_s": n / (ms / 1e3), "ms": ms,
                     "kernels": {k: round(v[2], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])}}
    ctx.set_option(sdl.OPT_BF16_FORM, 0)
    res = {"metric": METRIC, "workload": "coding_m256_K512_s8_n524288", "correlation_tflop": 2 * m * K * n / 1e12,
           "data": "synthetic (seeded; Sec. 3.1 data model)", **out}
    print(json.dumps(res), flush=True)


def run_coding_final(args):
    """The image-patch workload's final coding shape alone: 2^20 patches coded
    with s=16 against the 1024-atom overcomplete DCT (256 x 1024), with BF16
    correlations (Batch-OMP selection and the residual form), single-product
    TF32, FP32-accurate (F32X3) and FP32 CUDA-core ones.  The small case the
    s=16 selection kernel is profiled on; printed as its own line."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    p = si.config4(n_images=64, per_image=16384, L=64)
    Y = torch.from_numpy(p.Y).to(dev)
    D = torch.from_numpy(p.extra["D_merge0"]).to(dev)
    s = p.extra["s_final"]
    ctx = sdl.context(0)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, prec, form in (("bf16", sdl.PREC_BF16, 1), ("bf16_residual_form", sdl.PREC_BF16, 2),
                             ("tf32", sdl.PREC_TF32, 0), ("f32x3", sdl.PREC_F32X3, 0), ("fp32", sdl.PREC_F32, 0)):
        ctx.set_option(sdl.OPT_BF16_FORM, form)
        sdl.omp(D, Y, s, prec=prec, with_resid=False)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sdl.omp(D, Y, s, prec=prec, with_resid=False)
        e1.record(stream)
        e1.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        ms = e0.elapsed_time(e1)
        out[name] = {"signals_per_s": p.N / (ms / 1e3), "ms": ms,
                     "kernels": {k: round(v[2], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])}}
    ctx.set_option(sdl.OPT_BF16_FORM, 0)
    print(json.dumps({"metric": METRIC, "workload": f"coding_final_m256_K1024_s{s}_n{p.N}", **out}), flush=True)


def run_mod_local(args):
    """The local MOD update of the image-patch workload's shape, alone: 256
    subsets, K1=512 atoms, m=256, codes of s1=4 from the overcomplete DCT
    (by default 32 synthetic images of 16,384 patches, 2,048 per subset: the
    solve's cost does not depend on n; --mod-local-images sets the image count).  The
    third call of the default (checked mixed-precision) solve is bracketed by
    cudaProfilerStart/Stop, so a profiler started with profiling off captures
    exactly one accumulation, the FP32 pass, its check and the FP64 pass of
    what the check left, in the bench's launch configuration.  Then the FP64
    solve alone (SDL_OPT_MOD_MIXED 0) for comparison.  The small case the MOD
    kernels are profiled on; printed as its own line."""
    import torch

    import paper_1403_4781_gb300 as sdl

    dev = torch.device("cuda", 0)
    p = si.config4(n_images=args.mod_local_images, per_image=16384, L=256)
    Yp = sdl.split(torch.from_numpy(p.Y).to(dev), torch.from_numpy(p.perm).to(dev))
    D = torch.from_numpy(np.broadcast_to(p.extra["D_local0"], (p.L, p.K1, p.m)).copy()).to(dev)
    idx, val, _, _ = sdl.omp_batched(D, Yp, p.offsets, p.s1, prec=sdl.PREC_BF16, with_resid=False)
    ctx = sdl.context(0)
    flops = p.L * (p.K1 ** 3 / 3 + 2 * p.K1 ** 2 * p.m)
    out = {}
    for mixed in (1, 0):
        ctx.set_option(sdl.OPT_MOD_MIXED, mixed)
        for _ in range(2):   # the first call tunes the solve
            sdl.mod_update_batched(Yp, p.offsets, idx, val, D.clone())
        torch.cuda.synchronize()
        if mixed:
            torch.cuda.profiler.start()
            sdl.mod_update_batched(Yp, p.offsets, idx, val, D.clone())
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        ctx.profile(True)
        ctx.profile_reset()
        sdl.mod_update_batched(Yp, p.offsets, idx, val, D.clone())
        prof = ctx.profile_read()
        ctx.profile(False)
        kern = {k: round(v[2], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])}
        if mixed:
            ms32 = prof["mod_solve_fp32"][2]
            out["mixed"] = {"fp32_pass_ms": ms32, "fp32_pass_tflops": flops / (ms32 / 1e3) / 1e12,
                            "fp32_frac": flops / (ms32 / 1e3) / FP32_PEAK_FLOPS,
                            "check_ms": prof["mod_check"][2], "kernels": kern}
        else:
            ms = prof["mod_solve_fp64"][2]
            out["fp64"] = {"solve_ms": ms, "solve_tflops": flops / (ms / 1e3) / 1e12,
                           "fp64_frac": flops / (ms / 1e3) / FP64_PEAK_FLOPS, "kernels": kern}
    ctx.set_option(sdl.OPT_MOD_MIXED, 1)
    if args.mod_sweep:
        # the FP32 pass with the tile edge and cluster size set by hand (best of 3 calls)
        sweep = {}
        ctx.set_option(sdl.OPT_AUTOTUNE, 0)
        try:
            for ts in (32, 64):
                for C in (1, 2, 4, 8, 16):
                    ctx.set_option(sdl.OPT_MOD_TILE, ts)
                    ctx.set_option(sdl.OPT_CLUSTER, C)
                    sdl.mod_update_batched(Yp, p.offsets, idx, val, D.clone())
                    ctx.profile(True)
                    best = float("inf")
                    for _ in range(3):
                        ctx.profile_reset()
                        sdl.mod_update_batched(Yp, p.offsets, idx, val, D.clone())
                        best = min(best, ctx.profile_read()["mod_solve_fp32"][2])
                    ctx.profile(False)
                    sweep[f"tile{ts}_cluster{C}"] = round(best, 3)
        finally:
            ctx.set_option(sdl.OPT_MOD_TILE, 0)
            ctx.set_option(sdl.OPT_CLUSTER, 0)
            ctx.set_option(sdl.OPT_AUTOTUNE, 1)
        out["fp32_pass_ms_by_shape"] = sweep
    print(json.dumps({"metric": METRIC, "workload": f"mod_local_L{p.L}_K{p.K1}_m{p.m}_s{p.s1}_N{p.Y.shape[0]}", **out}),
          flush=True)


# ------------------------------------------------------------ CPU oracle ------
def _oracle_phases(p, name, Y, n_sub, local_iters, merge_iters, final_n, threads=None):
    """Run the oracle on a bounded sample of the workload, phase by phase: local
    training of the first n_sub subsets (`local_iters` iterations), a merge of
    their stacked scaled atoms (`merge_iters` iterations), the final coding of
    the first final_n signals, on `threads` host threads (default: all).
    Returns {phase: (coded signals, seconds)}, the threads used and the merge's
    last RMSE."""
    import oracle
    th = threads or oracle.default_threads()
    Yp = Y[p.perm[: p.offsets[n_sub]]].astype(np.float64)
    off = p.offsets[: n_sub + 1]
    if name == "patches":
        Dl = np.broadcast_to(p.extra["D_local0"].astype(np.float64), (n_sub, p.K1, p.m)).copy()
    else:
        Dl = np.stack([Yp[q] / np.linalg.norm(Yp[q], axis=1, keepdims=True) for q in p.picks[:n_sub]])
    out = {}
    t0 = time.perf_counter()
    loc = oracle.local_train(Yp, off, Dl, p.s1, local_iters, nthreads=th)
    out["local"] = (local_iters * int(off[-1]), time.perf_counter() - t0)
    t0 = time.perf_counter()
    if name == "patches":
        # Algorithm 1 step 3 from the overcomplete DCT: the scaled stack of the
        # local atoms trained from the given merge dictionary
        Yt = (loc["D"] * loc["xfro"][:, None, None]).reshape(-1, p.m)
        mer = oracle.train(Yt, p.extra["D_merge0"], p.s2, merge_iters, nthreads=th)
    else:
        # the whole workload merges from the GPU's initial columns; a sample
        # of fewer subsets from columns drawn among its own atoms
        pick = (p.mpick.astype(np.int32) if n_sub == p.L else
                np.random.default_rng(0).choice(n_sub * p.K1, p.K, replace=False).astype(np.int32))
        mer = oracle.merge(loc["D"], loc["xfro"], pick, p.K, p.s2, merge_iters, nthreads=th)
    out["merge"] = (merge_iters * n_sub * p.K1, time.perf_counter() - t0)
    t0 = time.perf_counter()
    fin = oracle.omp(mer["D"], Y[:final_n].astype(np.float64), p.s, nthreads=th)
    out["final"] = (final_n, time.perf_counter() - t0)
    return out, th, mer, fin


def _extrapolated_rate(p, phases):
    """Coded signals per second of a whole step, each phase's count of the
    workload at the per-signal time the sample measured for that phase."""
    whole = {"local": p.iters_local * p.N, "merge": p.iters_merge * p.L * p.K1, "final": p.N}
    step_s = sum(whole[k] * phases[k][1] / phases[k][0] for k in whole)
    return counts(p) / step_s, step_s


def cpu_baseline(p, name, Y):
    """The oracle timed on the host's cores: for the 200,000-signal workload
    one whole step (it finishes in seconds); for the image-patch workload a
    bounded sample (one subset per host thread for one local iteration, one
    merge iteration of their atoms, 8,000 final codings), extrapolated phase by
    phase to the whole step and labelled so."""
    import oracle
    th = oracle.default_threads()
    if name == "splitmerge":
        t0 = time.perf_counter()
        ph, th, mer, fin = _oracle_phases(p, name, Y, p.L, p.iters_local, p.iters_merge, p.N)
        dt = time.perf_counter() - t0
        r2 = float(oracle.residual(Y.astype(np.float64), mer["D"], fin["idx"], fin["val"])[0])
        c1 = _oracle_phases(p, name, Y, 4, p.iters_local, 4, 8000, threads=1)[0]
        v1, _ = _extrapolated_rate(p, c1)
        return {"value": counts(p) / dt, "unit": UNIT, "cores": th, "kind": "oracle",
                "sample": f"one whole step: {p.L} subsets x {p.iters_local} local iterations, merge of their "
                          f"{p.L * p.K1} atoms x {p.iters_merge} iterations, final coding of {p.N:,} signals "
                          f"({counts(p)} coded signals in {dt:.1f} s)",
                "oracle_rmse_final": float(np.sqrt(r2 / (p.m * p.N))),
                "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "extrapolated": True,
                                  "sample": "4 subsets x 20 local iterations, merge of their 1,024 atoms x 4 "
                                            "iterations, final coding of 8,000 signals, per-phase rates "
                                            "extrapolated to the whole step"}}
    n_sub = min(th, p.L)
    ph, th, _, _ = _oracle_phases(p, name, Y, n_sub, 1, 1, 8000)
    v, step_s = _extrapolated_rate(p, ph)
    return {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "extrapolated": True,
            "sample": f"{n_sub} of {p.L} subsets x 1 local iteration ({ph['local'][1]:.1f} s), one merge "
                      f"iteration of their {n_sub * p.K1} atoms ({ph['merge'][1]:.1f} s), final coding of 8,000 "
                      f"signals ({ph['final'][1]:.1f} s); each phase's per-signal time scaled to the whole "
                      f"step's count of that phase: {step_s:.0f} s per step",
            "extrapolated_step_s": step_s,
            "oracle_rmse_final": None,
            "oracle_rmse_note": "the oracle does not finish this workload within the bench; the 200,000-signal "
                                "workload's line reports the oracle's final RMSE beside the GPU's"}


def run_reference(args, rank, world):
    """The reference arm: the oracle (there is no reference implementation of
    this paper) on a bounded sample of the same workload every step, on every
    host core; rank 0 alone runs it."""
    if rank != 0:
        return
    name = args.workload if args.workload in WORKLOADS else "patches"
    p, host = make_workload(name)
    Y = host[0]
    import oracle
    # warm-up: the oracle's first calls (library load, page-in of the inputs)
    D_w = p.extra["D_merge0"] if name == "patches" else p.D0
    for _ in range(args.warmup):
        oracle.omp(D_w.astype(np.float64), Y[:500].astype(np.float64), p.s)
    th = oracle.default_threads()
    n_sub = min(th, p.L)
    li, mi, fn = (1, 1, 4000) if name == "patches" else (p.iters_local, 4, 8000)
    acc = {"local": [0, 0.0], "merge": [0, 0.0], "final": [0, 0.0]}
    t_all = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ph, th, _, _ = _oracle_phases(p, name, Y, n_sub, li, mi, fn)
        t_all += time.perf_counter() - t0
        for k, (c, s) in ph.items():
            acc[k][0] += c
            acc[k][1] += s
    value, step_s = _extrapolated_rate(p, {k: tuple(v) for k, v in acc.items()})
    sample = (f"per step: {n_sub} subsets x {li} local iterations, merge of their {n_sub * p.K1} atoms x {mi} "
              f"iterations, final coding of {fn:,} signals; per-phase rates extrapolated to the whole step "
              f"({step_s:.1f} s per whole step)")
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": workload_config(p, name, world),
        "form": "FP64 CPU oracle (plain C, every host core)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample,
                         "extrapolated": True},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-proposer", action="store_true", help="skip the proposer sub-benchmarks")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 200,000-signal split-and-merge workload's extra key")
    ap.add_argument("--chosen-prec", choices=["f32x3", "bf16", "tf32", "fp32"], default="bf16",
                    help="coding precision of the chosen form (the others are timed beside it)")
    ap.add_argument("--error-sample", type=int, default=2000,
                    help="signals of the final coding the oracle recodes for the precision error")
    ap.add_argument("--workload", choices=["patches", "splitmerge", "uneven-A", "uneven-B", "denoise", "coding",
                                           "coding-final",
                                           "conditioned", "proposer", "mod-local"],
                    default="patches",
                    help="the main line's workload (patches or splitmerge), or a parity workload measured alone")
    ap.add_argument("--mod-local-images", type=int, default=32,
                    help="--workload mod-local: synthetic images of 16,384 patches (256 at full size)")
    ap.add_argument("--mod-sweep", action="store_true",
                    help="--workload mod-local: also time the FP32 pass at every tile edge and cluster size")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed steps of the per-subset plain form (0 skips it)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload in WORKLOADS:
        run_ours(args, rank, world, local_rank)
    elif rank == 0:
        {"denoise": run_denoise, "coding": run_coding, "conditioned": run_conditioned, "proposer": run_proposer,
         "mod-local": run_mod_local, "coding-final": run_coding_final}.get(
            args.workload, lambda a: run_uneven(a, args.workload[-1]))(args)


if __name__ == "__main__":
    main()
