"""Learned support proposer (MLP 64 -> 512 -> 512 -> 256, GELU, BF16 tensor-core
products with FP32 accumulation) through the C ABI, against the FP64 oracle.

Gradients: BF16 rounding of weights and activations (u = 2^-9 per operand)
keeps the relative error of each parameter block's gradient within the BF16
tolerance 2e-2 used for every BF16 result.  Restricted OMP: for every signal it is OMP
on the sub-dictionary of its candidates, so it is compared with the oracle's
OMP on exactly that sub-dictionary."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
M, H1, H2, K, S = 64, 512, 512, 256, 6


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _data(seed, n):
    rng = np.random.default_rng(seed)
    D0 = si.unit_gaussian_atoms(rng, M, K).astype(np.float32)
    Y, sup, _ = si.sparse_signals(rng, D0.astype(np.float64), n, S, 0.01, dtype=np.float32)
    params = si.mlp_init(rng, M, H1, H2, K, S)
    return D0, Y, params


def test_gradient_matches_oracle():
    D0, Y, params = _data(500, 64)
    idx, *_ = sdl.omp(_t(D0), _t(Y), S)
    prop = sdl.Proposer(_t(params), M, H1, H2, K)
    loss, grad = prop.loss_grad(_t(Y), idx)
    torch.cuda.synchronize()
    lo, go = oracle.mlp_loss_grad(params.astype(np.float64), M, H1, H2, K, Y.astype(np.float64),
                                  idx.cpu().numpy())
    assert abs(float(loss) - lo) <= 2e-2 * abs(lo)
    g = grad.cpu().numpy().astype(np.float64)
    offs = oracle.mlp_sizes(M, H1, H2, K)
    for q, name in enumerate(["W1", "b1", "W2", "b2", "W3", "b3"]):
        a, b = offs[q], offs[q + 1]
        rel = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert rel <= 2e-2, (name, rel)


def test_loss_at_zero_weights():
    D0, Y, params = _data(501, 32)
    idx, *_ = sdl.omp(_t(D0), _t(Y), S)
    prop = sdl.Proposer(_t(np.zeros_like(params)), M, H1, H2, K)
    loss, grad = prop.loss_grad(_t(Y), idx)
    assert abs(float(loss) - K * np.log(2.0)) < 1e-4


def test_training_learns_supports_and_restricted_omp_matches_oracle():
    """Train on 2^20 (signal, plain-OMP support) pairs for 10 epochs (Adam, cosine
    learning rate from 2e-3).  The loss must fall well below the label-prior loss
    of the initial network, and the top-2s recall of the OMP supports must beat
    the untrained alternative, top-2s atoms by |d_j^T y|.  Then, for fresh signals,
    proposer-assisted OMP without fallback must equal the oracle's OMP on each
    signal's candidate sub-dictionary, and with the fallback threshold every
    accepted signal meets it while every other one carries plain OMP's code."""
    D0, Y, params = _data(502, 1 << 20)
    Dg, Yg = _t(D0), _t(Y)
    idx, *_ = sdl.omp(Dg, Yg, S)                       # labels: plain OMP supports
    prop = sdl.Proposer(_t(params), M, H1, H2, K)
    loss = torch.zeros(4, dtype=torch.float32, device=DEV)
    B, epochs, n = 4096, 10, Y.shape[0]
    first = None
    for epoch in range(epochs):
        lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * epoch / epochs))
        perm = torch.randperm(n, device=DEV)
        Ys, Is = Yg[perm], idx[perm]
        for a in range(0, n, B):
            prop.train_step(Ys[a:a + B], Is[a:a + B], lr, loss)
            if first is None:
                first = float(loss[0])
    last = float(loss[0])
    assert last < 0.6 * first, (first, last)
    rng = np.random.default_rng(503)
    Ye, _, _ = si.sparse_signals(rng, D0.astype(np.float64), 1500, S, 0.01, dtype=np.float32)
    Yeg = _t(Ye)
    ncand = 2 * S
    cand = np.argsort(-prop.scores(Yeg).cpu().numpy(), axis=1, kind="stable")[:, :ncand]
    plain = oracle.omp(D0.astype(np.float64), Ye.astype(np.float64), S)
    recall = np.mean([len(set(plain["idx"][i]) & set(cand[i])) / S for i in range(len(Ye))])
    corr = np.argsort(-np.abs(Ye @ D0.T), axis=1, kind="stable")[:, :ncand]
    recall0 = np.mean([len(set(plain["idx"][i]) & set(corr[i])) / S for i in range(len(Ye))])
    assert recall > recall0 + 0.05, (recall, recall0)
    # restricted OMP (no fallback) == oracle OMP on the candidate sub-dictionary
    gi, gv, gn, gr, nf = prop.omp(Dg, Yeg, S, ncand, 1e30)
    assert nf == 0
    gi, gv, gn, gr = (t.cpu().numpy() for t in (gi, gv, gn, gr))
    for i in range(len(Ye)):
        sub = D0[cand[i]].astype(np.float64)
        o = oracle.omp(sub, Ye[i:i + 1].astype(np.float64), S, nthreads=1)
        o["idx"] = np.where(o["idx"] >= 0, cand[i][np.maximum(o["idx"], 0)], -1)
        compare_codes(D0.astype(np.float64), Ye[i:i + 1].astype(np.float64), gi[i:i + 1], gv[i:i + 1],
                      gn[i:i + 1], gr[i:i + 1], o, fp32_gap_tol(M, np.linalg.norm(Ye[i:i + 1], axis=1)), 1e-4)
    # with the fallback threshold eps_fb = 8.5 sigma: accepted codes meet it, the rest are plain OMP
    eps_fb = 8.5 * 0.01
    fi, fv, fn, fr, nf = prop.omp(Dg, Yeg, S, ncand, eps_fb)
    fi, fr = fi.cpu().numpy(), fr.cpu().numpy()
    pi, pv, pn, pr = (t.cpu().numpy() for t in sdl.omp(Dg, Yeg, S))
    same_as_plain = (fi == pi).all(axis=1)
    accepted = np.sqrt(fr) <= eps_fb
    assert (accepted | same_as_plain).all()
    assert nf == int((~(np.sqrt(gr) <= eps_fb)).sum())
    print(f"proposer: recall@{ncand} {recall:.3f} (|D^T y| top-{ncand}: {recall0:.3f}), "
          f"fallback {nf}/{len(Ye)}")


def test_fallback_everywhere_reproduces_plain_omp():
    D0, Y, params = _data(504, 3000)
    Dg, Yg = _t(D0), _t(Y)
    prop = sdl.Proposer(_t(params), M, H1, H2, K)      # untrained: poor candidates
    gi, gv, gn, gr, nf = prop.omp(Dg, Yg, S, 2 * S, 0.0)
    assert nf == Y.shape[0]
    pi, pv, pn, pr = sdl.omp(Dg, Yg, S)
    np.testing.assert_array_equal(gi.cpu().numpy(), pi.cpu().numpy())
    np.testing.assert_allclose(gv.cpu().numpy(), pv.cpu().numpy(), rtol=0, atol=0)
