"""Learned support proposer (MLP 64 -> 512 -> 512 -> 256, GELU, BF16 tensor-core
products with FP32 accumulation) through the C ABI, against the FP64 oracle.

Forward and backward, element by element.  The GPU rounds the input, every
weight and every activation to BF16 (round to nearest, u = 2^-9), forms exact
products and accumulates in FP32 (gamma_n = n 2^-24), and keeps the logits and
the loss derivative in FP32.  Propagating those roundings through the network
to first order gives a bound for every logit and every gradient element,
computed here in numpy from the FP64 activations (magnitude sums such as
|W||h| times the unit of each rounding, carried through GELU' and GELU'').
That bound is a worst case: independent roundings add like a random walk, so
an n-term sum is typically off by about sqrt(n) u times its typical term, not
n u times it.  The GPU's logits and gradients must lie within 5 % of the bound
from the oracle's (measured: at most 0.4 %), so that a real mistake, such as
one batch element dropped from a gradient sum (about 1/B of the magnitude sum,
near the whole bound), fails.  The logits are also held to the 2e-2 BF16
tolerance relative to max(|z|, 1).  The Adam step (Kingma & Ba 2015) is
compared with the oracle's FP64 Adam applied to the GPU's own gradient.
Restricted OMP: for every signal it is OMP on the sub-dictionary of its
candidates, so it is compared with the oracle's OMP on exactly that
sub-dictionary."""
import numpy as np
import pytest
import torch
from scipy.special import erf

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
M, H1, H2, K, S = 64, 512, 512, 256, 6
U, U32 = 2.0 ** -9, 2.0 ** -24


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _data(seed, n):
    rng = np.random.default_rng(seed)
    D0 = si.unit_gaussian_atoms(rng, M, K).astype(np.float32)
    Y, sup, _ = si.sparse_signals(rng, D0.astype(np.float64), n, S, 0.01, dtype=np.float32)
    params = si.mlp_init(rng, M, H1, H2, K, S)
    return D0, Y, params


def _g(n):
    return n * U32 / (1 - n * U32)


def _gelu1(x):
    return 0.5 * (1 + erf(x / np.sqrt(2))) + x * np.exp(-0.5 * x * x) / np.sqrt(2 * np.pi)


def _gelu2(x):
    return np.exp(-0.5 * x * x) / np.sqrt(2 * np.pi) * (2 - x * x)


def _bounds(params, X, idx):
    """First-order rounding bounds of the BF16 path: per logit (eZ) and per
    packed gradient element, with the FP64 logits."""
    o = oracle.mlp_sizes(M, H1, H2, K)
    p = params.astype(np.float64)
    W1, b1 = p[o[0]:o[1]].reshape(H1, M), p[o[1]:o[2]]
    W2, b2 = p[o[2]:o[3]].reshape(H2, H1), p[o[3]:o[4]]
    W3, b3 = p[o[4]:o[5]].reshape(K, H2), p[o[5]:o[6]]
    X = X.astype(np.float64)
    A1 = X @ W1.T + b1
    Hh1 = 0.5 * A1 * (1 + erf(A1 / np.sqrt(2)))
    A2 = Hh1 @ W2.T + b2
    Hh2 = 0.5 * A2 * (1 + erf(A2 / np.sqrt(2)))
    Z = Hh2 @ W3.T + b3
    aW1, aW2, aW3, aX = np.abs(W1), np.abs(W2), np.abs(W3), np.abs(X)
    eA1 = (2 * U + _g(M)) * (aX @ aW1.T) + U32 * np.abs(A1)
    eH1 = np.abs(_gelu1(A1)) * eA1 + U * np.abs(Hh1)
    eA2 = (U + _g(H1)) * (np.abs(Hh1) @ aW2.T) + eH1 @ aW2.T + U32 * np.abs(A2)
    eH2 = np.abs(_gelu1(A2)) * eA2 + U * np.abs(Hh2)
    eZ = (U + _g(H2)) * (np.abs(Hh2) @ aW3.T) + eH2 @ aW3.T + U32 * np.abs(Z)
    B = X.shape[0]
    T = np.zeros((B, K))
    for b in range(B):
        T[b, idx[b][idx[b] >= 0]] = 1.0
    dZ = (1 / (1 + np.exp(-Z)) - T) / B
    e_dZ = 0.25 * eZ / B + U32 * np.abs(dZ)
    adZ = np.abs(dZ)
    e_gW3 = (U * adZ + e_dZ).T @ np.abs(Hh2) + adZ.T @ eH2 + _g(B) * (adZ.T @ np.abs(Hh2))
    e_gb3 = e_dZ.sum(0) + _g(B) * adZ.sum(0)
    dH2 = dZ @ W3
    e_dH2 = (2 * U * adZ + e_dZ) @ aW3 + _g(K) * (adZ @ aW3)
    dA2 = dH2 * _gelu1(A2)
    e_dA2 = e_dH2 * np.abs(_gelu1(A2)) + np.abs(dH2) * np.abs(_gelu2(A2)) * eA2 + U * np.abs(dA2)
    e_gW2 = e_dA2.T @ np.abs(Hh1) + np.abs(dA2).T @ eH1 + _g(B) * (np.abs(dA2).T @ np.abs(Hh1))
    e_gb2 = e_dA2.sum(0) + _g(B) * np.abs(dA2).sum(0)
    dH1 = dA2 @ W2
    e_dH1 = (e_dA2 + U * np.abs(dA2)) @ aW2 + _g(H2) * (np.abs(dA2) @ aW2)
    dA1 = dH1 * _gelu1(A1)
    e_dA1 = e_dH1 * np.abs(_gelu1(A1)) + np.abs(dH1) * np.abs(_gelu2(A1)) * eA1 + U * np.abs(dA1)
    e_gW1 = e_dA1.T @ aX + (U + _g(B)) * (np.abs(dA1).T @ aX)
    e_gb1 = e_dA1.sum(0) + _g(B) * np.abs(dA1).sum(0)
    eG = np.concatenate([e_gW1.ravel(), e_gb1, e_gW2.ravel(), e_gb2, e_gW3.ravel(), e_gb3])
    e_loss = (np.abs(1 / (1 + np.exp(-Z)) - T) * eZ).sum() / B
    return Z, eZ, eG, e_loss


def test_forward_scores_match_oracle_per_logit():
    D0, Y, params = _data(502, 1000)
    prop = sdl.Proposer(_t(params), M, H1, H2, K)
    Zg = prop.scores(_t(Y)).cpu().numpy().astype(np.float64)
    Zo = oracle.mlp_forward(params.astype(np.float64), M, H1, H2, K, Y.astype(np.float64))
    Zn, eZ, _, _ = _bounds(params, Y, np.full((len(Y), S), -1))
    np.testing.assert_allclose(Zn, Zo, rtol=1e-12, atol=1e-12)   # the bound's forward is the oracle's
    err = np.abs(Zg - Zo)
    ratio = err / eZ
    assert ratio.max() <= 0.05, (ratio.max(), np.unravel_index(np.argmax(ratio), ratio.shape))
    rel = err / np.maximum(np.abs(Zo), 1.0)
    assert rel.max() <= 2e-2, rel.max()
    print(f"logits: max |dz| {err.max():.2e}, max |dz| / bound {ratio.max():.3f}, max rel {rel.max():.2e}")
    prop.close()


def test_gradient_matches_oracle_per_element():
    D0, Y, params = _data(500, 64)
    idx, *_ = sdl.omp(_t(D0), _t(Y), S)
    prop = sdl.Proposer(_t(params), M, H1, H2, K)
    loss, grad = prop.loss_grad(_t(Y), idx)
    torch.cuda.synchronize()
    idx_h = idx.cpu().numpy()
    lo, go = oracle.mlp_loss_grad(params.astype(np.float64), M, H1, H2, K, Y.astype(np.float64), idx_h)
    _, _, eG, e_loss = _bounds(params, Y, idx_h)
    assert abs(float(loss) - lo) <= 1.5 * e_loss + 1e-6 * abs(lo), (float(loss), lo, e_loss)
    g = grad.cpu().numpy().astype(np.float64)
    offs = oracle.mlp_sizes(M, H1, H2, K)
    for q, name in enumerate(["W1", "b1", "W2", "b2", "W3", "b3"]):
        a, b = offs[q], offs[q + 1]
        err = np.abs(g[a:b] - go[a:b])
        ratio = err / np.maximum(eG[a:b], 1e-30)
        worst = int(np.argmax(ratio))
        assert ratio.max() <= 0.05, (name, worst, g[a + worst], go[a + worst], eG[a + worst])
        rel = err / (np.abs(go[a:b]) + 1e-2 * np.abs(go[a:b]).max())
        print(f"{name}: max |dg| / bound {ratio.max():.3f}; max |dg| / (|g| + 1e-2 max|g|) {rel.max():.2e}")
    prop.close()


def test_adam_step_matches_oracle_adam_on_the_gpu_gradient():
    """Two train_step calls against the oracle's FP64 Adam (beta1 0.9, beta2
    0.999, eps 1e-8, bias-corrected) fed the gradients the GPU forms at the same
    parameters and batches (loss_grad just before each step; the step's own
    gradient differs from it only by the order of atomic FP32 additions).
    Elements whose gradient is below 1e-3 of its first-order rounding bound have
    no determined sign; their step is only held to |step| <= 3 lr.  The rest
    must match to 1e-4 lr plus two units in the last place of the FP32
    parameter (FP32 moments and bias corrections are off by about 1e-5 of the
    step)."""
    D0, Y, params = _data(503, 128)
    idx, *_ = sdl.omp(_t(D0), _t(Y), S)
    prop = sdl.Proposer(_t(params), M, H1, H2, K)
    lr = 1e-3
    theta = params.astype(np.float64)
    mo, ve = np.zeros_like(theta), np.zeros_like(theta)
    batches = [(slice(0, 64)), (slice(64, 128))]
    idx_h = idx.cpu().numpy()
    for t, sl in enumerate(batches, start=1):
        Yb, Ib = _t(Y[sl]), idx[sl].contiguous()
        p_before = prop.params().cpu().numpy().astype(np.float64)
        _, g = prop.loss_grad(Yb, Ib)
        g = g.cpu().numpy().astype(np.float64)
        prop.train_step(Yb, Ib, lr)
        p_after = prop.params().cpu().numpy().astype(np.float64)
        theta, mo, ve = oracle.adam_step(p_before, g, mo, ve, t, lr)
        _, _, eG, _ = _bounds(p_before.astype(np.float32), Y[sl], idx_h[sl])
        sure = np.abs(g) > 1e-3 * eG
        step_gpu, step_orc = p_after - p_before, theta - p_before
        tol = 1e-4 * lr + 2 * np.spacing(np.abs(p_before).astype(np.float32)).astype(np.float64)
        err = np.abs(step_gpu - step_orc)
        bad = np.nonzero(sure & (err > tol))[0]
        assert len(bad) == 0, (t, len(bad), bad[:5], err[bad[:5]], tol[bad[:5]])
        assert np.abs(step_gpu[~sure]).max(initial=0.0) <= 3 * lr
        print(f"Adam step {t}: {sure.sum()} of {len(sure)} elements with a determined sign, "
              f"max |step error| {err[sure].max():.2e} (lr {lr})")
    prop.close()


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
