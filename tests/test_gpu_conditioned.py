"""Dictionary-conditioned support proposer through the C ABI: one network for
every dictionary of a batch, reading |D_t^T y| instead of y.

Features: each is an ordered FP32 FMA chain over the m entries of a unit atom
and the signal, within gamma_m ||y|| (gamma_m = m u / (1 - m u), u = 2^-24) of
the oracle's FP64 value.  The network's products are BF16 with FP32
accumulation (gradient tolerance 2e-2, as for the signal-input proposer).
Restricted OMP over a signal's candidates is OMP on the candidate
sub-dictionary of the signal's own dictionary, so it is compared with the
oracle's OMP there.  The fallback recodes with the batched full OMP, so with
eps_fb = 0 the codes equal sdl_omp_batched's bit for bit.  Batches above
65,536 signals cross the boundary of the feature chunks."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4781_gb300 as sdl
import sdl_inputs as si
from _parity import compare_codes, fp32_gap_tol

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
H1, H2 = 512, 512


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _gamma(m):
    u = 2.0 ** -24
    return m * u / (1 - m * u)


def _batch(seed, m, K, s, sizes, sigma=0.01):
    """One unit-atom dictionary per subset and signals sparse over it."""
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes])
    Y = np.concatenate([si.sparse_signals(rng, Ds[t], n_t, s, sigma)[0] if n_t else np.zeros((0, m))
                        for t, n_t in enumerate(sizes)])
    return rng, Ds.astype(np.float32), Y.astype(np.float32), off


@pytest.mark.parametrize("m,K", [(64, 256), (37, 130), (256, 1024), (8, 16)])
def test_features_match_oracle(m, K):
    rng = np.random.default_rng(950 + m + K)
    sizes = [517, 0, 1, 2000, 130]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Ds = np.stack([si.unit_gaussian_atoms(rng, m, K) for _ in sizes]).astype(np.float32)
    Y = rng.standard_normal((int(off[-1]), m)).astype(np.float32)
    F = sdl.corr_features(_t(Ds), _t(Y), off).cpu().numpy().astype(np.float64)
    want = oracle.corr_features(Ds.astype(np.float64), off, Y.astype(np.float64))
    tol = _gamma(m) * np.linalg.norm(Y.astype(np.float64), axis=1)
    err = np.abs(F - want)
    assert (err <= tol[:, None] + 1e-30).all(), (err / tol[:, None]).max()
    assert (F >= 0).all()


def test_gradient_with_correlation_inputs_matches_oracle():
    m, K, s = 64, 256, 6
    rng, Ds, Y, off = _batch(960, m, K, s, [40, 24])
    F = oracle.corr_features(Ds.astype(np.float64), off, Y.astype(np.float64)).astype(np.float32)
    idx, *_ = sdl.omp_batched(_t(Ds), _t(Y), off, s)
    params = si.mlp_init(rng, K, H1, H2, K, s)
    prop = sdl.Proposer(_t(params), K, H1, H2, K)
    loss, grad = prop.loss_grad(_t(F), idx)
    torch.cuda.synchronize()
    lo, go = oracle.mlp_loss_grad(params.astype(np.float64), K, H1, H2, K, F.astype(np.float64),
                                  idx.cpu().numpy())
    assert abs(float(loss) - lo) <= 2e-2 * abs(lo)
    g = grad.cpu().numpy().astype(np.float64)
    offs = oracle.mlp_sizes(K, H1, H2, K)
    for q, name in enumerate(["W1", "b1", "W2", "b2", "W3", "b3"]):
        a, b = offs[q], offs[q + 1]
        rel = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert rel <= 2e-2, (name, rel)
    prop.close()


def test_restricted_omp_uses_each_subsets_dictionary():
    """No fallback (eps_fb huge): every code is OMP over the signal's candidates
    from its own dictionary, the candidates being the top-2s scores of the
    network on |D_t^T y| (lowest atom index on ties)."""
    m, K, s = 64, 256, 6
    rng, Ds, Y, off = _batch(961, m, K, s, [700, 0, 1, 800])
    params = si.mlp_init(rng, K, H1, H2, K, s)
    prop = sdl.Proposer(_t(params), K, H1, H2, K)
    Dg, Yg = _t(Ds), _t(Y)
    ncand = 2 * s
    scores = prop.scores(sdl.corr_features(Dg, Yg, off)).cpu().numpy()
    cand = np.argsort(-scores, axis=1, kind="stable")[:, :ncand]
    gi, gv, gn, gr, nf = prop.omp_batched(Dg, Yg, off, s, ncand, 1e30)
    assert nf == 0
    gi, gv, gn, gr = (a.cpu().numpy() for a in (gi, gv, gn, gr))
    for t in range(len(off) - 1):
        D64 = Ds[t].astype(np.float64)
        for i in range(off[t], off[t + 1]):
            y = Y[i:i + 1].astype(np.float64)
            o = oracle.omp(D64[cand[i]], y, s, nthreads=1)
            o["idx"] = np.where(o["idx"] >= 0, cand[i][np.maximum(o["idx"], 0)], -1)
            compare_codes(D64, y, gi[i:i + 1], gv[i:i + 1], gn[i:i + 1], gr[i:i + 1], o,
                          fp32_gap_tol(m, np.linalg.norm(y, axis=1)), 1e-4)
    prop.close()


@pytest.mark.parametrize("features", [sdl.FEATURES_CORR, sdl.FEATURES_SIGNAL])
def test_fallback_everywhere_is_batched_omp(features):
    """eps_fb = 0 flags every signal, across empty subsets and the feature chunk
    boundary: the codes are sdl_omp_batched's, bit for bit."""
    m, K, s = 64, 256, 6
    sizes = [40000, 0, 1, 50000, 3000]
    rng, Ds, Y, off = _batch(962, m, K, s, sizes)
    n_in = K if features == sdl.FEATURES_CORR else m
    prop = sdl.Proposer(_t(si.mlp_init(rng, n_in, H1, H2, K, s)), n_in, H1, H2, K)
    Dg, Yg = _t(Ds), _t(Y)
    gi, gv, gn, gr, nf = prop.omp_batched(Dg, Yg, off, s, 2 * s, 0.0, features=features)
    assert nf == Y.shape[0]
    pi, pv, pn, pr = sdl.omp_batched(Dg, Yg, off, s)
    for a, b in zip((gi, gv, gn, gr), (pi, pv, pn, pr)):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    prop.close()


def test_partial_fallback_keeps_accepted_codes_and_recodes_the_rest():
    m, K, s = 64, 256, 6
    rng, Ds, Y, off = _batch(963, m, K, s, [3000, 1, 2000])
    prop = sdl.Proposer(_t(si.mlp_init(rng, K, H1, H2, K, s)), K, H1, H2, K)
    Dg, Yg = _t(Ds), _t(Y)
    ri, rv, rn, rr, nf0 = prop.omp_batched(Dg, Yg, off, s, 2 * s, 1e30)
    # an untrained network's candidates leave large residuals: put the threshold
    # midway between two neighbouring restricted residual norms near the median,
    # so that about half the signals are accepted and no norm sits at it
    rs = np.sort(np.sqrt(rr.cpu().numpy().astype(np.float64)))
    h = len(rs) // 2
    assert rs[h] - rs[h - 1] > 1e-5 * rs[h]
    eps_fb = 0.5 * (rs[h - 1] + rs[h])
    fi, fv, fn, fr, nf = prop.omp_batched(Dg, Yg, off, s, 2 * s, eps_fb)
    pi, pv, pn, pr = sdl.omp_batched(Dg, Yg, off, s)
    ri, rv, rr, fi, fv, fr, pi, pv, pr = (a.cpu().numpy() for a in (ri, rv, rr, fi, fv, fr, pi, pv, pr))
    acc = np.sqrt(rr.astype(np.float64)) <= eps_fb
    assert nf0 == 0 and nf == int((~acc).sum()) and 0 < nf < len(Y)
    np.testing.assert_array_equal(fi[acc], ri[acc])
    np.testing.assert_array_equal(fv[acc], rv[acc])
    np.testing.assert_array_equal(fr[acc], rr[acc])
    np.testing.assert_array_equal(fi[~acc], pi[~acc])
    np.testing.assert_array_equal(fv[~acc], pv[~acc])
    np.testing.assert_array_equal(fr[~acc], pr[~acc])
    prop.close()


def test_one_network_learns_across_dictionaries():
    """Sixteen dictionaries, 4,096 signals each: four epochs of Adam on
    (|D_t^T y|, plain-OMP support) pairs bring the loss well below its start
    (the label prior, where the output bias starts)."""
    m, K, s = 64, 256, 6
    rng, Ds, Y, off = _batch(964, m, K, s, [4096] * 16)
    Dg, Yg = _t(Ds), _t(Y)
    labels, *_ = sdl.omp_batched(Dg, Yg, off, s, with_resid=False)
    F = sdl.corr_features(Dg, Yg, off)
    prop = sdl.Proposer(_t(si.mlp_init(rng, K, H1, H2, K, s)), K, H1, H2, K)
    loss = torch.zeros(4, dtype=torch.float32, device=DEV)
    g = torch.Generator(device=DEV)
    g.manual_seed(5)
    first = None
    for epoch in range(4):
        order = torch.randperm(F.shape[0], device=DEV, generator=g)
        Fs, Ls = F[order], labels[order]
        for a in range(0, F.shape[0], 4096):
            prop.train_step(Fs[a:a + 4096], Ls[a:a + 4096], 2e-3, loss)
            if first is None:
                first = float(loss[0])
    print(f"conditioned proposer loss {first:.2f} -> {float(loss[0]):.2f}")
    assert float(loss[0]) < 0.9 * first, (first, float(loss[0]))
    prop.close()


def test_bad_arguments_are_rejected():
    m, K, s = 16, 32, 3
    rng, Ds, Y, off = _batch(965, m, K, s, [50, 30])
    prop = sdl.Proposer(_t(si.mlp_init(rng, m, 64, 64, K, s)), m, 64, 64, K)   # a signal-input network
    with pytest.raises(sdl.SdlError):
        prop.omp_batched(_t(Ds), _t(Y), off, s, 2 * s, 0.1, features=sdl.FEATURES_CORR)
    with pytest.raises(sdl.SdlError):
        prop.omp_batched(_t(Ds), _t(Y), off, s, 2 * s, 0.1, features=7)
    with pytest.raises(sdl.SdlError):
        prop.omp_batched(_t(Ds), _t(Y), off, s, s - 1, 0.1, features=sdl.FEATURES_SIGNAL)
    prop.close()


def test_largest_shapes_restricted_omp():
    """m = 256, K = 1024 (the largest compiled sizes), 32 candidates (the most a
    warp holds), s = 16, a network with 1,024 inputs: restricted OMP per subset
    against the oracle on each candidate sub-dictionary."""
    m, K, s, nc = 256, 1024, 16, 32
    rng, Ds, Y, off = _batch(966, m, K, s, [150, 0, 90])
    prop = sdl.Proposer(_t(si.mlp_init(rng, K, 64, 64, K, s)), K, 64, 64, K)
    Dg, Yg = _t(Ds), _t(Y)
    cand = np.argsort(-prop.scores(sdl.corr_features(Dg, Yg, off)).cpu().numpy(), axis=1, kind="stable")[:, :nc]
    gi, gv, gn, gr, nf = prop.omp_batched(Dg, Yg, off, s, nc, 1e30)
    assert nf == 0
    gi, gv, gn, gr = (a.cpu().numpy() for a in (gi, gv, gn, gr))
    for t in range(len(off) - 1):
        D64 = Ds[t].astype(np.float64)
        for i in range(off[t], off[t + 1]):
            y = Y[i:i + 1].astype(np.float64)
            o = oracle.omp(D64[cand[i]], y, s, nthreads=1)
            o["idx"] = np.where(o["idx"] >= 0, cand[i][np.maximum(o["idx"], 0)], -1)
            compare_codes(D64, y, gi[i:i + 1], gv[i:i + 1], gn[i:i + 1], gr[i:i + 1], o,
                          fp32_gap_tol(m, np.linalg.norm(y, axis=1)), 1e-3)
    prop.close()


def test_full_size_conditioned_sampled():
    """The bench's conditioned workload at full size: 64 dictionaries of 64 x 256,
    8,192 signals each (2^19 in all).  Sampled signals: features within
    gamma_m ||y|| of the oracle and restricted codes equal to the oracle's OMP
    on their candidate sub-dictionaries.  Every signal: with eps_fb = 8.5 sigma,
    the accepted ones keep their restricted code and the others carry plain
    batched OMP's code, bit for bit."""
    m, K, s, L, n_t = 64, 256, 6, 64, 8192
    rng, Ds, Y, off = _batch(967, m, K, s, [n_t] * L)
    prop = sdl.Proposer(_t(si.mlp_init(rng, K, H1, H2, K, s)), K, H1, H2, K)
    Dg, Yg = _t(Ds), _t(Y)
    F = sdl.corr_features(Dg, Yg, off)
    cand_all = torch.topk(prop.scores(F), 2 * s, dim=1).indices.cpu().numpy()
    F = F.cpu().numpy()
    ri, rv, rn, rr, nf0 = prop.omp_batched(Dg, Yg, off, s, 2 * s, 1e30)
    assert nf0 == 0
    ri, rv, rn, rr = (a.cpu().numpy() for a in (ri, rv, rn, rr))
    sample = np.sort(rng.choice(len(Y), 400, replace=False))
    for i in sample:
        t = int(np.searchsorted(off, i, side="right") - 1)
        D64, y = Ds[t].astype(np.float64), Y[i:i + 1].astype(np.float64)
        want = oracle.corr_features(D64[None], np.array([0, 1], np.int64), y)[0]
        assert (np.abs(F[i] - want) <= _gamma(m) * np.linalg.norm(y) + 1e-30).all()
        c = np.sort(cand_all[i])        # the candidate set (its order does not matter to OMP)
        o = oracle.omp(D64[c], y, s, nthreads=1)
        o["idx"] = np.where(o["idx"] >= 0, c[np.maximum(o["idx"], 0)], -1)
        compare_codes(D64, y, ri[i:i + 1], rv[i:i + 1], rn[i:i + 1], rr[i:i + 1], o,
                      fp32_gap_tol(m, np.linalg.norm(y, axis=1)), 1e-4)
    eps_fb = 8.5 * 0.01
    fi, fv, fn, fr, nf = prop.omp_batched(Dg, Yg, off, s, 2 * s, eps_fb)
    pi, pv, pn, pr = sdl.omp_batched(Dg, Yg, off, s)
    fi, fv, pi, pv = (a.cpu().numpy() for a in (fi, fv, pi, pv))
    acc = np.sqrt(rr.astype(np.float64)) <= eps_fb
    assert nf == int((~acc).sum())
    np.testing.assert_array_equal(fi[acc], ri[acc])
    np.testing.assert_array_equal(fv[acc], rv[acc])
    np.testing.assert_array_equal(fi[~acc], pi[~acc])
    np.testing.assert_array_equal(fv[~acc], pv[~acc])
    prop.close()
