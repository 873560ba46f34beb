"""The oracle's Adam step (Kingma & Ba 2015, Algorithm 1; the proposer's
optimiser) pinned by properties its definition fixes, none of them a retyping
of the update:
  * from zero moments the first step is alpha * g / (|g| + eps): the bias
    correction makes mhat = g and vhat = g^2 exactly;
  * under a constant gradient every step is that same move (the corrected
    moving averages of a constant equal it at every t);
  * scaling every gradient by c > 0 leaves the path unchanged when eps is
    negligible (v must track g^2, m must track g), and negating them mirrors it;
  * a gradient 1 then 0 gives, worked by hand, mhat = beta1 / (1 + beta1) and
    vhat = beta2 / (1 + beta2) at t = 2 (which pins the power t of the
    correction);
  * a zero gradient from zero moments moves nothing.
"""
import numpy as np

import oracle


def _run(g_seq, theta0, alpha, eps=1e-8):
    th = np.array(theta0, dtype=np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    path = [th.copy()]
    for t, g in enumerate(g_seq, start=1):
        th, m, v = oracle.adam_step(th, g, m, v, t, alpha, eps=eps)
        path.append(th.copy())
    return np.array(path)


def test_first_step_is_a_sign_step():
    rng = np.random.default_rng(0)
    g = rng.standard_normal(1000) * np.logspace(-6, 3, 1000)
    th0 = rng.standard_normal(1000)
    p = _run([g], th0, 1e-3)
    np.testing.assert_allclose(p[1], th0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_constant_gradient_gives_equal_steps():
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    p = _run([g] * 50, np.zeros(4), 2e-3)
    steps = np.diff(p, axis=0)
    np.testing.assert_allclose(steps, np.broadcast_to(-2e-3 * g / (np.abs(g) + 1e-8), steps.shape),
                               rtol=1e-12, atol=0)


def test_scale_and_sign_invariance():
    rng = np.random.default_rng(1)
    gs = [rng.standard_normal(64) for _ in range(12)]
    base = _run(gs, np.zeros(64), 1e-2, eps=0.0)
    for c in (1e-4, 3.0, 1e5):
        np.testing.assert_allclose(_run([c * g for g in gs], np.zeros(64), 1e-2, eps=0.0), base, rtol=1e-12,
                                   atol=1e-15)
    np.testing.assert_allclose(_run([-g for g in gs], np.zeros(64), 1e-2, eps=0.0), -base, rtol=1e-12, atol=1e-15)


def test_hand_worked_second_step():
    b1, b2, a = 0.9, 0.999, 0.01
    p = _run([np.array([1.0]), np.array([0.0])], np.zeros(1), a, eps=0.0)
    mhat, vhat = b1 / (1 + b1), b2 / (1 + b2)
    assert abs(p[1][0] - (-a)) < 1e-15
    assert abs((p[2][0] - p[1][0]) - (-a * mhat / np.sqrt(vhat))) < 1e-15


def test_zero_gradient_from_rest_moves_nothing():
    p = _run([np.zeros(5)] * 3, np.arange(5.0), 0.1)
    assert (p == np.arange(5.0)).all()
