"""Pins for the warm-start network's CPU reference (oracle/mlp_oracle.py)."""
import numpy as np

from oracle import mlp_oracle as N
from paper_0911_4348_gb300 import workloads as W


def _tiny(seed=0):
    rng = W.system_rng(80, seed)
    P = N.init_params(7, 6, 5, rng)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0.0, 0.1, P[k].shape)
    X = rng.normal(size=(9, 7))
    T = rng.normal(size=(9, 5))
    return P, X, T


def test_backward_matches_central_differences():
    P, X, T = _tiny()
    y, cache = N.forward(P, X)
    g = N.backward(P, cache, y, T)
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = N.loss(N.forward(P, X)[0], T)
            flat[idx] = old - h
            lm = N.loss(N.forward(P, X)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_first_adam_step_is_signed_learning_rate():
    # step 1: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps)
    P, X, T = _tiny(1)
    y, cache = N.forward(P, X)
    g = N.backward(P, cache, y, T)
    before = {k: v.copy() for k, v in P.items()}
    N.adam_step(P, g, {}, lr=1e-3)
    for k in P:
        want = before[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.max(np.abs(P[k] - want)) < 1e-15


def test_features_targets_scatter_roundtrip():
    rng = W.system_rng(81, 0)
    M, n = 5, 4
    S1 = W.random_symmetric_stack(rng, M, n, 1e-2)
    Ss = S1 + W.random_symmetric_stack(rng, M, n, 1e-3)
    G0 = W.random_symmetric_stack(rng, M, n)
    V = W.random_symmetric(rng, n)
    X = np.linspace(-2.0, 2.0, n)
    F, s = N.features(S1, G0, V, X, 10.0)
    assert F.shape == (n * (n + 1) // 2, 2 * M + 3) and s == np.max(np.abs(S1))
    pr = N.pair_index(n)
    k = 4  # pair (2, 1)
    a, b = pr[k]
    assert (a, b) == (2, 1)
    assert np.allclose(F[k, :M], S1[:, a, b] / s) and np.allclose(F[k, M:2 * M], G0[:, a, b])
    assert F[k, 2 * M] == V[a, b] and F[k, 2 * M + 1] == X[a] / 10.0
    T = N.targets(Ss, S1, s)
    # a perfect prediction reproduces Sigma* exactly, symmetric
    back = N.scatter_prediction(T, S1, s)
    assert np.allclose(back, Ss, atol=1e-17)
