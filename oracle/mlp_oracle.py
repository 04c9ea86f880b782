"""Plain FP64 CPU reference for the learned warm start of the second-Born
iteration. TEST INFRASTRUCTURE ONLY (same rules as fedvr_oracle: imported by
tests, the smoke check and the benchmark's CPU leg, never by the library).

The paper has no learned component; this is the reference for the library's
warm-start network: a per-(a, b)-pair MLP that maps the one-shot self-energy
Sigma^(2)[g^0]_ab(tau) and g^0_ab(tau) on the mesh (plus V_ab and the two node
positions) to the correction Delta_ab(tau) = Sigma*_ab(tau) - Sigma^(2)[g^0]_ab(tau)
of the converged self-energy, both scaled by s = max |Sigma^(2)[g^0]|.

Network: x (2M+3) -> relu(x W1 + b1) (H) -> relu(h1 W2 + b2) (H) -> h2 W3 + b3 (M);
loss L = sum (y - t)^2 / (2 * rows * M); Adam (beta1 0.9, beta2 0.999, eps 1e-8).
"""

from __future__ import annotations

import numpy as np


def pair_index(n: int) -> np.ndarray:
    """Pairs (a, b) with a >= b in row-major order of the lower triangle."""
    return np.array([(a, b) for a in range(n) for b in range(a + 1)], dtype=np.int64)


def features(S1: np.ndarray, G0: np.ndarray, V: np.ndarray, X: np.ndarray, L: float):
    """Feature rows, one per pair (a >= b):
    [S1_ab(tau_0..M-1)/s, g0_ab(tau_0..M-1), V_ab, X_a/L, X_b/L] with s = max|S1|.
    Returns (F [pairs][2M+3], s)."""
    M, n = S1.shape[0], S1.shape[1]
    s = float(np.max(np.abs(S1)))
    pr = pair_index(n)
    a, b = pr[:, 0], pr[:, 1]
    F = np.empty((len(pr), 2 * M + 3))
    F[:, :M] = (S1[:, a, b] / s).T
    F[:, M:2 * M] = G0[:, a, b].T
    F[:, 2 * M] = V[a, b]
    F[:, 2 * M + 1] = X[a] / L
    F[:, 2 * M + 2] = X[b] / L
    return F, s


def targets(Sstar: np.ndarray, S1: np.ndarray, s: float) -> np.ndarray:
    """(Sigma* - Sigma^(2)[g0])_ab(tau) / s per pair, [pairs][M]."""
    n = S1.shape[1]
    pr = pair_index(n)
    D = (Sstar - S1)[:, pr[:, 0], pr[:, 1]]
    return D.T / s


def scatter_prediction(Y: np.ndarray, S1: np.ndarray, s: float) -> np.ndarray:
    """Sigma_pred = S1 + s * Delta, Delta from the network output rows (symmetric)."""
    n = S1.shape[1]
    pr = pair_index(n)
    out = S1.copy()
    out[:, pr[:, 0], pr[:, 1]] += s * Y.T
    out[:, pr[:, 1], pr[:, 0]] = out[:, pr[:, 0], pr[:, 1]]
    return out


def init_params(din: int, hidden: int, dout: int, rng: np.random.Generator) -> dict:
    """He-normal weights (std sqrt(2/fan_in)), zero biases."""
    return {
        "W1": rng.normal(0.0, np.sqrt(2.0 / din), (din, hidden)), "b1": np.zeros(hidden),
        "W2": rng.normal(0.0, np.sqrt(2.0 / hidden), (hidden, hidden)), "b2": np.zeros(hidden),
        "W3": rng.normal(0.0, np.sqrt(2.0 / hidden), (hidden, dout)), "b3": np.zeros(dout),
    }


def forward(P: dict, X: np.ndarray):
    z1 = X @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"] + P["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.sum((y - t) ** 2) / (2.0 * y.shape[0] * y.shape[1]))


def backward(P: dict, cache, y: np.ndarray, t: np.ndarray) -> dict:
    """Gradients of ``loss`` with respect to every parameter (chain rule)."""
    X, z1, h1, z2, h2 = cache
    dy = (y - t) / (y.shape[0] * y.shape[1])
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dh2 = dy @ P["W3"].T
    dz2 = dh2 * (z2 > 0.0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ P["W2"].T
    dz1 = dh1 * (z1 > 0.0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return g


def adam_step(P: dict, g: dict, state: dict, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place (bias-corrected moments; state holds m, v, step)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = beta1 * m + (1.0 - beta1) * g[k]
        v[...] = beta2 * v + (1.0 - beta2) * g[k] ** 2
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        P[k] -= lr * mh / (np.sqrt(vh) + eps)
