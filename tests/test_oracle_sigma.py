"""Pins for the oracle's second-Born self-energy (Sec. 2.3, Eq. sigma2ndb)."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W


def test_hubbard_atom_half_filling():
    # one level at half filling: g = gb = 1/2 on [-beta, 0]; second Born gives
    # Sigma(tau) = U^2/8 for tau < 0, i.e. Sigma(i w) = U^2/(4 i w)
    U = 1.7
    g = np.array([[0.5]])
    S = O.sigma2_tau(g, g, np.array([[U]]), 2.0)
    assert abs(S[0, 0] - U * U / 8.0) < 1e-15


@pytest.mark.parametrize("sigma", [1.0, 2.0])
def test_single_level_reduces_to_sigma_minus_one(sigma):
    # n = 1: direct sigma V^2 g^2 gb minus exchange V^2 g gb g
    g, gb, U = np.array([[0.31]]), np.array([[0.77]]), np.array([[0.9]])
    S = O.sigma2_tau(g, gb, U, sigma)
    assert abs(S[0, 0] - (sigma - 1.0) * 0.81 * 0.31 ** 2 * 0.77) < 1e-15


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (5, 3)])
def test_two_index_equals_bruteforce_four_index(n, seed):
    rng = np.random.default_rng(seed)
    V = W.random_symmetric(rng, n)
    g = W.random_symmetric(rng, n)
    gb = W.random_symmetric(rng, n)
    eri = np.zeros((n, n, n, n))
    for a in range(n):
        for c in range(n):
            eri[a, a, c, c] = V[a, c]   # (ab|cd) = delta_ab delta_cd V_ac (Eq. umat1)
    S = O.sigma2_tau(g, gb, V, 2.0)
    B = O.sigma2_bruteforce(g, gb, eri, 2.0)
    assert np.max(np.abs(S - B)) < 1e-13 * max(1.0, np.max(np.abs(B)))


def test_exchange_term_by_explicit_loops():
    rng = np.random.default_rng(7)
    n = 4
    V, g, gb = (W.random_symmetric(rng, n) for _ in range(3))
    X = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            for k in range(n):
                for l in range(n):
                    X[a, b] += V[a, k] * V[b, l] * g[a, l] * gb[l, k] * g[k, b]
    D = 2.0 * g * (V @ (g * gb) @ V)
    np.testing.assert_allclose(O.sigma2_tau(g, gb, V, 2.0), D - X, atol=1e-14)


def test_sigma_symmetric():
    rng = np.random.default_rng(11)
    M, n = 5, 6
    G = W.random_symmetric_stack(rng, M, n)
    V = W.random_symmetric(rng, n)
    S = O.sigma2(G, V, 2.0)
    assert np.max(np.abs(S - S.transpose(0, 2, 1))) < 1e-14


def test_one_shot_correlation_energy_converges_to_twice_mp2():
    # With g^0 and Sigma^(2)[g^0], the Galitskii-Migdal correlation term equals
    # <V> at second order = 2 E_MP2 (the tau integral of exponentials is the
    # MP2 sum); the trapezoid error falls as h^2.
    s = W.he_small()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, 0)
    T, v = O.kinetic(b), O.potential(b["nodes"], s.Z, s.R, 1.0)
    V = O.interaction(b["nodes"], 1.0)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    e2 = 2.0 * O.mp2(hf["eps"], hf["C"], V, 1)
    errs = []
    for u in (4, 8, 16):
        mesh = O.power_mesh(s.beta, u, 16)
        G0 = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], s.beta)
        A = O.sigma2(G0, V, 2.0)
        ec = O.energy(h, V, 2.0, G0, A, mesh["w"]) - O.energy(h, V, 2.0, G0, 0 * A, mesh["w"])
        errs.append(abs(ec - e2) / abs(e2))
    assert errs[2] < 5e-4
    assert errs[0] > 3.0 * errs[1] > 9.0 * errs[2]
