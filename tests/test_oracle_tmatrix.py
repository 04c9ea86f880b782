"""Pins for the oracle's T-matrix self-energy (the particle-particle ladder of
the two-index interaction on the Matsubara mesh): the lowest order against
second Born, the pair-space convolution against the bubble's periodic
convolution, the fixed point against a dense linear solve, the third-order
scaling of the ladder correction, and the low-density limit of a single level,
where the ladder is exact to second order in the fugacity (the two-body
problem) and second Born is not."""
import numpy as np

from oracle import fedvr_oracle as O


def _random_system(seed, n, beta, u, p):
    rng = np.random.default_rng(seed)
    h = rng.normal(size=(n, n))
    h = 0.5 * (h + h.T)
    V = np.abs(rng.normal(size=(n, n)))
    V = 0.3 * (V + V.T)
    eps, C = np.linalg.eigh(h)
    mu = 0.5 * (eps[n // 2 - 1] + eps[n // 2])
    mesh = O.power_mesh(beta, u, p)
    G = O.g0_mesh(eps, C, mu, mesh["tau"], beta)
    return V, mesh, G, O.bose_lag_table(mesh["tau"], beta)


def test_lowest_order_is_second_born():
    # t = V^ K V^ closed with the hole line: the direct and exchange terms of Eq. sigma2ndb
    V, mesh, G, blag = _random_system(1, 4, 10.0, 2, 4)
    got = O.sigma_tmatrix(G, V, 2.0, mesh, blag, max_iter=0)["Sigma"]
    want = O.sigma2(G, V, 2.0)
    assert np.max(np.abs(got - want)) < 1e-15 * max(1.0, np.max(np.abs(want)))
    # and with the spin factor 1 (the exchange term enters with its own factor)
    got1 = O.sigma_tmatrix(G, V, 1.0, mesh, blag, max_iter=0)["Sigma"]
    assert np.max(np.abs(got1 - O.sigma2(G, V, 1.0))) < 1e-15 * max(1.0, np.max(np.abs(want)))


def test_pair_convolution_against_the_periodic_convolution():
    # t_j = phi_j delta_ab delta_kl: every element of K * t is the periodic
    # convolution of the scalar function g_ab(tau) g_kl(tau) with phi
    V, mesh, G, blag = _random_system(2, 3, 8.0, 2, 4)
    M, n = G.shape[0], G.shape[1]
    phi = np.cos(mesh["tau"])
    eye = np.einsum("ab,kl->akbl", np.eye(n), np.eye(n))
    t = phi[:, None, None, None, None] * eye[None]
    got = O.pair_conv(G, t, mesh, blag)
    for a, k, b, l in [(0, 0, 0, 0), (0, 1, 2, 0), (2, 1, 0, 2), (1, 2, 1, 0)]:
        Kel = (G[:, a, b] * G[:, k, l])[:, None, None]
        want = O.conv_bose(Kel, phi[:, None, None], mesh, blag)[:, 0, 0]
        assert np.max(np.abs(got[:, a, k, b, l] - want)) < 1e-14 * max(1.0, np.max(np.abs(want)))


def test_fixed_point_equals_direct_linear_solve():
    # the damped iteration solves (1 + V^ (K *)) t = V^ K V^
    V, mesh, G, blag = _random_system(3, 2, 6.0, 2, 2)
    M, n = G.shape[0], G.shape[1]
    out = O.ladder_t(G, V, 2.0, mesh, blag, tol=1e-15, max_iter=3000)
    N = M * n ** 4

    def apply(x):
        t = x.reshape(M, n, n, n, n)
        return (t + V[None, :, :, None, None] * O.pair_conv(G, t, mesh, blag)).ravel()

    A = np.stack([apply(e) for e in np.eye(N)], axis=1)
    direct = np.linalg.solve(A, out["S"].ravel()).reshape(M, n, n, n, n)
    assert np.max(np.abs(out["t"] - direct)) < 1e-12 * np.max(np.abs(direct))


def test_ladder_correction_is_third_order():
    # Sigma^T(lam V) - lam^2 Sigma^(2)(V) falls 8x per halving of lam
    V, mesh, G, blag = _random_system(4, 3, 10.0, 2, 4)
    D = O.sigma2(G, V, 2.0)
    errs = []
    for lam in (0.1, 0.05, 0.025):
        full = O.sigma_tmatrix(G, lam * V, 2.0, mesh, blag, tol=1e-16, max_iter=400)["Sigma"]
        errs.append(float(np.max(np.abs(full - lam * lam * D))))
    assert errs[0] / errs[1] > 7.3 and errs[1] / errs[2] > 7.6, errs


def test_low_density_single_level_is_exact_to_second_order_in_the_fugacity():
    # one spin-degenerate level at eps = mu + x with on-site U (n = 1): the
    # exact occupation per spin is (z + z^2 e^{-beta U}) / (1 + 2 z + z^2 e^{-beta U}),
    # z = e^{-beta x}; its interaction correction z^2 (e^{-beta U} - 1) + O(z^3)
    # is the two-body problem that the particle-particle ladder sums to all
    # orders in U. At beta U = 2 second Born's z^2 term (-beta U + (beta U)^2 / 2)
    # vanishes, the ladder's does not.
    beta, U, z = 1.0, 2.0, 0.01
    x = -np.log(z) / beta
    h, V = np.array([[x]]), np.array([[U]])
    rho = 0.0
    for _ in range(200):  # Hartree-Fock at fixed mu = 0 (Sigma^HF = U rho for one level)
        rho = 1.0 / (np.exp(beta * (x + U * rho)) + 1.0)
    hf = dict(eps=np.array([x + U * rho]), C=np.eye(1), mu=0.0, Sigma0=np.array([[U * rho]]))
    f = 1.0 / (np.exp(beta * x) + 1.0)
    n_exact = (z + z * z * np.exp(-beta * U)) / (1.0 + 2.0 * z + z * z * np.exp(-beta * U))
    d_exact = n_exact - f
    got = {}
    for se in ("tmatrix", "2b"):
        r = O.solve_2b(h, V, 2.0, hf, beta, 4, 16, 0.5, 1e-13, 200, self_energy=se)
        assert r["converged"]
        got[se] = r["N"] / 2.0 - f
    assert abs(got["tmatrix"] - d_exact) < 0.03 * abs(d_exact), (got, d_exact)
    assert abs(got["2b"] - d_exact) > 0.5 * abs(d_exact), (got, d_exact)
