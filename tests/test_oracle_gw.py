"""Pins for the oracle's GW self-energy (the two-index bubble series on the
Matsubara mesh): a single level in closed form, the lowest order against the
textbook one-level second-order terms, the periodic convolution against a
closed form with non-commuting matrices, the fixed-point iteration against a
direct linear solve, the third-order scaling of the bubble correction, and a
converged GW solve of the small He model."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W


def _one_level(beta, eps, V, u=2, p=4):
    mesh = O.power_mesh(beta, u, p)
    G = O.g0_mesh(np.array([eps]), np.eye(1), 0.0, mesh["tau"], beta)
    return mesh, G, np.array([[V]])


def test_single_level_screened_interaction_closed_form():
    # one level: Q(tau) = f (1 - f) is constant, so Q * w = Q int w and the
    # series sums to w = V^2 Q / (1 + sigma beta V Q) (the trapezoid is exact here)
    beta, eps, V = 10.0, 0.3, 0.7
    mesh, G, Vm = _one_level(beta, eps, V)
    f = 1.0 / (np.exp(beta * eps) + 1.0)
    Q = f * (1.0 - f)
    out = O.screened_w(G, Vm, 2.0, mesh, O.bose_lag_table(mesh["tau"], beta), tol=1e-15)
    want = V * V * Q / (1.0 + 2.0 * beta * V * Q)
    assert np.max(np.abs(out["w"] - want)) < 1e-13 * want


def test_lowest_order_is_the_direct_term():
    # w = V Q V (no bubble sum): for one level Sigma^GW = sigma V^2 g^2 gb while
    # second Born is (sigma - 1) V^2 g^2 gb, their difference the textbook
    # second-order exchange V^2 g^2 gb
    beta = 8.0
    mesh, G, Vm = _one_level(beta, -0.2, 0.9)
    M = G.shape[0]
    blag = O.bose_lag_table(mesh["tau"], beta)
    gw1 = O.sigma_gw(G, Vm, 2.0, mesh, blag, max_iter=0)["Sigma"]
    sb = O.sigma2(G, Vm, 2.0)
    g, gb = G[:, 0, 0], G[::-1, 0, 0]
    assert np.max(np.abs(gw1[:, 0, 0] - sb[:, 0, 0] - 0.81 * g * g * gb)) < 1e-15
    assert np.max(np.abs(gw1[:, 0, 0] - 2.0 * 0.81 * g * g * gb)) < 1e-15


def _conv_closed(tau, beta, CA, ya, CB, zb):
    # periodic A(x) = CA diag(cosh(y (x + beta/2))) CA^T (continuous across the period),
    # B(s) = CB diag(exp(-z s)) CB^T; int_{-beta}^0 A(tau - s) B(s) ds in closed form
    def piece(c, y, z, t):
        # int over [-beta, 0] of e_y(tau - s) e^{-z s}, e_y(x) = e^{c y (x + beta/2)} extended
        # periodically from [-beta, 0]
        a = c * y
        d = a + z  # e^{a (t - s) + a beta/2} e^{-z s} = e^{a t + a beta/2} e^{-d s}
        first = np.exp(a * t + a * beta / 2) * (np.exp(-d * t) - 1.0) / d        # s in [t, 0]
        second = np.exp(a * (t - beta) + a * beta / 2) * (np.exp(d * beta) - np.exp(-d * t)) / d
        return first + second
    out = np.zeros((len(tau),) + CA.shape)
    for i, t in enumerate(tau):
        acc = np.zeros(CA.shape)
        for p_, y in enumerate(ya):
            for q, z in enumerate(zb):
                sc = 0.5 * (piece(1.0, y, z, t) + piece(-1.0, y, z, t))
                acc += sc * np.outer(CA[:, p_], CA[:, p_]) @ np.outer(CB[:, q], CB[:, q])
        out[i] = acc
    return out


def test_periodic_convolution_closed_form_second_order():
    rng = np.random.default_rng(6)
    beta, n = 6.0, 3
    CA, _ = np.linalg.qr(rng.normal(size=(n, n)))
    CB, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ya, zb = np.array([0.3, 0.8, 1.3]), np.array([-0.5, 0.2, 0.9])
    errs = []
    for u in (4, 8, 16):
        mesh = O.power_mesh(beta, u, 4)
        tau = mesh["tau"]
        A = np.stack([CA @ np.diag(np.cosh(ya * (x + beta / 2))) @ CA.T for x in tau])
        B = np.stack([CB @ np.diag(np.exp(-zb * x)) @ CB.T for x in tau])
        got = O.conv_bose(A, B, mesh, O.bose_lag_table(tau, beta))
        want = _conv_closed(tau, beta, CA, ya, CB, zb)
        errs.append(float(np.max(np.abs(got - want)) / np.max(np.abs(want))))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_fixed_point_equals_direct_linear_solve():
    # the damped iteration solves (1 + sigma V (Q *)) w = V Q V: compare with
    # numpy's dense solve of the same linear map on a small mesh
    rng = np.random.default_rng(3)
    n, beta = 4, 20.0
    h = rng.normal(size=(n, n)); h = 0.5 * (h + h.T)
    V = np.abs(rng.normal(size=(n, n))); V = 0.3 * (V + V.T)
    eps, C = np.linalg.eigh(h)
    mu = 0.5 * (eps[1] + eps[2])
    mesh = O.power_mesh(beta, 2, 4)
    G = O.g0_mesh(eps, C, mu, mesh["tau"], beta)
    M = G.shape[0]
    blag = O.bose_lag_table(mesh["tau"], beta)
    out = O.screened_w(G, V, 2.0, mesh, blag, tol=1e-14, max_iter=2000)
    Q = out["Q"]

    def apply(x):
        w = x.reshape(M, n, n)
        c = O.conv_bose(Q, w, mesh, blag)
        return (w + 2.0 * np.stack([V @ c[j] for j in range(M)])).ravel()

    N = M * n * n
    Aop = np.stack([apply(e) for e in np.eye(N)], axis=1)
    w_direct = np.linalg.solve(Aop, out["VQV"].ravel()).reshape(M, n, n)
    assert np.max(np.abs(out["w"] - w_direct)) < 1e-11 * np.max(np.abs(w_direct))
    assert out["res"] < 1e-14


def test_bubble_correction_is_third_order():
    # Sigma^GW(lam V) - lam^2 D, D the lowest order, falls 8x per halving of lam
    s = W.he_small()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, 0)
    h = O.kinetic(b) + np.diag(O.potential(b["nodes"], s.Z, s.R, 1.0))
    V = O.interaction(b["nodes"], 1.0)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    mesh = O.power_mesh(s.beta, 2, 4)
    G = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], s.beta)
    blag = O.bose_lag_table(mesh["tau"], s.beta)
    D = O.sigma_gw(G, V, 2.0, mesh, blag, max_iter=0)["Sigma"]
    errs = []
    for lam in (0.2, 0.1, 0.05):
        full = O.sigma_gw(G, lam * V, 2.0, mesh, blag, tol=1e-16, max_iter=300)["Sigma"]
        errs.append(float(np.max(np.abs(full - lam * lam * D))))
    assert errs[0] / errs[1] > 7.0 and errs[1] / errs[2] > 7.5, errs


def test_gw_solve_of_the_small_he_model():
    s = W.he_small()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, 0)
    h = O.kinetic(b) + np.diag(O.potential(b["nodes"], s.Z, s.R, 1.0))
    V = O.interaction(b["nodes"], 1.0)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    # (the 129-point mesh: on coarser meshes the iteration diverges for second Born as well)
    res = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, 0.5, 1e-8, 100, self_energy="gw")
    assert res["converged"]
    G = res["G"]
    assert np.max(np.abs(G[-1] + G[0] - np.eye(G.shape[1]))) < 1e-12
    assert abs(res["N"] - 2.0) < 1e-3
    # GW sums the bubbles without the second-order exchange: more correlation
    # energy than second Born here, both below HF
    ref2 = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, 0.5, 1e-8, 100)
    assert res["E0"] < ref2["E0"] < hf["E_hf"]
    # the inner iteration is warm-started: later outer steps need fewer inner steps
    assert res["gw_inner"][-1] < res["gw_inner"][0]
