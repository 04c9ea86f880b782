"""Pins for the oracle's mesh, lag interpolation, convolutions and the
self-consistency loop (Sec. 2.3 Eq. deq, Sec. 3.1)."""
import math

import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W


@pytest.mark.parametrize("beta,u,p", [(100.0, 4, 16), (10.0, 3, 5), (37.5, 16, 16)])
def test_power_mesh_structure(beta, u, p):
    m = O.power_mesh(beta, u, p)
    tau, w = m["tau"], m["w"]
    M = 2 * u * p + 1
    assert m["M"] == M and len(tau) == M
    assert tau[0] == -beta and tau[-1] == 0.0 and np.all(np.diff(tau) > 0)
    for j in range(M):  # mirror tau_{M-1-j} = -beta - tau_j (built from the same offsets)
        assert -tau[M - 1 - j] == pytest.approx(beta + tau[j], abs=1e-13)
    assert abs(w.sum() - beta) < 1e-12 * beta
    np.testing.assert_allclose(m["wm"] + m["wp"], w, rtol=1e-15, atol=1e-300)
    # finest spacing at both ends: (beta/2) 2^(1-p) / u
    assert abs((tau[1] - tau[0]) - (beta / 2) * 2.0 ** (1 - p) / u) < 1e-12 * beta
    # trapezoid integrates linear functions exactly
    assert abs(np.sum(w * (3.0 * tau + 1.0)) - (-1.5 * beta ** 2 + beta)) < 1e-9 * beta ** 2


def test_lag_bracket_and_linear_interpolation_exact():
    beta = 20.0
    m = O.power_mesh(beta, 3, 6)
    tau = m["tau"]
    lag = O.lag_table(tau, beta)
    M = len(tau)
    a, c = 0.7, -0.2
    for i in range(M):
        for j in range(M):
            if i == j:
                continue
            y, sg = O.lag_point(tau, beta, i, j)
            k = int(lag["k"][i, j])
            assert k == min(int(np.searchsorted(tau, y, side="right")) - 1, M - 2)
            assert -beta <= y <= 0.0 and 0.0 <= lag["t"][i, j] <= 1.0
            assert sg == (1.0 if j > i else -1.0)
            t = lag["t"][i, j]
            val = (1 - t) * (a * tau[k] + c) + t * (a * tau[k + 1] + c)
            assert abs(val - (a * y + c)) < 1e-12


def _phi_scalar(x, y, beta):
    return float(O.phi(x, np.array([y]), beta)[0])


def _closed_form(tau, ya, yb, beta):
    # int_{-beta}^{0} phi_a(tau - s) phi_b(s) ds with phi_a anti-periodic
    fa = 1.0 / (math.exp(beta * ya) + 1.0)
    fb = 1.0 / (math.exp(beta * yb) + 1.0)
    d = ya - yb
    first = fa * fb * math.exp(-tau * ya) * (1.0 - math.exp(tau * d)) / d
    second = (1.0 - fa) * fb * math.exp(-tau * ya) * (math.exp(tau * d) - math.exp(-beta * d)) / d
    return first - second


def test_conv2_matches_closed_form_at_second_order():
    beta, ya, yb = 10.0, 0.3, -0.4
    errs = []
    for u in (4, 8, 16):
        mesh = O.power_mesh(beta, u, 6)
        tau = mesh["tau"]
        I1 = np.array([[[_phi_scalar(t, yb, beta)]] for t in tau])
        I2 = O.conv2(I1, np.array([ya]), np.eye(1), 0.0, mesh, beta)
        ref = np.array([_closed_form(t, ya, yb, beta) for t in tau])
        errs.append(np.max(np.abs(I2[:, 0, 0] - ref)))
    assert errs[0] > 3.8 * errs[1] > 3.8 ** 2 * errs[2]
    assert errs[2] < 1e-3


def test_conv1_with_interpolated_lag_matches_closed_form_at_second_order():
    beta, ya, yb = 10.0, -0.25, 0.45
    errs = []
    for u in (4, 8, 16):
        mesh = O.power_mesh(beta, u, 6)
        tau = mesh["tau"]
        lag = O.lag_table(tau, beta)
        A = np.array([[[_phi_scalar(t, ya, beta)]] for t in tau])
        G = np.array([[[_phi_scalar(t, yb, beta)]] for t in tau])
        I1 = O.conv1(np.zeros((1, 1)), A, G, mesh, beta, lag)
        ref = np.array([_closed_form(t, ya, yb, beta) for t in tau])
        errs.append(np.max(np.abs(I1[:, 0, 0] - ref)))
    assert errs[0] > 3.8 * errs[1] > 3.8 ** 2 * errs[2]
    assert errs[2] < 1e-3


def _conv_closed_form(tau, CA, yA, CB, yB, beta):
    # int A(tau - s) B(s) ds for A(x) = CA diag(phi(x; yA)) CA^T and
    # B(x) = CB diag(phi(x; yB)) CB^T (all levels distinct): the projector
    # pairs times the scalar convolution _closed_form
    out = np.zeros((CA.shape[0], CA.shape[0]))
    for a in range(len(yA)):
        Pa = np.outer(CA[:, a], CA[:, a])
        for b in range(len(yB)):
            out += (Pa @ np.outer(CB[:, b], CB[:, b])) * _closed_form(tau, yA[a], yB[b], beta)
    return out


def test_convolutions_of_noncommuting_matrices_match_closed_form():
    # matrix-valued pins of both convolutions: A and B do not commute, so a
    # transposed or swapped factor in conv1 (Sigma at the lag times g) or conv2
    # (g^0 at the lag times I1) fails; second order in the mesh
    rng = np.random.default_rng(17)
    beta = 10.0
    CA, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    CB, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    yA, yB = np.array([-0.35, 0.2, 0.9]), np.array([-0.5, 0.1, 0.7])
    dHF = 0.1 * W.random_symmetric(rng, 3)
    e1, e2 = [], []
    for u in (4, 8, 16):
        mesh = O.power_mesh(beta, u, 6)
        tau = mesh["tau"]
        A = O.g0_mesh(yA, CA, 0.0, tau, beta)
        B = O.g0_mesh(yB, CB, 0.0, tau, beta)
        ref = np.array([_conv_closed_form(t, CA, yA, CB, yB, beta) for t in tau])
        I1 = O.conv1(dHF, A, B, mesh, beta, O.lag_table(tau, beta))
        e1.append(float(np.max(np.abs(I1 - (dHF @ B + ref)))))
        I2 = O.conv2(B, yA, CA, 0.0, mesh, beta)
        e2.append(float(np.max(np.abs(I2 - ref))))
    for e in (e1, e2):
        assert e[0] > 3.5 * e[1] > 3.5 ** 2 * e[2], e
        assert e[2] < 1e-3


def _closed_form_diag(tau, y, beta):
    # the y_b -> y_a limit of _closed_form (the diagonal of a first-order change)
    f = 1.0 / (math.exp(beta * y) + 1.0)
    return -tau * f * f * math.exp(-tau * y) - (1.0 - f) * f * math.exp(-tau * y) * (tau + beta)


def test_closed_form_diag_is_the_limit():
    beta, y = 8.0, 0.6
    for t in (-7.5, -3.0, -0.25):
        assert abs(_closed_form_diag(t, y, beta) - _closed_form(t, y, y + 1e-6, beta)) < 1e-6


def _static_problem(rng, n=3):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    eps = np.array([-0.9, 0.6, 1.3])
    dh = 0.05 * W.random_symmetric(rng, n)
    F = (Q * eps) @ Q.T
    # V = 0 makes Sigma^corr[g] and Sigma^HF[g] vanish identically, and
    # Sigma0 = -dh turns the HF change dHF = Sigma^HF[g(0^-)] - Sigma0 into the
    # fixed perturbation dh: the oracle's own driver runs unmodified
    hf = dict(eps=eps, C=Q, mu=0.0, Sigma0=-dh)
    return F, np.zeros((n, n)), dh, hf


def test_static_perturbation_first_step_is_first_order_change():
    # from g = g^0 one step gives g_1 = (1 - a) g^0 + a sym(g^0 + I2), so
    # (g_1 - g^0) / a is the first-order change of g under dh: in the eigenbasis
    # of F, dh'_ab J(tau; y_a, y_b) (closed form), up to O(h^2) quadrature error.
    # A wrong mixing weight, a dropped or transposed factor in either
    # convolution, or a missing symmetrisation fails it.
    rng = np.random.default_rng(3)
    F, V, dh, hf = _static_problem(rng)
    beta, a = 8.0, 0.3
    y, Cm = hf["eps"], hf["C"]
    dhp = Cm.T @ dh @ Cm
    errs = []
    for u in (4, 8, 16):
        mesh = O.power_mesh(beta, u, 5)
        tau = mesh["tau"]
        lag = O.lag_table(tau, beta)
        G0 = O.g0_mesh(y, Cm, 0.0, tau, beta)
        step = O.dyson_iteration(F, V, 2.0, hf, mesh, lag, beta, G0, G0, a)
        assert np.max(np.abs(step["Sigma"])) == 0.0
        got = (step["G"] - G0) / a
        want = []
        for t in tau:
            J = np.array([[_closed_form(t, y[i], y[k], beta) if i != k else
                           _closed_form_diag(t, y[i], beta) for k in range(3)] for i in range(3)])
            want.append(Cm @ (dhp * J) @ Cm.T)
        errs.append(float(np.max(np.abs(got - np.array(want)))))
        # the update is symmetric although the sequential integration is not
        gn = G0 + step["I2"]
        assert np.max(np.abs(gn - gn.transpose(0, 2, 1))) > 1e-6
        assert np.max(np.abs(step["G"] - step["G"].transpose(0, 2, 1))) < 1e-15
    assert errs[0] > 3.5 * errs[1] > 3.5 ** 2 * errs[2]
    assert errs[2] < 1e-4


@pytest.mark.parametrize("mixing", [0.3, 0.5])
def test_static_perturbation_dyson_fixed_point(mixing):
    # Sigma^corr = 0 and a static dHF = dh through the oracle's own driver
    # (solve_2b -> dyson_iteration, symmetrised mixed update): the fixed point
    # is the Green's function of F + dh at the same mu (closed form by
    # diagonalisation) up to O(h^2) quadrature error; the residual contracts
    # by (1 - mixing) per step up to O(mixing |dh| / gap); the jump invariant
    # g(0^-) + g(-beta) = 1 holds.
    rng = np.random.default_rng(3)
    F, V, dh, hf = _static_problem(rng)
    beta = 8.0
    e2, C2 = np.linalg.eigh(F + dh)
    errs = []
    for u in (3, 6):
        res = O.solve_2b(F, V, 2.0, hf, beta, u, 5, mixing=mixing, tol=1e-13, max_iter=400)
        assert res["converged"]
        G = res["G"]
        assert np.max(np.abs(G[-1] + G[0] - np.eye(3))) < 1e-13
        assert np.max(np.abs(G - G.transpose(0, 2, 1))) < 1e-15
        ref = O.g0_mesh(e2, C2, 0.0, res["mesh"]["tau"], beta)
        errs.append(float(np.max(np.abs(G - ref))))
        r = np.array([h[1] for h in res["history"]])
        ratio = r[6:16] / r[5:15]
        assert np.all(np.abs(ratio - (1.0 - mixing)) < 0.08), ratio
    assert errs[1] < 2e-3 and errs[0] > 3.0 * errs[1]


@pytest.fixture(scope="module")
def he_small_solution():
    s = W.he_small()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, 0)
    T, v = O.kinetic(b), O.potential(b["nodes"], s.Z, s.R, 1.0)
    V = O.interaction(b["nodes"], 1.0)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    res = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, s.mixing, s.tol, 100)
    return s, b, T, v, V, h, hf, res


def test_sigma_zero_limit_returns_hf(he_small_solution):
    s, b, T, v, V, h, hf, res = he_small_solution
    mesh = res["mesh"]
    lag = O.lag_table(mesh["tau"], s.beta)
    G0 = res["G0"]
    step = O.dyson_iteration(h, V, 2.0, hf, mesh, lag, s.beta, G0, G0, 0.5, A=np.zeros_like(G0))
    assert np.max(np.abs(step["G"] - G0)) < 1e-12
    assert abs(step["E0"] - hf["E_hf"]) < 1e-12


def test_second_born_energy_ordering_and_invariants(he_small_solution):
    s, b, T, v, V, h, hf, res = he_small_solution
    assert res["converged"]
    Eex = O.exact_ground(T, v, V)
    E2, Ehf = res["E0"], hf["E_hf"]
    assert Ehf > E2 > Eex
    frac = (E2 - Ehf) / (Eex - Ehf)
    assert 0.4 < frac < 0.9
    assert abs(res["N"] - 2.0) < 1e-4
    G = res["G"]
    assert np.max(np.abs(G[-1] + G[0] - np.eye(b["n"]))) < 1e-13
    assert np.max(np.abs(res["Sigma"] - res["Sigma"].transpose(0, 2, 1))) < 1e-14
    # the first iteration's energy is the one-shot (MP2-like) estimate
    E_first = res["history"][0][2]
    e2 = 2.0 * O.mp2(hf["eps"], hf["C"], V, 1)
    assert abs((E_first - Ehf) - e2) < 0.01 * abs(e2)
