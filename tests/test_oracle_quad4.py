"""Pins for the oracle's fourth-order variant of the Dyson integrals (Sec. 2.3,
Eq. deq; the paper's "direct integration" names no rule): the cubic-per-interval
weights, cubic lag interpolation, and fourth-order convergence of both
convolutions and of the static-perturbation fixed point to closed forms."""
import math

import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W
from tests.test_oracle_dyson import _closed_form, _closed_form_diag, _conv_closed_form


def test_quad4_weights_integrate_cubics_exactly():
    rng = np.random.default_rng(5)
    meshes = [np.sort(rng.uniform(-3.0, 2.0, m + 1)) for m in (1, 2, 3, 4, 9, 17)]
    meshes.append(O.power_mesh(10.0, 4, 6)["tau"][:23])  # a side of the power mesh
    for x in meshes:
        w = O.quad4_weights(x)
        a, b = float(x[0]), float(x[-1])
        deg = min(3, len(x) - 1)
        for d in range(deg + 1):
            exact = (b ** (d + 1) - a ** (d + 1)) / (d + 1)
            assert abs(np.sum(w * x ** d) - exact) < 1e-12 * max(1.0, abs(exact))


def test_cubic_lag_reproduces_cubics_and_mesh_values():
    beta = 10.0
    tau = O.power_mesh(beta, 3, 5)["tau"]
    f = lambda x: 0.3 * x ** 3 - x ** 2 + 2.0 * x - 0.7
    vals = f(tau)
    rng = np.random.default_rng(6)
    for y in list(rng.uniform(-beta, 0.0, 50)) + [float(tau[0]), float(tau[-1])]:
        s0, cl = O.cubic_lag(tau, y)
        assert 0 <= s0 <= len(tau) - 4
        assert abs(sum(c * vals[s0 + q] for q, c in enumerate(cl)) - f(y)) < 1e-11
    for k in range(len(tau)):  # at a mesh point the value itself, exactly
        s0, cl = O.cubic_lag(tau, float(tau[k]))
        assert sum(c * vals[s0 + q] for q, c in enumerate(cl)) == vals[k]


def _phi_scalar(x, y, beta):
    return float(O.phi(x, np.array([y]), beta)[0])


def test_convolutions_converge_at_fourth_order():
    beta = 10.0
    rng = np.random.default_rng(17)
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
        I1 = O.conv1(dHF, A, B, mesh, beta, None, quad="cubic4")
        e1.append(float(np.max(np.abs(I1 - (dHF @ B + ref)))))
        I2 = O.conv2(B, yA, CA, 0.0, mesh, beta, quad="cubic4")
        e2.append(float(np.max(np.abs(I2 - ref))))
    for e in (e1, e2):  # ratios approach 16 per mesh halving (the default rule: 4)
        assert e[0] > 10.0 * e[1] and e[1] > 12.0 * e[2], e
        assert e[2] < 1e-6
    # and well below the default rule's error on the finest mesh
    mesh = O.power_mesh(beta, 16, 6)
    tau = mesh["tau"]
    A = O.g0_mesh(yA, CA, 0.0, tau, beta)
    B = O.g0_mesh(yB, CB, 0.0, tau, beta)
    ref = np.array([_conv_closed_form(t, CA, yA, CB, yB, beta) for t in tau])
    trap = O.conv1(dHF, A, B, mesh, beta, O.lag_table(tau, beta))
    assert e1[2] < 0.01 * float(np.max(np.abs(trap - (dHF @ B + ref))))


def test_static_perturbation_fixed_point_at_fourth_order():
    # the whole loop (solve_2b -> dyson_iteration with quad="cubic4"), Sigma^corr = 0
    # and dHF = dh as in the default-rule pin: fourth-order convergence to the
    # Green's function of F + dh, jump invariant exact
    rng = np.random.default_rng(3)
    n, beta = 3, 8.0
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    eps = np.array([-0.9, 0.6, 1.3])
    dh = 0.05 * W.random_symmetric(rng, n)
    F = (Q * eps) @ Q.T
    hf = dict(eps=eps, C=Q, mu=0.0, Sigma0=-dh)
    e2, C2 = np.linalg.eigh(F + dh)
    errs = []
    for u in (3, 6):
        res = O.solve_2b(F, np.zeros((n, n)), 2.0, hf, beta, u, 5, mixing=0.5, tol=1e-13,
                         max_iter=400, quad="cubic4")
        assert res["converged"]
        G = res["G"]
        assert np.max(np.abs(G[-1] + G[0] - np.eye(n))) < 1e-13
        ref = O.g0_mesh(e2, C2, 0.0, res["mesh"]["tau"], beta)
        errs.append(float(np.max(np.abs(G - ref))))
    assert errs[0] > 10.0 * errs[1], errs
    assert errs[1] < 2e-5
