"""Pins for the oracle's basis, one-body and interaction matrices (Sec. 2.1-2.2)."""
import math

import numpy as np
import pytest

from oracle import fedvr_oracle as O
from tests.conftest import load_golden

PAPER = load_golden("paper_values.txt")


@pytest.mark.parametrize("order,xi_ref,w_ref", [
    # textbook Lobatto rules (Abramowitz & Stegun 25.4.32)
    (2, [-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
     [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_gll_closed_forms(order, xi_ref, w_ref):
    xi, w = O.gll(order)
    np.testing.assert_allclose(xi, xi_ref, atol=2e-16, rtol=0)
    np.testing.assert_allclose(w, w_ref, rtol=4e-15, atol=0)


@pytest.mark.parametrize("order", [1, 5, 7, 10, 15])
def test_gll_roots_match_legendre_derivative_roots_and_exactness(order):
    xi, w = O.gll(order)
    assert len(xi) == order + 1 and xi[0] == -1.0 and xi[-1] == 1.0
    assert np.all(np.diff(xi) > 0)
    if order >= 2:
        ref = np.sort(np.polynomial.legendre.Legendre.basis(order).deriv().roots().real)
        np.testing.assert_allclose(xi[1:-1], ref, atol=1e-13)
    assert abs(w.sum() - 2.0) < 1e-14
    # Lobatto quadrature with order+1 points is exact up to degree 2*order - 1
    for deg in range(0, 2 * order):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * xi ** deg) - exact) < 1e-13, deg


def test_lagrange_derivative_differentiates_polynomials():
    xi, _ = O.gll(6)
    d = O.lagrange_deriv(xi)
    # sum_m p(xi_m) f'_m(xi_k) = p'(xi_k) for deg p <= 6
    for deg in range(7):
        p = xi ** deg
        dp = deg * xi ** (deg - 1) if deg else np.zeros_like(xi)
        np.testing.assert_allclose(p @ d, dp, atol=1e-11)


def test_basis_dimension_matches_paper():
    # n_b = n_e n_g - 1 (Eq. basisdim) with the paper's grids
    b = O.fedvr_basis(int(PAPER["he_case2_n_elem"]), int(PAPER["he_case2_order"]),
                      -100.0, 100.0, 1)
    assert b["n"] == int(PAPER["he_case2_n_b"])
    assert 13 * 11 - 1 == int(PAPER["h3p_n_b"])
    b = O.fedvr_basis(13, 11, -25.0, 25.0, 1)
    assert b["n"] == int(PAPER["h3p_n_b"])


def test_nodes_weights_index_map():
    b = O.fedvr_basis(5, 4, -3.0, 7.0, 0)
    n = b["n"]
    assert n == 5 * 4 - 1
    X, W = b["nodes"], b["weights"]
    assert np.all(np.diff(X) > 0) and X[0] > -3.0 and X[-1] < 7.0
    # quadrature sum of all weights (box ends excluded) integrates 1 over the box
    wl = b["wloc"]
    assert abs(W.sum() + wl[0][0] + wl[-1][-1] - 10.0) < 1e-13
    # bridge nodes are exactly the element edges
    for a in range(n):
        if b["local"][a] == 4:
            assert X[a] == b["edges"][b["elem"][a] + 1]
    # graded grid (case II) centre element is 1 a.u. wide
    e = np.array(O.element_edges(7, -10.0, 10.0, 1))
    w = np.diff(e)
    assert abs(w[3] - 1.0) < 1e-14 and np.all(np.diff(w[3:]) > 0)
    assert abs(w.sum() - 20.0) < 1e-13


def test_kinetic_symmetric_and_element_sparse():
    b = O.fedvr_basis(6, 5, -5.0, 5.0, 0)
    T = O.kinetic(b)
    assert np.array_equal(T, T.T)
    n, N = b["n"], b["order"]
    for a in range(n):
        for c in range(n):
            qa, qc = a + 1, c + 1
            share = any(i * N <= qa <= (i + 1) * N and i * N <= qc <= (i + 1) * N
                        for i in range(b["n_elem"]))
            if not share:
                assert T[a, c] == 0.0


def test_particle_in_box_spectrum():
    L = 10.0
    b = O.fedvr_basis(8, 8, 0.0, L, 0)
    ev = np.linalg.eigvalsh(O.kinetic(b))
    ref = np.array([(k * math.pi / L) ** 2 / 2 for k in range(1, 6)])
    np.testing.assert_allclose(ev[:5], ref, rtol=1e-10)


def test_particle_in_box_converges_spectrally_in_order():
    L = 10.0
    ref = (3 * math.pi / L) ** 2 / 2
    errs = []
    for order in (3, 5, 7):
        b = O.fedvr_basis(4, order, 0.0, L, 0)
        errs.append(abs(np.linalg.eigvalsh(O.kinetic(b))[2] - ref))
    assert errs[0] > 50 * errs[1] > 0 and errs[1] > 50 * errs[2]


def test_harmonic_oscillator_spectrum():
    b = O.fedvr_basis(20, 10, -9.0, 9.0, 0)
    h = O.kinetic(b) + np.diag(0.5 * b["nodes"] ** 2)
    ev = np.linalg.eigvalsh(h)
    np.testing.assert_allclose(ev[:6], np.arange(6) + 0.5, atol=1e-12)


def test_potential_and_interaction_values():
    X = np.array([-1.5, 0.0, 2.0])
    v = O.potential(X, [1.0, 2.0], [-1.0, 1.0], 1.0)
    ref = [-(1 / math.sqrt(0.25 + 1) + 2 / math.sqrt(6.25 + 1)),
           -(1 / math.sqrt(2.0) + 2 / math.sqrt(2.0)),
           -(1 / math.sqrt(10.0) + 2 / math.sqrt(2.0))]
    np.testing.assert_allclose(v, ref, rtol=1e-15)
    V = O.interaction(X, 1.0)
    assert np.array_equal(V, V.T) and np.all(np.diag(V) == 1.0)
    assert abs(V[0, 2] - 1 / math.sqrt(3.5 ** 2 + 1)) < 1e-16


@pytest.mark.parametrize("ne,order,kind", [(4, 4, 0), (6, 7, 1), (9, 5, 0)])
def test_interaction_eigen_route_equals_direct(ne, order, kind):
    b = O.fedvr_basis(ne, order, -20.0, 20.0, kind)
    V = O.interaction(b["nodes"], 1.0)
    Vr = O.interaction_eigen_route(b, 1.0)
    assert np.max(np.abs(Vr - V)) / np.max(np.abs(V)) < 1e-12
