"""Pins for the oracle's real-time Kadanoff-Baym propagation (Sec. 2, Eqs.
kbe, skkbe, skkbesigma): free propagation in closed form, conservation of N
and E, and agreement with exact two-electron dynamics to third order in the
interaction (time-dependent HF only to second)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fedvr_oracle as O


def _model():
    b = O.fedvr_basis(2, 2, -3.0, 3.0, 0)
    T = O.kinetic(b)
    v = O.potential(b["nodes"], [2.0], [0.0], 1.0)
    V = O.interaction(b["nodes"], 1.0)
    h = T + np.diag(v)
    # a kicked initial determinant: the lowest orbital of h + 0.3 x, evolved under h
    e, C = np.linalg.eigh(h + 0.3 * np.diag(b["nodes"]))
    return h, V, C[:, 0], b


def test_free_propagation_matches_closed_form_at_second_order():
    h, V, phi0, _ = _model()
    rho0 = np.outer(phi0, phi0)
    errs = []
    for dt in (0.1, 0.05):
        ns = int(round(1.0 / dt))
        r = O.kbe_propagate(h, 0.0 * V, 2.0, rho0, dt, ns)
        U = sla.expm(-1j * h)
        errs.append(max(float(np.max(np.abs(r["rho"][ns] - U @ rho0 @ U.conj().T))),
                        float(np.max(np.abs(r["L"][ns, 0] - U @ rho0)))))
    assert errs[0] > 3.8 * errs[1] and errs[1] < 1e-3


def test_second_born_conserves_particle_number_and_energy():
    h, V, phi0, _ = _model()
    rho0 = np.outer(phi0, phi0)
    drift = []
    for dt in (0.1, 0.05):
        r = O.kbe_propagate(h, V, 2.0, rho0, dt, int(round(2.0 / dt)))
        assert np.max(np.abs(r["N"] - 2.0)) < 1e-12
        assert np.max(np.abs(r["rho"] - r["rho"].conj().transpose(0, 2, 1))) < 1e-14
        drift.append(float(np.max(r["E"]) - np.min(r["E"])))
        # the correlation energy builds up from zero: the conserved total is not trivially flat
        assert abs(r["E"][-1] - r["E"][0]) < 1e-3 < float(np.max(np.abs(np.diff(r["rho"], axis=0))))
    assert drift[0] > 3.0 * drift[1] and drift[1] < 1e-4


def test_second_born_dynamics_exact_to_third_order_in_the_interaction():
    # from an uncorrelated determinant the exact self-energy is HF + second Born
    # up to O(V^3): the KBE error against exact two-electron dynamics falls 8x per
    # halving of the coupling, time-dependent HF's only 4x. The free evolution
    # is subtracted on both sides, so the time-step error of the O(1) part drops out.
    h, V, phi0, _ = _model()
    rho0 = np.outer(phi0, phi0)
    dt, ns = 0.02, 50
    times = np.arange(ns + 1) * dt
    free_exact = O.exact_dynamics(h, 0.0 * V, phi0, times)
    free_kbe = O.kbe_propagate(h, 0.0 * V, 2.0, rho0, dt, ns)["rho"]
    e2, e1 = [], []
    for lam in (0.4, 0.2, 0.1):
        ex = O.exact_dynamics(h, lam * V, phi0, times) - free_exact
        r2 = O.kbe_propagate(h, lam * V, 2.0, rho0, dt, ns)["rho"] - free_kbe
        r1 = O.kbe_propagate(h, lam * V, 2.0, rho0, dt, ns, second_born=False)["rho"] - free_kbe
        e2.append(float(np.max(np.abs(r2 - ex))))
        e1.append(float(np.max(np.abs(r1 - ex))))
    for k in range(2):
        assert e2[k] > 6.5 * e2[k + 1], e2
        assert 3.5 < e1[k] / e1[k + 1] < 4.5, e1
    assert e2[-1] < 0.05 * e1[-1]


def test_realtime_self_energy_reduces_to_matsubara_form_for_symmetric_arguments():
    # for real symmetric arguments (the Matsubara case) the real-time form is the
    # same function as sigma2_tau
    rng = np.random.default_rng(4)
    n = 5
    g = rng.normal(size=(n, n)); g = g + g.T
    gb = rng.normal(size=(n, n)); gb = gb + gb.T
    V = rng.normal(size=(n, n)); V = V + V.T
    assert np.max(np.abs(O.sigma2_realtime(g, gb, V, 2.0) - O.sigma2_tau(g, gb, V, 2.0))) < 1e-12
