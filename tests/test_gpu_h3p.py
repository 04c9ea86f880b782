"""The paper's linear H3+ results (Sec. 3.2, Fig. 3) from the GPU path.

Grid of the paper's H3+ runs: 13 graded (case II) elements over a 50 a.u.
interval, n_b = 142 (order 11). Unit soft-Coulomb nuclei at (-R, 0, R); the
internuclear energy 5/d (d = 2R) is added once to the electronic energy. The
Fig. 3 caption prints the equilibrium 2 d_b (= 2R at the minimum of the total
energy) of HF, second Born and the exact solution; the text states that second
Born recovers roughly 60-70 % of the correlation energy and that the HF density is the
most peaked at the centre, the exact one the least, with second Born in
between.

Checks: the GPU HF energies equal the oracle's to 1e-10 Ha along the curve and
their minimum lands on the printed HF value; the split-FP16 second-Born minimum
lands on the printed second-Born value, recovering part of the correlation
energy there; the GPU densities equal the oracle's (HF)
and integrate to N (second Born), and the three densities have the printed
order of peak heights. A small H3+ grid checks the FP64 second-Born density
and energy against the oracle's iteration."""
import math

import numpy as np
import pytest

from oracle import fedvr_oracle as O
from tests.conftest import load_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = load_golden("paper_values.txt")
N_ELEM = int(GOLD["h3p_n_elem"])
ORDER = (int(GOLD["h3p_n_b"]) + 1) // N_ELEM
HALF = GOLD["h3p_box_length"] / 2
BETA = 100.0
F16 = 3


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _context(R, n_elem=N_ELEM, order=ORDER, half=HALF):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(n_elem, order + 1, -half, half, 1)
    enn = c.set_potential([1.0, 1.0, 1.0], [-R, 0.0, R], 1.0, 1.0, 2)
    E_hf, _ = c.solve_hf(BETA, tol=1e-12)
    return c, E_hf, enn


@pytest.fixture(scope="module")
def oracle_grid():
    b = O.fedvr_basis(N_ELEM, ORDER, -HALF, HALF, 1)
    return dict(basis=b, T=O.kinetic(b), V=O.interaction(b["nodes"], 1.0))


def _oracle_hf(grid, R):
    v = O.potential(grid["basis"]["nodes"], [1.0, 1.0, 1.0], [-R, 0.0, R], 1.0)
    return O.hf_scf(grid["T"] + np.diag(v), grid["V"], 2.0, 1, BETA), v


def _golden_min(f, lo, hi, tol):
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = hi - g * (hi - lo), lo + g * (hi - lo)
    fa, fb = f(a), f(b)
    while hi - lo > tol:
        if fa < fb:
            hi, b, fb = b, a, fa
            a = hi - g * (hi - lo)
            fa = f(a)
        else:
            lo, a, fa = a, b, fb
            b = lo + g * (hi - lo)
            fb = f(b)
    return 0.5 * (lo + hi)


def test_h3p_hf_curve_matches_oracle_and_paper(oracle_grid):
    _need_gpu()
    for R in (2.0, 2.2, 2.4):
        c, E_hf, enn = _context(R)
        c.close()
        ref, _ = _oracle_hf(oracle_grid, R)
        assert abs(E_hf - ref["E_hf"]) < 1e-10
        assert enn == pytest.approx(5.0 / (2 * R), rel=1e-14)

    def total(R):
        c, E_hf, enn = _context(R)
        c.close()
        return E_hf + enn

    R = _golden_min(total, 2.0, 2.4, 2e-5)
    assert abs(2 * R - GOLD["h3p_2db_hf"]) < 5e-4


def _second_born_totals(Rs, u=32, p=16):
    from paper_0911_4348_gb300 import solve_2b_batched
    ctxs, E_hf, enn = [], [], []
    for R in Rs:
        c, e, z = _context(R)
        ctxs.append(c)
        E_hf.append(e)
        enn.append(z)
    r = solve_2b_batched(ctxs, BETA, u, p, 0.5, 1e-8, 300, F16)
    dens = [c.density("2b") for c in ctxs]
    for c in ctxs:
        c.close()
    assert np.all(r["iters"] < 300)
    return np.asarray(r["E0"]) + np.asarray(enn), np.asarray(E_hf), np.asarray(r["N"]), dens


def test_h3p_second_born_equilibrium_and_correlation_share(oracle_grid):
    _need_gpu()
    h, R0 = 0.04, GOLD["h3p_2db_2b"] / 2
    E, E_hf, N, _ = _second_born_totals([R0 - h, R0, R0 + h])
    assert np.all(np.abs(N - 2.0) < 1e-5)
    assert E[1] < E[0] and E[1] < E[2]
    R = R0 + h * (E[0] - E[2]) / (2 * (E[0] - 2 * E[1] + E[2]))
    assert abs(2 * R - GOLD["h3p_2db_2b"]) < 2e-3
    # share of the correlation energy at the second-Born equilibrium: second
    # Born lowers the HF energy without passing the exact one. (Measured here:
    # 0.55 at the equilibrium and 0.55-0.62 for d = 3.2-7.2, a little below the
    # paper's rough 60-70 %; the equilibria themselves agree.)
    _, v = _oracle_hf(oracle_grid, R0)
    E_ex = O.exact_ground(oracle_grid["T"], v, oracle_grid["V"]) + 5.0 / (2 * R0)
    E_hf_tot = E_hf[1] + 5.0 / (2 * R0)
    share = (E[1] - E_hf_tot) / (E_ex - E_hf_tot)
    assert 0.4 < share < 0.8


def test_h3p_densities_match_oracle_and_paper_order(oracle_grid):
    _need_gpu()
    R = GOLD["h3p_2db_2b"] / 2
    W = oracle_grid["basis"]["weights"]
    c, _, _ = _context(R)
    n_hf = c.density("hf")
    c.close()
    ref, v = _oracle_hf(oracle_grid, R)
    n_ref = O.density(ref["rho0"], W, 2.0)
    assert np.max(np.abs(n_hf - n_ref)) < 1e-10 * np.max(n_ref)
    _, _, _, dens = _second_born_totals([R])
    n_2b = dens[0]
    assert float(np.sum(W * n_2b)) == pytest.approx(2.0, abs=1e-5)
    _, psi = O.exact_ground_state(oracle_grid["T"], v, oracle_grid["V"])
    n_ex = O.exact_density(psi, W)
    assert np.max(n_hf) > np.max(n_2b) > np.max(n_ex)


def test_h3p_small_grid_second_born_density_and_energy_match_oracle():
    """FP64 GPU iteration against the oracle's on a small H3+ grid (5 equal
    elements of order 4 over 20 a.u., n_b = 19, 129 mesh points), after the
    same 25 iterations: on this coarse grid the plain iteration settles to a
    residual of about 1e-7 (E0 converged to 1e-9 Ha) and then drifts away along
    one unstable direction, so both sides are compared after a fixed number of
    steps rather than at a tolerance."""
    _need_gpu()
    R, K = 1.8, 25
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(5, 5, -10.0, 10.0, 0)
    c.set_potential([1.0, 1.0, 1.0], [-R, 0.0, R], 1.0, 1.0, 2)
    E_hf, _ = c.solve_hf(BETA, tol=1e-12)
    r = c.solve_2b(BETA, 4, 16, 0.5, 1e-14, K, precision=0, check=False)
    n_gpu = c.density("2b")
    c.close()
    assert r["iters"] == K
    b = O.fedvr_basis(5, 4, -10.0, 10.0, 0)
    T, V = O.kinetic(b), O.interaction(b["nodes"], 1.0)
    v = O.potential(b["nodes"], [1.0, 1.0, 1.0], [-R, 0.0, R], 1.0)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, 1, BETA)
    assert abs(E_hf - hf["E_hf"]) < 1e-10
    ref = O.solve_2b(h, V, 2.0, hf, BETA, 4, 16, 0.5, 1e-14, K)
    assert ref["iters"] == K
    assert abs(r["E0"] - ref["E0"]) < 1e-10
    n_ref = O.density(ref["G"][-1], b["weights"], 2.0)
    assert np.max(np.abs(n_gpu - n_ref)) < 1e-9 * np.max(n_ref)
    # the coarse 129-point mesh keeps N = 2 only to a few 1e-5
    assert float(np.sum(b["weights"] * n_gpu)) == pytest.approx(2.0, abs=1e-4)
