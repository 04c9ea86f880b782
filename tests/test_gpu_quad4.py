"""The fourth-order variant of the Dyson integrals (fedvr_set_quadrature(4),
FP64 path) against the oracle's quad="cubic4", its order of accuracy, and the
chemical-potential override (fedvr_set_mu) against the oracle at the same mu."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W
from tests._systems import maxrel, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.set_quadrature(4)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("n,u,p,beta,seed", [(8, 2, 3, 10.0, 0), (37, 3, 4, 25.0, 1),
                                             (70, 1, 3, 100.0, 2)])
def test_conv1_quad4_random(ctx, n, u, p, beta, seed):
    rng = W.system_rng(94, seed)
    M = 2 * u * p + 1
    A = W.random_symmetric_stack(rng, M, n)
    G = W.random_symmetric_stack(rng, M, n)
    dHF = W.random_symmetric(rng, n, 0.1)
    I1 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_sigma_g(beta, u, p, _dev(dHF), _dev(A), _dev(G), I1)
    torch.cuda.synchronize()
    want = O.conv1(dHF, A, G, O.power_mesh(beta, u, p), beta, None, quad="cubic4")
    assert maxrel(I1.cpu().numpy(), want) < TOL


@pytest.mark.parametrize("n,u,p,beta,seed", [(8, 2, 3, 10.0, 0), (37, 2, 4, 25.0, 1)])
def test_conv2_quad4_random(ctx, n, u, p, beta, seed):
    rng = W.system_rng(93, seed)
    M = 2 * u * p + 1
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    eps = np.sort(rng.uniform(-1.0, 2.0, n))
    mu = 0.5 * (eps[0] + eps[1])
    I1 = W.random_symmetric_stack(rng, M, n)
    I2 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_g0(beta, u, p, _dev(eps), _dev(Q), mu, _dev(I1), I2)
    torch.cuda.synchronize()
    want = O.conv2(I1, eps, Q, mu, O.power_mesh(beta, u, p), beta, quad="cubic4")
    assert maxrel(I2.cpu().numpy(), want) < TOL


def _small_he():
    # He on a coarse grid with a short mesh: the oracle's fourth-order solve
    # finishes in seconds
    return W.System("He n=11 M=49", -8.0, 8.0, 3, 4, [2.0], [0.0], beta=10.0, u=4, p=6)


def _oracle_solve(s, quad, mu=None):
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    T, v = O.kinetic(b), O.potential(b["nodes"], s.Z, s.R, s.soft_en)
    V = O.interaction(b["nodes"], s.soft_ee)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, s.n_elec // 2, s.beta, tol=1e-13)
    if mu is not None:
        hf = dict(hf, mu=mu)
    return O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, s.mixing, s.tol, 100, quad=quad), hf


def _gpu_solve(s, quad, mu=None, u=None):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-13)
    c.set_quadrature(quad)
    if mu is not None:
        c.set_mu(mu)
    r = c.solve_2b(s.beta, s.u if u is None else u, s.p, s.mixing, s.tol, 200)
    hist = c.get_history()
    c.close()
    return r, hist


def test_solve_2b_quad4_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = _small_he()
    ref, _ = _oracle_solve(s, "cubic4")
    got, hist = _gpu_solve(s, 4)
    assert ref["converged"] and got["status"] == 0
    assert abs(got["E0"] - ref["E0"]) < 1e-10
    assert abs(got["N"] - ref["N"]) < 1e-10
    assert got["iters"] == ref["iters"]
    for (k, res, e, nel), row in zip(ref["history"], hist):
        assert abs(row[2] - e) < 1e-10 and abs(row[3] - nel) < 1e-10


def test_quad4_energy_converges_faster_in_the_mesh():
    # the fourth-order rule at a coarse mesh lands closer to the converged
    # energy than the trapezoid at a four times finer mesh
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = W.he_small()  # n_b = 15, beta = 100, p = 16
    e = {}
    for quad, u in ((2, 4), (2, 16), (4, 4), (4, 8), (4, 16)):
        r, _ = _gpu_solve(s, quad, u=u)
        assert r["status"] == 0
        e[quad, u] = r["E0"]
    ref = e[4, 16]
    assert abs(e[4, 8] - ref) < abs(e[2, 16] - ref)
    assert abs(e[4, 4] - ref) < 0.5 * abs(e[2, 4] - ref)


def test_mu_override_matches_oracle():
    # beta = 10: thermal occupation across the gap makes N depend on mu, so the
    # override is a real change; the GPU solve equals the oracle's at that mu
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = _small_he()
    ref0, hf = _oracle_solve(s, "trap")
    e0, e1 = hf["eps"][0], hf["eps"][1]
    mu1 = e0 + 0.7 * (e1 - e0)
    ref1, _ = _oracle_solve(s, "trap", mu=mu1)
    assert abs(ref1["N"] - ref0["N"]) > 1e-4
    got1, _ = _gpu_solve(s, 2, mu=mu1)
    assert abs(got1["E0"] - ref1["E0"]) < 1e-10 and abs(got1["N"] - ref1["N"]) < 1e-10


def test_mu_dependence_inside_the_gap_is_quadrature_error():
    # beta = 100, He n_b = 15: the exact E0 does not depend on mu inside the HF
    # gap, but g(tau) ~ exp(-tau (eps - mu)) does, so the discrete tau integrals
    # carry a mu-dependent error. Its spread over mu = 1/4, 1/2, 3/4 of the gap
    # shrinks at fourth order with the fourth-order rule and is ten times below
    # the trapezoid's at the same mesh
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    s = W.he_small()
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-13)
    eps = c.get_hf()["eps"]
    spread = {}
    for quad, u in ((2, 8), (4, 4), (4, 8)):
        c.set_quadrature(quad)
        E = []
        for f in (0.25, 0.5, 0.75):
            c.set_mu(eps[0] + f * (eps[1] - eps[0]))
            r = c.solve_2b(s.beta, u, s.p, s.mixing, 1e-11, 300)
            E.append(r["E0"])
        spread[quad, u] = max(E) - min(E)
    c.close()
    assert spread[4, 8] < 0.1 * spread[2, 8]
    assert spread[4, 4] > 8.0 * spread[4, 8]
