"""T-matrix self-energy on the GPU (the particle-particle ladder of the
two-index interaction, FP64 path) against the oracle's ``sigma_tmatrix`` and
its self-consistent solve."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _he5():
    # He on 2 elements x 4 GLL points (n_b = 5), box [-6, 6], beta = 20, 33-point mesh
    return W.System("He n_b=5", -6.0, 6.0, 2, 3, [2.0], [0.0], beta=20.0, u=2, p=8)


def _oracle(s):
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    h = O.kinetic(b) + np.diag(O.potential(b["nodes"], s.Z, s.R, s.soft_en))
    V = O.interaction(b["nodes"], s.soft_ee)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    return h, V, hf


def _ctx(s):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-13)
    return c


@pytest.mark.parametrize("n,beta,u,p,seed", [(4, 10.0, 2, 4, 0), (7, 15.0, 2, 4, 1)])
def test_sigma_tmatrix_matches_oracle_and_restarts_from_its_ladder(n, beta, u, p, seed):
    _need_gpu()
    from paper_0911_4348_gb300 import Context
    rng = W.system_rng(97, seed)
    h = W.random_symmetric(rng, n, 1.0)
    V = np.abs(W.random_symmetric(rng, n, 0.3))
    eps, C = np.linalg.eigh(h)
    mu = 0.5 * (eps[n // 2 - 1] + eps[n // 2])
    mesh = O.power_mesh(beta, u, p)
    G = O.g0_mesh(eps, C, mu, mesh["tau"], beta)
    ref = O.sigma_tmatrix(G, V, 2.0, mesh, O.bose_lag_table(mesh["tau"], beta))
    M = G.shape[0]
    ctx = Context()
    Vd, Gd = torch.from_numpy(V).cuda(), torch.from_numpy(G).cuda()
    Sd = torch.empty_like(Gd)
    td = torch.empty((M, n, n, n, n), dtype=torch.float64, device="cuda")
    it = ctx.sigma_tmatrix(beta, u, p, Vd, Gd, Sd, t=td)
    assert abs(it - ref["iters"]) <= 1
    assert _rel(Sd.cpu().numpy(), ref["Sigma"]) < 1e-10
    # the library's ladder layout t[j][b][l][a][k] holds the oracle's t[j, a, k, b, l]
    assert _rel(td.cpu().numpy().transpose(0, 3, 4, 1, 2), ref["t"]) < 1e-10
    # restarted from its own converged ladder the iteration stops at once
    S2 = torch.empty_like(Gd)
    it2 = ctx.sigma_tmatrix(beta, u, p, Vd, Gd, S2, t=td, t_valid=True)
    assert it2 <= 2
    assert _rel(S2.cpu().numpy(), ref["Sigma"]) < 1e-10
    # lowest order: one damped step from V^ K V^ is not second Born, but the
    # ladder's source closed with the hole line is (the oracle's pin, on the GPU)
    S0 = torch.empty_like(Gd)
    ctx.sigma_tmatrix(beta, u, p, Vd, Gd, S0, t_mixing=1e-300, t_tol=1e300, t_max_iter=1)
    assert _rel(S0.cpu().numpy(), O.sigma2(G, V, 2.0)) < 1e-12
    ctx.close()


def test_tmatrix_solve_matches_oracle():
    # the self-consistent T-matrix iteration of a small He model: iterations,
    # energy, particle number and every iteration's E0 against the oracle; E0
    # lies between HF and second Born (the ladder weakens the repulsive
    # scattering that second Born treats to second order)
    _need_gpu()
    s = _he5()
    h, V, hf = _oracle(s)
    ref = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, 0.5, 1e-8, 100, self_energy="tmatrix")
    assert ref["converged"]
    ctx = _ctx(s)
    ctx.set_self_energy("tmatrix")
    got = ctx.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 100, precision=0)
    assert got["status"] == 0
    assert abs(got["iters"] - ref["iters"]) <= 1
    assert abs(got["E0"] - ref["E0"]) < 1e-9
    assert abs(got["N"] - ref["N"]) < 1e-9
    hist = ctx.get_history()
    k = min(hist.shape[0], len(ref["history"]))
    assert np.max(np.abs(hist[:k, 2] - np.array([r[2] for r in ref["history"]])[:k])) < 1e-9
    assert abs(ctx.gw_last_inner() - ref["gw_inner"][-1]) <= 1
    ctx.set_self_energy("2b")
    got2 = ctx.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 100, precision=0)
    assert hf["E_hf"] > got["E0"] > got2["E0"]
    ctx.close()


def test_tmatrix_argument_errors():
    _need_gpu()
    from paper_0911_4348_gb300 import Context, FedvrError
    s = _he5()
    ctx = _ctx(s)
    for bad in ((3, 0.3, 1e-12, 10), (2, 0.0, 1e-12, 10), (2, 0.3, -1.0, 10), (2, 0.3, 1e-12, 0)):
        with pytest.raises(FedvrError) as e:
            ctx.set_self_energy(*bad)
        assert e.value.code == -1
    ctx.set_self_energy("tmatrix")
    with pytest.raises(FedvrError) as e:  # split precisions keep second Born
        ctx.prepare_2b(s.beta, s.u, s.p, 3)
    assert e.value.code == -1
    ctx.close()
    big = Context()  # n_b = 35: pair space too large for the ladder
    big.build_fedvr(9, 5, -10.0, 10.0, 0)
    big.set_potential([2.0], [0.0], 1.0, 1.0, 2)
    big.solve_hf(20.0, tol=1e-10)
    big.set_self_energy("tmatrix")
    with pytest.raises(FedvrError) as e:
        big.prepare_2b(20.0, 2, 4, 0)
    assert e.value.code == -1
    Gd = torch.zeros((17, 33, 33), dtype=torch.float64, device="cuda")
    Vd = torch.zeros((33, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(FedvrError) as e:
        big.sigma_tmatrix(20.0, 2, 4, Vd, Gd, torch.empty_like(Gd))
    assert e.value.code == -1
    big.close()
