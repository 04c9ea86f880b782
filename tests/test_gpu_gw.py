"""GW self-energy on the GPU (the two-index bubble series of the screened
interaction, FP64 path) against the oracle's ``sigma_gw`` and GW solve."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _he_small():
    from paper_0911_4348_gb300 import Context
    s = W.he_small()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    h = O.kinetic(b) + np.diag(O.potential(b["nodes"], s.Z, s.R, s.soft_en))
    V = O.interaction(b["nodes"], s.soft_ee)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    ctx = Context()
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    ctx.solve_hf(s.beta, tol=1e-13)
    return s, h, V, hf, ctx


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_sigma_gw_matches_oracle_and_restarts_from_its_w():
    _need_gpu()
    s, h, V, hf, ctx = _he_small()
    u, p = s.u, s.p
    mesh = O.power_mesh(s.beta, u, p)
    G0 = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], s.beta)
    ref = O.sigma_gw(G0, V, 2.0, mesh, O.bose_lag_table(mesh["tau"], s.beta))
    Vd, Gd = torch.from_numpy(V).cuda(), torch.from_numpy(G0).cuda()
    Sd, wd = torch.empty_like(Gd), torch.empty_like(Gd)
    it = ctx.sigma_gw(s.beta, u, p, Vd, Gd, Sd, w=wd)
    assert abs(it - ref["iters"]) <= 1
    assert _rel(Sd.cpu().numpy(), ref["Sigma"]) < 1e-10
    assert _rel(wd.cpu().numpy(), ref["w"]) < 1e-10
    # restarted from its own converged w the iteration stops at once
    S2 = torch.empty_like(Gd)
    it2 = ctx.sigma_gw(s.beta, u, p, Vd, Gd, S2, w=wd, w_valid=True)
    assert it2 <= 2
    assert _rel(S2.cpu().numpy(), ref["Sigma"]) < 1e-10
    ctx.close()


def test_gw_argument_errors():
    _need_gpu()
    from paper_0911_4348_gb300 import FedvrError
    s, h, V, hf, ctx = _he_small()
    # (kind 2 is the T-matrix; 3 is no kind)
    for bad in ((3, 0.3, 1e-12, 10), (1, 0.0, 1e-12, 10), (1, 1.5, 1e-12, 10), (1, 0.3, 0.0, 10),
                (1, 0.3, 1e-12, 0)):
        with pytest.raises(FedvrError) as e:
            ctx.set_self_energy(*bad)
        assert e.value.code == -1
    ctx.set_self_energy("gw")
    with pytest.raises(FedvrError) as e:   # split precisions keep second Born
        ctx.prepare_2b(s.beta, s.u, s.p, 3)
    assert e.value.code == -1
    # an inner iteration that cannot converge in its budget is reported, not hidden
    ctx.set_self_energy("gw", w_mixing=0.3, w_tol=1e-14, w_max_iter=3)
    ctx.prepare_2b(s.beta, s.u, s.p, 0)
    with pytest.raises(FedvrError) as e:
        ctx.step_2b(0.5)
    assert e.value.code == -3
    ctx.close()


def test_gw_solve_matches_oracle():
    # the self-consistent GW iteration of the small He model (129-point mesh):
    # energy, particle number and every iteration's E0 against the oracle; then
    # the same context back on second Born reproduces that solve
    _need_gpu()
    s, h, V, hf, ctx = _he_small()
    ref = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, 0.5, 1e-8, 100, self_energy="gw")
    ctx.set_self_energy("gw")
    got = ctx.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 100, precision=0)
    assert got["status"] == 0
    assert abs(got["iters"] - ref["iters"]) <= 1
    assert abs(got["E0"] - ref["E0"]) < 1e-9
    assert abs(got["N"] - ref["N"]) < 1e-9
    hist = ctx.get_history()
    k = min(hist.shape[0], len(ref["history"]))
    assert np.max(np.abs(hist[:k, 2] - np.array([r[2] for r in ref["history"]])[:k])) < 1e-9
    assert abs(ctx.gw_last_inner() - ref["gw_inner"][-1]) <= 1
    ref2 = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, 0.5, 1e-8, 100)
    ctx.set_self_energy("2b")
    got2 = ctx.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 100, precision=0)
    assert abs(got2["E0"] - ref2["E0"]) < 1e-10
    assert got["E0"] < got2["E0"]
    ctx.close()
