"""GPU vs oracle: the two tau-convolutions (Eq. deq) and the full FP64
second-Born self-consistency, plus the error paths of the C ABI."""
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
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _empty(shape):
    return torch.empty(shape, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,u,p,beta,seed", [(1, 2, 3, 10.0, 0), (37, 2, 3, 25.0, 1),
                                             (70, 1, 4, 100.0, 2)])
def test_conv1_random(ctx, n, u, p, beta, seed):
    rng = W.system_rng(91, seed)
    M = 2 * u * p + 1
    A = W.random_symmetric_stack(rng, M, n)
    G = W.random_symmetric_stack(rng, M, n)
    dHF = W.random_symmetric(rng, n, 0.1)
    I1 = _empty((M, n, n))
    ctx.conv_sigma_g(beta, u, p, _dev(dHF), _dev(A), _dev(G), I1)
    torch.cuda.synchronize()
    mesh = O.power_mesh(beta, u, p)
    ref = O.conv1(dHF, A, G, mesh, beta, O.lag_table(mesh["tau"], beta))
    assert maxrel(I1.cpu().numpy(), ref) < TOL


@pytest.mark.parametrize("n,u,p,beta,seed", [(1, 2, 3, 10.0, 0), (37, 2, 3, 25.0, 1),
                                             (70, 1, 4, 100.0, 2)])
def test_conv2_random(ctx, n, u, p, beta, seed):
    rng = W.system_rng(92, seed)
    M = 2 * u * p + 1
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    eps = np.sort(rng.uniform(-1.0, 2.0, n))
    mu = 0.05
    I1 = W.random_symmetric_stack(rng, M, n)
    I2 = _empty((M, n, n))
    ctx.conv_g0(beta, u, p, _dev(eps), _dev(Q), mu, _dev(I1), I2)
    torch.cuda.synchronize()
    ref = O.conv2(I1, eps, Q, mu, O.power_mesh(beta, u, p), beta)
    assert maxrel(I2.cpu().numpy(), ref) < TOL


def test_conv1_conv2_he_small_full(ctx):
    ref = oracle_system("he_small")
    s, hf, mesh, G0 = ref["sys"], ref["hf"], ref["mesh"], ref["G0"]
    A = O.sigma2(G0, ref["V"], 2.0)
    dHF = O.hf_selfenergy(G0[-1], ref["V"], 2.0) - hf["Sigma0"]
    I1 = _empty(G0.shape)
    ctx.conv_sigma_g(s.beta, s.u, s.p, _dev(dHF), _dev(A), _dev(G0), I1)
    want1 = O.conv1(dHF, A, G0, mesh, s.beta, O.lag_table(mesh["tau"], s.beta))
    I2 = _empty(G0.shape)
    ctx.conv_g0(s.beta, s.u, s.p, _dev(hf["eps"]), _dev(hf["C"]), hf["mu"], _dev(want1), I2)
    torch.cuda.synchronize()
    assert maxrel(I1.cpu().numpy(), want1) < TOL
    want2 = O.conv2(want1, hf["eps"], hf["C"], hf["mu"], mesh, s.beta)
    assert maxrel(I2.cpu().numpy(), want2) < TOL


def test_conv1_conv2_he_medium_sampled_rows(ctx):
    ref = oracle_system("he_medium")
    s, hf, mesh, G0 = ref["sys"], ref["hf"], ref["mesh"], ref["G0"]
    M = G0.shape[0]
    rng = W.system_rng(93, 0)
    A = 1e-3 * W.random_symmetric_stack(rng, M, G0.shape[1])
    dHF = W.random_symmetric(rng, G0.shape[1], 1e-4)
    I1 = _empty(G0.shape)
    ctx.conv_sigma_g(s.beta, s.u, s.p, _dev(dHF), _dev(A), _dev(G0), I1)
    I2 = _empty(G0.shape)
    ctx.conv_g0(s.beta, s.u, s.p, _dev(hf["eps"]), _dev(hf["C"]), hf["mu"], I1, I2)
    torch.cuda.synchronize()
    got1, got2 = I1.cpu().numpy(), I2.cpu().numpy()
    rows = [0, 1, M // 2, M - 2, M - 1]
    lag = {"k": np.zeros((M, M), np.int32), "t": np.zeros((M, M)), "s": np.zeros((M, M))}
    for i in rows:
        for j in range(M):
            if i != j:
                y, sg = O.lag_point(mesh["tau"], s.beta, i, j)
                k, t = O.bracket(mesh["tau"], y)
                lag["k"][i, j], lag["t"][i, j], lag["s"][i, j] = k, t, sg
    want1 = O.conv1(dHF, A, G0, mesh, s.beta, lag, rows=rows)
    assert maxrel(got1[rows], want1) < TOL
    want2 = O.conv2(got1, hf["eps"], hf["C"], hf["mu"], mesh, s.beta, rows=rows)
    assert maxrel(got2[rows], want2) < 1e-11


@pytest.fixture(scope="module")
def he_small_2b():
    ref = oracle_system("he_small")
    s = ref["sys"]
    res = O.solve_2b(ref["h"], ref["V"], 2.0, ref["hf"], s.beta, s.u, s.p, s.mixing, s.tol, 100)
    return ref, res


def test_solve_2b_he_small_matches_oracle(ctx, he_small_2b):
    ref, res = he_small_2b
    s = ref["sys"]
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    ctx.solve_hf(s.beta, tol=1e-13)
    M, n = s.n_tau, s.n_b
    G, S, tau = np.empty((M, n, n)), np.empty((M, n, n)), np.empty(M)
    out = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100, G_out=G, Sigma_out=S, tau_out=tau)
    assert abs(out["E0"] - res["E0"]) < 1e-10
    assert abs(out["N"] - res["N"]) < 1e-10
    assert abs(out["iters"] - res["iters"]) <= 1
    assert np.array_equal(tau, res["mesh"]["tau"])
    # g(tau) inherits the HF eigenvalue conditioning (relative ~ beta * |d eps|)
    assert maxrel(G, res["G"]) < 1e-9
    assert maxrel(S, res["Sigma"]) < 1e-9
    assert np.max(np.abs(G[-1] + G[0] - np.eye(n))) < 1e-13
    hist = ctx.get_history()
    assert hist.shape == (out["iters"], 5) and hist[-1, 1] < s.tol
    assert np.allclose(hist[:, 2], [h[2] for h in res["history"][:len(hist)]], atol=1e-10)


def test_solve_2b_device_outputs_and_warm_start(ctx, he_small_2b):
    ref, res = he_small_2b
    s = ref["sys"]
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    ctx.solve_hf(s.beta, tol=1e-13)
    M, n = s.n_tau, s.n_b
    G, S = _empty((M, n, n)), _empty((M, n, n))
    out = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100, G_out=G, Sigma_out=S)
    # restart from the converged Sigma: same fixed point, fewer iterations
    ctx.set_initial_sigma(S)
    out2 = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100)
    assert abs(out2["E0"] - out["E0"]) < 1e-8
    assert out2["iters"] <= out["iters"]


def test_error_paths(ctx):
    from paper_0911_4348_gb300 import FedvrError, Context
    c = Context()
    with pytest.raises(FedvrError) as e:
        c.solve_hf(100.0)
    assert e.value.code == -7  # out of order
    with pytest.raises(FedvrError) as e:
        c.build_fedvr(0, 5, -1.0, 1.0)
    assert e.value.code == -1
    with pytest.raises(FedvrError) as e:
        c.build_fedvr(4, 5, 1.0, -1.0)
    assert e.value.code == -1
    c.build_fedvr(4, 5, -10.0, 10.0)
    with pytest.raises(FedvrError) as e:
        c.set_potential([2.0], [0.0], n_elec=3)
    assert e.value.code == -1
    c.set_potential([2.0], [0.0])
    c.solve_hf(100.0, tol=1e-13)
    with pytest.raises(FedvrError) as e:
        c.solve_2b(50.0, 4, 16)  # beta differs from the HF solution
    assert e.value.code == -1
    # non-convergence is reported, results still returned
    out = c.solve_2b(100.0, 2, 4, max_iter=2, check=False)
    assert out["status"] == -3 and out["iters"] == 2
    # a NaN in the starting self-energy is caught by the residual guard
    M, n = 17, 15
    bad = np.zeros((M, n, n))
    bad[3, 2, 2] = np.nan
    c.set_initial_sigma(bad)
    out = c.solve_2b(100.0, 2, 4, max_iter=5, check=False)
    assert out["status"] == -6
    c.close()
