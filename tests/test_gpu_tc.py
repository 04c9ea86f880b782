"""Tensor-core (split-TF32) path vs the FP64 oracle: Sigma^(2) to 1e-5
max-norm relative, E0 to 1e-6 Ha (the reduced-precision bounds)."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W
from tests._systems import maxrel, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
SIGMA_TOL = 1e-5
E0_TOL = 1e-6
TF32 = 1


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


@pytest.mark.parametrize("n,M,seed", [(8, 3, 0), (37, 3, 1), (130, 5, 2), (199, 3, 3),
                                      (257, 3, 4), (299, 3, 5)])
def test_sigma2_tf32_random(ctx, n, M, seed):
    rng = W.system_rng(96, seed)
    G = W.random_symmetric_stack(rng, M, n)
    V = W.random_symmetric(rng, n)
    S = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G), S, spin=2.0, precision=TF32)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    ref = O.sigma2(G, V, 2.0)
    assert maxrel(got, ref) < SIGMA_TOL
    assert np.array_equal(got, got.transpose(0, 2, 1))


def test_sigma2_tf32_he_small(ctx):
    ref = oracle_system("he_small")
    G0 = ref["G0"]
    S = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(ref["V"]), _dev(G0), S, precision=TF32)
    torch.cuda.synchronize()
    assert maxrel(S.cpu().numpy(), O.sigma2(G0, ref["V"], 2.0)) < SIGMA_TOL


@pytest.mark.parametrize("name", ["he_medium", "h3p_large"])
def test_sigma2_tf32_full_size_sampled(ctx, name):
    ref = oracle_system(name)
    G0, V = ref["G0"], ref["V"]
    M, n = G0.shape[0], G0.shape[1]
    S = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G0), S, precision=TF32)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    rng = np.random.default_rng(11)
    errs, scale = [], 0.0
    for j in [0, M // 2, M - 1] + list(rng.integers(0, M, 2)):
        full = O.sigma2_tau(G0[j], G0[M - 1 - j], V, 2.0)
        scale = max(scale, float(np.max(np.abs(full))))
        errs.append(float(np.max(np.abs(got[j] - full))))
    assert max(errs) / scale < SIGMA_TOL


def test_solve_2b_tf32_he_small_energy(ctx):
    ref = oracle_system("he_small")
    s = ref["sys"]
    res = O.solve_2b(ref["h"], ref["V"], 2.0, ref["hf"], s.beta, s.u, s.p, s.mixing, s.tol, 100)
    ctx.build_fedvr(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    ctx.solve_hf(s.beta, tol=1e-13)
    out = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100, precision=TF32)
    assert abs(out["E0"] - res["E0"]) < E0_TOL
    assert abs(out["N"] - res["N"]) < 1e-6
