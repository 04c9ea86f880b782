"""GPU vs oracle: Hartree-Fock (Sec. 2.3, Eqs. sigmahf, hamhf, hfgf) and the
FP64 second-Born self-energy (Eq. sigma2ndb). Tolerance: max-norm relative 1e-12."""
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


@pytest.mark.parametrize("name", ["he_small", "he_medium"])
def test_hf_matches_oracle(ctx, name):
    ref = oracle_system(name)
    s = ref["sys"]
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    E, mu = ctx.solve_hf(s.beta, tol=1e-13, max_iter=500)
    hf = ref["hf"]
    assert abs(E - hf["E_hf"]) < 1e-12
    got = ctx.get_hf()
    # eigenvalues carry the conditioning of the operator norm (kinetic ~1e2 Ha)
    assert np.max(np.abs(got["eps"] - hf["eps"])) < 1e-10 * max(1.0, np.max(np.abs(hf["eps"])))
    assert abs(mu - hf["mu"]) < 1e-10
    assert maxrel(got["rho0"], hf["rho0"]) < TOL
    assert maxrel(got["Sigma0"], hf["Sigma0"]) < 1e-11
    # orthonormal eigenvectors
    Cm = got["C"]
    assert np.max(np.abs(Cm.T @ Cm - np.eye(Cm.shape[0]))) < 1e-12


@pytest.mark.parametrize("n,M,seed", [(1, 3, 0), (37, 9, 1), (64, 5, 2), (70, 7, 3), (129, 3, 4)])
def test_sigma2_random_symmetric(ctx, n, M, seed):
    rng = W.system_rng(90, seed)
    G = W.random_symmetric_stack(rng, M, n)
    V = W.random_symmetric(rng, n)
    S = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G), S, spin=2.0)
    torch.cuda.synchronize()
    ref = O.sigma2(G, V, 2.0)
    assert maxrel(S.cpu().numpy(), ref) < TOL


def test_sigma2_he_small_full(ctx):
    ref = oracle_system("he_small")
    G0 = ref["G0"]
    S = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(ref["V"]), _dev(G0), S)
    torch.cuda.synchronize()
    want = O.sigma2(G0, ref["V"], 2.0)
    assert maxrel(S.cpu().numpy(), want) < TOL


@pytest.mark.parametrize("name", ["he_medium", "h3p_large"])
def test_sigma2_full_size_sampled(ctx, name):
    ref = oracle_system(name)
    G0, V = ref["G0"], ref["V"]
    M, n = G0.shape[0], G0.shape[1]
    S = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G0), S)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    rng = np.random.default_rng(7)
    js = [0, M // 2, M - 1] + list(rng.integers(0, M, 3))
    scale = 0.0
    errs = []
    for j in js:
        pairs = [(0, 0), (n - 1, n - 1), (n // 2, n // 3), (n - 1, 0)] + \
            [tuple(x) for x in rng.integers(0, n, (4, 2))]
        for a, b in pairs:
            want = O.sigma2_element(G0[j], G0[M - 1 - j], V, 2.0, a, b)
            errs.append(abs(got[j, a, b] - want))
        scale = max(scale, float(np.max(np.abs(O.sigma2_tau(G0[j], G0[M - 1 - j], V, 2.0)))))
    assert max(errs) / scale < TOL
    # exact symmetry of the mirrored lower triangle
    assert np.array_equal(got, got.transpose(0, 2, 1))
