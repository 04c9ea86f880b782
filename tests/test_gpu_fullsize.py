"""The benchmark system (He n_b = 199, M = 513) solved to convergence on the
GPU against the FP64 oracle's stored converged solution
(tests/golden/he_medium_2b.txt, written by make_he_medium_2b.py, which runs
only the oracle): the split-FP16 path (the benchmark's default) within the
reduced-precision bounds at every iteration and at convergence, and the
plain FP64 path's first iterations to rounding."""
import os

import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "he_medium_2b.txt")
F16, FP64 = 3, 0
E0_TOL = 1e-6      # the split paths' energy bound (FP32-level products)
SIGMA_TOL = 1e-5   # Sigma^(2) max-norm relative bound of the split paths


def _golden():
    vals, e_hist, r_hist = {}, [], []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()[:2]
            if k.startswith("E0_iter_"):
                e_hist.append(float(v))
            elif k.startswith("res_iter_"):
                r_hist.append(float(v))
            else:
                vals[k] = float(v)
    return vals, np.array(e_hist), np.array(r_hist)


def _ctx(s):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    E_hf, _ = c.solve_hf(s.beta, tol=1e-13)
    return c, E_hf


def test_split_f16_solve_converges_to_the_oracle_solution():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = W.he_medium()
    ref, e_hist, _ = _golden()
    assert ref["converged"] == 1
    ctx, E_hf = _ctx(s)
    assert abs(E_hf - ref["E_hf"]) < 1e-10
    M, n = s.n_tau, s.n_b
    G = np.empty((M, n, n))
    r = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 80, precision=F16, G_out=G)
    assert r["status"] == 0
    assert abs(r["E0"] - ref["E0"]) < E0_TOL
    assert abs(r["N"] - ref["N"]) < E0_TOL
    # the iteration tracks the oracle's step by step, not only at the end
    hist = ctx.get_history()
    k = min(hist.shape[0], e_hist.size)
    assert abs(hist.shape[0] - int(ref["iterations"])) <= 2
    assert np.max(np.abs(hist[:k, 2] - e_hist[:k])) < E0_TOL
    # the converged g keeps the anti-periodic jump g(0^-) + g(-beta) = 1
    assert np.max(np.abs(G[-1] + G[0] - np.eye(n))) < 1e-6
    # Sigma^(2) of the final g from the split kernels, sampled against the oracle
    V = ctx.get_operators()["V"]
    Gd = torch.from_numpy(G).cuda()
    S = torch.empty_like(Gd)
    ctx.sigma2(torch.from_numpy(V).cuda(), Gd, S, precision=F16)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    errs, scale = [], 0.0
    for j in (0, 1, M // 3, M // 2, M - 2, M - 1):
        full = O.sigma2_tau(G[j], G[M - 1 - j], V, 2.0)
        scale = max(scale, float(np.max(np.abs(full))))
        errs.append(float(np.max(np.abs(got[j] - full))))
    assert max(errs) / scale < SIGMA_TOL
    ctx.close()


def test_fp64_first_iterations_match_the_oracle_history():
    # three FP64 iterations (about 8 s each) against the oracle's recorded E0
    # and residual of the same iterations
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = W.he_medium()
    ref, e_hist, r_hist = _golden()
    ctx, _ = _ctx(s)
    ctx.prepare_2b(s.beta, s.u, s.p, FP64)
    for k in range(3):
        got = ctx.step_2b(s.mixing)
        assert abs(got["E0"] - e_hist[k]) < 1e-10, k
        # the residual is stored to 7 significant digits
        assert abs(got["res"] - r_hist[k]) < 1e-6 * r_hist[k], k
    ctx.close()
