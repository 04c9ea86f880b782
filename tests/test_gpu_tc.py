"""Tensor-core (split-TF32) path vs the FP64 oracle: Sigma^(2) to 1e-5
max-norm relative, E0 to 1e-6 Ha (the reduced-precision bounds)."""
import functools

import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W
from tests._systems import maxrel, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
SIGMA_TOL = 1e-5
E0_TOL = 1e-6
# I1 = sum_j B_ij g_j: the terms of the two anti-periodic branches cancel, so
# the split-TF32 product error (2^-21 relative per product) is amplified by
# sum|terms| / |I1| (about 20-40 on the He models). Bound: 2^-21 x 100.
# The same bound covers the FP32 block sums: the tensor core's FP32
# accumulation rounds like truncation (a CPU emulation with round-toward-zero
# after every MMA reproduces the measured errors, round-to-nearest gives 20x
# less), so a block of N accumulation steps carries up to N 2^-24 of its
# magnitude (N = 3 x 5 x 33 = 495 on the random n = 257 case: 3e-5).
CONV_TOL = 5e-5
TF32 = 1
F16 = 3


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
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    ctx.solve_hf(s.beta, tol=1e-13)
    out = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100, precision=TF32)
    assert abs(out["E0"] - res["E0"]) < E0_TOL
    assert abs(out["N"] - res["N"]) < 1e-6


@pytest.mark.parametrize("n,u,p,beta,seed", [(8, 2, 3, 10.0, 0), (37, 2, 3, 25.0, 1),
                                             (130, 1, 3, 100.0, 2), (257, 1, 2, 100.0, 3)])
def test_conv1_tf32_random(ctx, n, u, p, beta, seed):
    rng = W.system_rng(98, seed)
    M = 2 * u * p + 1
    A = W.random_symmetric_stack(rng, M, n)
    G = W.random_symmetric_stack(rng, M, n)
    dHF = W.random_symmetric(rng, n, 0.1)
    I1 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_sigma_g(beta, u, p, _dev(dHF), _dev(A), _dev(G), I1, precision=TF32)
    torch.cuda.synchronize()
    mesh = O.power_mesh(beta, u, p)
    ref = O.conv1(dHF, A, G, mesh, beta, O.lag_table(mesh["tau"], beta))
    assert maxrel(I1.cpu().numpy(), ref) < CONV_TOL


def test_conv1_tf32_he_small_full(ctx):
    ref = oracle_system("he_small")
    s, hf, mesh, G0 = ref["sys"], ref["hf"], ref["mesh"], ref["G0"]
    A = O.sigma2(G0, ref["V"], 2.0)
    dHF = O.hf_selfenergy(G0[-1], ref["V"], 2.0) - hf["Sigma0"]
    I1 = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.conv_sigma_g(s.beta, s.u, s.p, _dev(dHF), _dev(A), _dev(G0), I1, precision=TF32)
    torch.cuda.synchronize()
    want = O.conv1(dHF, A, G0, mesh, s.beta, O.lag_table(mesh["tau"], s.beta))
    assert maxrel(I1.cpu().numpy(), want) < CONV_TOL


def _lag_rows(mesh, beta, rows):
    """The oracle's lag table filled only for the output rows `rows`."""
    M = len(mesh["tau"])
    lag = {"k": np.zeros((M, M), np.int32), "t": np.zeros((M, M)), "s": np.zeros((M, M))}
    for i in rows:
        for j in range(M):
            if i != j:
                y, sg = O.lag_point(mesh["tau"], beta, i, j)
                k, t = O.bracket(mesh["tau"], y)
                lag["k"][i, j], lag["t"][i, j], lag["s"][i, j] = k, t, sg
    return lag


@functools.lru_cache(maxsize=None)
def _he_medium_conv1_case():
    """He n_b=199, M=513 g^0 with a random symmetric Sigma stack of the
    magnitude of Sigma^(2)[g^0], a small dHF, and the oracle's I1 on rows
    spread over the mesh (both ends, the middle and two random rows)."""
    ref = oracle_system("he_medium")
    s, mesh, G0 = ref["sys"], ref["mesh"], ref["G0"]
    M, n = G0.shape[0], G0.shape[1]
    A = O.sigma2(G0[[0, M // 3, M - 1]], ref["V"], 2.0)  # realistic magnitudes
    rng = W.system_rng(99, 0)
    Afull = (np.max(np.abs(A)) * W.random_symmetric_stack(rng, M, n))
    dHF = W.random_symmetric(rng, n, 1e-4)
    rows = sorted({0, M // 2, M - 1, *map(int, rng.integers(1, M - 1, 2))})
    want = O.conv1(dHF, Afull, G0, mesh, s.beta, _lag_rows(mesh, s.beta, rows), rows=rows)
    return s, G0, Afull, dHF, rows, want


def test_conv1_tf32_he_medium_sampled_rows(ctx):
    s, G0, Afull, dHF, rows, want = _he_medium_conv1_case()
    I1 = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.conv1_splits(1)
    ctx.conv_sigma_g(s.beta, s.u, s.p, _dev(dHF), _dev(Afull), _dev(G0), I1, precision=TF32)
    torch.cuda.synchronize()
    assert maxrel(I1.cpu().numpy()[rows], want) < CONV_TOL


@pytest.mark.parametrize("splits", [1, 2, 3])
def test_conv1_f16_he_medium_sampled_rows(ctx, splits):
    # the benchmark's size: every 128-row tile flushes 13 FP32 blocks of 41 mesh
    # points into FP64, spread over `splits` CTAs (partial stacks summed after)
    s, G0, Afull, dHF, rows, want = _he_medium_conv1_case()
    I1 = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.conv1_splits(splits)
    ctx.conv_sigma_g(s.beta, s.u, s.p, _dev(dHF), _dev(Afull), _dev(G0), I1, precision=F16)
    torch.cuda.synchronize()
    assert ctx.conv1_splits() == splits
    ctx.conv1_splits(1)
    assert maxrel(I1.cpu().numpy()[rows], want) < CONV_TOL


def test_tf32_and_fp64_steps_agree_at_full_size():
    # three iterations of the He n_b=199, M=513 workload in both precisions
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    s = W.he_medium()
    out = {}
    for prec in (0, TF32):
        c = Context()
        c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
        c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
        c.solve_hf(s.beta, tol=1e-12)
        c.prepare_2b(s.beta, s.u, s.p, prec)
        Es = [c.step_2b(s.mixing)["E0"] for _ in range(3)]
        G = np.empty((s.n_tau, s.n_b, s.n_b))
        c.read_2b(G_out=G)
        out[prec] = (Es, G)
        c.close()
    for e64, e32 in zip(out[0][0], out[TF32][0]):
        assert abs(e64 - e32) < E0_TOL
    assert maxrel(out[TF32][1], out[0][1]) < 1e-6


@pytest.mark.parametrize("prec,splits", [(TF32, 3), (TF32, 8), (F16, 3), (F16, 12)])
def test_conv1_splits_agree(prec, splits):
    # the first convolution cut into mesh-point ranges of whole FP32
    # accumulation blocks (partial stacks summed in a fixed order): the block
    # sums do not depend on the split count, only the order of their FP64
    # additions does, so the iterates agree to FP64 rounding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    s = W.he_small()
    out = {}
    for S in (1, splits):
        c = Context()
        c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
        c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
        c.solve_hf(s.beta, tol=1e-12)
        c.conv1_splits(S)
        c.prepare_2b(s.beta, s.u, s.p, prec)
        assert c.conv1_splits() == S
        Es = [c.step_2b(s.mixing)["E0"] for _ in range(3)]
        G = np.empty((s.n_tau, s.n_b, s.n_b))
        c.read_2b(G_out=G)
        out[S] = (Es, G)
        c.close()
    for e1, es in zip(out[1][0], out[splits][0]):
        assert abs(e1 - es) < 1e-13
    assert maxrel(out[splits][1], out[1][1]) < 1e-13


def test_conv1_measured_split_choice_is_a_candidate():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    s = W.he_small()
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-12)
    c.prepare_2b(s.beta, s.u, s.p, TF32)
    S = c.conv1_splits()
    assert S in (1, 2, 3, 4, 6, 8, 12, 16)
    r = c.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100, precision=TF32)
    assert r["status"] == 0
    c.close()


@pytest.mark.parametrize("n,u,p,beta,seed", [(8, 2, 3, 10.0, 0), (37, 2, 3, 25.0, 1),
                                             (130, 1, 3, 100.0, 2), (257, 1, 2, 100.0, 3),
                                             # packed last column slice: 8 / TU mesh points
                                             # per chunk, TU = 2, 3, 4 and 4 with no full
                                             # slice, accumulation blocks of 26, 9, 10 and 13
                                             # mesh points (partial last groups)
                                             (74, 4, 16, 40.0, 4), (84, 2, 16, 40.0, 5),
                                             (93, 2, 16, 40.0, 6), (31, 4, 16, 40.0, 7)])
def test_conv1_f16_random(ctx, n, u, p, beta, seed):
    # FP16-split operands scaled into FP16's range carry 22 significant bits,
    # like the TF32 split (and half the accumulation steps): the same bound
    rng = W.system_rng(98, seed)
    M = 2 * u * p + 1
    A = W.random_symmetric_stack(rng, M, n)
    G = W.random_symmetric_stack(rng, M, n)
    dHF = W.random_symmetric(rng, n, 0.1)
    I1 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_sigma_g(beta, u, p, _dev(dHF), _dev(A), _dev(G), I1, precision=F16)
    torch.cuda.synchronize()
    mesh = O.power_mesh(beta, u, p)
    ref = O.conv1(dHF, A, G, mesh, beta, O.lag_table(mesh["tau"], beta))
    assert maxrel(I1.cpu().numpy(), ref) < CONV_TOL


def test_conv1_f16_small_magnitudes(ctx):
    # Sigma five orders of magnitude below 1: the operand scale keeps FP16 normal
    rng = W.system_rng(98, 7)
    n, u, p, beta = 37, 2, 3, 25.0
    M = 2 * u * p + 1
    A = 1e-5 * W.random_symmetric_stack(rng, M, n)
    G = W.random_symmetric_stack(rng, M, n)
    dHF = W.random_symmetric(rng, n, 1e-6)
    I1 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_sigma_g(beta, u, p, _dev(dHF), _dev(A), _dev(G), I1, precision=F16)
    torch.cuda.synchronize()
    mesh = O.power_mesh(beta, u, p)
    ref = O.conv1(dHF, A, G, mesh, beta, O.lag_table(mesh["tau"], beta))
    assert maxrel(I1.cpu().numpy(), ref) < CONV_TOL


def test_conv1_f16_he_small_full(ctx):
    ref = oracle_system("he_small")
    s, hf, mesh, G0 = ref["sys"], ref["hf"], ref["mesh"], ref["G0"]
    A = O.sigma2(G0, ref["V"], 2.0)
    dHF = O.hf_selfenergy(G0[-1], ref["V"], 2.0) - hf["Sigma0"]
    I1 = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.conv_sigma_g(s.beta, s.u, s.p, _dev(dHF), _dev(A), _dev(G0), I1, precision=F16)
    torch.cuda.synchronize()
    want = O.conv1(dHF, A, G0, mesh, s.beta, O.lag_table(mesh["tau"], s.beta))
    assert maxrel(I1.cpu().numpy(), want) < CONV_TOL


def test_solve_2b_f16_he_small_energy(ctx):
    ref = oracle_system("he_small")
    s = ref["sys"]
    res = O.solve_2b(ref["h"], ref["V"], 2.0, ref["hf"], s.beta, s.u, s.p, s.mixing, s.tol, 100)
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    ctx.solve_hf(s.beta, tol=1e-13)
    out = ctx.solve_2b(s.beta, s.u, s.p, s.mixing, s.tol, 100, precision=F16)
    assert abs(out["E0"] - res["E0"]) < E0_TOL
    assert abs(out["N"] - res["N"]) < 1e-6


def test_f16_and_fp64_steps_agree_at_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    s = W.he_medium()
    out = {}
    for prec in (0, F16):
        c = Context()
        c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
        c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
        c.solve_hf(s.beta, tol=1e-12)
        c.prepare_2b(s.beta, s.u, s.p, prec)
        Es = [c.step_2b(s.mixing)["E0"] for _ in range(3)]
        G = np.empty((s.n_tau, s.n_b, s.n_b))
        c.read_2b(G_out=G)
        out[prec] = (Es, G)
        c.close()
    for e64, e16 in zip(out[0][0], out[F16][0]):
        assert abs(e64 - e16) < E0_TOL
    assert maxrel(out[F16][1], out[0][1]) < 1e-6


@pytest.mark.parametrize("n,M,seed", [(8, 3, 0), (37, 3, 1), (130, 5, 2), (199, 3, 3),
                                      (257, 3, 4), (299, 3, 5)])
def test_sigma2_f16_random(ctx, n, M, seed):
    # exchange on kind::f16: g V scaled by 2^(11 - e) (max|V| < 2^e), gb by 2^12,
    # 22 significant bits per split operand as in the TF32 split
    rng = W.system_rng(96, seed)
    G = W.random_symmetric_stack(rng, M, n)
    V = W.random_symmetric(rng, n)
    S = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G), S, spin=2.0, precision=F16)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    assert maxrel(got, O.sigma2(G, V, 2.0)) < SIGMA_TOL
    assert np.array_equal(got, got.transpose(0, 2, 1))


def test_sigma2_f16_large_interaction(ctx):
    # |V| up to 40 (a soft-Coulomb with a short softening length): the A scale
    # follows max|V| so that g V stays inside FP16's range
    rng = W.system_rng(96, 9)
    n, M = 61, 3
    G = W.random_symmetric_stack(rng, M, n)
    V = 40.0 * W.random_symmetric(rng, n)
    S = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G), S, spin=1.0, precision=F16)
    torch.cuda.synchronize()
    assert maxrel(S.cpu().numpy(), O.sigma2(G, V, 1.0)) < SIGMA_TOL


def test_sigma2_f16_he_small(ctx):
    ref = oracle_system("he_small")
    G0 = ref["G0"]
    S = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(ref["V"]), _dev(G0), S, precision=F16)
    torch.cuda.synchronize()
    assert maxrel(S.cpu().numpy(), O.sigma2(G0, ref["V"], 2.0)) < SIGMA_TOL


@pytest.mark.parametrize("name", ["he_medium", "h3p_large"])
def test_sigma2_f16_full_size_sampled(ctx, name):
    ref = oracle_system(name)
    G0, V = ref["G0"], ref["V"]
    M = G0.shape[0]
    S = torch.empty(G0.shape, dtype=torch.float64, device="cuda")
    ctx.sigma2(_dev(V), _dev(G0), S, precision=F16)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    rng = np.random.default_rng(12)
    errs, scale = [], 0.0
    for j in [0, M // 2, M - 1] + list(rng.integers(0, M, 2)):
        full = O.sigma2_tau(G0[j], G0[M - 1 - j], V, 2.0)
        scale = max(scale, float(np.max(np.abs(full))))
        errs.append(float(np.max(np.abs(got[j] - full))))
    assert max(errs) / scale < SIGMA_TOL


@pytest.mark.parametrize("n,u,p,beta,seed", [(96, 1, 3, 100.0, 0), (130, 2, 2, 25.0, 1),
                                             (257, 1, 2, 100.0, 2)])
def test_conv2_split_random(ctx, n, u, p, beta, seed):
    # the split iteration's second convolution: split TF32 on the tensor cores
    # (n >= 96), FP32 eigen-kernel table; against the oracle's naive FP64 loop
    rng = W.system_rng(97, seed)
    M = 2 * u * p + 1
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    eps = np.sort(rng.uniform(-1.0, 2.0, n))
    mu = 0.5 * (eps[0] + eps[1])
    I1 = W.random_symmetric_stack(rng, M, n)
    I2 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_g0(beta, u, p, _dev(eps), _dev(Q), mu, _dev(I1), I2, precision=TF32)
    torch.cuda.synchronize()
    want = O.conv2(I1, eps, Q, mu, O.power_mesh(beta, u, p), beta)
    assert maxrel(I2.cpu().numpy(), want) < CONV_TOL


def test_conv2_split_he_medium_sampled_rows(ctx):
    # the benchmark's size (n_b = 199, M = 513) on the HF eigenbasis, I1 of the
    # magnitude the iteration produces
    ref = oracle_system("he_medium")
    s, hf, mesh, G0 = ref["sys"], ref["hf"], ref["mesh"], ref["G0"]
    M, n = G0.shape[0], G0.shape[1]
    rng = W.system_rng(97, 7)
    I1 = 1e-2 * W.random_symmetric_stack(rng, M, n)
    I2 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    ctx.conv_g0(s.beta, s.u, s.p, _dev(hf["eps"]), _dev(hf["C"]), hf["mu"], _dev(I1), I2,
                precision=F16)
    torch.cuda.synchronize()
    rows = [0, 1, M // 2, M - 2, M - 1]
    want = O.conv2(I1, hf["eps"], hf["C"], hf["mu"], mesh, s.beta, rows=rows)
    assert maxrel(I2.cpu().numpy()[rows], want) < CONV_TOL


def test_f16_split_refuses_g_out_of_range(ctx):
    # |g| = 20 cannot be held by the FP16 split scaled by 2^12: the device check
    # makes both FP16 stage calls return FEDVR_ERR_ARG instead of Inf/NaN, and
    # the context stays usable
    from paper_0911_4348_gb300 import FedvrError
    rng = W.system_rng(96, 11)
    n, u, p, beta = 37, 2, 3, 25.0
    M = 2 * u * p + 1
    G = W.random_symmetric_stack(rng, M, n)
    G[M // 2, 3, 5] = G[M // 2, 5, 3] = 20.0
    V = W.random_symmetric(rng, n)
    S = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(FedvrError) as e:
        ctx.sigma2(_dev(V), _dev(G), S, spin=2.0, precision=F16)
    assert e.value.code == -1 and "16" in str(e.value)
    I1 = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(FedvrError) as e:
        ctx.conv_sigma_g(beta, u, p, _dev(0.1 * V), _dev(G), _dev(G), I1, precision=F16)
    assert e.value.code == -1
    # the same inputs in split TF32 are accepted, and the context still works
    ctx.sigma2(_dev(V), _dev(G), S, spin=2.0, precision=TF32)
    G[M // 2, 3, 5] = G[M // 2, 5, 3] = 0.5
    ctx.sigma2(_dev(V), _dev(G), S, spin=2.0, precision=F16)
    torch.cuda.synchronize()
    assert maxrel(S.cpu().numpy(), O.sigma2(G, V, 2.0)) < SIGMA_TOL


def test_bounded_wait_gives_up_and_fails_the_context():
    # the kernels' bounded mbarrier wait on a barrier that nothing releases
    # (1 ms limit): the call returns FEDVR_ERR_TIMEOUT instead of hanging, and
    # the context then refuses further work with FEDVR_ERR_STATE
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context, FedvrError
    c = Context()
    c.selftest_wait(True, 1e-3)          # released first: the wait succeeds
    with pytest.raises(FedvrError) as e:
        c.selftest_wait(False, 1e-3)
    assert e.value.code == -5
    with pytest.raises(FedvrError) as e:
        c.build_fedvr(4, 5, -10.0, 10.0)
    assert e.value.code == -7
    c.close()
    torch.cuda.synchronize()             # the device context is unharmed
    c2 = Context()
    c2.selftest_wait(True, 1e-3)
    c2.close()


def test_measured_split_counts_are_kept_per_precision():
    # the two split precisions have different accumulation blocks, hence
    # different candidate split counts: preparing one after the other on the
    # same (n_b, M) must measure each in its own right
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    s = W.warmstart_system(0)
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-12)
    for prec in (TF32, F16, TF32):
        c.prepare_2b(s.beta, s.u, s.p, prec)
        assert c.conv1_splits() in (1, 2, 3, 4, 6, 8, 12, 16)
        assert c.step_2b(s.mixing)["status"] == 0
    c.close()
