"""Learned warm start on the GPU vs its FP64 CPU reference (oracle/mlp_oracle.py):
loss and gradients, FP32/BF16 inference, features, and the iteration gain."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from oracle import mlp_oracle as N
from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _flat(P):
    return np.concatenate([P[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def _unflat(v, din, H, dout):
    out, o = {}, 0
    for k, shp in (("W1", (din, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                   ("W3", (H, dout)), ("b3", (dout,))):
        size = int(np.prod(shp))
        out[k] = v[o:o + size].reshape(shp)
        o += size
    return out


@pytest.fixture(scope="module")
def net():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import WarmStartNet
    M, H = 17, 32
    n = WarmStartNet(M, H, seed=5)
    yield n, M, H
    n.close()


def test_loss_and_gradient_match_oracle(net):
    n, M, H = net
    din = 2 * M + 3
    rng = W.system_rng(82, 0)
    P = N.init_params(din, H, M, rng)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0.0, 0.05, P[k].shape)
    X = rng.normal(size=(300, din))
    T = rng.normal(size=(300, M))
    n.set_params(_flat(P).astype(np.float32))
    P32 = _unflat(_flat(P).astype(np.float32).astype(np.float64), din, H, M)
    y, cache = N.forward(P32, X.astype(np.float32).astype(np.float64))
    want_loss = N.loss(y, T.astype(np.float32).astype(np.float64))
    want = N.backward(P32, cache, y, T.astype(np.float32).astype(np.float64))
    loss, grad = n.loss_grad(torch.from_numpy(X.astype(np.float32)).cuda(),
                             torch.from_numpy(T.astype(np.float32)).cuda())
    assert abs(loss - want_loss) < 1e-5 * want_loss
    got = _unflat(grad.astype(np.float64), din, H, M)
    for k in want:
        scale = np.max(np.abs(want[k]))
        assert np.max(np.abs(got[k] - want[k])) < 1e-4 * scale, k


def test_forward_fp32_and_bf16(net):
    n, M, H = net
    din = 2 * M + 3
    rng = W.system_rng(83, 0)
    P = N.init_params(din, H, M, rng)
    n.set_params(_flat(P).astype(np.float32))
    X = rng.normal(size=(129, din)).astype(np.float32)
    want = N.forward(P, X.astype(np.float64))[0]
    Y = torch.empty((129, M), dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    n.forward(Xd, Y, bf16=False)
    torch.cuda.synchronize()
    assert np.max(np.abs(Y.cpu().numpy() - want)) < 1e-5 * np.max(np.abs(want))
    n.forward(Xd, Y, bf16=True)
    torch.cuda.synchronize()
    # bf16 weights (8-bit significand): relative error of a few 2^-8
    assert np.max(np.abs(Y.cpu().numpy() - want)) < 3e-2 * np.max(np.abs(want))


def _he(z, seed):
    return W.System(f"He Z={z:.3f}", -20.0, 20.0, 10, 4, [z], [0.0], u=4, p=16)


def _ctx(s):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-12)
    return c


def test_collected_features_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import WarmStartNet
    s = _he(2.0, 0)
    M = s.n_tau
    net = WarmStartNet(M, 64, seed=1)
    c = _ctx(s)
    net.collect(c, s.beta, s.u, s.p)
    X, _ = net.get_rows(0, net.rows())
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, 0)
    T_, v = O.kinetic(b), O.potential(b["nodes"], s.Z, s.R, 1.0)
    V = O.interaction(b["nodes"], 1.0)
    hf = O.hf_scf(T_ + np.diag(v), V, 2.0, 1, s.beta, tol=1e-12)
    mesh = O.power_mesh(s.beta, s.u, s.p)
    G0 = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], s.beta)
    F, _ = N.features(O.sigma2(G0, V, 2.0), G0, V, b["nodes"], s.xmax - s.xmin)
    assert X.shape == F.shape
    # FP32 features of a split-TF32 one-shot Sigma (1e-5 relative) and FP64 g^0
    assert np.max(np.abs(X - F)) < 2e-5
    c.close()
    net.close()


def test_warm_start_reduces_iterations_on_held_out_systems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import WarmStartNet
    rng = W.system_rng(84, 0)
    train_z = rng.uniform(1.5, 2.5, 12)
    s0 = _he(2.0, 0)
    net = WarmStartNet(s0.n_tau, 128, seed=2)
    for k, z in enumerate(train_z):
        c = _ctx(_he(float(z), k))
        net.collect(c, s0.beta, s0.u, s0.p)
        c.close()
    loss = net.train(60, batch=1024, lr=1e-3)
    assert np.isfinite(loss)
    plain_it, warm_it = [], []
    for z in (1.77, 2.31):
        s = _he(z, 99)
        c = _ctx(s)
        ref = c.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 200, precision=1)
        hist = c.get_history()
        plain_it.append(next(i for i in range(len(hist))
                             if np.all(np.abs(hist[i:, 2] - ref["E0"]) <= 1e-6)) + 1)
        c.warm_start(net, s.beta, s.u, s.p, inner_steps=4)
        out = c.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 200, precision=1)
        assert abs(out["E0"] - ref["E0"]) < 1e-6  # same fixed point
        hw = c.get_history()
        warm_it.append(next(i for i in range(len(hw))
                            if np.all(np.abs(hw[i:, 2] - ref["E0"]) <= 1e-6)) + 1)
        c.close()
    print("iterations to E0 within 1e-6 Ha: plain", plain_it, "warm", warm_it)
    assert sum(warm_it) < sum(plain_it), (plain_it, warm_it)
    net.close()
