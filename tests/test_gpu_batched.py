"""Batched second Born: systems of different n_b and mesh size advanced
together by one tensor-core launch per kernel per iteration give exactly what
the same systems give one at a time, and match the FP64 oracle's energy."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TF32 = 1


def _systems():
    # meshes fine enough for the iteration to converge (coarse ones diverge in the
    # oracle as well: the scheme needs both p >= 10 and enough points per octave)
    a = W.he_small()                                                    # n=15,  M=129
    b = W.System("He n=39", -20.0, 20.0, 10, 4, [2.0], [0.0], u=4, p=16)    # n=39,  M=129
    c = W.System("H3+ n=59", -30.0, 30.0, 10, 6, [1.0, 1.0, 1.0], [-1.6, 0.0, 1.6], u=8, p=16)
    d = W.System("He n=139", -40.0, 40.0, 20, 7, [1.8], [0.0], u=4, p=16)   # two M tiles
    return [a, b, c, d]


def _ctx(s):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-12)
    return c


def test_batched_equals_single_system_solves():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import solve_2b_batched
    systems = _systems()
    single = []
    for s in systems:
        c = _ctx(s)
        c.conv1_splits(1)  # the batched queue runs unsplit convolution tiles
        single.append(c.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 150, precision=TF32, check=False))
        c.close()
    ctxs = [_ctx(s) for s in systems]
    ctxs[0].conv1_splits(1)  # the batch's own split count, as the single solves'
    out = solve_2b_batched(ctxs, [s.beta for s in systems], [s.u for s in systems],
                           [s.p for s in systems], 0.5, 1e-8, 150, TF32, check=False)
    assert out["status"] == min(r["status"] for r in single)
    for k, s in enumerate(systems):
        assert out["iters"][k] == single[k]["iters"], s.name
        assert out["E0"][k] == single[k]["E0"], s.name
        assert out["N"][k] == single[k]["N"], s.name
        hist = ctxs[k].get_history()
        assert hist.shape[0] == out["iters"][k]
        if single[k]["status"] == 0:
            assert hist[-1, 1] < 1e-8
    for c in ctxs:
        c.close()


def test_batched_energy_matches_oracle_he_small():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import solve_2b_batched
    s = W.he_small()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, 0)
    T, v = O.kinetic(b), O.potential(b["nodes"], s.Z, s.R, 1.0)
    V = O.interaction(b["nodes"], 1.0)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, 1, s.beta, tol=1e-13)
    ref = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, 0.5, 1e-8, 100)
    ctxs = [_ctx(s), _ctx(W.System("He n=39", -20.0, 20.0, 10, 4, [2.0], [0.0], u=4, p=16))]
    out = solve_2b_batched(ctxs, [s.beta, 100.0], [s.u, 4], [s.p, 16])
    assert abs(out["E0"][0] - ref["E0"]) < 1e-6
    for c in ctxs:
        c.close()


def test_batched_rejects_fp64_and_duplicates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import FedvrError, solve_2b_batched
    s = W.he_small()
    c = _ctx(s)
    with pytest.raises(FedvrError):
        solve_2b_batched([c], [s.beta], [s.u], [s.p], precision=0)
    with pytest.raises(FedvrError):
        solve_2b_batched([c, c], [s.beta] * 2, [s.u] * 2, [s.p] * 2)
    c.close()


def test_batched_graph_replay_is_bit_identical():
    # the batched iteration replayed from CUDA graphs (re-captured when a system
    # converges and leaves the active set) equals eager launches bit for bit
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Batch
    systems = _systems()[:3]
    runs = {}
    for graphs in (False, True):
        ctxs = [_ctx(s) for s in systems]
        ctxs[0].use_graphs(graphs)
        ctxs[0].conv1_splits(2)  # one split count for both runs (not a timed choice)
        b = Batch(ctxs, [s.beta for s in systems], [s.u for s in systems], [s.p for s in systems])
        rec, used = [], []
        for it in range(40):
            was = b.active.copy()
            r = b.step(0.5, tol=1e-8)
            m = was == 1  # systems stepped in this call (the others' outputs are not written)
            rec.append((r["res"][m].copy(), r["E0"][m].copy(), b.active.copy()))
            used.append(ctxs[0].use_graphs())
            if not b.active.any():
                break
        runs[graphs] = (rec, used, [c.get_history() for c in ctxs])
        b.close()
        for c in ctxs:
            c.close()
    (e_rec, e_used, e_hist), (g_rec, g_used, g_hist) = runs[False], runs[True]
    assert not any(e_used) and all(g_used)
    assert len(e_rec) == len(g_rec)
    for (er, ee, ea), (gr, ge, ga) in zip(e_rec, g_rec):
        assert np.array_equal(ea, ga)
        assert np.array_equal(er, gr) and np.array_equal(ee, ge)
    for he, hg in zip(e_hist, g_hist):
        assert np.array_equal(he[:, :4], hg[:, :4])


def test_batched_f16_equals_single_system_solves():
    # the FP16-split mode through the batched queue: same results as one system at a time
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import solve_2b_batched
    F16 = 3
    systems = _systems()[:3]
    single = []
    for s in systems:
        c = _ctx(s)
        c.conv1_splits(1)
        single.append(c.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 150, precision=F16, check=False))
        c.close()
    ctxs = [_ctx(s) for s in systems]
    ctxs[0].conv1_splits(1)
    out = solve_2b_batched(ctxs, [s.beta for s in systems], [s.u for s in systems],
                           [s.p for s in systems], 0.5, 1e-8, 150, F16, check=False)
    for k, s in enumerate(systems):
        assert out["iters"][k] == single[k]["iters"], s.name
        assert out["E0"][k] == single[k]["E0"], s.name
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("inner", [0, 3])
def test_batched_warm_start_equals_single_warm_starts(inner):
    # warm starts (an initial Sigma, optionally held fixed for `inner` full Dyson
    # steps) inside the batched iteration give what solve_2b gives one system at
    # a time; the initial Sigma is the oracle's Sigma^(2)[g^0] scaled by 0.9
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import solve_2b_batched
    F16 = 3
    systems = _systems()[:3]
    sig0 = []
    for s in systems:
        b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
        T, v = O.kinetic(b), O.potential(b["nodes"], s.Z, s.R, s.soft_en)
        V = O.interaction(b["nodes"], s.soft_ee)
        hf = O.hf_scf(T + np.diag(v), V, 2.0, s.n_elec // 2, s.beta, tol=1e-12)
        mesh = O.power_mesh(s.beta, s.u, s.p)
        G0 = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], s.beta)
        sig0.append(np.ascontiguousarray(0.9 * O.sigma2(G0, V, 2.0)))
    single = []
    for s, S0 in zip(systems, sig0):
        c = _ctx(s)
        c.conv1_splits(1)
        c.set_initial_sigma(S0, inner_steps=inner)
        single.append(c.solve_2b(s.beta, s.u, s.p, 0.5, 1e-8, 150, precision=F16, check=False))
        c.close()
    ctxs = [_ctx(s) for s in systems]
    ctxs[0].conv1_splits(1)
    for c, S0 in zip(ctxs, sig0):
        c.set_initial_sigma(S0, inner_steps=inner)
    out = solve_2b_batched(ctxs, [s.beta for s in systems], [s.u for s in systems],
                           [s.p for s in systems], 0.5, 1e-8, 150, F16, check=False)
    for k, s in enumerate(systems):
        assert single[k]["status"] == 0, s.name
        assert out["iters"][k] == single[k]["iters"], s.name
        assert out["E0"][k] == single[k]["E0"], s.name
        assert out["N"][k] == single[k]["N"], s.name
    for c in ctxs:
        c.close()
