"""Graph replay of the iteration gives bit-identical results to eager launches
(FP64 and split-TF32 paths, a change of mixing, warm-start inner steps)."""
import numpy as np
import pytest

from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(s):
    from paper_0911_4348_gb300 import Context
    c = Context()
    c.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    c.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    c.solve_hf(s.beta, tol=1e-12)
    return c


def _run(s, precision, graphs, mixings, Sigma0=None, inner=0):
    c = _ctx(s)
    c.use_graphs(graphs)
    if Sigma0 is not None:
        c.set_initial_sigma(Sigma0, inner_steps=inner)
    c.prepare_2b(s.beta, s.u, s.p, precision)
    rec, used = [], []
    for a in mixings:
        r = c.step_2b(a)
        rec.append((r["res"], r["E0"], r["N"]))
        used.append(c.use_graphs())
    st, launches = c.stage_times()
    G = np.empty((s.n_tau, s.n_b, s.n_b))
    S = np.empty_like(G)
    c.read_2b(G_out=G, Sigma_out=S)
    c.close()
    return np.array(rec), G, S, used, st, launches


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_is_bit_identical(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = W.he_small()
    mix = [0.5] * 4 + [0.7] * 2 + [0.5]
    e_rec, e_G, e_S, e_used, _, e_n = _run(s, precision, False, mix)
    g_rec, g_G, g_S, g_used, st, g_n = _run(s, precision, True, mix)
    assert not any(e_used)
    assert all(g_used)
    assert e_n == g_n
    assert np.array_equal(e_rec, g_rec)
    assert np.array_equal(e_G, g_G) and np.array_equal(e_S, g_S)
    # stage events are recorded inside the replayed graph
    assert all(v > 0 for v in st.values()) and st["step"] >= st["conv1"]


def test_graph_replay_after_warm_start_inner_steps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = W.he_small()
    _, _, S_ref, _, _, _ = _run(s, 1, False, [0.5] * 6)
    mix = [0.5] * 6
    e_rec, e_G, _, e_used, _, _ = _run(s, 1, False, mix, Sigma0=S_ref, inner=2)
    g_rec, g_G, _, g_used, _, _ = _run(s, 1, True, mix, Sigma0=S_ref, inner=2)
    assert g_used == [False, False, True, True, True, True]
    assert np.array_equal(e_rec, g_rec) and np.array_equal(e_G, g_G)
