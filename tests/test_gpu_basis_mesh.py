"""GPU vs oracle: basis, operators, mesh and lag table are bit-exact (Sec. 2.1-2.2, 3.1)."""
import numpy as np
import pytest

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context
    c = Context()
    yield c
    c.close()


GRIDS = [
    (4, 4, -10.0, 10.0, 0),     # He n_b=15
    (25, 8, -50.0, 50.0, 0),    # He n_b=199
    (30, 10, -60.0, 60.0, 0),   # H3+ n_b=299
    (29, 7, -100.0, 100.0, 1),  # paper's graded He grid, n_b=202
    (13, 11, -25.0, 25.0, 1),   # paper's graded H3+ grid, n_b=142
    (6, 3, -7.0, 5.5, 1),       # even graded grid
    (7, 1, -3.0, 4.0, 0),       # order 1 (no interior GLL roots)
    (3, 32, -2.0, 2.0, 0),      # maximum order
]


@pytest.mark.parametrize("ne,order,xmin,xmax,kind", GRIDS)
def test_basis_and_kinetic_bit_exact(ctx, ne, order, xmin, xmax, kind):
    nb = ctx.build_fedvr(ne, order + 1, xmin, xmax, kind)
    ref = O.fedvr_basis(ne, order, xmin, xmax, kind)
    assert nb == ref["n"] == ne * order - 1
    xi, om = ctx.get_gll()
    assert np.array_equal(xi, ref["xi"]) and np.array_equal(om, ref["omega"])
    got = ctx.get_basis()
    assert np.array_equal(got["nodes"], ref["nodes"])
    assert np.array_equal(got["weights"], ref["weights"])
    assert np.array_equal(got["elem"], ref["elem"]) and np.array_equal(got["local"], ref["local"])
    T = ctx.get_operators(potential=False)["T"]
    assert np.array_equal(T, O.kinetic(ref))


@pytest.mark.parametrize("maker", [W.he_small, W.he_medium, W.h3p_large])
def test_potential_interaction_hamiltonian_bit_exact(ctx, maker):
    s = maker()
    ctx.build_fedvr(s.n_elem, s.pts_per_elem, s.xmin, s.xmax, s.grid_kind)
    enn = ctx.set_potential(s.Z, s.R, s.soft_en, s.soft_ee, s.n_elec)
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    T = O.kinetic(b)
    v = O.potential(b["nodes"], s.Z, s.R, s.soft_en)
    V = O.interaction(b["nodes"], s.soft_ee)
    got = ctx.get_operators()
    assert np.array_equal(got["v"], v)
    assert np.array_equal(got["V"], V)
    assert np.array_equal(got["h"], T + np.diag(v))
    ref_enn = sum(s.Z[a] * s.Z[c] / abs(s.R[a] - s.R[c])
                  for a in range(len(s.Z)) for c in range(a + 1, len(s.Z)))
    assert abs(enn - ref_enn) < 1e-14 * max(1.0, ref_enn)


@pytest.mark.parametrize("beta,u,p,lag", [(100.0, 4, 16, True), (100.0, 16, 16, True),
                                          (100.0, 32, 16, False), (37.5, 3, 5, True),
                                          (1.0, 1, 1, True)])
def test_mesh_and_lag_table_bit_exact(ctx, beta, u, p, lag):
    M = 2 * u * p + 1
    dev = torch.device("cuda")
    tau, w, wm, wp = (torch.empty(M, dtype=torch.float64, device=dev) for _ in range(4))
    lk = torch.empty((M, M), dtype=torch.int32, device=dev) if lag else None
    lt = torch.empty((M, M), dtype=torch.float64, device=dev) if lag else None
    ctx.power_mesh(beta, u, p, tau, w, wm, wp, lk, lt)
    torch.cuda.synchronize()
    ref = O.power_mesh(beta, u, p)
    for name, t in (("tau", tau), ("w", w), ("wm", wm), ("wp", wp)):
        got = t.cpu().numpy()
        assert np.array_equal(got, ref[name]), name
        assert np.array_equal(np.signbit(got), np.signbit(ref[name])), name
    if lag:
        tab = O.lag_table(ref["tau"], beta)
        assert np.array_equal(lk.cpu().numpy(), tab["k"])
        assert np.array_equal(lt.cpu().numpy(), tab["t"])
