"""Host-side logic of the benchmark (no GPU): algorithmic flop counts, the
equilibrium estimate of a sampled binding curve, the traffic record lookup and
the workload definitions the bench lines name."""
import math

import numpy as np

import bench
from paper_0911_4348_gb300 import workloads as W


def test_algorithmic_counts():
    n, M = 199, 513
    assert bench.algorithmic("conv1", n, M) == 2.0 * M * M * n ** 3
    assert bench.algorithmic("sigma2", n, M) == M * (n ** 4 + 4.0 * n ** 3)
    # second convolution: left transform, eigen-kernel product, back transform
    assert bench.algorithmic("conv2", n, M) == 2.0 * M * M * n * n + 4.0 * M * n ** 3
    assert bench.algorithmic("update", n, M) == 0.0


def test_parabola_min_recovers_a_quadratic_vertex():
    x = np.linspace(3.0, 7.0, 11)
    y = 0.3 * (x - 4.57) ** 2 - 1.5
    assert math.isclose(bench._parabola_min(x, y), 4.57, abs_tol=1e-12)
    # a minimum at the end of the sampled range is not an estimate
    assert bench._parabola_min(x, (x - 2.0) ** 2) is None


def test_traffic_record_is_keyed_by_workload_and_source():
    assert bench.measured_traffic("conv1_f16_kernel", "some other workload") is None
    assert bench.measured_traffic("no_such_kernel", "He n_b=199 M=513") is None


def test_bench_workloads_have_the_stated_shapes():
    assert (W.he_small().n_b, W.he_small().n_tau) == (15, 129)
    assert (W.he_medium().n_b, W.he_medium().n_tau) == (199, 513)
    assert (W.h3p_large().n_b, W.h3p_large().n_tau) == (299, 1025)
    assert (W.he_paper().n_b, W.he_paper().n_tau) == (202, 1025)
    curve = W.h3p_curve()
    assert len(curve) == 11
    assert all((s.n_b, s.n_tau, s.grid_kind) == (142, 1025, 1) for s in curve)
    assert [round(2 * s.R[2], 6) for s in curve] == [round(3.2 + 0.4 * k, 6) for k in range(11)]
    batch = W.batch_systems(64)
    assert len(batch) == 64 and all(59 <= s.n_b <= 239 and 257 <= s.n_tau <= 513 for s in batch)
