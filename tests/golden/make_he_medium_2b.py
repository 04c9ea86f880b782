"""Write he_medium_2b.txt: the CPU oracle's converged second-Born solution of
the He n_b=199, M=513 workload (the benchmark's system), per-iteration E0 and
N included. Stored values for the full-size GPU parity tests and the
benchmark's reference energy E_ref (the FP64 solution at tol 1e-8).

Only the oracle runs here (basis, operators, HF, then the Dyson iteration of
Sec. 2.3, Eq. deq, on the power mesh of Sec. 3.1); the inputs come from the
seeded workload module. It takes about two hours on eight host cores:

    python tests/golden/make_he_medium_2b.py
"""

from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import fedvr_oracle as O  # noqa: E402
from paper_0911_4348_gb300 import workloads as W  # noqa: E402


def main(path: str = os.path.join(HERE, "he_medium_2b.txt")) -> None:
    s = W.he_medium()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    T = O.kinetic(b)
    v = O.potential(b["nodes"], s.Z, s.R, s.soft_en)
    V = O.interaction(b["nodes"], s.soft_ee)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, s.n_elec // 2, s.beta, tol=1e-13)
    t0 = time.time()
    res = O.solve_2b(h, V, 2.0, hf, s.beta, s.u, s.p, s.mixing, s.tol, 80)
    G = res["G"]
    jump = float(np.max(np.abs(G[-1] + G[0] - np.eye(G.shape[1]))))
    lines = [
        "# CPU oracle (oracle/fedvr_oracle.py, FP64) on the He n_b=199, M=513 workload:",
        "# Z=2, box [-50,50], 25 elements of order 8, beta=100, u=16, p=16, mixing 0.5,",
        "# tol 1e-8 (Sec. 2.3 Eq. deq; Sec. 3.1 power mesh). Written by",
        "# tests/golden/make_he_medium_2b.py; E0 excludes E_nn.",
        "# key                 value",
        f"E_hf                  {hf['E_hf']:.15f}",
        f"E0                    {res['E0']:.15f}",
        f"N                     {res['N']:.15f}",
        f"iterations            {res['iters']}",
        f"converged             {1 if res['converged'] else 0}",
        f"final_residual        {res['history'][-1][1]:.6e}",
        f"jump_invariant        {jump:.6e}",
        f"oracle_seconds        {time.time() - t0:.1f}",
    ]
    for it, r, e, nel in res["history"]:
        lines.append(f"E0_iter_{int(it):03d}          {e:.15f}")
    for it, r, e, nel in res["history"]:
        lines.append(f"res_iter_{int(it):03d}         {r:.6e}")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines[:13]))


if __name__ == "__main__":
    main()
