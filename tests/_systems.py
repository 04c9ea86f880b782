"""Oracle-side construction of the model systems used by the GPU parity tests
(basis, operators and HF from the oracle, cached per system)."""
import functools

import numpy as np

from oracle import fedvr_oracle as O
from paper_0911_4348_gb300 import workloads as W


@functools.lru_cache(maxsize=None)
def oracle_system(name: str, hf_tol: float = 1e-13):
    s = {"he_small": W.he_small, "he_medium": W.he_medium, "h3p_large": W.h3p_large}[name]()
    b = O.fedvr_basis(s.n_elem, s.order, s.xmin, s.xmax, s.grid_kind)
    T = O.kinetic(b)
    v = O.potential(b["nodes"], s.Z, s.R, s.soft_en)
    V = O.interaction(b["nodes"], s.soft_ee)
    h = T + np.diag(v)
    hf = O.hf_scf(h, V, 2.0, s.n_elec // 2, s.beta, tol=hf_tol)
    mesh = O.power_mesh(s.beta, s.u, s.p)
    G0 = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], s.beta)
    return dict(sys=s, basis=b, T=T, v=v, V=V, h=h, hf=hf, mesh=mesh, G0=G0)


def maxrel(x, ref):
    """Max-norm relative error max|x - ref| / max|ref|."""
    x, ref = np.asarray(x), np.asarray(ref)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))
