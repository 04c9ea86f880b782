"""Plain, slow FP64 CPU oracle for the FE-DVR second-Born Matsubara method.

TEST INFRASTRUCTURE ONLY. This module is the independent reference that the
CUDA library is checked against. Only the test suite, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it; the library and its
Python binding never do, and it imports nothing from them.

It follows Balzer, Bauch & Bonitz, "Finite elements and the discrete variable
representation in nonequilibrium Green's function calculations" (arXiv
0911.4348), step by step in the paper's order and notation:

* Sec. 2.1, Eqs. (xim), (wim) and the GLL definitions: ``gll``, ``fedvr_basis``.
* Sec. 2.2, Eqs. (vmat), (tmat): ``potential``, ``kinetic``.
* Sec. 2.2, Eqs. (umat)-(umatsep): ``interaction`` and ``interaction_eigen_route``.
* Sec. 2.3, Eq. (sigmahf): ``hf_selfenergy``; Eqs. (hamhf), (hfgf): ``hf_scf``,
  ``chemical_potential``, ``g0_mesh``.
* Sec. 2.3, Eq. (sigma2ndb): ``sigma2`` (two-index form) and
  ``sigma2_bruteforce`` (general four-index form, tiny n only).
* Sec. 2.3, Eq. (deq): ``conv1`` (I^(1)), ``conv2`` (I^(2)), ``solve_2b``.
* Sec. 3.1 (uniform power mesh, 2up+1 points): ``power_mesh``, ``lag_table``.
* Sec. 2.3 (total energy "as in" the cited references): ``energy``
  (Galitskii-Migdal form).
* A fourth-order variant of the "direct integration" of Eq. (deq) (the
  paper gives no quadrature; the trapezoid with linear lag interpolation is
  the default reading): ``quad4_weights``, ``cubic_lag``, ``quad="cubic4"``
  in ``conv1``, ``conv2``, ``energy``, ``solve_2b``.
* Sec. 2.3 and 3.2 observables: ``density`` (one-electron density from
  g(0^-)) and ``nuclear_repulsion`` (the internuclear term of Eq. h3pv).
* Sec. 4 (T-matrix named beside GW): ``pair_conv``, ``ladder_t``,
  ``sigma_tmatrix`` and ``solve_2b(self_energy="tmatrix")``.
* Sec. 4 (GW named as a further approximation the FE-DVR form simplifies):
  ``bose_lag_table``, ``conv_bose``, ``screened_w``, ``sigma_gw`` and
  ``solve_2b(..., self_energy="gw")`` (the screened interaction of the
  two-index bubble series on the same mesh; its lowest order is the direct
  term of Eq. sigma2ndb).
* Sec. 2, Eqs. (kbe), (skkbe), (skkbesigma) with (sigmahf), (sigma2ndb) on the
  Keldysh components: ``kbe_propagate`` (real-time two-time Kadanoff-Baym
  propagation from an uncorrelated initial state) and its self-energy
  ``sigma2_realtime``; pin only: ``exact_dynamics`` (two-electron
  Schroedinger evolution on the same grid).
* Pins only: ``mp2`` (closed-shell MP2), ``exact_ground`` /
  ``exact_ground_state`` / ``exact_density`` (exact two-electron ground state
  on the same grid).

Where the paper is silent or garbled the oracle takes one stated reading; each
is marked "Reading:" below. Every floating-point step of the basis, mesh and
lag-table construction uses only IEEE +, -, *, / and sqrt in a fixed order
(Python scalar arithmetic never fuses multiply-adds), so those results are
reproducible bit for bit by any implementation that performs the same
operations in the same order.

Every function is pinned by a test under ``tests/`` against something other
than itself (closed forms, special cases, brute force, printed paper values);
none is "parity unpinned".
"""

from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Sec. 2.1: Gauss-Lobatto-Legendre points and weights
# ---------------------------------------------------------------------------


def _legendre(N: int, x: float) -> tuple[float, float]:
    """(P_N(x), P_{N-1}(x)) by the three-term recurrence.

    P_{k+1} = ((2k+1) x P_k - k P_{k-1}) / (k+1), evaluated in exactly this
    order: a = (2k+1)*x; b = a*P_k; c = k*P_{k-1}; P_{k+1} = (b - c)/(k+1).
    """
    if N == 0:
        return 1.0, 0.0
    pm1, p = 1.0, x
    for k in range(1, N):
        a = float(2 * k + 1) * x
        b = a * p
        c = float(k) * pm1
        pm1, p = p, (b - c) / float(k + 1)
    return p, pm1


def _dlegendre(N: int, x: float) -> float:
    """P'_N(x) for |x| < 1 from (1 - x^2) P'_N = N (P_{N-1} - x P_N)."""
    p, pm1 = _legendre(N, x)
    num = float(N) * (pm1 - x * p)
    den = 1.0 - x * x
    return num / den


def _bisect_root(N: int, lo: float, hi: float, dlo: float) -> float:
    """Bisection for a sign change of P'_N in (lo, hi); stops when the
    midpoint can no longer move (the bracket is one ulp wide)."""
    mid = 0.5 * (lo + hi)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if not (lo < mid < hi):
            break
        dm = _dlegendre(N, mid)
        if dm == 0.0:
            break
        if (dm > 0.0) == (dlo > 0.0):
            lo = mid
        else:
            hi = mid
    return mid


GLL_SCAN_CELLS = 4096


def gll(order: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Lobatto-Legendre points xi_m and weights omega_m, m = 0..order.

    Sec. 2.1: the points are the roots of dP_{n_g}/dx plus the two end points
    +-1; the weights are omega_m = 2 / (n_g (n_g + 1) P_{n_g}(xi_m)^2).

    Reading (the paper's n_g): the root and weight formulas are those of the
    order-n_g rule, which has n_g + 1 points per element; with that reading
    n_b = n_e n_g - 1 (Eq. basisdim) reproduces the paper's 29*7-1 = 202 and
    13*11-1 = 142. ``order`` is therefore the polynomial order n_g and the
    element holds order + 1 points.

    Roots: P'_N is evaluated on the 4095 interior boundaries of a uniform
    4096-cell scan of [-1, 1]; an exact zero is a root, a strict sign change
    between neighbours is bisected to one ulp.
    """
    N = int(order)
    if N < 1:
        raise ValueError("order must be >= 1")
    roots: list[float] = []
    prev_x = prev_d = None
    for c in range(1, GLL_SCAN_CELLS):
        x = -1.0 + (2.0 * c) / GLL_SCAN_CELLS
        d = _dlegendre(N, x)
        if d == 0.0:
            roots.append(x)
        elif prev_d is not None and prev_d != 0.0 and ((d > 0.0) != (prev_d > 0.0)):
            roots.append(_bisect_root(N, prev_x, x, prev_d))
        prev_x, prev_d = x, d
    if len(roots) != N - 1:
        raise RuntimeError(f"GLL scan found {len(roots)} roots for order {N}")
    xi = [-1.0] + roots + [1.0]
    om = []
    nn1 = float(N * (N + 1))
    for x in xi:
        p, _ = _legendre(N, x)
        om.append(2.0 / (nn1 * (p * p)))
    return np.array(xi), np.array(om)


def lagrange_deriv(xi: np.ndarray) -> np.ndarray:
    """d[m, k] = f'_m(xi_k) for the Lagrange (Lobatto shape) functions of Sec. 2.1.

    k != m: (1/(xi_m - xi_k)) * prod_{l != m,k} (xi_k - xi_l)/(xi_m - xi_l), l ascending.
    k == m: sum_{l != m} 1/(xi_m - xi_l), l ascending.
    """
    xs = [float(v) for v in xi]
    n = len(xs)
    d = np.zeros((n, n))
    for m in range(n):
        for k in range(n):
            if k == m:
                s = 0.0
                for l in range(n):
                    if l != m:
                        s = s + 1.0 / (xs[m] - xs[l])
                d[m, k] = s
            else:
                prod = 1.0 / (xs[m] - xs[k])
                for l in range(n):
                    if l != m and l != k:
                        prod = prod * ((xs[k] - xs[l]) / (xs[m] - xs[l]))
                d[m, k] = prod
    return d


# ---------------------------------------------------------------------------
# Sec. 2.1 / Sec. 3.1: finite elements, nodes, weights, index map
# ---------------------------------------------------------------------------


def element_widths_graded(n_elem: int, L: float) -> list[float]:
    """Case II partition (Sec. 3.1): a central element 1 a.u. wide and widths
    growing linearly towards both box ends.

    Reading (the paper gives no law): odd n_e: K = (n_e-1)/2 elements per side
    of width 1 + k*delta (k = 1..K), delta = (L - 1 - 2K) / (K(K+1)); even n_e:
    K = n_e/2 per side of width 1 + (k-1)*delta, delta = (L/2 - K) / (K(K-1)/2).
    Widths are listed from the left box end to the right one.
    """
    ne = int(n_elem)
    if ne == 1:
        return [L]
    if ne % 2 == 1:
        K = (ne - 1) // 2
        delta = (L - 1.0 - 2.0 * K) / float(K * (K + 1))
        side = [1.0 + float(k) * delta for k in range(1, K + 1)]
        return side[::-1] + [1.0] + side
    K = ne // 2
    if K == 1:
        return [0.5 * L, 0.5 * L]
    delta = (0.5 * L - float(K)) / float((K * (K - 1)) // 2)
    side = [1.0 + float(k - 1) * delta for k in range(1, K + 1)]
    return side[::-1] + side


def element_edges(n_elem: int, xmin: float, xmax: float, grid_kind: int = 0) -> list[float]:
    """Element boundaries x^0 = xmin < ... < x^{n_e} = xmax (Sec. 2.1, Fig. 1).

    Case I (grid_kind 0, Sec. 3.1): e_i = xmin + (i * L) / n_e, e_{n_e} = xmax.
    Case II (grid_kind 1): e_0 = xmin, e_{i+1} = e_i + width_i, e_{n_e} = xmax.
    """
    ne = int(n_elem)
    L = xmax - xmin
    if grid_kind == 0:
        e = [xmin + (float(i) * L) / float(ne) for i in range(ne)]
    elif grid_kind == 1:
        wid = element_widths_graded(ne, L)
        if min(wid) <= 0.0:
            raise ValueError("graded widths must be positive")
        e = [xmin]
        for i in range(ne - 1):
            e.append(e[-1] + wid[i])
    else:
        raise ValueError("grid_kind must be 0 or 1")
    e.append(xmax)
    return e


def fedvr_basis(n_elem: int, order: int, xmin: float, xmax: float, grid_kind: int = 0) -> dict:
    """FE-DVR nodes, weights and index map (Sec. 2.1, Eqs. xim, wim, basis, basisdim).

    Global node q = i*order + m (element i, local point m = 0..order); the node
    shared by elements i and i+1 is element i+1's m = 0, i.e. exactly the edge
    e_{i+1}. Interior points: x = e_i + ((xi_m + 1) * h_i) * 0.5 with
    h_i = e_{i+1} - e_i (Eq. xim rearranged). The two box ends carry no basis
    function (G vanishes outside the interval), so the basis is q = 1 ..
    n_e*order - 1 and n_b = n_e n_g - 1 (Eq. basisdim); basis index a = q - 1.

    Element weight w^i_m = (omega_m * h_i) * 0.5 (Eq. wim); a bridge function
    carries W = w^i_{order} + w^{i+1}_0 (the normalisation in Eq. basis;
    Reading: the paper's f^i_{n_g-1} and w^i_{n_g-1} are the element's last
    point, index ``order`` here).
    """
    ne, N = int(n_elem), int(order)
    xi, om = gll(N)
    e = element_edges(ne, xmin, xmax, grid_kind)
    h = [e[i + 1] - e[i] for i in range(ne)]
    nq = ne * N + 1
    xq = [0.0] * nq
    for i in range(ne):
        xq[i * N] = e[i]
        for m in range(1, N):
            xq[i * N + m] = e[i] + ((float(xi[m]) + 1.0) * h[i]) * 0.5
    xq[ne * N] = e[ne]
    wloc = [[(float(om[m]) * h[i]) * 0.5 for m in range(N + 1)] for i in range(ne)]
    n = ne * N - 1
    X = np.zeros(n)
    W = np.zeros(n)
    elem = np.zeros(n, dtype=np.int32)
    local = np.zeros(n, dtype=np.int32)
    for a in range(n):
        q = a + 1
        i, m = divmod(q, N)
        X[a] = xq[q]
        if m == 0:  # bridge between elements i-1 and i
            W[a] = wloc[i - 1][N] + wloc[i][0]
            elem[a], local[a] = i - 1, N
        else:
            W[a] = wloc[i][m]
            elem[a], local[a] = i, m
    return dict(n=n, order=N, n_elem=ne, xi=xi, omega=om, edges=np.array(e),
                h=np.array(h), wloc=np.array(wloc), nodes=X, weights=W,
                elem=elem, local=local)


# ---------------------------------------------------------------------------
# Sec. 2.2: one- and two-body matrices
# ---------------------------------------------------------------------------


def kinetic(basis: dict) -> np.ndarray:
    """Kinetic matrix T (Sec. 2.2, Eq. tmat) assembled element by element.

    Element matrix t~^i_{m1 m2} = sum_k D^i_{m1 k} D^i_{m2 k} w^i_k with
    D^i = (2/h_i) d (d from ``lagrange_deriv``), k ascending. Then
    T_ab = (0.5 * S_ab) / sqrt(W_a * W_b), S_ab = sum of t~^i over the elements
    i that contain both nodes, i ascending. This is the paper's four-case table
    written as one assembly rule (Reading: the table's deltas and weight
    normalisations are those of the bridge/element functions of Eq. basis).
    """
    ne, N, n = basis["n_elem"], basis["order"], basis["n"]
    d = lagrange_deriv(basis["xi"])
    S = np.zeros((n, n))
    for i in range(ne):
        hi = float(basis["h"][i])
        s = 2.0 / hi
        D = [[s * float(d[m, k]) for k in range(N + 1)] for m in range(N + 1)]
        wk = [float(basis["wloc"][i][k]) for k in range(N + 1)]
        for m1 in range(N + 1):
            qa = i * N + m1
            if qa < 1 or qa > ne * N - 1:
                continue
            for m2 in range(N + 1):
                qb = i * N + m2
                if qb < 1 or qb > ne * N - 1:
                    continue
                acc = 0.0
                for k in range(N + 1):
                    acc = acc + (D[m1][k] * D[m2][k]) * wk[k]
                S[qa - 1, qb - 1] = S[qa - 1, qb - 1] + acc
    W = basis["weights"]
    T = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            if S[a, b] != 0.0:
                T[a, b] = (0.5 * float(S[a, b])) / math.sqrt(float(W[a]) * float(W[b]))
    return T


def potential(nodes: np.ndarray, Z, R, soft_en: float) -> np.ndarray:
    """Diagonal potential v_a (Sec. 2.2, Eq. vmat; Sec. 3 model potentials).

    v_a = sum_A (-Z_A) / sqrt((X_a - R_A)^2 + soft_en), A ascending. At a
    bridge both terms of the paper's weighted average sample v at the same
    point, so v~ = v(node) exactly (Reading).
    """
    v = np.zeros(len(nodes))
    for a, x in enumerate(nodes):
        acc = 0.0
        for z, r in zip(Z, R):
            dx = float(x) - float(r)
            acc = acc + (-float(z)) / math.sqrt(dx * dx + float(soft_en))
        v[a] = acc
    return v


def interaction(nodes: np.ndarray, soft_ee: float) -> np.ndarray:
    """Two-index interaction V_ab = u(|x_a - x_b|) = 1/sqrt((x_a-x_b)^2 + soft_ee).

    Sec. 2.2, Eqs. (umat1)-(umatsep): the four-index integrals collapse to
    delta delta u~ and, in exact arithmetic, u~_ab = u(|x_a - x_b|) (Reading;
    ``interaction_eigen_route`` computes the paper's route for the check).
    """
    x = np.asarray(nodes, dtype=np.float64)
    dx = x[:, None] - x[None, :]
    return 1.0 / np.sqrt(dx * dx + float(soft_ee))


def interaction_eigen_route(basis: dict, soft_ee: float) -> np.ndarray:
    """u~ by the paper's separable route (Eqs. umatred, umatsep): diagonalise U
    over the element-local point list, average the two coincident bridge rows
    with the element weights, and sum alpha beta beta."""
    ne, N = basis["n_elem"], basis["order"]
    e, xi = basis["edges"], basis["xi"]
    pts = []
    for i in range(ne):
        hi = e[i + 1] - e[i]
        for m in range(N + 1):
            if m == 0:
                pts.append(e[i])
            elif m == N:
                pts.append(e[i + 1])
            else:
                pts.append(e[i] + ((xi[m] + 1.0) * hi) * 0.5)
    pts = np.array(pts)
    U = 1.0 / np.sqrt((pts[:, None] - pts[None, :]) ** 2 + soft_ee)
    alpha, Bt = np.linalg.eigh(U)
    n = basis["n"]
    beta = np.zeros((n, len(pts)))
    wl = basis["wloc"]
    for a in range(n):
        i, m = basis["elem"][a], basis["local"][a]
        if m == N:  # bridge: average rows (i, N) and (i+1, 0)
            r1, r2 = i * (N + 1) + N, (i + 1) * (N + 1)
            beta[a] = (Bt[r1] * wl[i][N] + Bt[r2] * wl[i + 1][0]) / (wl[i][N] + wl[i + 1][0])
        else:
            beta[a] = Bt[i * (N + 1) + m]
    return (beta * alpha) @ beta.T


# ---------------------------------------------------------------------------
# Sec. 2.3: Hartree-Fock, chemical potential, HF Matsubara Green's function
# ---------------------------------------------------------------------------


def hf_selfenergy(rho: np.ndarray, V: np.ndarray, sigma: float) -> np.ndarray:
    """Sigma^HF[rho] = sigma diag(V diag rho) - V o rho (Sec. 2.3, Eq. sigmahf).

    Reading: g(t, t^+) in Eq. (sigmahf) is the density matrix rho = g(0^-) of
    the Matsubara branch; the -i prefactor belongs to the real-time contour.
    """
    hartree = V @ np.diag(rho)
    return sigma * np.diag(hartree) - V * rho


def fermi(y: np.ndarray, beta: float) -> np.ndarray:
    """Fermi function f_beta(y) = 1/(exp(beta y) + 1) in overflow-free form."""
    y = np.asarray(y, dtype=np.float64)
    out = np.empty_like(y)
    pos = beta * y > 0.0
    e = np.exp(-beta * y[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(beta * y[~pos]))
    return out


def _softplus(z: float) -> float:
    return max(z, 0.0) + math.log1p(math.exp(-abs(z)))


def _lse(vals: list[float]) -> float:
    m = max(vals)
    s = 0.0
    for v in vals:
        s = s + math.exp(v - m)
    return m + math.log(s)


def _balance(mu: float, eps: np.ndarray, nocc: int, beta: float) -> float:
    holes = [-_softplus(beta * (mu - float(e))) for e in eps[:nocc]]
    parts = [-_softplus(beta * (float(e) - mu)) for e in eps[nocc:]]
    return _lse(holes) - _lse(parts)


def chemical_potential(eps: np.ndarray, nocc: int, beta: float) -> float:
    """mu from the Fermi normalisation N/sigma = sum_a f_beta(eps_a - mu) (Sec. 2.3).

    Reading: the equation is solved in its balanced form, holes = particles,
    sum_{a<nocc} f(mu - eps_a) = sum_{a>=nocc} f(eps_a - mu), compared as
    log-sum-exps. It is the same equation rearranged; in the direct form the
    residual changes by ~1e-14 per unit mu inside the HOMO-LUMO gap at
    beta = 100, so FP64 cannot locate mu there, while the balanced form has
    slope ~ -2 beta. Bisection on [eps_min - 1, eps_max + 1] until the midpoint
    no longer moves. ``eps`` must be ascending.
    """
    eps = np.asarray(eps, dtype=np.float64)
    if not (0 < nocc < len(eps)):
        raise ValueError("need 0 < nocc < n")
    lo, hi = float(eps[0]) - 1.0, float(eps[-1]) + 1.0
    mid = 0.5 * (lo + hi)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if not (lo < mid < hi):
            break
        if _balance(mid, eps, nocc, beta) > 0.0:
            lo = mid
        else:
            hi = mid
    return mid


def hf_energy(h: np.ndarray, V: np.ndarray, rho: np.ndarray, sigma: float) -> float:
    """E_HF = sigma Tr[h rho] + (sigma/2) Tr[Sigma^HF[rho] rho]."""
    return float(sigma * np.sum(h * rho) + 0.5 * sigma * np.sum(hf_selfenergy(rho, V, sigma) * rho))


def hf_scf(h: np.ndarray, V: np.ndarray, sigma: float, nocc: int, beta: float,
           tol: float = 1e-12, max_iter: int = 500, mixing: float = 0.5) -> dict:
    """Self-consistent HF at inverse temperature beta (Sec. 2.3, Eq. hamhf).

    Reading (start, mixing and stop are not given): rho starts as the
    projector on the nocc lowest eigenvectors of h; each step builds
    F = h + Sigma^HF[rho], diagonalises it, fixes mu, forms
    rho' = C diag f C^T; stop when max|rho' - rho| < tol, otherwise
    rho <- (1 - a) rho + a rho'. The returned eps, C, mu, F belong to the last
    rho; rho0 = C diag f C^T = g^0(0^-) and Sigma0 = F - h.
    """
    eps, C = np.linalg.eigh(h)
    rho = C[:, :nocc] @ C[:, :nocc].T
    it = 0
    for it in range(1, max_iter + 1):
        F = h + hf_selfenergy(rho, V, sigma)
        eps, C = np.linalg.eigh(F)
        mu = chemical_potential(eps, nocc, beta)
        f = fermi(eps - mu, beta)
        rho_new = (C * f) @ C.T
        r = float(np.max(np.abs(rho_new - rho)))
        if r < tol:
            break
        rho = (1.0 - mixing) * rho + mixing * rho_new
    else:
        raise RuntimeError("HF did not converge")
    return dict(eps=eps, C=C, mu=mu, f=f, F=F, Sigma0=F - h, rho0=rho_new,
                E_hf=hf_energy(h, V, rho_new, sigma), iters=it)


# ---------------------------------------------------------------------------
# Sec. 3.1: uniform power mesh on [-beta, 0]
# ---------------------------------------------------------------------------


def power_mesh(beta: float, u: int, p: int) -> dict:
    """Uniform power mesh with 2up + 1 points (Sec. 3.1, Fig. 2b).

    Reading (the mesh is defined only by reference): offsets s on [0, beta/2]:
    B_p = beta/2, B_{k-1} = 0.5 B_k, B_0 = 0; segment k = 1..p spans
    [B_{k-1}, B_k] (width B_1 for k = 1, else B_{k-1}) and is cut into u
    equal parts: s = B_{k-1} + (width * r) / u, r = 1..u. Then
    tau_j = -beta + s_j for j <= up and tau_{M-1-m} = -s_m: the mesh is dense
    at both ends and tau_{M-1-j} = -beta - tau_j holds bit for bit.

    Weights: trapezoid w_j = (tau_{j+1} - tau_{j-1}) * 0.5 (one-sided at the
    ends), and the halves wm_j = (tau_j - tau_{j-1}) * 0.5,
    wp_j = (tau_{j+1} - tau_j) * 0.5 used where the integrand jumps.
    """
    u, p = int(u), int(p)
    if u < 1 or p < 1:
        raise ValueError("u, p >= 1")
    half = 0.5 * beta
    B = [0.0] * (p + 1)
    B[p] = half
    for k in range(p, 1, -1):
        B[k - 1] = 0.5 * B[k]
    s = [0.0]
    for k in range(1, p + 1):
        width = B[1] if k == 1 else B[k - 1]
        for r in range(1, u + 1):
            s.append(B[k - 1] + (width * float(r)) / float(u))
    up = u * p
    M = 2 * up + 1
    tau = [0.0] * M
    for j in range(up + 1):
        tau[j] = -beta + s[j]
    for m in range(up + 1):
        tau[M - 1 - m] = -s[m]
    w = [0.0] * M
    wm = [0.0] * M
    wp = [0.0] * M
    for j in range(M):
        if j > 0:
            wm[j] = (tau[j] - tau[j - 1]) * 0.5
        if j < M - 1:
            wp[j] = (tau[j + 1] - tau[j]) * 0.5
        if j == 0:
            w[j] = (tau[1] - tau[0]) * 0.5
        elif j == M - 1:
            w[j] = (tau[M - 1] - tau[M - 2]) * 0.5
        else:
            w[j] = (tau[j + 1] - tau[j - 1]) * 0.5
    return dict(tau=np.array(tau), w=np.array(w), wm=np.array(wm), wp=np.array(wp), M=M)


def lag_point(tau: np.ndarray, beta: float, i: int, j: int) -> tuple[float, float]:
    """Mesh argument y in [-beta, 0] and sign for the lag tau_i - tau_j, i != j.

    Reading (the Dyson integrals run over a full period, Eq. deq): functions
    are extended anti-periodically, F(x) = -F(x - beta) for x in (0, beta].
    j > i: x = tau_i - tau_j < 0, y = x, sign +1; j < i: y = (tau_i - tau_j) - beta,
    sign -1.
    """
    x = float(tau[i]) - float(tau[j])
    if j > i:
        return x, 1.0
    return x - beta, -1.0


def bracket(tau: np.ndarray, y: float) -> tuple[int, float]:
    """k = largest index in [0, M-2] with tau_k <= y (binary search) and the
    linear-interpolation weight t = (y - tau_k) / (tau_{k+1} - tau_k)."""
    lo, hi = 0, len(tau) - 1
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if float(tau[mid]) <= y:
            lo = mid
        else:
            hi = mid
    t = (y - float(tau[lo])) / (float(tau[lo + 1]) - float(tau[lo]))
    return lo, t


def lag_table(tau: np.ndarray, beta: float) -> dict:
    """(k, t, sign) for every off-diagonal pair (i, j); diagonal entries are
    k = -1, t = 0, sign = 0 (the jump at lag 0 is handled separately)."""
    M = len(tau)
    K = np.full((M, M), -1, dtype=np.int32)
    T = np.zeros((M, M))
    S = np.zeros((M, M))
    for i in range(M):
        for j in range(M):
            if i == j:
                continue
            y, sg = lag_point(tau, beta, i, j)
            k, t = bracket(tau, y)
            K[i, j], T[i, j], S[i, j] = k, t, sg
    return dict(k=K, t=T, s=S)


# ---------------------------------------------------------------------------
# Sec. 2.3, Eq. (hfgf): HF Matsubara Green's function
# ---------------------------------------------------------------------------


def phi(x: float, y: np.ndarray, beta: float) -> np.ndarray:
    """Eigenbasis factor of Eq. (hfgf): phi_a(x) = f_beta(y_a) exp(-x y_a),
    x in [-beta, 0], y_a = eps_a - mu, in the overflow-free forms
    y >= 0: exp(-(beta + x) y) / (1 + exp(-beta y)); y < 0: exp(-x y)/(1 + exp(beta y))."""
    y = np.asarray(y, dtype=np.float64)
    out = np.empty_like(y)
    pos = y >= 0.0
    yp, yn = y[pos], y[~pos]
    out[pos] = np.exp(-((beta + x) * yp)) / (1.0 + np.exp(-(beta * yp)))
    out[~pos] = np.exp(-(x * yn)) / (1.0 + np.exp(beta * yn))
    return out


def g0_mesh(eps: np.ndarray, C: np.ndarray, mu: float, tau: np.ndarray, beta: float) -> np.ndarray:
    """g^0(tau_j) = C diag(phi(tau_j)) C^T for every mesh point (Eq. hfgf)."""
    y = np.asarray(eps) - mu
    return np.stack([(C * phi(float(t), y, beta)) @ C.T for t in tau])


# ---------------------------------------------------------------------------
# Sec. 2.3, Eq. (sigma2ndb): second-Born self-energy
# ---------------------------------------------------------------------------


def sigma2_tau(g: np.ndarray, gb: np.ndarray, V: np.ndarray, sigma: float) -> np.ndarray:
    """Sigma^corr at one mesh point from g = g(tau_j) and gb = g(-beta - tau_j).

    Direct term sigma g o (V Q V) with the polarisation Q = g o gb, and the
    second-order exchange X_ab = sum_{k,l} V_ak V_bl g_al gb_lk g_kb;
    Sigma^corr = sigma g o (V Q V) - X.

    Reading (Eq. sigma2ndb prints u_14 u_23 with g(t,t') and g(t',t); the
    interaction is instantaneous, so the time-consistent pairing is u_13 u_24,
    which leaves the direct term unchanged and makes the exchange the diagram
    above, O(n_b^2) per element as the paper states). Sign: with the paper's
    g > 0 on [-beta, 0] the direct term enters with + and the exchange with -
    (the Hubbard-atom and MP2 pins fix this).
    """
    Q = g * gb
    D = sigma * g * (V @ Q @ V)
    n = g.shape[0]
    X = np.empty_like(g)
    for b in range(n):
        P = g @ (V[b][:, None] * gb)      # P_ak = sum_l g_al V_bl gb_lk
        X[:, b] = (V * P) @ g[:, b]       # X_ab = sum_k V_ak P_ak g_kb
    return D - X


def sigma2_element(g: np.ndarray, gb: np.ndarray, V: np.ndarray, sigma: float, a: int,
                   b: int) -> float:
    """One element Sigma^corr_ab from the two sums of ``sigma2_tau`` written
    out, O(n^2): sigma g_ab sum_kl V_ak g_kl gb_lk V_lb - sum_kl V_ak V_bl g_al gb_lk g_kb."""
    direct = sigma * g[a, b] * float(np.einsum("k,kl,l->", V[a], g * gb, V[:, b]))
    exch = float(np.einsum("k,l,l,lk,k->", V[a], V[b], g[a], gb, g[:, b]))
    return direct - exch


def sigma2(G: np.ndarray, V: np.ndarray, sigma: float) -> np.ndarray:
    """Sigma^corr(tau_j) for every j; gb_j = G[M-1-j] (mesh mirror symmetry)."""
    M = G.shape[0]
    return np.stack([sigma2_tau(G[j], G[M - 1 - j], V, sigma) for j in range(M)])


def sigma2_bruteforce(g: np.ndarray, gb: np.ndarray, eri: np.ndarray, sigma: float) -> np.ndarray:
    """General-basis second Born with all four-index integrals (chemist
    notation eri[a,b,c,d] = (ab|cd)), O(n^6) (Sec. 2.3 text after Eq.
    sigma2ndb):

    Sigma_ij = sum_{abcdef} (ia|cd)(bj|ef) [sigma g_ab g_de gb_fc - g_ae gb_fc g_db].
    With (ab|cd) = delta_ab delta_cd V_ac (Eq. umat1) it must equal ``sigma2_tau``.
    """
    direct = sigma * np.einsum("iacd,bjef,ab,de,fc->ij", eri, eri, g, g, gb, optimize=True)
    exch = np.einsum("iacd,bjef,ae,fc,db->ij", eri, eri, g, gb, g, optimize=True)
    return direct - exch


# ---------------------------------------------------------------------------
# Sec. 2.3, Eq. (deq): the two tau-convolutions
# ---------------------------------------------------------------------------


def _lagrange(xs, x: float) -> list:
    """Values at x of the Lagrange basis polynomials of the nodes xs."""
    out = []
    for p in range(len(xs)):
        v = 1.0
        for q in range(len(xs)):
            if q != p:
                v *= (x - float(xs[q])) / (float(xs[p]) - float(xs[q]))
        out.append(v)
    return out


def quad4_weights(x: np.ndarray) -> np.ndarray:
    """Weights of a fourth-order rule for the integral of f over [x_0, x_m] on
    the points x (any spacing): on each interval [x_q, x_q+1], f is replaced by
    its cubic through the four points x_s0 .. x_s0+3 with s0 = q - 1 clamped to
    [0, m - 3] (the stencil is shifted inward at the ends), and the cubic is
    integrated exactly with the two-point Gauss-Legendre rule (exact for
    cubics). With fewer than four points the interpolant through all of them
    is used. Error O(h^4) for smooth f.

    Variant (the paper's "direct integration" gives no rule; the trapezoid is
    the default reading): it serves the fourth-order Dyson integrals below."""
    x = np.asarray(x, dtype=np.float64)
    m = len(x) - 1
    w = np.zeros(m + 1)
    g = 1.0 / math.sqrt(3.0)
    for q in range(m):
        s0 = 0 if m < 3 else min(max(q - 1, 0), m - 3)
        st = list(range(s0, min(s0 + 4, m + 1)))
        h = float(x[q + 1]) - float(x[q])
        mid = 0.5 * (float(x[q]) + float(x[q + 1]))
        for node in (mid - 0.5 * h * g, mid + 0.5 * h * g):
            for p, l in zip(st, _lagrange(x[st], node)):
                w[p] += 0.5 * h * l
    return w


def cubic_lag(tau: np.ndarray, y: float) -> tuple[int, list]:
    """Cubic interpolation at y in [-beta, 0] on the mesh: the stencil start s0
    (the bracket k of y, minus one, clamped to [0, M - 4]) and the Lagrange
    coefficients of the four mesh points tau_s0 .. tau_s0+3."""
    k, _ = bracket(tau, y)
    s0 = min(max(k - 1, 0), len(tau) - 4)
    return s0, _lagrange(tau[s0:s0 + 4], y)


def conv1(dHF: np.ndarray, A: np.ndarray, G: np.ndarray, mesh: dict, beta: float,
          lag: dict, rows=None, quad: str = "trap") -> np.ndarray:
    """I^(1)(tau_i) = (Sigma^HF - Sigma^0) g(tau_i) + int Sigma^corr(tau_i - t) g(t) dt.

    Eq. (deq), second line. Reading (the quadrature of the "direct
    integration" is not given): trapezoid on the mesh, split at t = tau_i
    where Sigma^corr jumps: for j != i the weight is w_j and Sigma^corr at the
    lag is linearly interpolated on the mesh (anti-periodic beyond 0); at
    j = i the left half-interval uses Sigma^corr(0^+) = -A_0 with weight wm_i
    and the right one Sigma^corr(0^-) = A_{M-1} with weight wp_i.
    ``rows`` restricts the output to a subset of i (sampled checks).

    quad="cubic4" (fourth-order variant): each side of the split, [-beta, tau_i]
    and [tau_i, 0], is integrated with ``quad4_weights`` on its own mesh points,
    and Sigma^corr at the lags is interpolated by ``cubic_lag`` (``lag`` is then
    not used).
    """
    M = G.shape[0]
    w, wm, wp = mesh["w"], mesh["wm"], mesh["wp"]
    tau = mesh["tau"]
    rows = range(M) if rows is None else rows
    out = []
    for i in rows:
        acc = dHF @ G[i]
        if quad == "cubic4":
            wl, wr = quad4_weights(tau[:i + 1]), quad4_weights(tau[i:])
            acc = acc + (-wl[i] * A[0] + wr[0] * A[M - 1]) @ G[i]
            for j in range(M):
                if j == i:
                    continue
                y, s = lag_point(tau, beta, i, j)
                s0, cl = cubic_lag(tau, y)
                wj = wl[j] if j < i else wr[j - i]
                B = (s * wj) * sum(c * A[s0 + q] for q, c in enumerate(cl))
                acc = acc + B @ G[j]
            out.append(acc)
            continue
        acc = acc + (-wm[i] * A[0] + wp[i] * A[M - 1]) @ G[i]
        for j in range(M):
            if j == i:
                continue
            k, t, s = int(lag["k"][i, j]), float(lag["t"][i, j]), float(lag["s"][i, j])
            B = (s * w[j]) * ((1.0 - t) * A[k] + t * A[k + 1])
            acc = acc + B @ G[j]
        out.append(acc)
    return np.stack(out)


def conv2(I1: np.ndarray, eps: np.ndarray, C: np.ndarray, mu: float, mesh: dict,
          beta: float, rows=None, quad: str = "trap") -> np.ndarray:
    """I^(2)(tau_i) = int g^0(tau_i - t) I^(1)(t) dt (Eq. deq, first integral).

    Same split trapezoid as ``conv1``; g^0 at every lag is evaluated from
    Eq. (hfgf) (no interpolation): lag < 0 gives C phi(lag) C^T, lag > 0 gives
    -C phi(lag - beta) C^T; at j = i the halves use g^0(0^+) = -g^0(-beta) and
    g^0(0^-). Plain O(M^2 n^3) loop. quad="cubic4": the two sides of the split
    with ``quad4_weights`` (g^0 stays exact at every lag).
    """
    tau, w, wm, wp = mesh["tau"], mesh["w"], mesh["wm"], mesh["wp"]
    M = len(tau)
    y = np.asarray(eps) - mu
    g0_0m = (C * phi(0.0, y, beta)) @ C.T          # g^0(0^-)
    g0_0p = -((C * phi(-beta, y, beta)) @ C.T)     # g^0(0^+)
    rows = range(M) if rows is None else rows
    out = []
    for i in rows:
        if quad == "cubic4":
            wl, wr = quad4_weights(tau[:i + 1]), quad4_weights(tau[i:])
            wj_of = lambda j, wl=wl, wr=wr, i=i: wl[j] if j < i else wr[j - i]
            acc = (wl[i] * g0_0p + wr[0] * g0_0m) @ I1[i]
        else:
            wj_of = lambda j: w[j]
            acc = (wm[i] * g0_0p + wp[i] * g0_0m) @ I1[i]
        for j in range(M):
            if j == i:
                continue
            yl, sg = lag_point(tau, beta, i, j)
            gl = sg * ((C * phi(yl, y, beta)) @ C.T)
            acc = acc + (wj_of(j) * gl) @ I1[j]
        out.append(acc)
    return np.stack(out)


# ---------------------------------------------------------------------------
# Sec. 2.3: total energy and the self-consistency loop
# ---------------------------------------------------------------------------


def energy(h: np.ndarray, V: np.ndarray, sigma: float, G: np.ndarray, A: np.ndarray,
           w: np.ndarray) -> float:
    """Galitskii-Migdal energy (the paper computes it "as in" its refs; Reading):

    E0 = sigma Tr[h rho] + (sigma/2) Tr[Sigma^HF[rho] rho]
         - (sigma/2) sum_j w_j Tr[Sigma^corr(tau_{M-1-j}) g(tau_j)],  rho = g(0^-).

    The last term is (sigma/2) Tr[(Sigma^corr * g)(0^-)]: the lag 0^- - tau_j
    is positive, so Sigma^corr there is -Sigma^corr(-beta - tau_j), which is
    the mirrored mesh point. E0 excludes the nuclear repulsion.
    """
    M = G.shape[0]
    rho = G[M - 1]
    e = sigma * float(np.sum(h * rho))
    e += 0.5 * sigma * float(np.sum(hf_selfenergy(rho, V, sigma) * rho))
    ec = 0.0
    for j in range(M):
        ec += float(w[j]) * float(np.sum(A[M - 1 - j] * G[j]))
    return e - 0.5 * sigma * ec


def dyson_iteration(h, V, sigma, hf, mesh, lag, beta, G0, G, mixing, A=None,
                    quad: str = "trap") -> dict:
    """One step of the second-Born self-consistency (Eq. deq):
    A = Sigma^corr[g] (unless given), dHF = Sigma^HF[g(0^-)] - Sigma^0,
    I1 = conv1, I2 = conv2, g_new = g^0 + I2, g' = (1 - a) g + a sym(g_new),
    r = max|g' - g|, E0 and N from (g, A).

    Reading: G(tau) of a real symmetric Hamiltonian is a symmetric matrix; the
    sequential direct integration g^0 * (Sigma * g) breaks that at the level
    of the quadrature error, so the update takes the symmetric part
    sym(X)_ab = 0.5 (X_ab + X_ba) of g_new. The jump invariant
    g(0^-) + g(-beta) = 1 is unaffected.

    quad="cubic4": the fourth-order variant of both integrals and of the
    energy's tau integral (``quad4_weights`` over the whole mesh)."""
    M = G.shape[0]
    if A is None:
        A = sigma2(G, V, sigma)
    dHF = hf_selfenergy(G[M - 1], V, sigma) - hf["Sigma0"]
    wE = quad4_weights(mesh["tau"]) if quad == "cubic4" else mesh["w"]
    E = energy(h, V, sigma, G, A, wE)
    Nel = sigma * float(np.trace(G[M - 1]))
    I1 = conv1(dHF, A, G, mesh, beta, lag, quad=quad)
    I2 = conv2(I1, hf["eps"], hf["C"], hf["mu"], mesh, beta, quad=quad)
    Gnew = G0 + I2
    Gnew = 0.5 * (Gnew + Gnew.transpose(0, 2, 1))
    Gnext = (1.0 - mixing) * G + mixing * Gnew
    r = float(np.max(np.abs(Gnext - G)))
    return dict(G=Gnext, Sigma=A, E0=E, N=Nel, res=r, I1=I1, I2=I2)


def bose_lag_table(tau: np.ndarray, beta: float) -> dict:
    """(k, t) of the lag tau_i - tau_j for every (i, j), functions extended
    periodically, F(x) = F(x - beta) for x in (0, beta] (bosonic: the bubble
    and the screened interaction). j >= i: y = tau_i - tau_j (y = 0 at i = j,
    the last mesh point); j < i: y = tau_i - tau_j - beta."""
    M = len(tau)
    K = np.zeros((M, M), dtype=np.int32)
    T = np.zeros((M, M))
    for i in range(M):
        for j in range(M):
            x = float(tau[i]) - float(tau[j])
            y = x if j >= i else x - beta
            K[i, j], T[i, j] = bracket(tau, y)
    return dict(k=K, t=T)


def conv_bose(A: np.ndarray, B: np.ndarray, mesh: dict, blag: dict) -> np.ndarray:
    """(A * B)(tau_i) = int over one period of A(tau_i - s) B(s) ds for
    periodic A: trapezoid on the mesh (weights w_j), A at the lag linearly
    interpolated (``bose_lag_table``); a periodic A has no jump at lag 0, so
    the trapezoid is not split there."""
    M = A.shape[0]
    w = mesh["w"]
    out = []
    for i in range(M):
        # A at the lags tau_i - tau_j for every j, each times w_j, then the sum over j of
        # those matrices times B_j
        k = blag["k"][i]
        t = blag["t"][i][:, None, None]
        Al = w[:, None, None] * ((1.0 - t) * A[k] + t * A[k + 1])
        out.append(np.einsum("jab,jbc->ac", Al, B))
    return np.stack(out)


def screened_w(G: np.ndarray, V: np.ndarray, sigma: float, mesh: dict, blag: dict, w0=None,
               mixing: float = 0.3, tol: float = 1e-12, max_iter: int = 500) -> dict:
    """Correlated screened interaction of the two-index bubble series.

    In the FE-DVR form the interaction is two-index (V_ab between the nodes a
    and b), so the polarisation bubble is too: with this code's g > 0 on
    [-beta, 0] it is -sigma Q with Q_j = g_j o gb_j (gb_j = g(-beta - tau_j)),
    and the correlated part of the screened interaction, W^c = V P V + V P * W^c,
    becomes -sigma w with

        w = V Q V - sigma V (Q * w),        Sigma^GW = sigma g o w,

    whose lowest order w = V Q V gives the direct term of Eq. sigma2ndb.
    Reading (the paper names GW without equations): the linear equation is
    solved by the damped fixed-point iteration w <- (1 - a) w + a w_new from w0
    (default V Q V) until max|w_new - w| < tol; the operator
    w -> sigma V (Q * w) has real non-negative eigenvalues here (bounded by
    about 5 on the He models at beta = 100), so a = 0.3 contracts where the
    plain series diverges. Returns w, the iterations and the last residual."""
    M = G.shape[0]
    Q = np.stack([G[j] * G[M - 1 - j] for j in range(M)])
    VQV = np.stack([V @ Q[j] @ V for j in range(M)])
    w = VQV.copy() if w0 is None else np.array(w0, dtype=np.float64)
    r = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        C = conv_bose(Q, w, mesh, blag)
        new = VQV - sigma * np.stack([V @ C[j] for j in range(M)])
        r = float(np.max(np.abs(new - w)))
        w = (1.0 - mixing) * w + mixing * new
        if r < tol:
            break
    return dict(w=w, iters=it, res=r, Q=Q, VQV=VQV)


def sigma_gw(G: np.ndarray, V: np.ndarray, sigma: float, mesh: dict, blag: dict, w0=None,
             mixing: float = 0.3, tol: float = 1e-12, max_iter: int = 500) -> dict:
    """GW correlation self-energy Sigma^GW_j = sigma g_j o w_j (``screened_w``);
    no exchange term (GW sums the bubbles, second Born adds the second-order
    exchange)."""
    sw = screened_w(G, V, sigma, mesh, blag, w0, mixing, tol, max_iter)
    sw["Sigma"] = sigma * G * sw["w"]
    return sw


def pair_conv(G: np.ndarray, t: np.ndarray, mesh: dict, blag: dict) -> np.ndarray:
    """(K * t)(tau_i) for the particle-particle propagator K(tau) = g(tau) (x) g(tau)
    acting on the row pair of a pair-space function t[j, a, k, b, l] (rows
    (a, k), columns (b, l)):

        (K * t)_i[a, k, b, l] = sum_j w_j sum_{a' k'} K(tau_i - tau_j)_{(a k),(a' k')} t_j[a', k', b, l],
        K(x)_{(a k),(a' k')} = g_{a a'}(x) g_{k k'}(x).

    K is periodic (the product of two anti-periodic functions), so the lag is
    wrapped as for the bubble (``bose_lag_table``) and K at the lag is the
    linear interpolation of K between the bracketing mesh points."""
    M = G.shape[0]
    w = mesh["w"]
    # (g_r (x) g_r) t_j for every mesh point r and j: Z[r, j] = g_r X g_r^T per column (b, l)
    Z = np.einsum("rac,rkd,jcdbl->rjakbl", G, G, t, optimize=True)
    jj = np.arange(M)[None, :]
    kk, tt = blag["k"], blag["t"]
    lower = (w[None, :] * (1.0 - tt))[:, :, None, None, None, None] * Z[kk, jj]
    upper = (w[None, :] * tt)[:, :, None, None, None, None] * Z[kk + 1, jj]
    return (lower + upper).sum(axis=1)


def ladder_t(G: np.ndarray, V: np.ndarray, sigma: float, mesh: dict, blag: dict, t0=None,
             mixing: float = 0.3, tol: float = 1e-12, max_iter: int = 500) -> dict:
    """Correlated particle-particle T-matrix of the two-index interaction.

    Reading (the paper names the T-matrix approximation without equations;
    this follows the Matsubara Feynman rules in this code's g > 0 convention,
    G(tau) = g(tau) and G(-tau) = -gb(tau) on [-beta, 0]): a pair of particles
    at the nodes (a, k) scatters through V_ak without changing nodes, so the
    ladder lives on node pairs with the pair propagator K = g (x) g, and with
    V^ the diagonal pair-space matrix of the V_ak the correlated part of the
    T-matrix, T^c = -V^ K V^ - V^ (K * T^c), is -t with

        t = V^ K V^ - V^ (K * t),      t_j[a, k, b, l] = V_ak g_ab g_kl V_bl - V_ak (K * t)_j[a, k, b, l].

    No spin factor enters (no closed loop). Solved like the screened
    interaction: damped fixed-point iteration from t0 (default the lowest
    order V^ K V^) until max|t_new - t| < tol. Pair-space arrays are
    [M][n][n][n][n]; small n only."""
    M = G.shape[0]
    S = np.einsum("ak,jab,jkl,bl->jakbl", V, G, G, V)
    t = S.copy() if t0 is None else np.array(t0, dtype=np.float64)
    r = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        C = pair_conv(G, t, mesh, blag)
        new = S - V[None, :, :, None, None] * C
        r = float(np.max(np.abs(new - t)))
        t = (1.0 - mixing) * t + mixing * new
        if r < tol:
            break
    return dict(t=t, iters=it, res=r, S=S)


def sigma_tmatrix(G: np.ndarray, V: np.ndarray, sigma: float, mesh: dict, blag: dict, t0=None,
                  mixing: float = 0.3, tol: float = 1e-12, max_iter: int = 500) -> dict:
    """T-matrix correlation self-energy: the ladder closed with a hole line, the
    direct term with the spin factor and the exchange term without,

        Sigma^T_ab(tau_j) = sum_kl [sigma t_j[a, k, b, l] - t_j[a, k, l, b]] gb_j[l, k],

    gb_j = g(-beta - tau_j) (``ladder_t``). At lowest order (t = V^ K V^) this
    is Eq. sigma2ndb term by term: the direct term sigma g_ab (V Q V)_ab and the
    exchange sum_kl V_ak V_bl g_al gb_lk g_kb."""
    lt = ladder_t(G, V, sigma, mesh, blag, t0, mixing, tol, max_iter)
    t = lt["t"]
    M = G.shape[0]
    gb = G[::-1]
    lt["Sigma"] = (sigma * np.einsum("jakbl,jlk->jab", t, gb)
                   - np.einsum("jaklb,jlk->jab", t, gb))
    return lt


def solve_2b(h, V, sigma, hf, beta, u, p, mixing=0.5, tol=1e-8, max_iter=200,
             sigma_init=None, quad: str = "trap", self_energy: str = "2b",
             gw_mixing: float = 0.3, gw_tol: float = 1e-12, gw_max_iter: int = 500) -> dict:
    """Second-Born Matsubara self-consistency (Sec. 2.3 and 3.1).

    Reading (the iteration scheme is not given): start from g = g^0; linear
    mixing of g with weight ``mixing``; stop when max|g_{k+1} - g_k| < tol.
    ``sigma_init`` replaces Sigma^corr[g^0] in the first iteration only (warm
    start). Returns the final g_{k+1}, Sigma_k = Sigma^corr[g_k], and E0 and N
    evaluated on (g_k, Sigma_k).

    self_energy="gw": Sigma^corr = ``sigma_gw`` instead of second Born; the
    inner iteration for w starts from the previous outer iteration's w (V Q V
    at the first) and ``gw_inner`` lists its iterations per outer step.
    self_energy="tmatrix": Sigma^corr = ``sigma_tmatrix``, its ladder iteration
    warm-started the same way (``gw_*`` name the inner iteration's controls).
    """
    mesh = power_mesh(beta, u, p)
    lag = lag_table(mesh["tau"], beta)
    blag = bose_lag_table(mesh["tau"], beta) if self_energy in ("gw", "tmatrix") else None
    G0 = g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], beta)
    G = G0.copy()
    hist = []
    step = None
    converged = False
    w_state = None
    gw_inner = []
    for it in range(max_iter):
        A = sigma_init if (it == 0 and sigma_init is not None) else None
        if A is None and self_energy == "gw":
            sg = sigma_gw(G, V, sigma, mesh, blag, w_state, gw_mixing, gw_tol, gw_max_iter)
            A, w_state = sg["Sigma"], sg["w"]
            gw_inner.append(sg["iters"])
        elif A is None and self_energy == "tmatrix":
            sg = sigma_tmatrix(G, V, sigma, mesh, blag, w_state, gw_mixing, gw_tol, gw_max_iter)
            A, w_state = sg["Sigma"], sg["t"]
            gw_inner.append(sg["iters"])
        step = dyson_iteration(h, V, sigma, hf, mesh, lag, beta, G0, G, mixing, A=A, quad=quad)
        hist.append((it, step["res"], step["E0"], step["N"]))
        G = step["G"]
        if step["res"] < tol:
            converged = True
            break
    return dict(G=G, Sigma=step["Sigma"], E0=step["E0"], N=step["N"], iters=len(hist),
                converged=converged, history=hist, mesh=mesh, G0=G0, gw_inner=gw_inner)


# ---------------------------------------------------------------------------
# Sec. 2, Eqs. (kbe), (skkbe), (skkbesigma): real-time Kadanoff-Baym equations
# ---------------------------------------------------------------------------


def sigma2_realtime(g: np.ndarray, gb: np.ndarray, V: np.ndarray, sigma: float) -> np.ndarray:
    """Second-Born self-energy of Eq. (sigma2ndb) for complex two-time
    matrices: g = the Green's function at (t, t'), gb = minus the other
    Keldysh component at (t', t) (indices kept: gb_lk is line l -> k from t'
    back to t), in the convention L = -i G^< (so L(t, t) = rho) and
    Gt = -i G^>:

      -i Sigma^<(t, t') = S(L(t, t'), -Gt(t', t)),
      -i Sigma^>(t, t') = S(Gt(t, t'), -L(t', t)),
      S(g, gb) = sigma g o (V (g o gb^T) V) - X,  X_ab = sum_kl V_ak V_bl g_al gb_lk g_kb.

    The polarisation bubble pairs g_kl(t, t') with the reversed line
    gb_lk(t', t), hence the transpose; for the real symmetric Matsubara
    functions of ``sigma2_tau`` (g(tau) and gb = g(-beta - tau)) the two forms
    coincide. Reading (as for the Matsubara form): the time-consistent pairing
    u_13 u_24 of Eq. (sigma2ndb)."""
    Q = g * gb.T
    D = sigma * g * (V @ Q @ V)
    n = g.shape[0]
    X = np.empty_like(g)
    for b in range(n):
        P = g @ (V[b][:, None] * gb)      # P_ak = sum_l g_al V_bl gb_lk
        X[:, b] = (V * P) @ g[:, b]       # X_ab = sum_k V_ak P_ak g_kb
    return D - X


def kbe_propagate(h: np.ndarray, V: np.ndarray, sigma: float, rho0: np.ndarray, dt: float,
                  n_steps: int, dv: np.ndarray = None, second_born: bool = True) -> dict:
    """Two-time Kadanoff-Baym propagation (Eqs. kbe, skkbe with the self-energy
    of Eq. skkbesigma: the time-local HF part of Eq. sigmahf plus second Born)
    on the uniform grid t_k = k dt, k = 0 .. n_steps.

    Reading (the paper states the equations, with initial correlations by the
    mixed Green's function, and runs only the equilibrium problem): the
    initial state is uncorrelated, L(0, 0) = rho0 (the one-particle density
    matrix per spin of a Slater determinant or thermal HF state), so the
    contour reduces to the real-time branches and the collision integrals start
    at t = 0. With L = -i G^< and Gt = -i G^> (L(t, t) = rho(t),
    Gt(t, t) = rho(t) - 1, L(t', t) = L(t, t')^H, Gt likewise) the equation for
    the first time argument reads

      d/dt F(t, t') = -i h_HF(t) F(t, t') + K_F(t, t'),   F = L or Gt,
      K_L = int_0^t [s^> - s^<](t, s) L(s, t') ds + int_0^t' s^<(t, s) [L - Gt](s, t') ds,
      K_G = int_0^t [s^> - s^<](t, s) Gt(s, t') ds + int_0^t' s^>(t, s) [L - Gt](s, t') ds,

    s^x = -i Sigma^x (``sigma2_realtime``), h_HF(t) = h + diag(dv(t)) +
    Sigma^HF[rho(t)]; the equal-time density follows
    d rho/dt = X + X^H with X = -i h_HF rho + K_L(t, t) (the adjoint equation
    gives the second argument). The integrals use the trapezoid on the grid and
    each step is Heun's predictor-corrector (second order in dt): the new time
    row F(t_N+1, t_j) and rho(t_N+1) from the right-hand sides at t_N, then
    again with those at the predicted t_N+1.

    Returns rho [n_steps+1][n][n] (complex), L, Gt [T][T][n][n], the energy
    E(t) = sigma Tr[h rho] + (sigma/2) Tr[Sigma^HF rho] + (sigma/2) Re Tr[i K_L(t, t)]
    (the one-body part with h(t), the HF interaction and the correlation
    energy from the collision integral; conserved without dv) and
    N(t) = sigma Tr rho. ``second_born`` False: time-dependent HF."""
    n = h.shape[0]
    T = n_steps + 1
    L = np.zeros((T, T, n, n), complex)
    G = np.zeros((T, T, n, n), complex)
    sL = np.zeros((T, T, n, n), complex)
    sG = np.zeros((T, T, n, n), complex)
    hHF = np.zeros((T, n, n), complex)
    ident = np.eye(n)
    L[0, 0] = rho0
    G[0, 0] = rho0 - ident

    def h_at(i):
        return h + (np.diag(dv[i]) if dv is not None else 0.0)

    def self_energies(i):
        hHF[i] = h_at(i) + hf_selfenergy(L[i, i], V, sigma)
        if second_born:
            for k in range(i + 1):
                sL[i, k] = sigma2_realtime(L[i, k], -G[i, k].conj().T, V, sigma)
                sG[i, k] = sigma2_realtime(G[i, k], -L[i, k].conj().T, V, sigma)

    def weights(m):
        w = np.full(m + 1, dt)
        w[0] = w[-1] = 0.5 * dt
        return w * (m > 0)

    def rhs(i, j):
        wi, wj = weights(i), weights(j)
        A = sG[i, :i + 1] - sL[i, :i + 1]
        D = L[:j + 1, j] - G[:j + 1, j]
        KL = (np.einsum("s,sab,sbc->ac", wi, A, L[:i + 1, j])
              + np.einsum("s,sab,sbc->ac", wj, sL[i, :j + 1], D))
        KG = (np.einsum("s,sab,sbc->ac", wi, A, G[:i + 1, j])
              + np.einsum("s,sab,sbc->ac", wj, sG[i, :j + 1], D))
        return -1j * hHF[i] @ L[i, j] + KL, -1j * hHF[i] @ G[i, j] + KG, KL

    def observe(i):
        rho = L[i, i]
        KL = rhs(i, i)[2]
        e = sigma * np.trace(h_at(i) @ rho).real
        e += 0.5 * sigma * np.trace(hf_selfenergy(rho, V, sigma) @ rho).real
        e += 0.5 * sigma * (1j * np.trace(KL)).real
        return e, sigma * np.trace(rho).real

    def mirror(i):
        for j in range(i):
            L[j, i] = L[i, j].conj().T
            G[j, i] = G[i, j].conj().T

    self_energies(0)
    obs = [observe(0)]
    for N in range(n_steps):
        r0 = [rhs(N, j) for j in range(N + 1)]
        d0 = r0[N][0] + r0[N][0].conj().T
        for j in range(N + 1):   # predictor
            L[N + 1, j] = L[N, j] + dt * r0[j][0]
            G[N + 1, j] = G[N, j] + dt * r0[j][1]
        L[N + 1, N + 1] = L[N, N] + dt * d0
        G[N + 1, N + 1] = L[N + 1, N + 1] - ident
        mirror(N + 1)
        self_energies(N + 1)
        r1 = [rhs(N + 1, j) for j in range(N + 2)]
        d1 = r1[N + 1][0] + r1[N + 1][0].conj().T
        for j in range(N + 1):   # corrector
            L[N + 1, j] = L[N, j] + 0.5 * dt * (r0[j][0] + r1[j][0])
            G[N + 1, j] = G[N, j] + 0.5 * dt * (r0[j][1] + r1[j][1])
        L[N + 1, N + 1] = L[N, N] + 0.5 * dt * (d0 + d1)
        G[N + 1, N + 1] = L[N + 1, N + 1] - ident
        mirror(N + 1)
        self_energies(N + 1)
        obs.append(observe(N + 1))
    rho = np.array([L[i, i] for i in range(T)])
    return dict(rho=rho, L=L, Gt=G, E=np.array([o[0] for o in obs]),
                N=np.array([o[1] for o in obs]))


def exact_dynamics(h: np.ndarray, V: np.ndarray, phi0: np.ndarray, times) -> np.ndarray:
    """Pin only: the two-electron singlet evolved exactly on the grid, from the
    doubly occupied orbital phi0 (spatial wave function Psi_ab = phi0_a phi0_b)
    under H = h (x) 1 + 1 (x) h + diag(V_ab); returns the density matrix per
    spin rho_ab(t) = sum_c Psi_ac(t) Psi_bc(t)^* for each time."""
    import scipy.linalg as sla
    n = h.shape[0]
    ident = np.eye(n)
    H2 = np.kron(h, ident) + np.kron(ident, h) + np.diag(np.asarray(V).ravel())
    psi0 = np.outer(phi0, phi0).ravel().astype(complex)
    out = []
    for t in times:
        psi = (sla.expm(-1j * H2 * float(t)) @ psi0).reshape(n, n)
        out.append(psi @ psi.conj().T)
    return np.array(out)


# ---------------------------------------------------------------------------
# Pins: MP2 and the exact two-electron ground state on the same grid
# ---------------------------------------------------------------------------


def mp2(eps: np.ndarray, C: np.ndarray, V: np.ndarray, nocc: int) -> float:
    """Closed-shell MP2 energy with FE-DVR integrals (pq|rs) = delta_pq delta_rs V_pr:
    E = sum_{ij occ, ab virt} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b),
    (ia|jb) = sum_{pq} C_pi C_pa V_pq C_qj C_qb."""
    occ, vir = C[:, :nocc], C[:, nocc:]
    L = np.einsum("pi,pa->iap", occ, vir)
    ovov = np.einsum("iap,pq,jbq->iajb", L, V, L, optimize=True)
    eo, ev = eps[:nocc], eps[nocc:]
    den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return float(np.sum(ovov * (2.0 * ovov - ovov.transpose(0, 3, 2, 1)) / den))


def exact_ground(T: np.ndarray, v: np.ndarray, V: np.ndarray) -> float:
    """Lowest eigenvalue of the two-electron grid Hamiltonian
    H = T (x) 1 + 1 (x) T + diag(v_a + v_b + V_ab) on n^2 product points.
    In 1D the spatially symmetric (singlet) state is the ground state."""
    n = T.shape[0]
    diag = (v[:, None] + v[None, :] + V).ravel()
    if n <= 40:
        I = np.eye(n)
        H = np.kron(T, I) + np.kron(I, T) + np.diag(diag)
        return float(np.linalg.eigvalsh(H)[0])
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    Ts = sp.csr_matrix(T)
    I = sp.identity(n, format="csr")
    H = sp.kron(Ts, I) + sp.kron(I, Ts) + sp.diags(diag)
    val = spl.eigsh(H.tocsr(), k=1, which="SA", tol=1e-12)[0]
    return float(val[0])


def exact_ground_state(T: np.ndarray, v: np.ndarray, V: np.ndarray) -> tuple[float, np.ndarray]:
    """Lowest eigenpair of the two-electron grid Hamiltonian of ``exact_ground``:
    the energy and the eigenvector as DVR coefficients Psi[a, b] of the two
    electrons at nodes x_a and x_b (sum |Psi|^2 = 1, Psi symmetric)."""
    n = T.shape[0]
    diag = (v[:, None] + v[None, :] + V).ravel()
    if n <= 40:
        I = np.eye(n)
        H = np.kron(T, I) + np.kron(I, T) + np.diag(diag)
        vals, vecs = np.linalg.eigh(H)
        return float(vals[0]), vecs[:, 0].reshape(n, n)
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    Ts = sp.csr_matrix(T)
    I = sp.identity(n, format="csr")
    H = sp.kron(Ts, I) + sp.kron(I, Ts) + sp.diags(diag)
    vals, vecs = spl.eigsh(H.tocsr(), k=1, which="SA", tol=1e-12)
    return float(vals[0]), vecs[:, 0].reshape(n, n)


def exact_density(psi: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """One-electron density of the two-electron ground state at the nodes:
    n(x_a) = 2 sum_b Psi_ab^2 / W_a (each electron's marginal, the DVR
    function of node a being 1/sqrt(W_a) there); sum_a W_a n(x_a) = 2."""
    return 2.0 * np.sum(psi * psi, axis=1) / weights


# ---------------------------------------------------------------------------
# Sec. 2.3 and 3.2: observables
# ---------------------------------------------------------------------------


def density(g0m: np.ndarray, weights: np.ndarray, sigma: float) -> np.ndarray:
    """One-electron density at the nodes from g(0^-) (Sec. 2.3: n(x) is the sum
    over basis pairs of chi chi g(0^-)). A DVR function is 1/sqrt(W_a) at its own
    node and zero at every other node, so only the diagonal survives there:
    n(x_a) = sigma g_aa(0^-) / W_a.

    Reading: g is the Green's function of one spin (sigma Tr g(0^-) = N, as in
    the particle number), so the density carries sigma and integrates to N:
    sum_a W_a n(x_a) = N."""
    return sigma * np.diag(g0m) / weights


def nuclear_repulsion(Z, R) -> float:
    """E_nn = sum_{A<B} Z_A Z_B / |R_A - R_B| (bare Coulomb).

    Reading (Eq. h3pv): the offset 5/d of the H3+ model collects the
    internuclear energy; for unit charges at (-d/2, 0, d/2) it is exactly
    1/(d/2) + 1/(d/2) + 1/d = 5/d. It is added once to the electronic energy
    (not to the one-electron potential, which would count it per electron)."""
    e = 0.0
    for A in range(len(Z)):
        for B in range(A + 1, len(Z)):
            e += float(Z[A]) * float(Z[B]) / abs(float(R[A]) - float(R[B]))
    return e
