"""GB300-native FE-DVR second-Born Green's functions (arXiv:0911.4348).

Thin Python binding over the C ABI of ``libfedvr_negf.so`` (declared in
include/fedvr_negf.h). Every call marshals arguments and forwards to the CUDA
library; no numerical step runs in Python. Device buffers are float64 torch
tensors on the context's device; host buffers are numpy arrays.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native

FP64, SPLIT_TF32, SPLIT_BF16, SPLIT_F16 = 0, 1, 2, 3
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_NOCONV", -4: "ERR_DIVERGED",
          -5: "ERR_TIMEOUT", -6: "ERR_NAN", -7: "ERR_STATE"}


class FedvrError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code


def _dptr(arr):
    """ctypes double* for a host numpy array (or None)."""
    if arr is None:
        return None
    assert arr.dtype == np.float64 and arr.flags["C_CONTIGUOUS"]
    return arr.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(arr):
    if arr is None:
        return None
    assert arr.dtype == np.int32 and arr.flags["C_CONTIGUOUS"]
    return arr.ctypes.data_as(C.POINTER(C.c_int))


def _dev(t, shape=None, dtype=None):
    """Raw device address of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if dtype is None and t.dtype != torch.float64:
        raise ValueError("expected float64")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _host_or_dev(x):
    if x is None:
        return None, False
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data), False
    return _dev(x), True


class Context:
    """A library context (``fedvr_create``) bound to a CUDA stream."""

    def __init__(self, stream=None):
        self._lib = _native.lib()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._h = C.c_void_p()
        code = self._lib.fedvr_create(C.byref(self._h), C.c_void_p(stream))
        if code != 0:
            raise FedvrError(code, "fedvr_create failed")
        self.n_b = 0

    def close(self):
        if self._h:
            self._lib.fedvr_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _check(self, code):
        if code != 0:
            msg = self._lib.fedvr_last_error(self._h)
            raise FedvrError(code, msg.decode() if msg else "")
        return code

    def last_error(self) -> str:
        return self._lib.fedvr_last_error(self._h).decode()

    # -- basis and operators -------------------------------------------------
    def build_fedvr(self, n_elem, pts_per_elem, xmin, xmax, grid_kind=0) -> int:
        """FE-DVR basis with n_elem elements of pts_per_elem GLL points each
        (polynomial order pts_per_elem - 1); returns n_b."""
        nb = C.c_int()
        self._check(self._lib.build_fedvr(self._h, n_elem, pts_per_elem, xmin, xmax, grid_kind,
                                          C.byref(nb)))
        self.n_b = nb.value
        self.order = pts_per_elem - 1
        return nb.value

    def set_potential(self, Z, R, soft_en=1.0, soft_ee=1.0, n_elec=2) -> float:
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        enn = C.c_double()
        self._check(self._lib.set_potential(self._h, len(Z), _dptr(Z), _dptr(R), soft_en, soft_ee,
                                            n_elec, C.byref(enn)))
        return enn.value

    def get_basis(self):
        n = self.n_b
        x, w = np.empty(n), np.empty(n)
        e, m = np.empty(n, np.int32), np.empty(n, np.int32)
        self._check(self._lib.fedvr_get_basis(self._h, _dptr(x), _dptr(w), _iptr(e), _iptr(m)))
        return dict(nodes=x, weights=w, elem=e, local=m)

    def get_gll(self):
        xi, om = np.empty(self.order + 1), np.empty(self.order + 1)
        self._check(self._lib.fedvr_get_gll(self._h, _dptr(xi), _dptr(om)))
        return xi, om

    def get_operators(self, potential=True):
        n = self.n_b
        T = np.empty((n, n))
        if not potential:
            self._check(self._lib.fedvr_get_operators(self._h, _dptr(T), None, None, None))
            return dict(T=T)
        v, V, h = np.empty(n), np.empty((n, n)), np.empty((n, n))
        self._check(self._lib.fedvr_get_operators(self._h, _dptr(T), _dptr(v), _dptr(V), _dptr(h)))
        return dict(T=T, v=v, V=V, h=h)

    # -- Hartree-Fock -----------------------------------------------------------
    def solve_hf(self, beta, tol=1e-12, max_iter=500):
        e, mu = C.c_double(), C.c_double()
        self._check(self._lib.solve_hf(self._h, beta, tol, max_iter, C.byref(e), C.byref(mu)))
        return e.value, mu.value

    def get_hf(self):
        n = self.n_b
        eps, Cm, rho, S0 = np.empty(n), np.empty((n, n)), np.empty((n, n)), np.empty((n, n))
        self._check(self._lib.fedvr_get_hf(self._h, _dptr(eps), _dptr(Cm), _dptr(rho), _dptr(S0)))
        return dict(eps=eps, C=Cm, rho0=rho, Sigma0=S0)

    def density(self, source="2b"):
        """One-electron density at the nodes, spin * g_aa(0^-) / W_a
        (``fedvr_density``): source "hf" (last HF solution) or "2b" (current
        second-Born iterate)."""
        src = {"hf": 0, "2b": 1}[source]
        out = np.empty(self.n_b)
        self._check(self._lib.fedvr_density(self._h, src, _dptr(out)))
        return out

    # -- second Born ------------------------------------------------------------
    def solve_2b(self, beta, u, p, mixing=0.5, tol=1e-8, max_iter=200, precision=FP64,
                 G_out=None, Sigma_out=None, tau_out=None, check=True):
        """Run the self-consistency. Outputs may be numpy arrays (host) or CUDA
        tensors (device); all given outputs must be of the same kind."""
        outs = [_host_or_dev(x) for x in (G_out, Sigma_out, tau_out)]
        kinds = {d for (p_, d) in outs if p_ is not None}
        if len(kinds) > 1:
            raise ValueError("outputs must all be host or all be device")
        on_dev = 1 if kinds == {True} else 0
        E0, N, it = C.c_double(), C.c_double(), C.c_int()
        code = self._lib.solve_2b(self._h, beta, u, p, mixing, tol, max_iter, precision, on_dev,
                                  outs[0][0], outs[1][0], outs[2][0], C.byref(E0), C.byref(N),
                                  C.byref(it))
        if check:
            self._check(code)
        return dict(E0=E0.value, N=N.value, iters=it.value, status=code)

    def prepare_2b(self, beta, u, p, precision=FP64):
        self._check(self._lib.fedvr_2b_prepare(self._h, beta, u, p, precision))
        self.M = 2 * u * p + 1

    def step_2b(self, mixing=0.5, G_in=None, check=True):
        """One iteration; G_in (host numpy or CUDA tensor) replaces the iterate first."""
        ptr, dev = _host_or_dev(G_in)
        res, E0, N = C.c_double(), C.c_double(), C.c_double()
        code = self._lib.fedvr_2b_step(self._h, mixing, ptr, 1 if dev else 0, C.byref(res),
                                       C.byref(E0), C.byref(N))
        if check:
            self._check(code)
        return dict(res=res.value, E0=E0.value, N=N.value, status=code)

    def use_graphs(self, enable=None) -> bool:
        """Switch graph replay of the iteration on/off (None: leave it); returns
        whether the last step ran as a graph replay."""
        last = C.c_int()
        self._check(self._lib.fedvr_use_graphs(self._h, -1 if enable is None else int(bool(enable)),
                                               C.byref(last)))
        return bool(last.value)

    def conv1_splits(self, request=None) -> int:
        """Request the first convolution's split count (0 = measured choice,
        None = leave); returns the count of the prepared run."""
        cur = C.c_int()
        self._check(self._lib.fedvr_conv1_splits(self._h, -1 if request is None else int(request),
                                                 C.byref(cur)))
        return cur.value

    def set_mu(self, mu):
        """Chemical potential of the next second-Born run (``fedvr_set_mu``)."""
        self._check(self._lib.fedvr_set_mu(self._h, float(mu)))

    def set_self_energy(self, kind, w_mixing=0.3, w_tol=1e-12, w_max_iter=500):
        """Correlation self-energy of the next prepare/solve: "2b" (second Born),
        "gw" or "tmatrix" (``fedvr_set_self_energy``)."""
        k = {"2b": 0, "gw": 1, "tmatrix": 2}.get(kind, kind)
        self._check(self._lib.fedvr_set_self_energy(self._h, int(k), float(w_mixing),
                                                    float(w_tol), int(w_max_iter)))

    def gw_last_inner(self) -> int:
        it = C.c_int()
        self._check(self._lib.fedvr_gw_last_inner(self._h, C.byref(it)))
        return it.value

    def sigma_gw(self, beta, u, p, V, G, Sigma, spin=2.0, w=None, w_valid=False, w_mixing=0.3,
                 w_tol=1e-12, w_max_iter=500):
        """Stage-level GW self-energy of the CUDA stack G into Sigma
        (``fedvr_sigma_gw``); returns the inner iterations."""
        M, n = G.shape[0], G.shape[1]
        assert M == 2 * u * p + 1
        it = C.c_int()
        self._check(self._lib.fedvr_sigma_gw(
            self._h, n, float(beta), int(u), int(p), float(spin), _dev(V, (n, n)),
            _dev(G, (M, n, n)), _dev(Sigma, (M, n, n)), _dev(w, (M, n, n)) if w is not None else None,
            1 if w_valid else 0, float(w_mixing), float(w_tol), int(w_max_iter), C.byref(it)))
        return it.value

    def sigma_tmatrix(self, beta, u, p, V, G, Sigma, spin=2.0, t=None, t_valid=False,
                      t_mixing=0.3, t_tol=1e-12, t_max_iter=500):
        """Stage-level T-matrix self-energy of the CUDA stack G into Sigma
        (``fedvr_sigma_tmatrix``); t (optional) is the ladder [M][n][n][n][n] in
        the library's layout t[j][b][l][a][k]; returns the inner iterations."""
        M, n = G.shape[0], G.shape[1]
        assert M == 2 * u * p + 1
        it = C.c_int()
        self._check(self._lib.fedvr_sigma_tmatrix(
            self._h, n, float(beta), int(u), int(p), float(spin), _dev(V, (n, n)),
            _dev(G, (M, n, n)), _dev(Sigma, (M, n, n)),
            _dev(t, (M, n, n, n, n)) if t is not None else None, 1 if t_valid else 0,
            float(t_mixing), float(t_tol), int(t_max_iter), C.byref(it)))
        return it.value

    def set_quadrature(self, order):
        """Quadrature of the Dyson integrals (``fedvr_set_quadrature``): 2 = split
        trapezoid with linear lag interpolation, 4 = the fourth-order variant
        (FP64 path)."""
        self._check(self._lib.fedvr_set_quadrature(self._h, int(order)))

    def stage_times(self):
        """Device milliseconds of the last step's stages: sigma2, hf+energy,
        conv1, conv2, update, whole step; and its kernel launch count."""
        ms = np.empty(6)
        ln = C.c_int()
        self._check(self._lib.fedvr_stage_times(self._h, _dptr(ms), C.byref(ln)))
        return dict(zip(("sigma2", "hf_energy", "conv1", "conv2", "update", "step"), ms)), ln.value

    def read_2b(self, G_out=None, Sigma_out=None, tau_out=None):
        outs = [_host_or_dev(x) for x in (G_out, Sigma_out, tau_out)]
        kinds = {d for (p_, d) in outs if p_ is not None}
        if len(kinds) > 1:
            raise ValueError("outputs must all be host or all be device")
        on_dev = 1 if kinds == {True} else 0
        self._check(self._lib.fedvr_2b_read(self._h, on_dev, outs[0][0], outs[1][0], outs[2][0]))

    def set_initial_sigma(self, Sigma0, M=None, inner_steps=0):
        if Sigma0 is None:
            self._check(self._lib.fedvr_set_initial_sigma(self._h, None, 0, 0, 0))
            return
        ptr, dev = _host_or_dev(Sigma0)
        M = Sigma0.shape[0] if M is None else M
        self._check(self._lib.fedvr_set_initial_sigma(self._h, ptr, M, 1 if dev else 0,
                                                      inner_steps))

    def warm_start(self, mlp, beta, u, p, inner_steps=4):
        """Predict the converged Sigma with the network and set it as the warm
        start of the next solve_2b (``fedvr_warm_start``)."""
        code = self._lib.fedvr_warm_start(self._h, mlp.handle, beta, u, p, inner_steps)
        if code != 0:
            raise FedvrError(code, mlp.last_error() or self.last_error())

    def get_history(self) -> np.ndarray:
        ln = C.c_int()
        self._check(self._lib.fedvr_get_history(self._h, None, 0, C.byref(ln)))
        buf = np.empty(5 * max(ln.value, 1))
        self._check(self._lib.fedvr_get_history(self._h, _dptr(buf), ln.value, C.byref(ln)))
        return buf[: 5 * ln.value].reshape(-1, 5)

    # -- stage-level calls on device buffers -----------------------------------------
    def power_mesh(self, beta, u, p, tau=None, w=None, wm=None, wp=None, lag_k=None, lag_t=None):
        import torch
        self._check(self._lib.fedvr_power_mesh(self._h, beta, u, p, _dev(tau), _dev(w), _dev(wm),
                                               _dev(wp), _dev(lag_k, dtype=torch.int32),
                                               _dev(lag_t)))

    def sigma2(self, V, G, Sigma, spin=2.0, precision=FP64):
        M, n = G.shape[0], G.shape[1]
        self._check(self._lib.fedvr_sigma2(self._h, n, M, spin, _dev(V, (n, n)), _dev(G, (M, n, n)),
                                           _dev(Sigma, (M, n, n)), precision))

    def conv_sigma_g(self, beta, u, p, dHF, Sigma, G, I1, precision=FP64):
        M, n = G.shape[0], G.shape[1]
        assert M == 2 * u * p + 1
        self._check(self._lib.fedvr_conv_sigma_g(self._h, n, beta, u, p, _dev(dHF, (n, n)),
                                                 _dev(Sigma, (M, n, n)), _dev(G, (M, n, n)),
                                                 _dev(I1, (M, n, n)), precision))

    def conv_g0(self, beta, u, p, eps, Cmat, mu, I1, I2, precision=FP64):
        M, n = I1.shape[0], I1.shape[1]
        assert M == 2 * u * p + 1
        self._check(self._lib.fedvr_conv_g0(self._h, n, beta, u, p, _dev(eps, (n,)),
                                            _dev(Cmat, (n, n)), mu, _dev(I1, (M, n, n)),
                                            _dev(I2, (M, n, n)), precision))

    def selftest_wait(self, release, limit_seconds=1e-3):
        """Run the bounded device-wait self-test (``fedvr_selftest_wait``):
        release=True must return normally; release=False raises FedvrError
        with code -5 (timeout) and leaves the context failed."""
        self._check(self._lib.fedvr_selftest_wait(self._h, 1 if release else 0, limit_seconds))

    def kbe_propagate(self, dt, n_steps, second_born=True, rho0=None, dv=None, want_rho=True,
                      precision=FP64):
        """Real-time two-time Kadanoff-Baym propagation (``fedvr_kbe_propagate``)
        from rho0 (complex [n][n]; None: the HF density of the last solve_hf)
        under h + diag(dv[k]) (dv: [n_steps+1][n] or None); precision FP64 or
        SPLIT_TF32 (collision integrals on the tensor cores). Returns a dict
        with rho [n_steps+1][n][n] complex (if want_rho), E and N [n_steps+1]."""
        n = self.n_b
        T = n_steps + 1
        r0 = None
        if rho0 is not None:
            r0 = np.ascontiguousarray(np.asarray(rho0, dtype=np.complex128)).view(np.float64)
            assert r0.shape == (n, 2 * n)
        d = None
        if dv is not None:
            d = np.ascontiguousarray(dv, dtype=np.float64)
            assert d.shape == (T, n)
        rho = np.empty((T, n, n), dtype=np.complex128) if want_rho else None
        E = np.empty(T)
        N = np.empty(T)
        self._check(self._lib.fedvr_kbe_propagate(
            self._h, float(dt), int(n_steps), 1 if second_born else 0, int(precision), _dptr(r0),
            _dptr(d),
            _dptr(rho.view(np.float64)) if want_rho else None, _dptr(E), _dptr(N)))
        return {"rho": rho, "E": E, "N": N}

    def kbe_block(self, which, i, j):
        """Block (i, j) of L = -i G^< (which 0 or "L") or Gt = -i G^> (1 or "G")
        of the last propagation, complex [n][n]."""
        w = {"L": 0, "G": 1}.get(which, which)
        out = np.empty((self.n_b, self.n_b), dtype=np.complex128)
        self._check(self._lib.fedvr_kbe_get_block(self._h, int(w), int(i), int(j),
                                                  _dptr(out.view(np.float64))))
        return out

    def kbe_stats(self):
        """Timing of the last propagation: total, collision and self-energy ms,
        their algorithmic flops, and the kernel launches."""
        out = np.zeros(8)
        self._check(self._lib.fedvr_kbe_stats(self._h, _dptr(out)))
        return {"ms": out[0], "collision_ms": out[1], "sigma_ms": out[2],
                "collision_flops": out[3], "sigma_flops": out[4], "launches": int(out[5]),
                "products_ms": out[6], "products_bytes": out[7]}


def solve_2b_batched(contexts, beta, u, p, mixing=0.5, tol=1e-8, max_iter=200,
                     precision=SPLIT_TF32, check=True):
    """Second-Born self-consistency of several prepared contexts (HF solved)
    advanced together: one tensor-core launch per kernel per iteration covers
    every system (``solve_2b_batched``). Returns per-system E0, N, iterations."""
    lib = _native.lib()
    k = len(contexts)
    handles = (C.c_void_p * k)(*[c.handle.value for c in contexts])
    beta = np.ascontiguousarray(np.broadcast_to(beta, (k,)), dtype=np.float64)
    u = np.ascontiguousarray(np.broadcast_to(u, (k,)), dtype=np.int32)
    p = np.ascontiguousarray(np.broadcast_to(p, (k,)), dtype=np.int32)
    E0, N, it = np.empty(k), np.empty(k), np.empty(k, dtype=np.int32)
    code = lib.solve_2b_batched(handles, k, _dptr(beta), _iptr(u), _iptr(p), mixing, tol, max_iter,
                                precision, _dptr(E0), _dptr(N), _iptr(it))
    if check and code != 0:
        raise FedvrError(code, contexts[0].last_error())
    return dict(E0=E0, N=N, iters=it, status=code)


class Batch:
    """A batch of prepared contexts stepped together (``fedvr_batch_*``)."""

    def __init__(self, contexts, beta, u, p, precision=SPLIT_TF32):
        self._lib = _native.lib()
        self.contexts = list(contexts)
        k = len(self.contexts)
        handles = (C.c_void_p * k)(*[c.handle.value for c in self.contexts])
        beta = np.ascontiguousarray(np.broadcast_to(beta, (k,)), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (k,)), dtype=np.int32)
        p = np.ascontiguousarray(np.broadcast_to(p, (k,)), dtype=np.int32)
        self._h = C.c_void_p()
        code = self._lib.fedvr_batch_create(C.byref(self._h), handles, k, _dptr(beta), _iptr(u),
                                            _iptr(p), precision)
        if code != 0:
            raise FedvrError(code, self.contexts[0].last_error())
        self.active = np.ones(k, dtype=np.int32)

    def step(self, mixing=0.5, tol=0.0):
        k = len(self.contexts)
        res, E0, N = np.empty(k), np.empty(k), np.empty(k)
        code = self._lib.fedvr_batch_step(self._h, mixing, tol, _iptr(self.active), _dptr(res),
                                          _dptr(E0), _dptr(N))
        if code != 0:
            raise FedvrError(code, self.contexts[0].last_error())
        return dict(res=res, E0=E0, N=N)

    def close(self):
        if self._h:
            self._lib.fedvr_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fptr(arr):
    if arr is None:
        return None
    assert arr.dtype == np.float32 and arr.flags["C_CONTIGUOUS"]
    return arr.ctypes.data_as(C.POINTER(C.c_float))


class WarmStartNet:
    """The per-pair warm-start network (``fedvr_mlp_*``)."""

    def __init__(self, M, hidden=512, seed=9114348, stream=None):
        self._lib = _native.lib()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._h = C.c_void_p()
        code = self._lib.fedvr_mlp_create(C.byref(self._h), M, hidden, seed, C.c_void_p(stream))
        if code != 0:
            raise FedvrError(code, "fedvr_mlp_create failed")
        self.M, self.hidden = M, hidden

    @property
    def handle(self):
        return self._h

    def last_error(self):
        return self._lib.fedvr_mlp_last_error(self._h).decode()

    def _check(self, code):
        if code != 0:
            raise FedvrError(code, self.last_error())

    def num_params(self):
        n = C.c_long()
        self._check(self._lib.fedvr_mlp_num_params(self._h, C.byref(n)))
        return n.value

    def get_params(self):
        out = np.empty(self.num_params(), dtype=np.float32)
        self._check(self._lib.fedvr_mlp_get_params(self._h, _fptr(out), out.size))
        return out

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._lib.fedvr_mlp_set_params(self._h, _fptr(params), params.size))

    def loss_grad(self, X, T):
        """X, T: float32 CUDA tensors [rows][2M+3], [rows][M]."""
        grad = np.empty(self.num_params(), dtype=np.float32)
        loss = C.c_double()
        self._check(self._lib.fedvr_mlp_loss_grad(self._h, C.c_void_p(X.data_ptr()),
                                                  C.c_void_p(T.data_ptr()), X.shape[0],
                                                  _fptr(grad), C.byref(loss)))
        return loss.value, grad

    def forward(self, X, Y, bf16=False):
        self._check(self._lib.fedvr_mlp_forward(self._h, C.c_void_p(X.data_ptr()), X.shape[0],
                                                C.c_void_p(Y.data_ptr()), 1 if bf16 else 0))

    def collect(self, ctx, beta, u, p, mixing=0.5, tol=1e-8, max_iter=200):
        it = C.c_int()
        self._check(self._lib.fedvr_mlp_collect(self._h, ctx.handle, beta, u, p, mixing, tol,
                                                max_iter, C.byref(it)))
        return it.value

    def rows(self):
        n = C.c_long()
        self._check(self._lib.fedvr_mlp_rows(self._h, C.byref(n)))
        return n.value

    def get_rows(self, start, count):
        X = np.empty((count, 2 * self.M + 3), dtype=np.float32)
        T = np.empty((count, self.M), dtype=np.float32)
        self._check(self._lib.fedvr_mlp_get_rows(self._h, start, count, _fptr(X), _fptr(T)))
        return X, T

    def train(self, epochs, batch=4096, lr=1e-3):
        loss = C.c_double()
        self._check(self._lib.fedvr_mlp_train(self._h, epochs, batch, lr, C.byref(loss)))
        return loss.value

    def close(self):
        if self._h:
            self._lib.fedvr_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sigma2_noalloc(V, G, Sigma, spin=2.0, stream=None):
    """Allocation-free FP64 Sigma^(2) build (``fedvr_sigma2_noalloc``) for callers
    that cannot let the library allocate device memory. Limit M*n*n <= 2^19;
    concurrent calls race on the library's one workspace array."""
    M, n = G.shape[0], G.shape[1]
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    code = _native.lib().fedvr_sigma2_noalloc(n, M, spin, _dev(V, (n, n)), _dev(G, (M, n, n)),
                                              _dev(Sigma, (M, n, n)), C.c_void_p(stream))
    if code != 0:
        raise FedvrError(code, "fedvr_sigma2_noalloc failed")


__all__ = ["WarmStartNet", "Batch", "solve_2b_batched", "sigma2_noalloc", "Context", "FedvrError", "FP64", "SPLIT_TF32", "SPLIT_BF16",
           "SPLIT_F16"]
