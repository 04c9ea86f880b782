#!/usr/bin/env python
"""Benchmark of the second-Born hot path: Sigma^(2) builds per second.

One step = one pass of the whole hot path over the workload: the Sigma^(2)
build for every mesh point (direct + exchange), the HF self-energy change and
the Galitskii-Migdal energy, the two Dyson convolutions and the mixed update
with its residual, i.e. one iteration of the self-consistency. Each step
contains exactly one Sigma^(2) build, so steps/s = builds/s.

Default workload (N=1): 1D He, Z=2, box [-50,50], 25 elements of order 8
(n_b = 199), beta = 100, 513-point power mesh (u=16, p=16), mixing 0.5.
Every rank runs its own replica of the workload (independent systems, weak
scaling); ranks only meet at the timing barrier.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|tf32|f16]
                    [--workload he_medium|he_small|h3p_large|he_paper|batch64|warmstart|h3p_curve|
                                combined|kbe] [--kbe-steps T]
                    [--no-time-to-e0] [--no-fp64-compare] [--no-cpu-baseline]
                    [--train-systems T] [--test-systems H] [--epochs E] [--hidden H]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_0911_4348_gb300 import workloads as W  # noqa: E402

METRIC = "Sigma^(2) builds/s (one build + its Dyson iteration per step)"
UNIT = "builds/s"
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16": 2, "f16": 3}
WORKLOADS = {"he_medium": W.he_medium, "he_small": W.he_small, "h3p_large": W.h3p_large,
             "he_paper": W.he_paper, "batch64": None, "warmstart": None, "h3p_curve": None,
             "combined": None, "kbe": None}
N_SM = 152
FP64_FLOP_PER_CLK_SM = 4  # 2 DFMA per clock per SM -> 1.26 TFLOP/s at 2070 MHz


def algorithmic(stage: str, n: int, M: int) -> float:
    """Algorithmic flops of one launch of a stage (one mesh, one system)."""
    if stage == "conv1":
        return 2.0 * M * M * n ** 3          # M^2 products of n x n matrices
    if stage == "sigma2":
        return M * (1.0 * n ** 4 + 4.0 * n ** 3)  # symmetric exchange half + direct term
    if stage == "conv2":
        return 2.0 * M * M * n * n + 4.0 * M * n ** 3  # left transform, eigen-kernel, back
    return 0.0


# Stored FP64 oracle solutions (written by tests/golden/make_*.py, which run
# only the oracle): workload name -> file of "key value" lines with E0.
GOLDEN = {"He n_b=199 M=513": "he_medium_2b.txt"}

PRECISION_BY_STAGE = {
    "f16": {
        "sigma2_exchange": "fp16 hi+lo split operands (22 significant bits, power-of-two scaled), "
                           "3 products (kind::f16), fp32 accumulation in TMEM, fp32 epilogue "
                           "k-sum, fp64 result",
        "sigma2_direct_VQV": "tf32 hi+lo split operands, 3 products (kind::tf32), fp32 accumulation",
        "conv1": "fp16 hi+lo split operands, 3 products (kind::f16), quadrature weights as "
                 "fp32 {c1, c2}, fp32 block sums of 512 MMA steps added in fp64",
        "conv2": "tf32 hi+lo split, 3 products (n_b >= 96; fp32 CUDA cores below), "
                 "fp32 eigen-kernel table",
        "update_residual_N_E0": "fp64",
        "basis_mesh_tables_hf": "fp64"},
    "tf32": {
        "sigma2_exchange": "tf32 hi+lo split operands, 3 products (kind::tf32), fp32 accumulation "
                           "in TMEM, fp32 epilogue k-sum, fp64 result",
        "sigma2_direct_VQV": "tf32 hi+lo split operands, 3 products (kind::tf32), fp32 accumulation",
        "conv1": "tf32 hi+lo split operands, 3 products, quadrature weights as fp32 {c1, c2}, "
                 "fp32 block sums of 512 MMA steps added in fp64",
        "conv2": "tf32 hi+lo split, 3 products (n_b >= 96; fp32 CUDA cores below), "
                 "fp32 eigen-kernel table",
        "update_residual_N_E0": "fp64",
        "basis_mesh_tables_hf": "fp64"},
    "fp64": {"all": "fp64"},
}


def golden_E_ref(workload: str):
    """E0 of the FP64 oracle's converged solution of this workload (tol 1e-8),
    read from its stored file, or None."""
    name = GOLDEN.get(workload)
    if not name:
        return None
    try:
        with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
            for line in fh:
                f = line.split()
                if len(f) >= 2 and f[0] == "E0":
                    return float(f[1])
    except OSError:
        return None
    return None


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or None
    if there is none for this workload or the kernel source changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            entry = json.load(fh).get(kernel)
        if not entry or entry.get("workload") != workload:
            return None
        with open(os.path.join(ROOT, entry["source"]), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != entry["source_sha256_16"]:
                return None
        return int(entry["dram_read_bytes"]) + int(entry["dram_write_bytes"])
    except (OSError, ValueError, KeyError):
        return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.dev = device_id
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.dev:
            cmd += ["-i", self.dev]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist(backend: str = "nccl"):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def max_over_ranks(dist, x: float, device: str = "cuda") -> float:
    """The largest of the ranks' values of x (the whole job ends with its
    slowest rank); x itself when running alone."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def split_precision(args) -> int:
    """The library code of a split precision (the batched and warm-start paths run
    only on the tensor-core kernels)."""
    if args.precision not in ("tf32", "f16"):
        raise SystemExit(f"--precision {args.precision}: this workload runs split tf32 or f16")
    return PRECISIONS[args.precision]


def rank_config(config_id: int, rank: int) -> int:
    """Seed stream of a rank's share of a family of independent systems: every
    rank draws its own systems (weak scaling, no data exchanged)."""
    return config_id + 100 * rank


def _cpu_cores() -> int:
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(sys_: W.System, n_sigma: int, n_rows: int, prepared=None):
    """Time the CPU oracle on a bounded sample of one iteration of the
    workload and scale it to builds/s: n_sigma mesh points of the Sigma^(2)
    build and n_rows output rows of each convolution, extrapolated to all M."""
    from oracle import fedvr_oracle as O
    if prepared is None:
        b = O.fedvr_basis(sys_.n_elem, sys_.order, sys_.xmin, sys_.xmax, sys_.grid_kind)
        T, v = O.kinetic(b), O.potential(b["nodes"], sys_.Z, sys_.R, sys_.soft_en)
        V = O.interaction(b["nodes"], sys_.soft_ee)
        h = T + np.diag(v)
        hf = O.hf_scf(h, V, 2.0, sys_.n_elec // 2, sys_.beta, tol=1e-12)
        mesh = O.power_mesh(sys_.beta, sys_.u, sys_.p)
        G0 = O.g0_mesh(hf["eps"], hf["C"], hf["mu"], mesh["tau"], sys_.beta)
        prepared = (V, hf, mesh, G0)
    V, hf, mesh, G0 = prepared
    M = G0.shape[0]
    rng = np.random.default_rng(0)
    js = rng.choice(M, size=min(n_sigma, M), replace=False)
    rows = rng.choice(M, size=min(n_rows, M), replace=False)
    t0 = time.perf_counter()
    A = np.empty_like(G0)
    for j in js:
        A[j] = O.sigma2_tau(G0[j], G0[M - 1 - j], V, 2.0)
    t1 = time.perf_counter()
    A[:] = A[js[0]]  # stand-in values elsewhere: only the timing of the sample matters
    lag = {"k": np.zeros((M, M), np.int32), "t": np.zeros((M, M)), "s": np.zeros((M, M))}
    for i in rows:
        for j in range(M):
            if i != j:
                y, sg = O.lag_point(mesh["tau"], sys_.beta, i, j)
                k, t = O.bracket(mesh["tau"], y)
                lag["k"][i, j], lag["t"][i, j], lag["s"][i, j] = k, t, sg
    t2 = time.perf_counter()
    I1 = np.zeros_like(G0)
    I1[rows] = O.conv1(np.zeros_like(G0[0]), A, G0, mesh, sys_.beta, lag, rows=list(rows))
    t3 = time.perf_counter()
    O.conv2(I1, hf["eps"], hf["C"], hf["mu"], mesh, sys_.beta, rows=list(rows))
    t4 = time.perf_counter()
    per_iter = (t1 - t0) / len(js) * M + ((t3 - t2) + (t4 - t3)) / len(rows) * M
    sample = (f"oracle Sigma^(2) at {len(js)} of {M} mesh points and both convolutions for "
              f"{len(rows)} of {M} output rows, extrapolated to one full iteration")
    return 1.0 / per_iter, sample, t4 - t0, prepared


def run_reference(args, rank: int):
    """The reference arm: the CPU oracle as it stands, on this host's cores."""
    if rank != 0:
        return
    make = WORKLOADS[args.workload]
    if make is None:  # families: time the oracle on their first system
        make = {"warmstart": lambda: W.warmstart_system(0),
                "combined": lambda: W.warmstart_system(0),
                "h3p_curve": lambda: W.h3p_curve()[0]}.get(args.workload,
                                                           lambda: W.batch_systems(64)[0])
    sys_ = make()
    vals, prepared, spent = [], None, 0.0
    sample = ""
    for k in range(args.warmup + args.steps):
        v, sample, dt, prepared = oracle_sample(sys_, 2, 1, prepared)
        spent += dt
        if k >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sys_.name, "n_b": sys_.n_b, "n_tau": sys_.n_tau,
                       "beta": sys_.beta, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _parabola_min(x, y):
    """Abscissa of the vertex of the parabola through the lowest sample and its
    two neighbours (None at the ends of the sampled range)."""
    k = int(np.argmin(y))
    if k == 0 or k == len(y) - 1:
        return None
    h = x[k + 1] - x[k]
    return float(x[k] + h * (y[k - 1] - y[k + 1]) / (2 * (y[k - 1] - 2 * y[k] + y[k + 1])))


def run_batch(args, dist, rank, world, local):
    """Systems advanced together, a step being one batched iteration of every
    system. batch64: 64 uneven systems (32 He, 32 H3+; n_b 59-239, 257-513
    mesh points). h3p_curve: the paper's H3+ binding curve (Sec. 3.2), 11
    bond lengths on its n_b = 142 grid with 1025 mesh points."""
    import torch
    from paper_0911_4348_gb300 import Batch, Context, solve_2b_batched
    curve = args.workload == "h3p_curve"
    systems = W.h3p_curve() if curve else W.batch_systems(64, config_id=rank_config(4, rank))
    stream = torch.cuda.current_stream()
    e_hf, e_nn = [], []

    def make():
        ctxs = []
        e_hf.clear()
        e_nn.clear()
        for s_ in systems:
            c = Context(stream.cuda_stream)
            c.build_fedvr(s_.n_elem, s_.pts_per_elem, s_.xmin, s_.xmax, s_.grid_kind)
            e_nn.append(c.set_potential(s_.Z, s_.R, s_.soft_en, s_.soft_ee, s_.n_elec))
            e_hf.append(c.solve_hf(s_.beta, tol=1e-12)[0])
            ctxs.append(c)
        return ctxs

    ctxs = make()
    betas = [s_.beta for s_ in systems]
    us, ps = [s_.u for s_ in systems], [s_.p for s_ in systems]
    prec = split_precision(args)
    batch = Batch(ctxs, betas, us, ps, prec)
    for _ in range(args.warmup):
        batch.step(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        batch.step(0.5)
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1)
    elapsed = max_over_ranks(dist, elapsed)
    batch.close()
    n_sys = len(systems)
    value = world * n_sys * args.steps / (elapsed / 1000.0)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": elapsed / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
           "config": {"workload": ("H3+ binding curve: R = 1.6..3.6 step 0.2, 13 x 11 graded "
                                   "(n_b=142), M=1025") if curve else
                                  "batch of 64: 32 He (Z~U[1.5,2.5]) + 32 H3+ (R~U[1.2,3.0])",
                      "n_b": [s_.n_b for s_ in systems], "n_tau": [s_.n_tau for s_ in systems],
                      "precision": args.precision, "parallelism": f"replicas x{world}"}}
    if not args.no_time_to_e0:
        ctxs2 = make()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = solve_2b_batched(ctxs2, betas, us, ps, 0.5, 1e-8, 200, prec, check=False)
        torch.cuda.synchronize()
        out["time_to_converge_all"] = {"seconds": time.perf_counter() - t0,
                                       "max_iterations": int(np.max(r["iters"])),
                                       "status": r["status"]}
        if curve:
            d = np.array([2.0 * s_.R[2] for s_ in systems])
            tot_hf = np.array(e_hf) + np.array(e_nn)
            tot_2b = np.asarray(r["E0"]) + np.array(e_nn)
            out["h3p_curve"] = {"d": d.tolist(), "E_hf_total": tot_hf.tolist(),
                                "E_2b_total": tot_2b.tolist(), "N": np.asarray(r["N"]).tolist(),
                                "d_b_hf": _parabola_min(d, tot_hf),
                                "d_b_2b": _parabola_min(d, tot_2b)}
        for c in ctxs2:
            c.close()
    for c in ctxs:
        c.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _context(stream, s_):
    from paper_0911_4348_gb300 import Context
    c = Context(stream.cuda_stream)
    c.build_fedvr(s_.n_elem, s_.pts_per_elem, s_.xmin, s_.xmax, s_.grid_kind)
    c.set_potential(s_.Z, s_.R, s_.soft_en, s_.soft_ee, s_.n_elec)
    c.solve_hf(s_.beta, tol=1e-12)
    return c


def _first_within(E, E_ref, tol=1e-6):
    """First index k from which every E[k:] lies within tol of E_ref (or None)."""
    E = np.asarray(E)
    return next((k for k in range(len(E)) if np.all(np.abs(E[k:] - E_ref) <= tol)), None)


def _timed_solve(c, s_, prec, tol, max_iter, stop_near=None):
    """prepare + steps through the public split API with host wall times; stops
    at res < tol, or (stop_near) two steps after E0 first comes within 1e-6 Ha
    of stop_near."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c.prepare_2b(s_.beta, s_.u, s_.p, prec)
    prep = time.perf_counter() - t0
    E, res, N, step_s = [], [], [], []
    hit = None
    converged = False
    for k in range(max_iter):
        t1 = time.perf_counter()
        r = c.step_2b(s_.mixing)
        step_s.append(time.perf_counter() - t1)
        E.append(r["E0"])
        res.append(r["res"])
        N.append(r["N"])
        if stop_near is not None:
            if hit is None and abs(r["E0"] - stop_near) <= 1e-6:
                hit = k
            if hit is not None and k >= hit + 2:
                break
        elif r["res"] < tol:
            converged = True
            break
    return dict(prepare_s=prep, E=E, res=res, N=N, step_s=np.array(step_s), converged=converged)


def _errors_vs_fp64(c, s_, prec, run, E_ref):
    """Errors of a split-precision solve (left in context c) against FP64:
    Sigma^(2) of its final g built by the split path and by the library's FP64
    path on the same g (max-norm relative over all mesh points), |E0 - E_ref|
    (the FP64 oracle's converged E0), |N - 2| and the jump invariant
    max|g(0^-) + g(-beta) - 1|."""
    import torch
    n, M = s_.n_b, s_.n_tau
    G = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    c.read_2b(G_out=G)
    V = torch.from_numpy(c.get_operators()["V"]).cuda()
    S_split = torch.empty_like(G)
    S_64 = torch.empty_like(G)
    c.sigma2(V, G, S_split, precision=prec)
    c.sigma2(V, G, S_64, precision=0)
    torch.cuda.synchronize()
    sig = float((S_split - S_64).abs().max() / S_64.abs().max())
    jump = float((G[M - 1] + G[0] - torch.eye(n, dtype=torch.float64, device="cuda")).abs().max())
    return {"sigma2_maxrel_vs_fp64_path_same_g": sig,
            "E0_abs_vs_fp64_oracle": None if E_ref is None else abs(run["E"][-1] - E_ref),
            "N_minus_2": abs(run["N"][-1] - 2.0), "jump_invariant": jump,
            "bounds": {"sigma2": 1e-5, "E0_Ha": 1e-6}}


def _to_e0(hist, E_ref, tol=1e-6):
    """Iterations and summed step wall time until E0 stays within tol of E_ref."""
    k = next((i for i in range(len(hist)) if np.all(np.abs(hist[i:, 2] - E_ref) <= tol)), None)
    if k is None:
        return None, None
    return int(k + 1), float(np.sum(hist[: k + 1, 4]) / 1000.0)


def run_warmstart(args, dist, rank, world, local):
    """Learned warm start on the family of 20 x 7-point systems (n_b = 119,
    257-point mesh): collect converged self-energies of T training systems,
    train the per-pair network (FP32 master weights), then time H held-out
    systems to a converged E0 (within 1e-6 Ha of their own converged E0) from
    (a) the plain start g = g^0, (b) Sigma^(2)[g^0] with the same fixed-Sigma
    inner steps (network output forced to zero) and (c) the network's
    prediction (BF16 inference). A step is one iteration of one system."""
    import torch
    from paper_0911_4348_gb300 import WarmStartNet
    stream = torch.cuda.current_stream()
    cid = rank_config(5, rank)
    train = [W.warmstart_system(k, cid) for k in range(args.train_systems)]
    test = [W.warmstart_system(50000 + k, cid) for k in range(args.test_systems)]
    M = train[0].n_tau
    net = WarmStartNet(M, args.hidden, seed=W.MASTER_SEED, stream=stream.cuda_stream)
    zero = WarmStartNet(M, args.hidden, seed=1, stream=stream.cuda_stream)
    zero.set_params(np.zeros(zero.num_params(), dtype=np.float32))
    t0 = time.perf_counter()
    collect_iters = []
    for s_ in train:
        c = _context(stream, s_)
        collect_iters.append(net.collect(c, s_.beta, s_.u, s_.p))
        c.close()
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = net.train(args.epochs, batch=4096, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    per = []
    steps_total, step_ms = 0, 0.0
    for s_ in test:
        row = {"system": s_.name}
        for mode, model in (("plain", None), ("sigma1", zero), ("network", net)):
            c = _context(stream, s_)
            torch.cuda.synchronize()
            t_ws = 0.0
            if model is not None:
                t1 = time.perf_counter()
                c.warm_start(model, s_.beta, s_.u, s_.p, inner_steps=4)
                torch.cuda.synchronize()
                t_ws = time.perf_counter() - t1
            r = c.solve_2b(s_.beta, s_.u, s_.p, s_.mixing, s_.tol, 200, split_precision(args),
                           check=False)
            hist = c.get_history()
            if mode == "plain":
                E_ref = r["E0"]
                steps_total += len(hist)
                step_ms += float(np.sum(hist[:, 4]))
            it, sec = _to_e0(hist, E_ref)
            row[mode] = {"iterations": it, "seconds": None if sec is None else sec + t_ws,
                         "predict_seconds": t_ws, "E0": r["E0"], "status": r["status"],
                         "dE0_vs_plain": abs(r["E0"] - E_ref)}
            c.close()
        per.append(row)
    net.close()
    zero.close()

    def total(mode, key):
        v = [r[mode][key] for r in per]
        return None if any(x is None for x in v) else float(np.sum(v))

    value = world * steps_total / (step_ms / 1000.0)
    s0 = train[0]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": steps_total, "warmup": 0, "ms_per_step": step_ms / steps_total,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
           "data": "synthetic",
           "config": {"workload": "warm-start family: He (Z~U[1.5,2.5]) / H3+ (R~U[1.2,3.0]), "
                                  f"20 x 7 points (n_b={s0.n_b}), M={M}",
                      "train_systems": len(train), "test_systems": len(test),
                      "hidden": args.hidden, "epochs": args.epochs, "precision": args.precision,
                      "parallelism": f"replicas x{world}"},
           "warm_start": {"collect_seconds": t_collect,
                          "collect_iterations_mean": float(np.mean(collect_iters)),
                          "train_seconds": t_train, "final_train_loss": loss,
                          "rows": len(train) * s0.n_b * (s0.n_b + 1) // 2,
                          "time_to_E0_seconds": {m: total(m, "seconds")
                                                 for m in ("plain", "sigma1", "network")},
                          "iterations_to_E0": {m: total(m, "iterations")
                                               for m in ("plain", "sigma1", "network")},
                          "max_dE0_network": max(r["network"]["dE0_vs_plain"] for r in per),
                          "per_system": per}}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_combined(args, dist, rank, world, local):
    """Time to a converged E0 (within 1e-6 Ha of each system's FP64 answer) on
    held-out systems of the warm-start family (20 x 7 points, n_b = 119, 257
    mesh points): (a) the plain FP64 GPU path, one system after another, run to
    tol 1e-8 (its converged E0 is the system's E_ref; its own time to E0 is read
    from its history); (b) the batched, warm-started (network trained on the
    largest training set), split-precision solver on all held-out systems at
    once. Also a learning curve: total iterations to E0 of the held-out systems
    solved one at a time from the network's warm start, for each training-set
    size. A step is one iteration of one system."""
    import torch
    from paper_0911_4348_gb300 import WarmStartNet, solve_2b_batched
    stream = torch.cuda.current_stream()
    cid = rank_config(5, rank)
    sizes = sorted({int(x) for x in args.curve.split(",") if x.strip()})
    test = [W.warmstart_system(50000 + k, cid) for k in range(args.test_systems)]
    M = test[0].n_tau
    prec = split_precision(args)
    # (a) FP64 reference solves
    e_ref, fp64 = [], []
    for s_ in test:
        c = _context(stream, s_)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = c.solve_2b(s_.beta, s_.u, s_.p, s_.mixing, s_.tol, 200, 0, check=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        hist = c.get_history()
        e_ref.append(r["E0"])
        it, sec = _to_e0(hist, r["E0"])
        fp64.append({"system": s_.name, "E0": r["E0"], "iterations": r["iters"],
                     "status": r["status"], "solve_seconds": wall,
                     "iterations_to_E0": it,
                     "seconds_to_E0": None if sec is None else sec + (wall - float(np.sum(hist[:, 4])) / 1000.0)})
        c.close()
    # learning curve: one network per training-set size (same seed, same epochs)
    curve, net = [], None
    for T in sizes:
        if net is not None:
            net.close()
        net = WarmStartNet(M, args.hidden, seed=W.MASTER_SEED, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        for k in range(T):
            s_ = W.warmstart_system(k, cid)
            c = _context(stream, s_)
            net.collect(c, s_.beta, s_.u, s_.p)
            c.close()
        t_collect = time.perf_counter() - t0
        t0 = time.perf_counter()
        loss = net.train(args.epochs, batch=4096, lr=1e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        iters, worst = 0, 0.0
        for s_, E in zip(test, e_ref):
            c = _context(stream, s_)
            c.warm_start(net, s_.beta, s_.u, s_.p, inner_steps=4)
            r = c.solve_2b(s_.beta, s_.u, s_.p, s_.mixing, s_.tol, 200, prec, check=False)
            it, _ = _to_e0(c.get_history(), E)
            iters += it if it is not None else 10 ** 6
            worst = max(worst, abs(r["E0"] - E))
            c.close()
        curve.append({"train_systems": T, "iterations_to_E0": iters, "max_dE0_vs_fp64": worst,
                      "collect_seconds": t_collect, "train_seconds": t_train,
                      "final_train_loss": loss})
    # (b) the combined solver: warm starts from the last network, one batched solve
    ctxs = [_context(stream, s_) for s_ in test]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, s_ in zip(ctxs, test):
        c.warm_start(net, s_.beta, s_.u, s_.p, inner_steps=4)
    torch.cuda.synchronize()
    t_ws = time.perf_counter() - t0
    r = solve_2b_batched(ctxs, [s_.beta for s_ in test], [s_.u for s_ in test],
                         [s_.p for s_ in test], 0.5, 1e-8, 200, prec, check=False)
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    hists = [c.get_history() for c in ctxs]
    n_it = max(h.shape[0] for h in hists)
    step_s = np.zeros(n_it)  # wall time of each batched iteration (the same for every system)
    for h in hists:
        step_s[: h.shape[0]] = np.maximum(step_s[: h.shape[0]], h[:, 4] / 1000.0)
    k_all = 0
    for h, E in zip(hists, e_ref):
        k, _ = _to_e0(h, E)
        k_all = max(k_all, k if k is not None else 10 ** 6)
    t_batch_e0 = t_ws + (t_all - t_ws - float(np.sum(step_s))) + float(np.sum(step_s[:k_all]))
    net.close()
    for c in ctxs:
        c.close()
    fp64_total = sum(x["seconds_to_E0"] or 0.0 for x in fp64)
    steps = int(sum(h.shape[0] for h in hists))
    value = world * steps / max(float(np.sum(step_s)), 1e-9)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
           "warmup": 0, "ms_per_step": 1000.0 * float(np.sum(step_s)) / max(steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.precision, "data": "synthetic",
           "config": {"workload": "combined solver on held-out warm-start systems: He "
                                  "(Z~U[1.5,2.5]) / H3+ (R~U[1.2,3.0]), 20 x 7 points "
                                  f"(n_b={test[0].n_b}), M={M}",
                      "test_systems": len(test), "train_sizes": sizes, "hidden": args.hidden,
                      "epochs": args.epochs, "precision": args.precision,
                      "parallelism": f"replicas x{world}"},
           "time_to_E0": {"E_ref": "each system's FP64 GPU solve at tol 1e-8",
                          "fp64_sequential_seconds": fp64_total,
                          "combined_seconds": t_batch_e0,
                          "combined_warm_start_seconds": t_ws,
                          "combined_iterations_to_E0": k_all,
                          "combined_solve_status": r["status"],
                          "max_dE0_vs_fp64": float(max(abs(a - b) for a, b in zip(r["E0"], e_ref))),
                          "speedup": fp64_total / t_batch_e0 if t_batch_e0 > 0 else None},
           "fp64_per_system": fp64, "learning_curve": curve}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_kbe(args, dist, rank, world, local):
    """Real-time two-time Kadanoff-Baym propagation (second Born, complex FP64):
    one step of this workload is one whole propagation of T time steps from
    the HF ground state under a dipole field; the metric is time steps per
    second. Each rank propagates its own replica (no exchange)."""
    import torch
    run = W.kbe_he(args.kbe_steps)
    s_ = run.system
    stream = torch.cuda.current_stream()
    ctx = _context(stream, s_)
    x = ctx.get_basis()["nodes"]
    dv = np.ascontiguousarray(np.outer(run.field(), x))
    T = run.n_steps + 1
    prec = PRECISIONS[args.kbe_precision]
    for _ in range(args.warmup):
        ctx.kbe_propagate(run.dt, run.n_steps, True, dv=dv, want_rho=False, precision=prec)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0] or None)
    clocks.start()
    dev_ms, coll_ms, sig_ms, prod_ms, launches, walls = 0.0, 0.0, 0.0, 0.0, 0, []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ctx.kbe_propagate(run.dt, run.n_steps, True, dv=dv, precision=prec)
        walls.append(time.perf_counter() - t0)
        st = ctx.kbe_stats()
        dev_ms += st["ms"]
        coll_ms += st["collision_ms"]
        sig_ms += st["sigma_ms"]
        prod_ms += st["products_ms"]
        launches += st["launches"]
    torch.cuda.nvtx.range_pop()
    ck = clocks.stop()
    dev_s = max_over_ranks(dist, dev_ms / 1000.0)
    wall_s = max_over_ranks(dist, float(sum(walls)))
    steps_total = world * args.steps * run.n_steps
    achieved = st["collision_flops"] / (coll_ms / args.steps / 1000.0)
    n = ctx.n_b
    if prec == 0:
        roof = {"bound": "alu", "kernel": "collision_kernel (FP64 pipe)",
                "peak": N_SM * FP64_FLOP_PER_CLK_SM * 2070e6 / 1e12,
                "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz"}
    else:
        # the split products stream the FP32 shadows of the two-time matrices: HBM roofline
        # on the bytes they read once, over the products' own CUDA-event time
        hbm = load_peaks().get("hbm_gbs")
        roof = {"bound": "hbm", "kernel": "collision products (gemm_tf32x3_kernel, split TF32)",
                "achieved": st["products_bytes"] / (prod_ms / args.steps / 1000.0) / 1e9,
                "peak": hbm, "unit": "GB/s", "peak_source": "measured copy bandwidth, of measured",
                "products_ms_per_step": prod_ms / args.steps,
                "collision_tflops_algorithmic": achieved / 1e12}
    if prec == 0:
        roof.update({"achieved": achieved / 1e12, "unit": "TFLOP/s"})
    roof["traffic"] = None
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["peak"] else None
    line = {"metric": "real-time KBE time steps/s (second Born, two-time)",
            "value": steps_total / dev_s, "unit": "time steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dev_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if prec == 0 else "c128 (collision integrals split tf32)",
            "data": "synthetic",
            "config": {"workload": f"{s_.name}: T={T} time points, dt={run.dt}, dipole field "
                                   f"{run.amp} a.u. at omega={run.omega}, HF initial state",
                       "two_time_bytes": 2 * (T * n) ** 2 * 16,
                       "parallelism": f"replicas x{world}",
                       "l2": "two-time matrices larger than L2 beyond T = 145 at n_b = 39"},
            "roofline": roof,
            "stage_ms_per_step": {"collision": coll_ms / args.steps,
                                  "self_energy": sig_ms / args.steps,
                                  "other": (dev_ms - coll_ms - sig_ms) / args.steps},
            "e2e": {"value": steps_total / wall_s, "unit": "time steps/s",
                    "h2d_bytes_per_step": int(dv.nbytes),
                    "d2h_bytes_per_step": int(T * n * n * 16 + 2 * T * 8)},
            "gpu_launches": launches,
            "observables": {"E_first": float(out["E"][0]), "E_last": float(out["E"][-1]),
                            "N_last": float(out["N"][-1])},
            "clocks": ck}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = kbe_cpu_baseline(ctx, run, dv)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def kbe_cpu_baseline(ctx, run, dv):
    """The oracle's propagation of the first steps of the same run (its cost
    per step grows as the square of the step index, like the GPU's), timed on
    the host cores."""
    from oracle import fedvr_oracle as O
    s_ = run.system
    b = O.fedvr_basis(s_.n_elem, s_.order, s_.xmin, s_.xmax, s_.grid_kind)
    h = O.kinetic(b) + np.diag(O.potential(b["nodes"], s_.Z, s_.R, s_.soft_en))
    V = O.interaction(b["nodes"], s_.soft_ee)
    rho0 = ctx.get_hf()["rho0"].astype(np.complex128)
    ns = min(run.n_steps, 24)
    t0 = time.perf_counter()
    O.kbe_propagate(h, V, 2.0, rho0, run.dt, ns, dv=dv[: ns + 1])
    sec = time.perf_counter() - t0
    return {"value": ns / sec, "unit": "time steps/s", "cores": _cpu_cores(), "kind": "oracle",
            "sample": f"first {ns} of {run.n_steps} time steps of the same run"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=tuple(PRECISIONS), default="f16")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="he_medium")
    ap.add_argument("--no-time-to-e0", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch each iteration's kernels eagerly instead of replaying a CUDA graph")
    ap.add_argument("--train-systems", type=int, default=48)
    ap.add_argument("--test-systems", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--curve", default="12,48,192",
                    help="training-set sizes of the combined workload's learning curve")
    ap.add_argument("--kbe-steps", type=int, default=100,
                    help="time steps of one propagation of the kbe workload")
    ap.add_argument("--kbe-precision", choices=("fp64", "tf32"), default="fp64",
                    help="kbe workload: collision integrals in FP64 or as split-TF32 products")
    ap.add_argument("--self-energy", choices=("2b", "gw", "tmatrix"), default="2b",
                    help="correlation self-energy of the Matsubara iteration (gw, tmatrix: "
                         "FP64 path; tmatrix: n_b <= 32, e.g. --workload he_small)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    # the reference arm is the CPU oracle: its ranks meet (if at all) over gloo
    dist, rank, world, local = _dist("gloo" if args.impl == "reference" else "nccl")
    if args.impl == "reference":
        run_reference(args, rank)
        if dist:
            dist.destroy_process_group()
        return

    import torch
    from paper_0911_4348_gb300 import Context

    torch.cuda.set_device(local)
    if args.workload in ("batch64", "warmstart", "h3p_curve", "combined", "kbe"):
        {"warmstart": run_warmstart, "combined": run_combined,
         "kbe": run_kbe}.get(args.workload, run_batch)(
            args, dist, rank, world, local)
        if dist:
            dist.destroy_process_group()
        return
    sys_ = WORKLOADS[args.workload]()
    prec = PRECISIONS[args.precision]
    stream = torch.cuda.current_stream()
    ctx = Context(stream.cuda_stream)
    ctx.build_fedvr(sys_.n_elem, sys_.pts_per_elem, sys_.xmin, sys_.xmax, sys_.grid_kind)
    ctx.set_potential(sys_.Z, sys_.R, sys_.soft_en, sys_.soft_ee, sys_.n_elec)
    E_hf, _ = ctx.solve_hf(sys_.beta, tol=1e-12)
    ctx.use_graphs(not args.no_graphs)
    gw = args.self_energy in ("gw", "tmatrix")  # an inner iteration per outer step
    if gw:
        if prec != 0:
            raise SystemExit(f"--self-energy {args.self_energy} runs on the FP64 path: "
                             "add --precision fp64")
        if args.self_energy == "tmatrix" and sys_.n_b > 32:
            raise SystemExit("--self-energy tmatrix needs n_b <= 32 (e.g. --workload he_small)")
        ctx.set_self_energy(args.self_energy)
        args.no_fp64_compare = True   # the FP64 path is the one timed
        args.no_cpu_baseline = True   # the oracle sample below is second Born's
    ctx.prepare_2b(sys_.beta, sys_.u, sys_.p, prec)
    n, M = sys_.n_b, sys_.n_tau
    inner = []

    for _ in range(args.warmup):
        ctx.step_2b(sys_.mixing)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    dev_id = None
    try:
        dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        dev_id = None
    clocks = ClockSampler(dev_id)
    stage_ms = {}
    launches = 0
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.step_2b(sys_.mixing)
        st, nl = ctx.stage_times()
        launches += nl
        if gw:
            inner.append(ctx.gw_last_inner())
        for k, v in st.items():
            stage_ms.setdefault(k, []).append(v)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1)
    elapsed = max_over_ranks(dist, elapsed)
    value = world * args.steps / (elapsed / 1000.0)

    # end to end through the public API: each step takes its input g from
    # pinned host memory and returns its scalars to the host
    G_host = torch.empty((M, n, n), dtype=torch.float64, pin_memory=True)
    ctx.read_2b(G_out=G_host.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.step_2b(sys_.mixing, G_in=G_host.numpy())
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s)
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": M * n * n * 8, "d2h_bytes_per_step": 3 * 8}

    avg = {k: float(np.mean(v)) for k, v in stage_ms.items()}
    dom = max(("sigma2", "conv1", "conv2"), key=lambda k: avg.get(k, 0.0))
    if gw:
        dom = "sigma2"  # the inner iteration's periodic convolutions
    peaks = load_peaks()
    if prec == 0:
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = N_SM * FP64_FLOP_PER_CLK_SM * sm_max * 1e6 / 1e12
        bound, punit, psrc = "alu", "TFLOP/s", ("FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x "
                                               f"{sm_max:.0f} MHz (unit counts and clocks)")
    elif dom == "conv2":  # the second convolution's GEMMs run on the FP32 pipe
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = N_SM * 128 * 2 * sm_max * 1e6 / 1e12
        bound, punit, psrc = "alu", "TFLOP/s", ("FP32 pipe: 152 SMs x 128 FMA/clk x 2 flop x "
                                               f"{sm_max:.0f} MHz (unit counts and clocks)")
    else:
        # burst peak for a timed region under a few seconds with no power cap
        # seen; the sustained (power-capped) figure otherwise
        burst = elapsed < 3000.0 and not (clk and "sw_power_cap" in clk.get("reasons", []))
        key = "bf16_tflops" if burst else "bf16_tflops_sustained"
        base = float(peaks.get(key, 1946.4 if burst else 1721.8))
        kind = "burst" if burst else "sustained"
        if args.precision == "f16" and dom in ("conv1", "sigma2"):  # both run kind::f16
            peak = base
            bound, punit, psrc = "tensor", "TFLOP/s", f"measured bf16 {kind} (fp16 dense rate = bf16)"
        else:
            peak = base / 2.0
            bound, punit, psrc = "tensor", "TFLOP/s", f"measured bf16 {kind} x 1/2 (tf32 ratio)"
    dom_flops = algorithmic(dom, n, M)
    if args.self_energy == "gw":  # one periodic convolution (2 M^2 n^3) per inner iteration
        dom_flops = float(np.mean(inner)) * algorithmic("conv1", n, M)
    elif args.self_energy == "tmatrix":
        # per inner iteration the ladder's convolution applies, for every (i, j)
        # and column pair, the two interpolation points' g_r X g_r^T: 8 M^2 n^5
        dom_flops = float(np.mean(inner)) * 8.0 * M * M * float(n) ** 5
    achieved = dom_flops / (avg[dom] / 1000.0) / 1e12
    # keys of profiles/ncu_traffic.json: the kernel of the stage in this precision
    kernel_name = {("conv1", "f16"): "conv1_f16_kernel", ("conv1", "tf32"): "conv1_tc_kernel",
                   ("sigma2", "f16"): "exchange_tc_kernel<f16>",
                   ("sigma2", "tf32"): "exchange_tc_kernel<tf32>"}.get((dom, args.precision))
    traffic = measured_traffic(kernel_name, sys_.name) if (prec != 0 and kernel_name) else None
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": punit,
            "frac": achieved / peak, "traffic": traffic, "kernel": dom,
            "algorithmic_flops_per_launch": dom_flops, "peak_source": psrc,
            "stage_ms": avg}
    if gw:
        roof["kernel"] = ("GW screened interaction (conv1_fp64_kernel, periodic table)"
                          if args.self_energy == "gw" else
                          "T-matrix ladder (tm_ladder_kernel, periodic table)")
        roof["inner_iterations_mean"] = float(np.mean(inner))

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == 0 else args.precision,
           "data": "synthetic",
           "config": {"workload": sys_.name, "n_b": n, "n_tau": M, "beta": sys_.beta,
                      "precision": args.precision, "parallelism": f"replicas x{world}",
                      "self_energy": args.self_energy,
                      "graphs": ctx.use_graphs(), "conv1_splits": ctx.conv1_splits(),
                      "l2": "inputs larger than L2 (g stack %.0f MB)" % (M * n * n * 8 / 1e6)},
           "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clk,
           "E_hf": E_hf, "precision_by_stage": PRECISION_BY_STAGE[args.precision if prec else "fp64"]}

    E_ref = None if gw else golden_E_ref(sys_.name)
    if not args.no_time_to_e0:
        # time to a converged E0 through the public API (prepare included):
        # E_ref is the FP64 oracle's converged E0 where it is stored, else this
        # run's own converged value
        ctx2 = _context(stream, sys_)
        if gw:
            ctx2.set_self_energy(args.self_energy)
        run = _timed_solve(ctx2, sys_, prec, sys_.tol, 200)
        ref = E_ref if E_ref is not None else run["E"][-1]
        k = _first_within(run["E"], ref)
        out["time_to_E0"] = {
            "seconds": None if k is None else run["prepare_s"] + float(np.sum(run["step_s"][:k + 1])),
            "iterations": None if k is None else k + 1, "prepare_seconds": run["prepare_s"],
            "E_ref": ref, "E_ref_source": ("FP64 oracle, converged at tol 1e-8 (stored)"
                                           if E_ref is not None else "this run's final E0"),
            "solve_seconds": run["prepare_s"] + float(np.sum(run["step_s"])),
            "solve_iterations": len(run["E"]), "E0": run["E"][-1], "converged": run["converged"]}
        if prec != 0:
            out["error_vs_fp64"] = _errors_vs_fp64(ctx2, sys_, prec, run, E_ref)
        ctx2.close()

    if prec != 0 and not args.no_fp64_compare:
        # the plain FP64 GPU path on the same system: its per-step time, and its
        # measured time to E0 within 1e-6 Ha of E_ref (run until there and two
        # steps beyond, to see that it stays)
        ctx3 = _context(stream, sys_)
        if E_ref is not None and not args.no_time_to_e0:
            run3 = _timed_solve(ctx3, sys_, 0, 0.0, 60, stop_near=E_ref)
            k3 = _first_within(run3["E"], E_ref)
            st3, _ = ctx3.stage_times()
            fp64_ms = 1000.0 * float(np.median(run3["step_s"]))
            out["fp64_path"] = {
                "ms_per_step": fp64_ms, "builds_per_s": 1000.0 / fp64_ms, "stage_ms": st3,
                "speedup_per_step": fp64_ms / (elapsed / args.steps),
                "time_to_E0": {
                    "seconds": None if k3 is None else
                    run3["prepare_s"] + float(np.sum(run3["step_s"][:k3 + 1])),
                    "iterations": None if k3 is None else k3 + 1,
                    "E0_at_stop": run3["E"][-1], "E_ref": E_ref,
                    "stays_within_2_more_steps": k3 is not None and k3 + 3 <= len(run3["E"])}}
            if "time_to_E0" in out and out["time_to_E0"]["seconds"] and k3 is not None:
                out["fp64_path"]["time_to_E0_speedup"] = (
                    out["fp64_path"]["time_to_E0"]["seconds"] / out["time_to_E0"]["seconds"])
        else:  # one warm-up and one timed step
            ctx3.prepare_2b(sys_.beta, sys_.u, sys_.p, 0)
            ctx3.step_2b(sys_.mixing)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx3.step_2b(sys_.mixing)
            e1.record(stream)
            barrier()
            fp64_ms = e0.elapsed_time(e1)
            st3, _ = ctx3.stage_times()
            out["fp64_path"] = {"ms_per_step": fp64_ms, "builds_per_s": 1000.0 / fp64_ms,
                                "stage_ms": st3,
                                "speedup_per_step": fp64_ms / (elapsed / args.steps)}
        ctx3.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample, _, _ = oracle_sample(sys_, 6, 3)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": _cpu_cores(), "kind": "oracle",
                               "sample": sample}
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
