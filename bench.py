"""Benchmark of the R-ChFSI eigensolver on one GB300 (or N independent replicas).

Default workload (the largest configuration that runs on one GPU at its stated size): the
finite-element generalized problem on a periodic mesh of 16^3 Q4 cells (262,144 dofs), A = 0.5
stiffness + mass weighted by a potential of 8 seeded Gaussian wells, B = consistent mass,
D^-1 = GLL-lumped inverse of B; nev = 500, block 600, degree 25; TF32 tensor-core filter
products, FP64 residuals and Rayleigh-Ritz.  One step = one complete solve from the same seeded
initial block to the relative residual 1e-8 (time-to-tolerance).  `--workload dense` runs the
dense generalized problem instead (m = 4000, dense SPD B, D^-1 = diag(B)^-1, nev 200, block 240,
degree 30).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload fe|dense|...]

Prints one JSON line (rank 0).  The reference arm (--impl reference) times the FP64 CPU oracle on
this machine's host cores: a full solve per step on the dense problem, a bounded sample of one
outer iteration per step on the finite-element problem (whose full oracle solve takes hours).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

DENSE = dict(m=4000, nev=200, block=240, degree=30, tol=1e-8)
FE = dict(n=16, nev=500, block=600, degree=25, tol=1e-8)
METRIC = "R-ChFSI time-to-1e-8 relative residual"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="fe", choices=["fe", "dense", "kpoints", "serving", "psweep"])
    ap.add_argument("--precision", default="tf32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison runs")
    ap.add_argument("--rr", default="emulated", choices=["fp64", "emulated"],
                    help="FP64 products of residual / Rayleigh-Ritz: DFMA or BF16-slice emulation")
    ap.add_argument("--eig", default="tridiag", choices=["syevd", "jacobi", "tridiag"],
                    help="N x N projected eigensolver: cuSOLVER dsyevd, or this library's Jacobi or tridiagonal kernels")
    ap.add_argument("--quick", action="store_true",
                    help="timed solves only: no comparisons, no end-to-end run, no CPU baseline (profiling runs)")
    ap.add_argument("--fe-n", type=int, default=None,
                    help="FE workload: n^3 cells instead of 16^3 (a smaller case for ncu captures)")
    a = ap.parse_args()
    if a.fe_n is not None:
        FE["n"] = int(a.fe_n)
    return a


def workload_desc(kind, prec):
    if kind == "dense":
        return ("dense generalized A x = lambda B x, m=4000 (A: spectrum linspace(-1,10) + 0.05 gap after "
                "index 50; B = S^1/2 (I + 0.1 G) S^1/2, diag(B)=S log-uniform[0.5,50]; D^-1 = diag(B)^-1), "
                "nev=200, block=240, degree=30, %s filter products, FP64 Rayleigh-Ritz" % prec)
    n = FE["n"]
    return ("FE generalized problem, periodic %d^3 Q4 cells (%s dofs), A = 0.5 K + V-mass (8 seeded "
            "wells), B = consistent mass, D^-1 = GLL-lumped inverse, nev=500, block=600, degree=25, "
            "%s filter products, FP64 Rayleigh-Ritz" % (n, format((4 * n) ** 3, ","), prec))


# Batched k-point workload: the structure of the 16-k-point configuration (Bloch problems on
# periodic Q4 meshes of different sizes, complex Hermitian, nev and block per problem) at reduced
# mesh sizes (6^3..10^3 cells instead of 8^3..20^3, nev 25..200 instead of 100..800): the full sizes
# need ~470 GB of solver workspace.
KPOINTS = dict(n_problems=16, seed=7, nmin=6, nmax=10, nev_range=(25, 200), degree=25, tol=1e-8)


def kpoint_problems():
    specs = wl.fe_config4_list(n_problems=KPOINTS["n_problems"], seed=KPOINTS["seed"], nmin=KPOINTS["nmin"],
                               nmax=KPOINTS["nmax"], nev_range=KPOINTS["nev_range"])
    out = []
    for i, sp in enumerate(specs):
        p = wl.fe_kpoint_problem(sp["n"], sp["kappa"])
        rng = np.random.default_rng(100 + i)
        X0 = rng.standard_normal((p["m"], sp["block"])) + 1j * rng.standard_normal((p["m"], sp["block"]))
        out.append((sp, p, X0))
    return out


def kpoints_desc(prec):
    return ("16 Bloch k-point problems (complex Hermitian FE, periodic Q4 meshes of 6^3..10^3 cells = "
            "13,824..64,000 complex dofs, kappa in [-0.5,0.5)^3, nev 25..200, block ceil(1.2 nev/16)*16, "
            "degree 25, %s cell products), seeds 7 / 100+i" % prec)


def kpoints_run(args, torch, dev):
    """Batched solve of the k-point list vs the same problems solved one after the other."""
    from paper_2503_22652_gb300 import Solver, solve_batch
    prec = args.precision if args.precision in ("tf32", "bf16") else "tf32"
    probs = kpoint_problems()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    solvers, X0 = [], []
    for sp, p, x0 in probs:
        s = Solver(p["m"], nev=sp["nev"], block=sp["block"], degree=KPOINTS["degree"], precision=prec,
                   field="complex", max_iter=300, tol=KPOINTS["tol"], rr_mode=args.rr, eig_mode=args.eig)
        s.set_fe(T(p["cell_dofs"]), T(p["A_cells"]), T(p["B_cell"]), T(p["Dinv"]))
        solvers.append(s)
        X0.append(T(x0))

    def batched():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = solve_batch(solvers, X0)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3, out

    def sequential():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = [s.solve(x) for s, x in zip(solvers, X0)]
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3, out

    batched()  # warm-up: tile tuning, graph capture, workspaces
    sequential()
    solvers[0].profile(True)
    tb, ob = batched()
    fe = solvers[0].profile_read("fe_cell")
    launches = solvers[0].profile_read("all")["launches"]
    solvers[0].profile(False)
    ts, osq = sequential()
    worst = max(st["max_rel_residual"] for _, _, _, st in ob)
    iters = [st["iterations"] for _, _, _, st in ob]
    flops = sum(st["filter_flops"] for _, _, _, st in ob)
    filt_ms = max(st["t_filter_ms"] for _, _, _, st in ob)
    dev_ev = max(float(np.max(np.abs(a[1][:sp["nev"]] - b[1][:sp["nev"]]) / np.maximum(np.abs(b[1][:sp["nev"]]),
                                                                                         1.0)))
                 for a, b, (sp, _, _) in zip(ob, osq, probs))
    hbm = peaks().get("hbm_gbs", 6800.0)
    roof = None
    if fe["launches"] and fe["ms"] > 0:
        ach = fe["bytes"] / (fe["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                "traffic": None, "peak_source": "measured HBM copy (of measured)", "kernel": "fe_tc_kernel (batched)",
                "per_launch_ms": fe["ms"] / fe["launches"],
                "tflops": round(fe["flops"] / (fe["ms"] * 1e-3) / 1e12, 2)}
    for s in solvers:
        s.close()
    return {"batched_ms": round(tb, 1), "sequential_ms": round(ts, 1), "speedup": round(ts / tb, 2),
            "problems": len(probs), "problems_per_s": round(len(probs) / (tb * 1e-3), 2),
            "iterations": iters, "max_rel_residual": worst, "max_rel_eval_diff_batched_vs_alone": dev_ev,
            "filter_tflops": round(flops / (filt_ms * 1e-3) / 1e12, 2) if filt_ms > 0 else None,
            "roofline": roof, "gpu_launches": int(launches), "precision": prec,
            "workload": kpoints_desc(prec)}


# Serving stream: Poisson arrivals of requests from four outer-loop chains (real FE meshes of 6^3 and
# 8^3 cells, complex k-point meshes of 6^3 and 8^3 cells), each request a 1% drift of the well depths
# of the chain's previous operator, warm-started from the chain's last subspace kept on the device;
# arrival rate 0.8 x the measured warm single-stream solve rate.  The full-size stream (up to 32^3
# cells, nev 2000) needs ~200 GB per request and minutes per solve.
SERVING = dict(chains=[(6, None, 40, 48), (8, None, 60, 80), (6, (0.2, -0.1, 0.3), 30, 48),
                       (8, (-0.3, 0.25, 0.1), 50, 64)], per_chain=16, slots=2, load=0.8, degree=25, tol=1e-8,
               seed_arrivals=8)


def serving_desc(prec):
    return ("serving stream: %d requests, Poisson arrivals at %.1f x the warm single-stream solve rate, 4 chains "
            "of 1%%-drifting FE operators (real 6^3 / 8^3 Q4 cells, complex k-point 6^3 / 8^3; nev 40 / 60 / 30 / "
            "50), warm starts kept on the device, %d server slots, degree 25, %s filter"
            % (SERVING["per_chain"] * len(SERVING["chains"]), SERVING["load"], SERVING["slots"], prec))


def serving_run(args):
    """Serving stream through rchfsi_server_create / rchfsi_submit / rchfsi_poll."""
    from paper_2503_22652_gb300 import Server
    prec = args.precision
    chains = []
    for ci, (n, kp, nev, blk) in enumerate(SERVING["chains"]):
        kpoint = None if kp is None else 2.0 * np.pi / (n * 0.5) * np.asarray(kp)
        probs = wl.fe_scf_chain(n, SERVING["per_chain"] + 1, seed_wells=6 + ci, seed_pert=100 + ci, kpoint=kpoint)
        rng = np.random.default_rng(200 + ci)
        m = probs[0]["m"]
        X0 = rng.standard_normal((m, blk))
        if kp is not None:
            X0 = X0 + 1j * rng.standard_normal((m, blk))
        chains.append(dict(probs=probs, nev=nev, block=blk, X0=X0, field="real" if kp is None else "complex"))
    srv = Server(slots=SERVING["slots"])

    def submit(ci, k, key):
        c = chains[ci]
        p = c["probs"][k]
        fe = dict(cell_dofs=p["cell_dofs"], A_cells=p["A_cells"], B_cells=p["B_cell"], Dinv=p["Dinv"])
        return srv.submit(p["m"], c["nev"], c["block"], X0=c["X0"], warm_key=key, fe=fe, field=c["field"],
                          precision=prec, degree=SERVING["degree"], max_iter=300, tol=SERVING["tol"])

    def wait(t):
        while True:
            r = srv.poll(t)
            if r is not None:
                return r
            time.sleep(0.001)

    # calibration (own warm keys): a cold then a warm solve per chain, one at a time
    warm_ms = []
    for ci in range(len(chains)):
        wait(submit(ci, 0, 1000 + ci))
        warm_ms.append(wait(submit(ci, 1, 1000 + ci))["latency_ms"])
    S = float(np.mean(warm_ms)) / 1e3
    rate = SERVING["load"] / S
    # the stream: request k of every chain (k = 1..per_chain, operator k), in a seeded random order
    order = [(ci, k) for k in range(1, SERVING["per_chain"] + 1) for ci in range(len(chains))]
    rng = np.random.default_rng(SERVING["seed_arrivals"])
    gaps = rng.exponential(1.0 / rate, len(order))
    t_arr = np.cumsum(gaps) - gaps[0]
    pending, results = {}, []
    t0 = time.perf_counter()
    i = 0
    while i < len(order) or pending:
        now = time.perf_counter() - t0
        while i < len(order) and t_arr[i] <= now:
            ci, k = order[i]
            pending[submit(ci, k, 1 + ci)] = (ci, k, now)
            i += 1
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                ci, k, ta = pending.pop(t)
                r["done_s"] = time.perf_counter() - t0
                r["chain"], r["step"] = ci, k
                results.append(r)
        time.sleep(0.0005)
    t_end = max(r["done_s"] for r in results)
    srv.close()
    lat = np.array([r["latency_ms"] for r in results])
    its = {ci: [r["iterations"] for r in sorted(results, key=lambda x: x["step"]) if r["chain"] == ci]
           for ci in range(len(chains))}
    return {"p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "mean_ms": round(float(lat.mean()), 2), "queue_ms_p50": round(float(np.median([r["queue_ms"] for r in results])), 2),
            "solves_per_s": round(len(results) / t_end, 3), "requests": len(results),
            "arrival_rate_per_s": round(rate, 3), "warm_service_ms": [round(v, 1) for v in warm_ms],
            "statuses_ok": int(sum(r["status"] == 0 for r in results)),
            "statuses": {str(k): int(v) for k, v in zip(*np.unique([r["status"] for r in results], return_counts=True))},
            "failed": [(r["chain"], r["step"], r["status"], r["error"][:100]) for r in results if r["status"] != 0],
            "max_rel_residual": float(max(r["max_rel_residual"] for r in results)),
            "iterations_first_vs_rest": {str(ci): [v[0], round(float(np.mean(v[1:])), 1)] for ci, v in its.items()},
            "precision": prec, "workload": serving_desc(prec)}


def run_serving(args, rank, world, local_rank):
    import torch
    import paper_2503_22652_gb300.build as B
    torch.cuda.set_device(local_rank)
    B.build()
    clk = ClockSampler(local_rank)
    clk.start()
    r = serving_run(args)
    clocks = clk.stop()
    if rank != 0:
        return None
    return {"metric": "serving latency p50 (Poisson arrivals, warm-started outer-loop chains)", "value": r["p50_ms"],
            "unit": "ms", "n_gpus": world, "steps": r["requests"], "warmup": 8, "ms_per_step": r["mean_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "%s+f64" % r["precision"],
            "data": "synthetic", "config": {"workload": r["workload"], "parallelism": "single GPU"},
            "roofline": None, "gpu_launches": None, "clocks": clocks, "e2e": None, "cpu_baseline": None,
            "serving": {k: v for k, v in r.items() if k != "workload"}}


def psweep_run(args, torch, dev):
    """Degree sweep on the dense benchmark problem: time to 1e-8 and iterations per degree and
    precision (where the reduced-precision filter stops paying for higher degrees)."""
    from paper_2503_22652_gb300 import Solver
    prob = make_problem("dense")
    c = prob["dense"]
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    dA, dB, dD, X0 = T(c["A"]), T(c["B"]), T(c["Dinv"]), T(prob["X0"])
    out = []
    for prec in ("tf32", "bf16", "fp32"):
        for p in (10, 20, 30, 40, 60, 80, 100, 120):
            s = Solver(prob["m"], nev=prob["nev"], block=prob["block"], degree=p, precision=prec, max_iter=300,
                       tol=prob["tol"], rr_mode=args.rr, eig_mode=args.eig)
            s.set_dense(dA, B=dB, Dinv=dD)
            s.solve(X0.clone(), allow_not_converged=True)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ev, res, st = s.solve(X0.clone(), allow_not_converged=True)
            torch.cuda.synchronize()
            out.append({"precision": prec, "degree": p, "ms": round((time.perf_counter() - t0) * 1e3, 1),
                        "iterations": st["iterations"], "status": st["status"],
                        "max_rel_residual": st["max_rel_residual"], "t_filter_ms": round(st["t_filter_ms"], 1),
                        "cholqr_retries": st.get("cholqr_retries")})
            s.close()
    return out


def run_psweep(args, rank, world, local_rank):
    import torch
    import paper_2503_22652_gb300.build as B
    torch.cuda.set_device(local_rank)
    B.build()
    r = psweep_run(args, torch, torch.device("cuda", local_rank))
    if rank != 0:
        return None
    best = min((x for x in r if x["status"] == 0), key=lambda x: x["ms"])
    return {"metric": "R-ChFSI time-to-1e-8 relative residual, best degree", "value": best["ms"], "unit": "ms",
            "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": best["ms"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "%s+f64" % best["precision"], "data": "synthetic",
            "config": {"workload": workload_desc("dense", "swept") + "; degree swept 10..120",
                       "parallelism": "single GPU"},
            "roofline": None, "gpu_launches": None, "clocks": None, "e2e": None, "cpu_baseline": None,
            "best": best, "sweep": r}


def max_over_ranks(x, device):
    """The largest of every rank's x (the job's time is its slowest rank's); collective over the
    default process group (NCCL on GPUs, gloo on host tensors)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_problem(kind):
    if kind == "dense":
        c = wl.dense_config2(m=DENSE["m"])
        X0 = wl.gaussian_block(DENSE["m"], DENSE["block"], seed=2)
        return {"dense": c, "X0": X0, **DENSE}
    p = wl.fe_config3(n=FE["n"])
    X0 = wl.gaussian_block(p["m"], FE["block"], seed=2)
    return {"fe": p, "X0": X0, "m": p["m"], **FE}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- reference arm
def cpu_cores():
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        th = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if th:
            return int(th[0])
    except Exception:
        pass
    return n


def oracle_fe_iterations():
    """Outer iterations of the oracle's own FP64 R-ChFSI solve of the finite-element construction
    (8^3 cells, energy window of the 16^3 problem; tests/golden/oracle_iterations.json, written by
    tests/golden/make_oracle_iterations.py from oracle/ alone)."""
    with open(os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")) as f:
        g = json.load(f)["fe_8cubed_energy_matched"]
    return int(g["iterations"]), g


def oracle_sample_fe(prob):
    """Bounded sample of the FP64 oracle on the FE workload at full size: one sparse operator
    product A D^-1 R on a 60-column slice (scaled to the block width), one Gram product Y^T Z of the
    full block and one block x block dense generalized eigensolve.  Returns (seconds per outer
    iteration, setup seconds, measured seconds) with the model: an iteration = (p - 1) filter
    products + 2 Rayleigh-Ritz products (A Y, B Y) + 5 Gram-sized products (2 Gram matrices, 3
    rotations) + the eigensolve; setup = one Rayleigh-Ritz step."""
    import scipy.linalg as sla
    from oracle import fe as ofe
    p = prob["fe"]
    t_all = time.perf_counter()
    As = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    d = p["Dinv"]
    X0 = prob["X0"]
    N = X0.shape[1]
    cols = min(60, N)
    t0 = time.perf_counter()
    As @ (d[:, None] * X0[:, :cols])
    t_prod = (time.perf_counter() - t0) * N / cols
    t0 = time.perf_counter()
    G = X0.T @ X0
    t_gram = time.perf_counter() - t0
    t0 = time.perf_counter()
    sla.eigh(G + G.T + N * np.eye(N), np.eye(N) * N)
    t_eig = time.perf_counter() - t0
    t_rr = 2 * t_prod + 5 * t_gram + t_eig
    return (prob["degree"] - 1) * t_prod + t_rr, t_rr, time.perf_counter() - t_all


def oracle_dense_solve(prob):
    """The oracle's own time-to-tolerance on the dense workload: Lanczos bounds, initial
    Rayleigh-Ritz and Algorithm 1 with Algorithm 3 in FP64 until the relative residual of the
    first nev columns is <= tol.  Returns (seconds, iterations, final relative residual)."""
    from oracle import lanczos, solver
    c = prob["dense"]
    A = lambda v: c["A"] @ v  # noqa: E731
    B = lambda v: c["B"] @ v  # noqa: E731
    d = c["Dinv"]
    X0 = prob["X0"]
    t0 = time.perf_counter()
    lmax = lanczos.upper_bound(A, d, X0[:, 0], 10)
    normA = lanczos.norm_estimate(A, X0[:, 0], 10)
    r = solver.solve(A, B, X0, prob["nev"], prob["degree"], prob["tol"], 200, lmax, normA, method="rchfsi",
                     Dinv=lambda R: d[:, None] * R)
    return time.perf_counter() - t0, int(r["iters"]), float(r["history_rel"][-1])


def oracle_dense_warmup(prob):
    """A short untimed oracle run (one Rayleigh-Ritz step of the initial block)."""
    from oracle import rr
    c = prob["dense"]
    rr.rayleigh_ritz(prob["X0"], lambda v: c["A"] @ v, lambda v: c["B"] @ v)


def run_reference(args, rank):
    if rank != 0:
        return None
    if args.workload in ("kpoints", "serving", "psweep"):
        return {"impl": "reference", "unavailable": "the oracle arm times the dense and FE workloads only"}
    prob = make_problem(args.workload)
    cores = cpu_cores()
    extra = {}
    if args.workload == "dense":
        for _ in range(args.warmup):
            oracle_dense_warmup(prob)
        samples = []
        for _ in range(args.steps):
            t, iters, res = oracle_dense_solve(prob)
            samples.append(t)
        val = statistics.mean(samples) * 1e3
        desc = ("FP64 NumPy oracle, one complete solve per step (Lanczos bounds, initial Rayleigh-Ritz, Algorithm 1 "
                "with Algorithm 3 to relative residual %.0e): %d iterations, final residual %.2e"
                % (prob["tol"], iters, res))
        extra = {"oracle_iterations": iters, "oracle_max_rel_residual": res}
    else:
        iters, g = oracle_fe_iterations()
        for _ in range(args.warmup):
            oracle_sample_fe(prob)
        samples, measured = [], []
        for _ in range(args.steps):
            per_it, setup, took = oracle_sample_fe(prob)
            samples.append(setup + per_it * iters)
            measured.append(took)
        val = statistics.mean(samples) * 1e3
        desc = ("FP64 NumPy/SciPy oracle, bounded sample per step (%.1f s measured): one sparse A D^-1 R product "
                "on 60 columns (scaled to the block), one Gram product and one dense eigensolve at full size; "
                "value = setup + %d outer iterations x [(p-1) + 2 products + 5 Gram-sized products + eigensolve], "
                "%d = the oracle's own iteration count on the same construction at %d^3 cells (nev %d, block %d: "
                "same energy window), tests/golden/oracle_iterations.json"
                % (statistics.mean(measured), iters, iters, g["cells_per_dim"], g["nev"], g["block"]))
        extra = {"oracle_iterations": iters, "sample_seconds_per_step": round(statistics.mean(measured), 2),
                 "value_is": "model: measured per-iteration pieces x the oracle's measured iteration count"}
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "ms", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(val, 3), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(args.workload, "fp64"), "parallelism": "host cores"},
           "cpu_baseline": {"value": round(val, 3), "unit": "ms", "cores": cores, "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": round(val, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    out.update(extra)
    return out


# ----------------------------------------------------------------------------- GPU arm
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def roofline(prof, solve_ms_total, pk, precision, rr_mode="emulated"):
    """Roofline entry of the kernel class with the largest device time in the timed region."""
    best = max(prof.items(), key=lambda kv: kv[1]["ms"])
    return class_roofline(best[0], best[1], solve_ms_total, pk, precision, rr_mode)


def class_roofline(name, r, solve_ms_total, pk, precision, rr_mode="emulated"):
    """Roofline entry of one kernel class: its algorithmic work over its device time."""
    per_launch_ms = r["ms"] / max(r["launches"], 1)
    hbm = pk.get("hbm_gbs", 6800.0)
    bf16 = pk.get("bf16_tflops_sustained", 1700.0)
    if name == "filter_tc":
        # tensor-bound when the dense operator stays in L2 across the degree loop
        ratio = {"tf32": 0.5, "bf16": 1.0}.get(precision, 0.5)
        ach = r["flops"] / (r["ms"] * 1e-3) / 1e12
        peak = bf16 * ratio
        return name, {"bound": "tensor", "achieved": round(ach, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                      "frac": round(ach / peak, 4), "traffic": None,
                      "peak_source": "measured bf16 sustained x nominal %s/bf16 ratio %.2f (of measured)" % (
                          precision, ratio),
                      "share_of_solve": round(r["ms"] / solve_ms_total, 4), "per_launch_ms": per_launch_ms}
    if name == "gemm_f64_emu":
        # the 28 BF16 slice products per FP64-accurate product run on the tensor cores
        ach = r["flops"] / (r["ms"] * 1e-3) / 1e12
        return name, {"bound": "tensor", "achieved": round(ach, 2), "peak": round(bf16, 1), "unit": "TFLOP/s",
                      "frac": round(ach / bf16, 4), "traffic": None,
                      "peak_source": "measured bf16 sustained (of measured)",
                      "fp64_equivalent_tflops": round(ach / 28.0, 2),
                      "share_of_solve": round(r["ms"] / solve_ms_total, 4), "per_launch_ms": per_launch_ms}
    if name == "fe_cell_f64" and rr_mode == "emulated":
        # FP64-accurate cell products from BF16 slices: 28 slice products per FP64 product on the
        # tensor cores (the recorded flops are the FP64-equivalent 2 n_c^2 C N)
        ach = 28.0 * r["flops"] / (r["ms"] * 1e-3) / 1e12
        return name, {"bound": "tensor", "achieved": round(ach, 2), "peak": round(bf16, 1), "unit": "TFLOP/s",
                      "frac": round(ach / bf16, 4), "traffic": None,
                      "peak_source": "measured bf16 sustained (of measured)",
                      "fp64_equivalent_tflops": round(ach / 28.0, 2),
                      "share_of_solve": round(r["ms"] / solve_ms_total, 4), "per_launch_ms": per_launch_ms}
    if name in ("gemm_f64", "filter_simt", "fe_cell_f64", "eig", "small_dense"):
        ach = r["flops"] / (r["ms"] * 1e-3) / 1e12
        peak = 69.8 if name == "filter_simt" else 1.25
        return name, {"bound": "alu", "achieved": round(ach, 4), "peak": peak, "unit": "TFLOP/s",
                      "frac": round(ach / peak, 4), "traffic": None,
                      "peak_source": ("FP32 FFMA 69.8 TFLOP/s (measured, cuBLAS SGEMM)" if name == "filter_simt" else
                                      "nominal FP64 1.25 TFLOP/s (a DFMA loop measured 1.198 TFLOP/s)"),
                      "share_of_solve": round(r["ms"] / solve_ms_total, 4), "per_launch_ms": per_launch_ms}
    ach = r["bytes"] / (r["ms"] * 1e-3) / 1e9
    return name, {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                  "frac": round(ach / hbm, 4), "traffic": None, "peak_source": "measured HBM copy (of measured)",
                  "share_of_solve": round(r["ms"] / solve_ms_total, 4), "per_launch_ms": per_launch_ms}


def run_kpoints(args, rank, world, local_rank):
    """--workload kpoints: one JSON line for the batched k-point solve (replicas under torchrun)."""
    import torch
    import paper_2503_22652_gb300.build as B
    torch.cuda.set_device(local_rank)
    B.build()
    dev = torch.device("cuda", local_rank)
    clk = ClockSampler(local_rank)
    clk.start()
    r = kpoints_run(args, torch, dev)
    clocks = clk.stop()
    if rank != 0:
        return None
    return {"metric": "batched k-point time-to-1e-8 relative residual (16 problems)", "value": r["batched_ms"],
            "unit": "ms", "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": r["batched_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "%s+f64" % r["precision"],
            "data": "synthetic", "config": {"workload": r["workload"], "parallelism": "single GPU"},
            "roofline": r["roofline"], "gpu_launches": r["gpu_launches"], "clocks": clocks, "e2e": None,
            "cpu_baseline": None, "kpoints": {k: v for k, v in r.items() if k not in ("roofline", "workload")}}


def filter_step_roofline(prof, prob, pk, steps_per_solve):
    """Roofline of one degree step of the filter (the hot path of Algorithm 3) on the FE workload:
    the fused tensor-core kernel does the whole step (gather of D^-1 R_Y, cell products, recurrence
    terms and scatter into R_X), so its launches are the steps.  Algorithmic bytes per step:
    4 block streams (R_Y gathered, R_X read and written, W read) of m N FP32 values plus the cell
    matrices in the operand precision, C n_c^2 s."""
    r = prof.get("fe_cell")
    if not r or not r["launches"] or r["ms"] <= 0:
        return None
    hbm = pk.get("hbm_gbs", 6800.0)
    per_ms = r["ms"] / r["launches"]
    per_bytes = r["bytes"] / r["launches"]
    ach = per_bytes / (per_ms * 1e-3) / 1e9
    # DRAM traffic of the kernel from the ncu capture of profiles/fe_step_kernel_fe12_n600.md (12^3 cells,
    # 1.227 GB per launch), scaled by the units processed (cells x columns) to this launch
    units = prob["fe"]["cell_dofs"].shape[0] * prob["block"]
    traffic = 1.227e9 * units / (1728 * 600)
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
            "traffic": traffic, "traffic_source": "ncu dram__bytes_read+write of fe_step_kernel at 12^3 cells x 600 "
                                                  "columns, scaled by cells x columns",
            "peak_source": "measured HBM copy, MEASURED_PEAKS.json (of measured)",
            "kernel": "fe_step_kernel (one launch = one degree step of Algorithm 3)",
            "algorithmic_bytes_per_step": per_bytes, "per_launch_ms": round(per_ms, 4),
            "launches_per_solve": r["launches"], "tflops": round(r["flops"] / (r["ms"] * 1e-3) / 1e12, 2)}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2503_22652_gb300 import Solver
    import paper_2503_22652_gb300.build as B
    from paper_2503_22652_gb300._lib import KERNEL_CLASSES
    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        B.build()
    dev = torch.device("cuda", local_rank)
    prob = make_problem(args.workload)
    m, N = prob["m"], prob["block"]
    # one non-default stream for torch's work and the library's (the handle of the legacy default
    # stream would read as NULL, a library-owned stream): the CUDA events below then bracket
    # exactly the library's work, and torch's writes to the inputs are ordered before it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    s = Solver(m, nev=prob["nev"], block=N, degree=prob["degree"], precision=args.precision, max_iter=200,
               tol=prob["tol"], stream=stream.cuda_stream, rr_mode=args.rr, eig_mode=args.eig)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    if "dense" in prob:
        c = prob["dense"]
        dA, dB, dD = T(c["A"]), T(c["B"]), T(c["Dinv"])
        s.set_dense(dA, B=dB, Dinv=dD)
    else:
        p = prob["fe"]
        s.set_fe(T(p["cell_dofs"]), T(p["A_cells"]), T(p["B_cell"]), T(p["Dinv"]))
    X0 = T(prob["X0"])
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2 (flush buffer)

    def one_solve():
        X = X0.clone()
        return s.solve(X)

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local_rank)
    clk.start()
    # timed region: clean solves, no per-launch timers (rchfsi_profile(h, 0) only restarts the
    # library's launch counter)
    s.profile(False)
    times, iters, resid = [], [], []
    for _ in range(args.steps):
        l2.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, ev, res, st = one_solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        iters.append(st["iterations"])
        resid.append(st["max_rel_residual"])
    launches = s.profile_read("all")["launches"]
    clocks = clk.stop()
    total = sum(times)
    if world > 1:
        total = max_over_ranks(total, dev)
    ms = total / args.steps
    st_last = st
    # one more solve, outside the timed region, with the per-kernel-class device timers
    s.profile(True)
    l2.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    one_solve()
    e1.record(stream)
    torch.cuda.synchronize()
    prof_ms = e0.elapsed_time(e1)
    prof = {k: s.profile_read(k) for k in KERNEL_CLASSES}
    s.profile(False)
    pk = peaks()
    kname, roof_dom = roofline(prof, prof_ms, pk, args.precision, args.rr)
    roof_all = {k: class_roofline(k, v, prof_ms, pk, args.precision, args.rr)[1] for k, v in prof.items()
                if v["launches"]}
    roof_step = filter_step_roofline(prof, prob, pk, None) if "fe" in prob else None
    extras = {}
    if not (args.no_extras or args.quick) and rank == 0:
        extras = comparisons(s, prob, args, torch, dev, stream, ms)
    e2e = end_to_end(prob, args, torch) if rank == 0 and not args.quick else None
    if rank != 0:
        return None
    sorted_t = sorted(times)
    p99 = sorted_t[min(len(sorted_t) - 1, int(np.ceil(0.99 * len(sorted_t))) - 1)]
    if roof_step is not None:
        roof = dict(roof_step)
        roof["dominant_kernel_class"] = kname
        roof["dominant_share_of_solve"] = roof_dom["share_of_solve"]
        roof["share_of_solve"] = round(prof["fe_cell"]["ms"] / prof_ms, 4)
    else:
        roof = roof_dom
    out = {"metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "%s+f64" % args.precision, "data": "synthetic",
           "config": {"workload": workload_desc(args.workload, args.precision),
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "flushed (256 MB write) before every timed step"},
           "p50_ms": round(statistics.median(times), 3), "p99_ms": round(p99, 3),
           "solves_per_s": round(world * args.steps / (total * 1e-3), 3),
           "iterations": iters[-1], "max_rel_residual": max(resid),
           "t_filter_ms": round(st_last["t_filter_ms"], 3), "t_rr_ms": round(st_last["t_rr_ms"], 3),
           "filter_tflops_in_solve": (round(st_last["filter_flops"] / (st_last["t_filter_ms"] * 1e-3) / 1e12, 2)
                                      if st_last["t_filter_ms"] > 0 else None),
           "solve_status": st_last["status"],
           "roofline_kernel": "filter degree step" if roof_step is not None else kname, "roofline": roof,
           "roofline_by_class": {k: {kk: v[kk] for kk in ("bound", "achieved", "unit", "frac", "share_of_solve")}
                                 for k, v in roof_all.items()},
           "kernel_classes_ms": {k: round(v["ms"], 3) for k, v in prof.items() if v["launches"]},
           "profiled_solve_ms": round(prof_ms, 3),
           "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e}
    out.update(extras)
    out["cpu_baseline"] = None if args.quick else cpu_baseline(prob, iters[-1])
    rr_other = st_last["t_rr_ms"] - (prof["gemm_f64"]["ms"] + prof["fe_cell_f64"]["ms"] + prof["gemm_f64_emu"]["ms"])
    out["config"]["rr_products"] = args.rr
    out["config"]["eigensolver"] = args.eig
    out["rr_non_gemm_ms"] = round(rr_other, 3)
    return out


def timed_solve(s, X0, torch, stream, **kw):
    """One solve bracketed by CUDA events on the library's stream: (ms, stats)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, _, _, st = s.solve(X0, allow_not_converged=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), st


def comparisons(s, prob, args, torch, dev, stream, rchfsi_ms):
    """The FP64 baselines on the same GPU (outside the timed region):
    * filter throughput of R-ChFSI in the chosen precision vs the FP64 ChFSI filter (Algorithm 2);
    * plain FP64 ChFSI time-to-tolerance (Algorithm 1 with Algorithm 2, FP64 products): with the
      exact inverse B^-1 (dense workload: formed once in FP64), which converges, and with the
      approximate inverse D^-1 of the workload, which stagnates at a floor set by ||D^-1 - B^-1||;
    * FP64 R-ChFSI time-to-tolerance (dense workload; on the FE workload an FP64 solve takes minutes)."""
    out = {}
    m, N, p = prob["m"], prob["block"], prob["degree"]
    X = torch.from_numpy(np.linalg.qr(prob["X0"])[0]).to(dev)
    lam = torch.linspace(-1.0, 0.5, N, dtype=torch.float64, device=dev)
    W = torch.randn(m, N, dtype=torch.float64, device=dev) * 1e-3
    bounds = (-1.5, 1.0, 80.0)
    per = (2.0 * m * m * N) if "dense" in prob else 2.0 * 125 * 125 * prob["fe"]["cell_dofs"].shape[0] * N

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    t_r = timed(lambda: s.filter(X, lam, W, *bounds, p))
    out["rchfsi_filter_ms"] = round(t_r, 3)
    out["rchfsi_filter_tflops"] = round(per * (p - 1) / (t_r * 1e-3) / 1e12, 2)
    s.set_params(precision="fp64")
    t_c = timed(lambda: s.chfsi_filter(X, *bounds, p))
    out["fp64_chfsi_filter_ms"] = round(t_c, 3)
    out["fp64_chfsi_filter_tflops"] = round(per * p / (t_c * 1e-3) / 1e12, 3)
    out["filter_speedup_vs_fp64_chfsi"] = round(t_c / t_r, 2)
    X0 = torch.from_numpy(prob["X0"]).to(dev)
    from paper_2503_22652_gb300 import Solver, _lib
    status_name = {_lib.OK: "converged", _lib.ERR_STAGNATED: "stagnated", _lib.ERR_NOT_CONVERGED: "not converged"}
    if "dense" in prob:
        # FP64 R-ChFSI on the same handle
        t, st = timed_solve(s, X0.clone(), torch, stream)
        out["fp64_rchfsi_time_ms"] = round(t, 3)
        out["fp64_rchfsi_iterations"] = st["iterations"]
        # plain FP64 ChFSI with the exact inverse: the time-to-tolerance denominator
        c = prob["dense"]
        Binv = np.linalg.inv(c["B"])
        Binv = 0.5 * (Binv + Binv.T)
        sx = Solver(m, nev=prob["nev"], block=N, degree=p, precision="fp64", method="chfsi", max_iter=200,
                    tol=prob["tol"], stream=stream.cuda_stream, rr_mode=args.rr, eig_mode=args.eig)
        sx.set_dense(torch.from_numpy(c["A"]).to(dev), B=torch.from_numpy(c["B"]).to(dev),
                     Dinv_dense=torch.from_numpy(Binv).to(dev))
        t, st = timed_solve(sx, X0.clone(), torch, stream)
        sx.close()
        out["fp64_chfsi_time_to_tol_ms"] = round(t, 3) if st["status"] == _lib.OK else None
        out["fp64_chfsi_exact_inverse"] = {"status": status_name.get(st["status"], st["status"]),
                                           "iterations": st["iterations"], "ms": round(t, 3),
                                           "max_rel_residual": st["max_rel_residual"],
                                           "inverse": "B^-1 formed once in FP64 (host LAPACK), dense"}
        if st["status"] == _lib.OK:
            out["speedup_vs_fp64_chfsi_time_to_tol"] = round(t / rchfsi_ms, 2)
        stall_max = (5, 60)
    else:
        out["fp64_chfsi_time_to_tol_ms"] = None
        out["fp64_chfsi_exact_inverse"] = {"status": "not run", "why": "B^-1 of the consistent mass is dense "
                                           "(262,144^2); this library applies only the lumped D^-1"}
        stall_max = (4, 12)
    # plain FP64 ChFSI with the workload's approximate inverse: stagnates
    s.set_params(precision="fp64", method="chfsi", stall_iters=stall_max[0], max_iter=stall_max[1])
    t, st = timed_solve(s, X0.clone(), torch, stream)
    out["fp64_chfsi_lumped"] = {"status": status_name.get(st["status"], st["status"]), "iterations": st["iterations"],
                                "max_iter": stall_max[1], "ms": round(t, 3),
                                "residual_at_exit": st["max_rel_residual"],
                                "inverse": "the workload's approximate inverse D^-1 (%s)" % (
                                    "diag(B)^-1" if "dense" in prob else "GLL-lumped mass")}
    s.set_params(precision=args.precision, method="rchfsi", stall_iters=0, max_iter=200)
    return out


def end_to_end(prob, args, torch):
    """Same solve through the C ABI with HOST (pinned) buffers: operator upload, initial block and
    results cross PCIe/C2C inside the timed region."""
    from paper_2503_22652_gb300 import Solver
    m, N = prob["m"], prob["block"]

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64 if a.dtype == np.float64 else torch.int32, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    s = Solver(m, nev=prob["nev"], block=N, degree=prob["degree"], precision=args.precision, max_iter=200,
               tol=prob["tol"], rr_mode=args.rr, eig_mode=args.eig)
    if "dense" in prob:
        c = prob["dense"]
        args_op = dict(A=pinned(c["A"]), B=pinned(c["B"]), Dinv=pinned(c["Dinv"]))
        h2d = sum(a.nbytes for a in args_op.values())
        setop = lambda: s.set_dense(**args_op)  # noqa: E731
    else:
        p = prob["fe"]
        ops = (pinned(p["cell_dofs"]), pinned(p["A_cells"]), pinned(p["B_cell"]), pinned(p["Dinv"]))
        h2d = sum(a.nbytes for a in ops)
        setop = lambda: s.set_fe(*ops)  # noqa: E731
    X0 = pinned(prob["X0"])
    Xw = pinned(prob["X0"])  # the in/out block of rchfsi_solve, refilled before every step
    h2d += X0.nbytes
    d2h = X0.nbytes + 2 * N * 8
    setop()
    s.solve(Xw, inplace=True)
    ts = []
    for _ in range(max(1, min(args.steps, 3))):
        np.copyto(Xw, X0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        setop()
        X, ev, res, st = s.solve(Xw, inplace=True)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    s.close()
    return {"value": round(statistics.mean(ts), 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h),
            "includes": "rchfsi_set_operator + rchfsi_solve from pinned host buffers (X0 in, Ritz vectors out)"}


def cpu_baseline(prob, gpu_iters):
    """The FP64 oracle on the host cores, as it stands: on the dense workload one complete solve to
    the tolerance (measured); on the FE workload the bounded sample of oracle_sample_fe, scaled by
    the oracle's own iteration count (tests/golden/oracle_iterations.json)."""
    if "dense" in prob:
        t, iters, res = oracle_dense_solve(prob)
        return {"value": round(t * 1e3, 1), "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
                "sample": "FP64 NumPy oracle, one complete solve to relative residual %.0e (measured): %d "
                          "iterations (GPU: %d), final residual %.2e" % (prob["tol"], iters, gpu_iters, res)}
    iters, g = oracle_fe_iterations()
    per_it, setup, took = oracle_sample_fe(prob)
    val = (setup + per_it * iters) * 1e3
    return {"value": round(val, 1), "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
            "sample": ("FP64 NumPy/SciPy oracle, %.1f s measured: one sparse A D^-1 R product on 60 columns (scaled "
                       "to the block), one Gram product and one dense eigensolve at full size; modelled as setup + "
                       "%d iterations x [(p-1) + 2 products + 5 Gram-sized products + eigensolve]; %d = the oracle's "
                       "own count on the %d^3-cell construction with the same energy window (GPU: %d iterations)"
                       % (took, iters, iters, g["cells_per_dim"], gpu_iters))}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "gb300":
            torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank)
    elif args.workload == "kpoints":
        out = run_kpoints(args, rank, world, local_rank)
    elif args.workload == "serving":
        out = run_serving(args, rank, world, local_rank)
    elif args.workload == "psweep":
        out = run_psweep(args, rank, world, local_rank)
    else:
        out = run_gpu(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
