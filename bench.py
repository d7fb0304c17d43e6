"""Benchmark of the RFF-preconditioned KRR solve on GB300.

One step = the whole hot path on the 65,536-point, 64-dimensional Gaussian
mixture workload (sigma = 8, lambda = 1e-4, s = 2,048 random Fourier
features, tolerance 1e-6): features, Gram matrix, FP64 Cholesky, Woodbury
factors, mixed-precision PCG with iterative refinement to a true relative
residual of 1e-6, and prediction at 8,192 held-out points.  Inputs are
resident in HBM when a step starts; the L2 cache is flushed between steps.

Also reported: the plain FP32 solve of the same system (its time and the
residual floor it reaches), the fused BF16 kernel product timed alone
(pairs/s, TFLOP/s and its exp-bound roofline), the same step through the C
ABI with host buffers (e2e), and the FP64 oracle timed on a bounded sample
on the host cores (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank solves its own
replica of the workload: the path has no exchange step (replicas only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import krr_synth as ks  # noqa: E402

METRIC = "KRR PCG time-to-rel-residual 1e-6 (mixed vs FP32); kernel-matvec TFLOP/s"
WORKLOAD = ("gaussian-mixture n=65536 d=64 (10 centres N(0,4I), unit spread), sigma=8, "
            "lambda=1e-4, s=2048 RFF, tol 1e-6, predict m=8192")
M_TEST = 8192
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one fused FP16 product
# launch at n = 65536, d = 64, from an ncu capture of `bench.py --profile fp16`; ncu does
# not run inside the bench, so the figure is carried here and applies to that size only.
TC_DRAM_BYTES_N65536 = 8679424


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", "--n", dest="n", type=int, default=None,
                    help="override n (smaller instance)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the plain FP32 comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the d = 784, k = 10 product (workload 3's shape)")
    ap.add_argument("--profile", default=None,
                    choices=["step", "bf16", "fp16", "fp16sym", "hp", "fp32", "apply", "batch"],
                    help="short run for ncu: 'step' = one mixed and one FP32 solve of "
                         "--profile-iters PCG iterations with the host-driven loop (every "
                         "launch listed); 'batch' = 3 one-launch products of the 16 largest "
                         "problems of the uneven batch; otherwise 3 launches of that kernel "
                         "product / apply")
    ap.add_argument("--workload", type=int, default=None, choices=[3, 4, 5, 6],
                    help="solve one other workload at full size (mixed, tol 1e-6) and print "
                         "one JSON line of its results instead of the bench line; 6 is the "
                         "65,536-point workload with the random-features method and "
                         "Algorithm 1 at several preconditioner ridges lambda_p")
    ap.add_argument("--oracle-config1", action="store_true",
                    help="internal: time the oracle's Algorithm 1 on workload 1 and print it")
    ap.add_argument("--profile-iters", type=int, default=12)
    ap.add_argument("--profile-k", type=int, default=1,
                    help="right-hand sides of the --profile bf16/fp16/hp/fp32 products")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest `value` over the ranks of the initialised process group."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def bench_config(P, n: int, world: int) -> dict:
    """The `config` object of the bench line (both arms)."""
    return {"workload": WORKLOAD, "n": n, "d": P.d, "s": P.s, "sigma": P.sigma,
            "lambda": P.lam, "tol": P.tol, "m_predict": M_TEST,
            "l2": "flushed between steps (512 MiB write)",
            "parallelism": "replicas" if world > 1 else "single-gpu"}


def tensor_peak_tflops() -> tuple[float, str]:
    """Dense FP16/BF16 tensor peak for a kernel timed alone: the measured cuBLAS
    BF16 burst figure when the measured-peaks file is present (FP16 runs at the
    BF16 rate), else the fallback of 1,900 TFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops"])
        return v, "of measured (cuBLAS BF16 burst; FP16 runs at the BF16 rate)"
    except Exception:
        return 1900.0, "of fallback (1.9 PFLOP/s BF16 burst)"


def blas_threads() -> int:
    """Threads the oracle's BLAS calls use (threadpoolctl when present)."""
    try:
        from threadpoolctl import threadpool_info
        n = sum(i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas")
        if n > 0:
            return n
    except Exception:
        pass
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or (os.cpu_count() or 1)


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        # the raw samples go to KRR_CLOCKS_DIR (default: the system temp directory)
        out = os.environ.get("KRR_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_gpu{gpu}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- oracle leg --
def oracle_product_seconds(P, rows: int) -> float:
    """Seconds for one full FP64 oracle kernel product on this workload, timed on
    `rows` rows (the blocked product is row-parallel, so time scales with rows)."""
    from oracle import krr_oracle as O
    V = np.random.default_rng(0).standard_normal((P.n, 1))
    t0 = time.perf_counter()
    O.kernel_matvec_blocked(P.X[:rows], P.X, V, P.sigma)
    return (time.perf_counter() - t0) * P.n / rows


def oracle_alg1(P) -> dict:
    """The oracle's Algorithm 1 (RFF features, Woodbury preconditioner, FP64 PCG)
    end to end on P, timed, with its own iteration count and true residual."""
    from oracle import krr_oracle as O
    t0 = time.perf_counter()
    out = O.krr_pcg_solve(P.X, P.Y, P.sigma, P.lam, P.W, P.b, tol=P.tol, max_iter=5000)
    t = time.perf_counter() - t0
    res = float(O.true_rel_residual(P.X, P.Y, out["x"], P.sigma, P.lam)[0])
    return {"n": P.n, "s": P.s, "seconds": t, "iters": int(out["iters"][0]), "rel_res": res,
            "status": out["status"]}


def oracle_direct(P) -> dict:
    from oracle import krr_oracle as O
    t0 = time.perf_counter()
    C = O.direct_solve(P.X, P.Y, P.sigma, P.lam)
    t = time.perf_counter() - t0
    return {"n": P.n, "seconds": t,
            "rel_res": float(O.true_rel_residual(P.X, P.Y, C, P.sigma, P.lam)[0])}


def oracle_one_core_config1() -> dict | None:
    """Workload 1 (n = 2,000) through the oracle's Algorithm 1 on one core: a
    child process with every BLAS/OpenMP pool limited to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-config1"],
                           env=env, capture_output=True, text=True, timeout=600)
        return json.loads(p.stdout.strip().splitlines()[-1])
    except Exception as e:  # the baseline is reported, not required
        return {"error": str(e)[:200]}


def cpu_baseline(P) -> dict:
    """The FP64 oracle timed on the host cores (measured parts and one labelled
    extrapolation to the benched size)."""
    cores = blas_threads()
    cfg1 = oracle_alg1(ks.make_config(1))
    cfg1_one = oracle_one_core_config1()
    P8 = ks.make_config(2, n=8192)          # same recipe, same W and b
    alg8 = oracle_alg1(P8)
    direct4 = oracle_direct(ks.make_config(2, n=4096))
    rows = min(512, P.n)
    t_mv = oracle_product_seconds(P, rows)
    est_ms = alg8["iters"] * t_mv * 1e3
    return {"value": est_ms, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": (f"extrapolated: the oracle's own Algorithm 1 iteration count on the "
                       f"8,192-point instance ({alg8['iters']}) x one full {P.n}-point FP64 "
                       f"product ({t_mv:.1f} s, timed on {rows} rows); iterations grow with n, "
                       f"so this underestimates the full solve"),
            "measured": {"config1_all_cores": cfg1, "config1_one_core": cfg1_one,
                         "alg1_n8192": alg8, "direct_n4096": direct4,
                         "full_product_s": t_mv, "full_product_rows_timed": rows}}


def run_reference(args, rank, world):
    """The oracle, timed on the host cores (rank 0 only; other ranks exit at once).

    One step = the oracle's Algorithm 1 end to end on a 2,048-point instance of
    the benched workload (same recipe, same W and b) plus one full-size FP64
    kernel product timed on 256 rows; the step's value scales the full-size
    product time by the sample solve's own iteration count."""
    if rank != 0:
        return
    n = args.n or ks.CONFIGS[2]
    P = ks.make_config(2, n=n, m=M_TEST)
    Ps = ks.make_config(2, n=min(2048, n))
    vals, last = [], None
    for i in range(args.warmup + args.steps):
        alg = oracle_alg1(Ps)
        t_mv = oracle_product_seconds(P, min(256, n))
        if i >= args.warmup:
            vals.append(alg["iters"] * t_mv * 1e3)
            last = (alg, t_mv)
    v = statistics.mean(vals)
    alg, t_mv = last
    cores = blas_threads()
    sample = (f"extrapolated per step: oracle Algorithm 1 on a {Ps.n}-point instance "
              f"({alg['seconds']:.2f} s, {alg['iters']} iterations, residual "
              f"{alg['rel_res']:.1e}) x one full {n}-point FP64 product ({t_mv:.1f} s, timed "
              f"on 256 rows)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(P, n, world),
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": sample, "measured": {"alg1_sample": alg,
                                                        "full_product_s": t_mv}},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# --------------------------------------------------------------- profile --
def run_profile(args):
    """Short, launch-bounded runs for Nsight Compute (no timing is reported)."""
    import torch
    from paper_1611_03220_gb300 import build
    build()
    from paper_1611_03220_gb300 import _krr as K

    n = args.n or ks.CONFIGS[2]
    P = ks.make_config(2, n=n)
    X = torch.from_numpy(P.X).cuda()
    Y = torch.from_numpy(P.Y).cuda()
    W = torch.from_numpy(P.W).cuda()
    b = torch.from_numpy(P.b).cuda()
    h = K.Handle()
    if args.profile == "step":
        C = torch.zeros_like(Y)
        for prec in ("mixed", "fp32"):
            o = K.default_opts(tol=P.tol, precision=prec, max_iter=args.profile_iters,
                               use_graph=0)
            rep = K.krr_pcg_solve(h, X, P.sigma, P.lam, W, b, Y, C, o, check=False)
            torch.cuda.synchronize()
            print(prec, rep["status"], rep["iters"], rep["matvecs"], flush=True)
    elif args.profile == "batch":
        probs = sorted(ks.make_uneven(), key=lambda q: -q.n)[:16]
        rng = np.random.default_rng(4)
        items = []
        for q in probs:
            Vb = torch.from_numpy(rng.standard_normal((q.n, 1)).astype(np.float32)).cuda()
            items.append((torch.from_numpy(q.X).cuda(), q.sigma, q.lam, Vb, torch.empty_like(Vb)))
        for _ in range(3):
            K.krr_kernel_matvec_batched(h, items)
    elif args.profile == "apply":
        Z = torch.empty((n, P.s), dtype=torch.float32, device="cuda")
        K.krr_rff_features(h, X, W, b, Z)
        K.krr_precond_setup(h, Z, P.lam, "zl", z_format="bf16")
        R = torch.randn((n, 1), dtype=torch.float64, device="cuda")
        Zo = torch.empty_like(R)
        for _ in range(3):
            K.krr_precond_apply(h, R, Zo)
    else:
        dt = torch.float64 if args.profile == "hp" else torch.float32
        V = torch.randn((n, args.profile_k), dtype=dt, device="cuda")
        Q = torch.empty_like(V)
        prec = args.profile
        if prec == "fp16sym":   # the symmetric product (plan mode 2)
            h.set_autotune(2)
            prec = "fp16"
        for _ in range(3):
            K.krr_kernel_matvec(h, X, X, P.sigma, P.lam, V, Q, prec)
    torch.cuda.synchronize()
    h.close()


# ---------------------------------------------------------- workloads ---
def run_workload(args):
    """Full-size solves of the multi-RHS (3), uneven-batch (4) and gradient (5)
    workloads: wall time, iterations and the solver's residual certificate."""
    import torch
    from paper_1611_03220_gb300 import build
    build()
    from paper_1611_03220_gb300 import _krr as K

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    h = K.Handle()
    opts = K.default_opts(tol=1e-6, precision="mixed", max_iter=60000, max_outer=60)
    out = {"workload": args.workload, "precision": "mixed", "tol": 1e-6}
    if args.workload == 6:
        # the random-features method (features as the model) against kernel
        # ridge regression solved by Algorithm 1, and Algorithm 1 at larger
        # preconditioner ridges (Table 2's lambda_p)
        P = ks.make_config(2, m=M_TEST)
        X, W, b, Y, Xte = dev(P.X), dev(P.W), dev(P.b), dev(P.Y), dev(P.Xte)
        Yte = P.Yte
        Wf = torch.empty((P.s, 1), dtype=torch.float64, device="cuda")
        Fr = torch.empty((M_TEST, 1), dtype=torch.float64, device="cuda")
        K.krr_rfm_fit(h, X, W, b, P.lam, Y, Wf)   # warm-up (allocations)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        K.krr_rfm_fit(h, X, W, b, P.lam, Y, Wf)
        torch.cuda.synchronize()
        t_fit = time.perf_counter() - t0
        t0 = time.perf_counter()
        K.krr_rfm_predict(h, Xte, W, b, Wf, Fr)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
        fr = Fr.cpu().numpy()
        sweep = []
        fk = None
        for lp in (P.lam, 1e-2, 1.0):
            Cc = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
            o = K.default_opts(tol=1e-6, precision="mixed", max_iter=60000, max_outer=60,
                               lambda_p=lp)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = K.krr_pcg_solve(h, X, P.sigma, P.lam, W, b, Y, Cc, o, check=False)
            torch.cuda.synchronize()
            sweep.append({"lambda_p": lp, "s": time.perf_counter() - t0, "iters": r["iters"][0],
                          "outer_steps": r["outer_steps"], "status": r["status"],
                          "rel_res": r["rel_res"][0]})
            if fk is None:
                Fk = torch.empty((M_TEST, 1), dtype=torch.float64, device="cuda")
                K.krr_predict(h, X, Xte, P.sigma, Cc, Fk, "fp32")
                fk = Fk.cpu().numpy()
        rmse = lambda f: float(np.sqrt(np.mean((f - Yte) ** 2)))
        out.update({"n": P.n, "d": P.d, "s": P.s, "lambda": P.lam, "m": M_TEST,
                    "rfm_fit_s": t_fit, "rfm_predict_s": t_pred,
                    "heldout_rmse_rfm": rmse(fr), "heldout_rmse_krr": rmse(fk),
                    "rfm_vs_krr_rel": float(np.linalg.norm(fr - fk) / np.linalg.norm(fk)),
                    "pcg_lambda_p": sweep})
        h.close()
        print(json.dumps(out))
        return
    if args.workload == 4:
        probs = ks.make_uneven()
        items, cs = [], []
        for P in probs:
            Cc = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
            cs.append(Cc)
            items.append((dev(P.X), P.sigma, P.lam, dev(P.W), dev(P.b), dev(P.Y), Cc))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = K.krr_pcg_solve_batched(h, items, opts, check=False)
        torch.cuda.synchronize()
        out.update({"s": time.perf_counter() - t0, "ms_setup": reps[0]["ms_setup"],
                    "problems": len(probs),
                    "converged": sum(r["status_code"] == K.KRR_OK for r in reps),
                    "max_iters": max(r["iters"][0] for r in reps),
                    "max_rel_res": max(r["rel_res"][0] for r in reps),
                    "sum_n2": float(sum(P.n ** 2 for P in probs)),
                    "not_converged": [
                        {"problem": i, "n": P.n, "d": P.d, "lam": P.lam, "s": P.s,
                         "status": r["status"], "iters": r["iters"][0],
                         "outer_steps": r["outer_steps"], "rel_res": r["rel_res"][0]}
                        for i, (P, r) in enumerate(zip(probs, reps))
                        if r["status_code"] != K.KRR_OK]})
    else:
        P = ks.make_config(args.workload)
        Cc = torch.zeros((P.n, P.k), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = K.krr_pcg_solve(h, dev(P.X), P.sigma, P.lam, dev(P.W), dev(P.b), dev(P.Y), Cc, opts,
                            check=False)
        torch.cuda.synchronize()
        out.update({"n": P.n, "d": P.d, "k": P.k, "s": P.s, "solve_s": time.perf_counter() - t0,
                    "status": r["status"], "iters": r["iters"], "outer_steps": r["outer_steps"],
                    "ms_setup": r["ms_setup"], "rel_res": max(r["rel_res"])})
        if args.workload == 5:
            # the held-out loss gradient: adjoint solve and (D o K) products
            m = P.Xte.shape[0]
            F = torch.empty((m, 1), dtype=torch.float64, device="cuda")
            K.krr_predict(h, dev(P.X), dev(P.Xte), P.sigma, Cc, F, "hp")
            GF = (2.0 / m) * (F - dev(P.Yte))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            (gs, gl), rg = K.krr_hypergrad(h, dev(P.X), dev(P.Xte), P.sigma, P.lam, dev(P.W),
                                           dev(P.b), Cc, GF, opts, check=False)
            torch.cuda.synchronize()
            out.update({"grad_s": time.perf_counter() - t0, "dlogsigma": gs, "dloglambda": gl,
                        "adjoint_status": rg["status"], "adjoint_iters": rg["iters"]})
    h.close()
    print(json.dumps(out))


# ----------------------------------------------------------------- ours ---
def run_ours(args, rank, world, local):
    import torch
    from paper_1611_03220_gb300 import build
    build()
    from paper_1611_03220_gb300 import _krr as K

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n or ks.CONFIGS[2]
    P = ks.make_config(2, n=n, m=M_TEST)
    X = torch.from_numpy(P.X).to(dev)
    Y = torch.from_numpy(P.Y).to(dev)
    W = torch.from_numpy(P.W).to(dev)
    b = torch.from_numpy(P.b).to(dev)
    Xte = torch.from_numpy(P.Xte).to(dev)
    C = torch.zeros_like(Y)
    F = torch.zeros((M_TEST, 1), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    h = K.Handle()
    # Algorithm 1 needs a few thousand PCG iterations on this workload (the
    # preconditioner is weak here, see the plain-CG entry), hence the budget.
    opts = K.default_opts(tol=P.tol, precision="mixed", max_iter=20000, max_outer=60)

    def step():
        C.zero_()
        rep = K.krr_pcg_solve(h, X, P.sigma, P.lam, W, b, Y, C, opts, check=False)
        K.krr_predict(h, X, Xte, P.sigma, C, F, "fp32")
        return rep

    for _ in range(args.warmup):
        rep = step()
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    launches0 = K._lib.krr_launch_count()
    st = torch.cuda.current_stream()
    times, reps = [], []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rep = step()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        reps.append(rep)
        flush.zero_()
    torch.cuda.synchronize()
    launches = K._lib.krr_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(times), world, dev)
    if world > 1:
        torch.distributed.barrier()
    rep = reps[-1]

    # ------------------------------------------ fused product, timed alone
    # (the inner solves' product: FP16 points on the tensor cores)
    Vf = torch.randn((n, 1), dtype=torch.float32, device=dev)
    Qf = torch.empty_like(Vf)
    for _ in range(3):
        K.krr_kernel_matvec(h, X, X, P.sigma, P.lam, Vf, Qf, "fp16")
    mv_ms = []
    for _ in range(10):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        K.krr_kernel_matvec(h, X, X, P.sigma, P.lam, Vf, Qf, "fp16")
        e1.record(st)
        e1.synchronize()
        mv_ms.append(e0.elapsed_time(e1))
    t_mv = statistics.median(mv_ms) * 1e-3
    pairs = float(n) * n
    d_pad = 64 * math.ceil(P.d / 64)
    n_pad = 256 * math.ceil(n / 256)
    alg_flops = 2.0 * pairs * (P.d + 1)
    # exp-bound roofline: the best measured rate of base-2 exponentials with the
    # MUFU ex2 and the FMA-pipe polynomial running side by side, over splits
    import ctypes
    r = ctypes.c_double()
    kms = ctypes.c_double()
    mix = {}
    for f in (0, 2, 4, 6, 8, 10, 12, 16):
        if K._lib.krr_bench_ex2_mix(h.ptr, 2048, f, ctypes.byref(r), ctypes.byref(kms)) == 0:
            mix[f] = r.value
    best_f = max(mix, key=mix.get)
    peak = mix[best_f]
    clk_mhz = clk.get("sm_mhz") or 2070.0
    achieved = pairs / t_mv
    # algorithmic bytes of one product: the FP16 points once, w, and the row sums
    alg_bytes = n_pad * d_pad * 2 + n * 4 + n * 4
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                "unit": "Gexp/s", "frac": achieved / peak,
                "frac_of_mufu_only": achieved / mix[0],
                "traffic": TC_DRAM_BYTES_N65536 if n == 65536 and P.d == 64 else None,
                "traffic_unit": "DRAM bytes per launch (ncu capture of bench.py --profile fp16)",
                "alg_bytes": alg_bytes,
                "kernel": "tc_matvec_kernel (+ w/reduce helpers)",
                "peak_basis": (f"measured: best combined MUFU ex2 + FMA-pipe polynomial exp2 "
                               f"rate over splits ({best_f} of 32 on the FMA pipe), "
                               f"152 SMs, clocks median {clk_mhz:.0f} MHz in the timed region"),
                "exp2_rates_by_fma_per_32": {str(k): v / 1e9 for k, v in mix.items()}}
    mv = {"ms": t_mv * 1e3, "pairs_per_s": achieved, "alg_tflops": alg_flops / t_mv / 1e12,
          "tensor_tflops": 2.0 * n_pad * n_pad * d_pad / t_mv / 1e12}

    # ------------- the tensor-bound product: workload 3's shape (d = 784, k = 10)
    c3 = None
    if n == ks.CONFIGS[2] and not args.no_c3:
        P3 = ks.make_config(3)
        X3 = torch.from_numpy(P3.X).to(dev)
        V3 = torch.randn((P3.n, P3.k), dtype=torch.float32, device=dev)
        Q3 = torch.empty_like(V3)
        for _ in range(3):
            K.krr_kernel_matvec(h, X3, X3, P3.sigma, P3.lam, V3, Q3, "fp16")
        c3_ms = []
        for _ in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            K.krr_kernel_matvec(h, X3, X3, P3.sigma, P3.lam, V3, Q3, "fp16")
            e1.record(st)
            e1.synchronize()
            c3_ms.append(e0.elapsed_time(e1))
        t3 = statistics.median(c3_ms) * 1e-3
        fl3 = 2.0 * P3.n * P3.n * (P3.d + P3.k)
        tpk, tpk_basis = tensor_peak_tflops()
        c3 = {"workload": f"n={P3.n} d={P3.d} k={P3.k} sigma={P3.sigma} (FP16 points)",
              "ms": t3 * 1e3, "alg_tflops": fl3 / t3 / 1e12,
              "roofline": {"bound": "tensor", "achieved": fl3 / t3 / 1e12, "peak": tpk,
                           "unit": "TFLOP/s", "frac": fl3 / t3 / 1e12 / tpk,
                           "peak_basis": tpk_basis,
                           "flops": "2 n^2 (d + k) per product"}}
        del X3, V3, Q3

    # ------------------------------------------------ FP32 comparator ------
    fp32 = None
    if not args.no_fp32:
        C32 = torch.zeros_like(Y)
        o32 = K.default_opts(tol=P.tol, precision="fp32")
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r32 = K.krr_pcg_solve(h, X, P.sigma, P.lam, W, b, Y, C32, o32, check=False)
        torch.cuda.synchronize()
        fp32 = {"ms": (time.perf_counter() - t0) * 1e3, "status": r32["status"],
                "iters": r32["iters"][0], "rel_res_fp64_check": r32["rel_res"][0]}

    # ---------------------------------- plain CG (M = I, Table 4's comparator)
    plain_cg = {}
    for prec in ("mixed",) + (() if args.no_fp32 else ("fp32",)):
        Cc = torch.zeros_like(Y)
        oc = K.default_opts(tol=P.tol, precision=prec, precond=0)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = K.krr_pcg_solve(h, X, P.sigma, P.lam, W, b, Y, Cc, oc, check=False)
        torch.cuda.synchronize()
        plain_cg[prec] = {"ms": (time.perf_counter() - t0) * 1e3, "status": rc["status"],
                          "iters": rc["iters"][0], "outer_steps": rc["outer_steps"],
                          "rel_res_fp64_check": rc["rel_res"][0]}

    # --------------------- Algorithm 1 with a larger preconditioner ridge ---
    # (Table 2's lambda_p; the timed headline keeps lambda_p = lambda)
    Ct = torch.zeros_like(Y)
    ot = K.default_opts(tol=P.tol, precision="mixed", max_iter=20000, max_outer=60, lambda_p=1.0)
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rt = K.krr_pcg_solve(h, X, P.sigma, P.lam, W, b, Y, Ct, ot, check=False)
    torch.cuda.synchronize()
    tuned = {"lambda_p": 1.0, "ms": (time.perf_counter() - t0) * 1e3, "status": rt["status"],
             "iters": rt["iters"][0], "outer_steps": rt["outer_steps"],
             "rel_res_fp64_check": rt["rel_res"][0]}

    # ------------------------------------------------ end to end (host) ----
    Xh, Yh, Wh, bh = P.X, P.Y, P.W, P.b
    Xteh = P.Xte
    Ch = np.zeros((n, 1))
    Fh = np.zeros((M_TEST, 1))
    e2e_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        K.krr_pcg_solve(h, Xh, P.sigma, P.lam, Wh, bh, Yh, Ch, opts, check=False)
        K.krr_predict(h, Xh, Xteh, P.sigma, Ch, Fh, "fp32")
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = Xh.nbytes + Yh.nbytes + Wh.nbytes + bh.nbytes + Xh.nbytes + Xteh.nbytes + Ch.nbytes
    d2h = Ch.nbytes + Fh.nbytes

    cpu = None
    rel_res_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the headline solution's true residual recomputed by the FP64 oracle
        from oracle import krr_oracle as O
        rel_res_oracle = float(O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma,
                                                   P.lam)[0])
        cpu = cpu_baseline(P)

    if rank == 0:
        out = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp16+f64",
            "data": "synthetic",
            "config": bench_config(P, n, world),
            "solve": {"status": rep["status"], "iters": rep["iters"][0],
                      "kappa_estimate": rep["kappa"][0],
                      "outer_steps": rep["outer_steps"], "matvecs": rep["matvecs"],
                      "rel_res_fp64": rep["rel_res"][0], "rel_res_oracle": rel_res_oracle,
                      "ms_setup": rep["ms_setup"],
                      "ms_solve": rep["ms_solve"], "step_ms_all": times},
            "fp32": fp32, "plain_cg": plain_cg, "pcg_lambda_p_1": tuned, "kernel_matvec": mv, "roofline": roofline,
            "kernel_matvec_c3": c3,
            "cpu_baseline": cpu,
            "e2e": {"value": statistics.mean(e2e_ms), "unit": "ms", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clk, "gpu_launches": launches,
        }
        if world > 1:
            out["aggregate_solves_per_s"] = world * 1000.0 / ms
        print(json.dumps(out))
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.oracle_config1:
        print(json.dumps(oracle_alg1(ks.make_config(1))))
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile:
        run_profile(args)
        return
    if args.workload:
        run_workload(args)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
