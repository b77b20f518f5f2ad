"""Benchmark: Hopf solves/sec at duality gap <= 1e-5 on one GB300 (or N).

Workload (one step): the batched FP32 value solve of the generalized Hopf
formula for 65,536 query points x ~ N(0, 4 I) of one random n=10, m=2 system
(A ~ N(0, 1/n) - 0.5 I, B ~ N(0, 1), unit-ball control, ellipsoid target
Q = diag U[1, 4]) at horizon t = 2 with 256 left-Riemann nodes: node-table
build, warm-start network prediction of p*, persistent primal-dual kernel
(accelerated steps, two phases) from the prediction, and a cold re-solve of
any point the warm solve leaves uncertified; every point is certified to
relative gap <= 1e-5.  The network is trained before timing on 262,144 other
points labelled by the solver itself.  The same line reports the cold-start
solves (the paper's iteration of Eq. 15, and the accelerated one) on the same
GB300 for comparison.  Inputs are seeded and synthetic.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --workload chain|dimension ...   (secondary workloads: the
       100-mass spring chain on the tiled large-state kernel; 60 stacked
       double-integrator copies on the structured stacked-copy kernel)
Under torchrun each rank solves its own 65,536 points (weak scaling, no
collective on the data path; one barrier and a max-reduction of the timings).
The reference arm times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from inputs import workloads as wl  # noqa: E402

METRIC = "Hopf solves/sec at gap<=1e-5: warm-start batched vs plain cold PDHG, same GB300"
POINTS = 65536
TOL = 1e-5
MAX_ITER_DEFAULT = 400000
TAU_ACCEL = 2.0
TAU_TERM = 0.5       # Eq. 15 in terminal-time variables (oracle sweep: mean 80 iterations vs 110 at 0.3)
# the learned warm start on the 100-mass chain (n = 200, m = 10 box, N = 512):
# value solves at T = 10 for 65,536 fresh points (seed 5); labels from seed 4
C4 = dict(points=65536, T=10.0, N=512, tau=0.1, tau_paper=0.5, train_points=262144, train_epochs=150,
          plain_points=2048)
PARK_TERM = 256
TRAIN_POINTS = 262144
TRAIN_EPOCHS = 60


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload(rank, points=POINTS):
    # rank r solves its own seeded points; rank 0 is the standard point set
    from paper_1712_08226_gb300 import shard
    return wl.workload_random10(points, seed_sys=1, seed_pts=shard.rank_point_seed(rank))


def flops_per_point_iter(n, m, N):
    """Algorithmic FLOPs of one primal-dual iteration for one point: the two
    node-table products K pbar and K^T y (2 N m n each) and the n x n prox
    product S v (2 n^2)."""
    return 4 * N * m * n + 2 * n * n


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(n_points, seconds_hint=20.0):
    """Times the FP64 oracle (as it stands) on the first n_points of the
    workload in a fresh single-threaded process.  Returns (solves/s, desc)."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
from inputs import workloads as wl
from oracle import hopf as oh
w = wl.workload_random10({n_points})
t0 = time.perf_counter()
r = oh.value(w["system"], w["x"], w["t"], w["N"], w["rule"], tau=w["tau"], tol={TOL}, max_iter=100000)
dt = time.perf_counter() - t0
print(json.dumps(dict(dt=dt, ok=int((r["status"] == 0).sum()), iters=float(r["iters"].mean()))))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=max(600, 20 * seconds_hint))
    if out.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + out.stderr[-2000:])
    d = json.loads(out.stdout.strip().splitlines()[-1])
    return d["ok"] / d["dt"], d


def _oracle_slice(job):
    """Worker of the all-core oracle timing: solves points [lo, hi) of the
    headline workload with the FP64 oracle (one thread) and reports the time."""
    lo, hi = job
    from oracle import hopf as oh
    w = wl.workload_random10(hi)
    t0 = time.perf_counter()
    r = oh.value(w["system"], w["x"][lo:hi], w["t"], w["N"], w["rule"], tau=w["tau"], tol=TOL, max_iter=100000)
    return time.perf_counter() - t0, int((r["status"] == 0).sum()), float(r["iters"].sum())


def _oracle_chain_slice(job):
    """Worker of the all-core oracle timing for the chain workload: points
    [lo, hi) of the fresh C4 points (seed 5), value at T = 10, the iteration
    of Eq. 15 in terminal-time variables (tau 0.1, the GPU's cold iteration;
    in the paper's variable the oracle needs ~14,000 iterations, ~60 s, per
    point)."""
    lo, hi = job
    from oracle import hopf as oh
    x = wl.normal_points(5, hi, 200, 1.0)[lo:hi]
    t0 = time.perf_counter()
    r = oh.value(wl.spring_chain(), x, C4["T"], C4["N"], oh.LEFT_RIEMANN, tau=C4["tau"], tol=TOL,
                 max_iter=400000, variables="terminal")
    return time.perf_counter() - t0, int((r["status"] == 0).sum()), float(r["iters"].sum())


def _oracle_warm(_):
    from oracle import hopf  # noqa: F401
    return 0


class OraclePool:
    """One single-threaded oracle process per host core (spawned before any
    CUDA work); a step hands each process its own slice of the points."""

    def __init__(self, procs=None, fn=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                                "CUDA_VISIBLE_DEVICES")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
        self.pool = mp.get_context("spawn").Pool(self.procs)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        self.fn = fn or _oracle_slice
        self.pool.map(_oracle_warm, range(self.procs))                # imports

    def step(self, per_proc):
        """Wall time and certified solves of procs x per_proc points."""
        jobs = [(k * per_proc, (k + 1) * per_proc) for k in range(self.procs)]
        t0 = time.perf_counter()
        out = self.pool.map(self.fn, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        return wall, sum(o[1] for o in out), sum(o[2] for o in out) / (self.procs * per_proc)

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference_c4(args):
    """Reference arm for the default workload: the FP64 oracle on the host
    cores, one process per core, one chain point per process and step."""
    pool = OraclePool(fn=_oracle_chain_slice)
    times, ok_total, t_all, its = [], 0, 0.0, []
    for step in range(args.warmup + args.steps):
        dt, ok, it = pool.step(1)
        if step >= args.warmup:
            times.append(dt)
            ok_total += ok
            t_all += dt
            its.append(it)
    pool.close()
    value = ok_total / t_all
    desc = (f"FP64 numpy oracle (Eq. 15 in terminal-time variables, tau {C4['tau']}), one process per host core "
            f"({pool.procs} cores, 1 thread each), {pool.procs} of the {C4['points']} chain points per step, "
            f"gap<=1e-5, mean {statistics.mean(its):.0f} iterations")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"c4_warm_start_spring_chain_n200_m10_box_N512_T10_value_{C4['points']}pts",
                       "n": 200, "m": 10, "N": C4["N"], "t": C4["T"], "points": C4["points"],
                       "sample_points_per_step": pool.procs, "tol_gap": TOL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": pool.procs, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    if args.workload == "c4":
        run_reference_c4(args)
        return
    pool = OraclePool()
    per_proc = 48
    sample = per_proc * pool.procs
    times, ok_total, t_all = [], 0, 0.0
    for step in range(args.warmup + args.steps):
        dt, ok, _ = pool.step(per_proc)
        if step >= args.warmup:
            times.append(dt)
            ok_total += ok
            t_all += dt
    pool.close()
    value = ok_total / t_all
    desc = (f"FP64 numpy oracle (the paper's iteration, Eq. 15), one process per host core "
            f"({pool.procs} cores, 1 thread each), {sample} of the {POINTS} points per step, "
            f"gap<=1e-5, same system/t/N/tau")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "random_n10_m2_t2_N256_65536pts", "n": 10, "m": 2, "N": 256, "t": 2.0,
                       "points": POINTS, "sample_points_per_step": sample, "tol_gap": TOL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": pool.procs, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def train_warm_start(H, sysd, w, rank):
    """Untimed set-up: label 262,144 fresh points with the GPU solver (cold,
    terminal-time variables, gap 2e-6) and train the warm-start network on
    them with the library's own forward/backward/Adam kernels."""
    import torch
    from paper_1712_08226_gb300.warmstart import WarmStartNet
    t0 = time.perf_counter()
    xtr = torch.tensor(wl.normal_points(40 + 1000 * rank, TRAIN_POINTS, 10, 2.0), dtype=torch.float32,
                       device="cuda")
    lab = H.value(sysd, xtr, w["t"], H.Options(N=w["N"], tau=TAU_TERM, tol_gap=2e-6,
                                               variables=H.VARS_TERMINAL))
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    net = WarmStartNet(10, 10, hidden=256, seed=0)
    net.set_normalisation(xtr, lab["p"])
    t0 = time.perf_counter()
    hist = net.fit(xtr, lab["p"], epochs=TRAIN_EPOCHS, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    info = {"train_points": TRAIN_POINTS, "label_s": round(t_label, 2), "epochs": TRAIN_EPOCHS, "batch": 4096,
            "train_s": round(time.perf_counter() - t0, 2), "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
            "network": "10-256-256-10 GELU, bf16 weights, fp32 accumulation"}
    return net, info


def oracle_sample_seconds(code_body, timeout=900):
    """Runs an oracle timing snippet in a fresh single-threaded process; it
    prints one JSON dict with dt (s) and ok (certified points)."""
    code = f"import os, sys, time, json\nsys.path.insert(0, {ROOT!r})\n" + code_body
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


SECONDARY = {
    # 100-mass spring chain, value at a shared horizon: the tiled large-state kernel
    "chain": dict(points=4096, T=10.0, N=512, tau=0.5, tau_terminal=0.1, cpu_points=1),
    # 60 double-integrator samples sharing one control (d = 120): the structured
    # stacked-copy solve, with the dense stacked system as comparison
    "dimension": dict(points=16384, T=2.5, d=120, cpu_points=2),
    # the first --systems of the 64 random systems (n = 4..128, m = ceil(n/8),
    # 1000-4000 points each, t = 2, N = 256), solved one system per call
    # (terminal-time variables unless --paper-variables: tau 0.5 for n <= 16,
    # 1.0 above, from an oracle sweep of 0.15-6 on four of the systems)
    "ragged": dict(T=2.0, N=256, tau=0.15, tau_small=0.5, tau_large=1.0, cpu_points=1),
}


def ragged_tau(cfg, n, paper_variables):
    """Primal step of one ragged system: the paper's variable keeps one tau;
    terminal-time variables take 0.5 for n <= 16 and 1.0 above."""
    if paper_variables:
        return cfg["tau"]
    return cfg["tau_small"] if n <= 16 else cfg["tau_large"]


def run_secondary(args):
    """One JSON line for a secondary workload (same timing rules as the
    headline: W warm-up steps, K timed steps, L2 flushed before each, CUDA
    events on the launching stream, clocks sampled)."""
    cfg = SECONDARY[args.workload]
    rank, world, local = rank_env()
    points = args.points if args.points != POINTS else cfg.get("points", 0)
    if args.workload == "chain":
        sysd = wl.spring_chain()
        x = wl.normal_points(3 + 1000 * rank, points, 200, 1.0)
        n, m, N, T = 200, 10, cfg["N"], cfg["T"]
        tau = cfg["tau"] if args.paper_variables else cfg["tau_terminal"]
        fpi = flops_per_point_iter(n, m, N)
        wname = f"spring_chain_n200_m10_box_N512_T10_{points}pts"
        kernel = "pdhg_tile_kernel<10,1>"
        cpu_code = (f"from inputs import workloads as wl\nfrom oracle import hopf as oh\n"
                    f"x = wl.normal_points(3, {cfg['cpu_points']}, 200, 1.0)\nt0 = time.perf_counter()\n"
                    f"r = oh.value(wl.spring_chain(), x, {T}, {N}, oh.LEFT_RIEMANN, tau={cfg['tau']}, tol={TOL}, "
                    f"max_iter=200000, accel={bool(args.accel)})\n"
                    f"print(json.dumps(dict(dt=time.perf_counter() - t0, ok=int((r['status'] == 0).sum()))))\n")
    elif args.workload == "ragged":
        wr = wl.workload_ragged()
        items = wr["items"][:args.systems]
        N, T, tau, m = cfg["N"], cfg["T"], cfg["tau"], None
        n = max(it["system"]["A"].shape[0] for it in items)
        points = sum(len(it["x"]) for it in items)
        fpi = None
        wname = f"ragged_random_systems_first{len(items)}_of_64_N256_t2_{points}pts"
        kernel = "pdhg_tile_kernel (n > 16) / pdhg_small_kernel (n <= 16)"
        s0 = items[0]["system"]
        tau0 = ragged_tau(cfg, s0["A"].shape[0], args.paper_variables)
        cpu_code = (f"from inputs import workloads as wl\nfrom oracle import hopf as oh\n"
                    f"it = wl.workload_ragged()['items'][0]\nt0 = time.perf_counter()\n"
                    f"r = oh.value(it['system'], it['x'][:{cfg['cpu_points']}], {T}, {N}, oh.LEFT_RIEMANN, "
                    f"tau={tau0}, tol={TOL}, max_iter=200000, "
                    f"variables={'initial' if args.paper_variables else 'terminal'!r})\n"
                    f"print(json.dumps(dict(dt=time.perf_counter() - t0, ok=int((r['status'] == 0).sum()))))\n")
        x = None
    else:
        w = wl.workload_dimension(cfg["d"], points, seed=13 + 1000 * rank)
        sysd = w["system"]
        x = w["x"]
        nb, k, m, N, T, tau = 2, cfg["d"] // 2, 1, w["N"], cfg["T"], w["tau"]
        n = nb * k
        fpi = 4 * N * m * nb + 2 * k * nb * nb
        wname = f"dimension_scaling_d{cfg['d']}_N100_T2.5_{points}pts"
        kernel = "pdhg_stacked_kernel<float>"
        cpu_code = (f"from inputs import workloads as wl\nfrom oracle import hopf as oh\n"
                    f"w = wl.workload_dimension({cfg['d']}, {cfg['cpu_points']})\nt0 = time.perf_counter()\n"
                    f"r = oh.value(w['system'], w['x'], {T}, w['N'], w['rule'], tau=w['tau'], tol={TOL}, "
                    f"max_iter=200000)\n"
                    f"print(json.dumps(dict(dt=time.perf_counter() - t0, ok=int((r['status'] == 0).sum()))))\n")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        d = oracle_sample_seconds(cpu_code)
        cpu = {"value": d["ok"] / d["dt"], "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"FP64 numpy oracle{' (dense stacked system)' if args.workload == 'dimension' else ''}, "
                         f"1 thread, {cfg['cpu_points']} point(s) of the workload"
                         f"{' (first system)' if args.workload == 'ragged' else ''}, gap<=1e-5, {d['dt']:.1f} s"}
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://", device_id=torch.device("cuda", local))
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    H._lib.load()
    accel = bool(args.accel)
    if args.workload == "ragged":
        run_ragged(args, H, items, cfg, cpu, rank, world, local, dist, wname, kernel, N, T, tau)
        return
    x_dev = torch.tensor(x, dtype=torch.float32, device="cuda")
    variables = H.VARS_TERMINAL if (args.workload == "chain" and not args.paper_variables) else H.VARS_INITIAL
    opts = H.Options(N=N, tau=tau, tol_gap=TOL, max_iter=args.max_iter, profile=True, accel=accel,
                     variables=variables, kernel={"auto": 0, "tensor": 2, "tile": 3}[args.kernel])
    warm_info = None
    if args.workload == "chain" and args.warm:
        # untimed set-up: label seeded training points with the GPU solver
        # (certified ones only) and train the 200-256-256-200 network
        from paper_1712_08226_gb300.warmstart import WarmStartNet, value_warm
        S = H.System.from_dict(sysd)
        t0 = time.perf_counter()
        xtr = torch.tensor(wl.normal_points(4 + 1000 * rank, args.train_points, n, 1.0), dtype=torch.float32,
                           device="cuda")
        lab = H.value(S, xtr, T, H.Options(N=N, tau=tau, tol_gap=TOL, max_iter=60000))
        okm = lab["status"] == 0
        xtr, ptr = xtr[okm].contiguous(), lab["p"][okm].contiguous()
        torch.cuda.synchronize()
        t_label = time.perf_counter() - t0
        net = WarmStartNet(n, n, hidden=256, seed=0)
        net.set_normalisation(xtr, ptr)
        t0 = time.perf_counter()
        hist = net.fit(xtr, ptr, epochs=args.train_epochs, batch=1024, lr=2e-3)
        torch.cuda.synchronize()
        warm_info = {"train_points": int(xtr.shape[0]), "label_s": round(t_label, 1), "epochs": args.train_epochs,
                     "train_s": round(time.perf_counter() - t0, 1), "loss_first_epoch": hist[0],
                     "loss_last_epoch": hist[-1], "network": "200-256-256-200 GELU, bf16 weights, fp32 accumulation"}
        call = lambda xx: value_warm(S, xx, T, net, opts)     # noqa: E731
        dense_call = None
    elif args.workload == "chain":
        S = H.System.from_dict(sysd)
        call = lambda xx: H.value(S, xx, T, opts)            # noqa: E731
        dense_call = None
    else:
        base = H.System.from_dict(sysd["base"])
        Sd = H.System.from_dict(sysd)
        call = lambda xx: H.value_stacked(base, sysd["W_blocks"], xx, T, opts)   # noqa: E731
        dense_call = lambda xx: H.value(Sd, xx, T, opts)                         # noqa: E731
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(f, steps):
        ms, sv, un, ok, its = [], [], 0, 0, None
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = f(x_dev)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            # the value path records events around its solve kernel; the
            # stacked path is one table build and one kernel: use the step
            sv.append(H.last_profile()[1] if f is not call or args.workload == "chain" else ms[-1])
            it = r["iters"].to(torch.int64)
            un += int((it + 1).sum().item())
            ok += int((r["status"] == 0).sum().item())
            its = it.cpu().numpy()
        return dict(ms=ms, solve_ms=sv, units=un, ok=ok, iters=its)

    for _ in range(args.warmup):
        call(x_dev)
    torch.cuda.synchronize()
    compare = None
    if dense_call is not None and not args.no_compare:
        dense_call(x_dev)
        rd = timed(dense_call, 1)
        compare = {"dense_stacked_solves_per_s": rd["ok"] / (rd["ms"][0] * 1e-3), "dense_ms": rd["ms"][0],
                   "dense_mean_iters": float(rd["iters"].mean()), "kernel": "pdhg_tile_kernel<1,2>"}
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    res = timed(call, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    x_pin = torch.tensor(x, dtype=torch.float32).pin_memory()
    e2e_s, ok_e2e = [], 0
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        t0 = time.perf_counter()
        xd = x_pin.to("cuda", non_blocking=True)
        rh = call(xd)
        phi_h, st_h = rh["phi"].cpu(), rh["status"].cpu()
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_s.append(dt)
            ok_e2e = int((st_h == 0).sum())
    if not e2e_s:
        e2e_s = [float("nan")]
    from paper_1712_08226_gb300 import shard
    t_local = shard.reduce_max([statistics.mean(res["ms"]), statistics.mean(e2e_s) * 1e3], dist,
                               device="cuda" if dist else None)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    value = shard.job_throughput(res["ok"] / args.steps, world, t_local[0] * 1e-3)
    achieved = res["units"] / args.steps * fpi / (statistics.mean(res["solve_ms"]) * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    line = {
        "metric": f"Hopf solves/sec at gap<=1e-5 ({args.workload} workload)", "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(t_local[0]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded)",
        "config": {"workload": wname, "n": n, "m": m, "N": N, "t": T, "points_per_gpu": points, "tol_gap": TOL,
                   "tau": tau, "iteration": "accelerated (strongly convex G)" if accel else "Eq. 15 (theta = 1)",
                   "variables": "terminal-time q (p = e^{TA^T} q)" if variables else "paper's p",
                   "l2": "flushed between timed steps (512 MB write)",
                   "mean_iters": float(res["iters"].mean()), "max_iters": int(res["iters"].max()),
                   "certified_per_step": res["ok"] / args.steps, "ms_solve": statistics.mean(res["solve_ms"]),
                   "comparison": compare, "warm_start": warm_info},
        "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {max_mhz:.0f} MHz (max SM clock)",
                     "flops_per_point_iter": fpi,
                     "point_iters_per_s": res["units"] / args.steps / (statistics.mean(res["solve_ms"]) * 1e-3)},
        "cpu_baseline": cpu,
        "e2e": {"value": shard.job_throughput(ok_e2e, world, t_local[1] * 1e-3), "unit": "solves/s",
                "h2d_bytes_per_step": points * n * 4, "d2h_bytes_per_step": points * 8},
        # chain: horizons, tables, pad, tiled solve, tail; dimension: horizons,
        # expand, tables, stacked solve.  The warm start adds the network
        # (standardise + 3 tensor-core GEMMs), 3 ordering kernels, the fallback
        # list and a second pad + solve + tail
        "gpu_launches": (16 if warm_info else (5 if args.workload == "chain" else 4)) * args.steps
                        + (2 * args.steps if variables else 0),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_ragged(args, H, items, cfg, cpu, rank, world, local, dist, wname, kernel, N, T, tau):
    """Secondary line for the ragged systems: one hopf_value call per system
    per step (each with its own node table), timed together."""
    import torch
    xs = [torch.tensor(it["x"], dtype=torch.float32, device="cuda") for it in items]
    systems = [H.System.from_dict(it["system"]) for it in items]
    variables = H.VARS_INITIAL if args.paper_variables else H.VARS_TERMINAL
    taus = [ragged_tau(cfg, S.n, args.paper_variables) for S in systems]
    opts_of = [H.Options(N=N, tau=tu, tol_gap=TOL, max_iter=args.max_iter, profile=True, variables=variables)
               for tu in taus]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # systems overlap on the GPU: one stream per system slot (the library
    # keeps one workspace per stream), joined before the end event
    side = [torch.cuda.Stream() for _ in range(min(args.streams, len(systems)))]

    def step():
        out = []
        ev0 = torch.cuda.Event()
        ev0.record(stream)
        for i, (S, xd) in enumerate(zip(systems, xs)):
            st = side[i % len(side)]
            st.wait_event(ev0)
            with torch.cuda.stream(st):
                out.append(H.value(S, xd, T, opts_of[i], stream=st))
        for st in side:
            stream.wait_stream(st)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, ok, flops, its = [], 0, 0.0, []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        for S, r in zip(systems, rs):
            it = r["iters"].to(torch.int64)
            ok += int((r["status"] == 0).sum().item())
            flops += float((it + 1).sum().item()) * flops_per_point_iter(S.n, S.m, N)
            its.append(it.cpu().numpy())
    clk = clocks.stop()
    if rank != 0:
        return
    t = statistics.mean(ms) * 1e-3
    achieved = flops / args.steps / t / 1e12
    props = torch.cuda.get_device_properties(0)
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * max_mhz * 1e6 / 1e12
    its = np.concatenate(its)
    ns = [S.n for S in systems]
    line = {
        "metric": "Hopf solves/sec at gap<=1e-5 (ragged workload)", "value": ok / args.steps / t,
        "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": wname, "systems": len(systems), "n_per_system": ns, "N": N, "t": T,
                   "tau": "0.15" if args.paper_variables else "0.5 (n <= 16), 1.0 (n > 16)",
                   "variables": "paper's p" if args.paper_variables else "terminal-time q",
                   "tol_gap": TOL, "points": int(sum(len(x) for x in xs)), "streams": len(side),
                   "mean_iters": float(its.mean()),
                   "max_iters": int(its.max()), "certified_per_step": ok / args.steps,
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 FLOP x {max_mhz:.0f} MHz (max SM clock)",
                     "timing": "whole step (tables + solves; systems overlap on the side streams)"},
        "cpu_baseline": cpu,
        "e2e": None,
        # per system: horizons, tables and either pad + tiled solve + tail or
        # the three small-state phases
        "gpu_launches": 5 * len(systems) * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_chain_ttr(args):
    """Secondary line: minimum time to reach for the 100-mass chain (§IV),
    bisection or (--newton) the Newton hybrid on [0, --t-max], float32 solves
    to gap 1e-5, tol_T 1e-5, terminal-time variables (tau 0.1).  Default: the
    fixed-step rule (one table of 512 nodes on [0, 40]) for all 4,096 chain
    points with the accelerated steps (near phi = 0 at these horizons the
    plain iteration of Eq. 15 is far slower); --ttr-rule paper: Eq. 17 with
    N = 512 and one table per point and candidate (64 points;
    --paper-variables runs it in the paper's variable)."""
    rank, world, local = rank_env()
    import torch
    torch.cuda.set_device(local)
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    H._lib.load()
    fixed = args.ttr_rule == "fixed"
    P = args.points if args.points != POINTS else (4096 if fixed else 64)
    n, m = 200, 10
    N = 512
    sysd = H.System.from_dict(wl.spring_chain())
    x = torch.tensor(wl.normal_points(3 + 1000 * rank, P, n, 1.0), dtype=torch.float32, device="cuda")
    variables = H.VARS_INITIAL if (args.paper_variables and not fixed) else H.VARS_TERMINAL
    # per-solve cap: 40,000 unless given (each round waits for its slowest point)
    max_iter = args.max_iter if args.max_iter != MAX_ITER_DEFAULT else 40000
    o = H.Options(rule=H.LEFT_FIXED if fixed else H.LEFT_RIEMANN, N=N,
                  tau=0.5 if variables == H.VARS_INITIAL else 0.1, tol_gap=TOL, t_max=args.t_max, tol_T=1e-5,
                  max_iter=max_iter, newton=args.newton, variables=variables, accel=fixed)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        H.time_to_reach(sysd, x, o)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, ok, steps = [], 0, 0
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = H.time_to_reach(sysd, x, o)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        st = r["status"].cpu().numpy()
        ok += int(np.isin(st, (0, 4)).sum())
        steps = r["steps"]
    clk = clocks.stop()
    t = statistics.mean(ms) * 1e-3
    Tv = r["T"].cpu().numpy()
    line = {
        "metric": "time-to-reach solves/sec (chain workload)", "value": ok / args.steps / t, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": f"spring_chain_n200_m10_ttr_tmax{args.t_max:g}_"
                               f"{'fixedstep' if fixed else 'N'}{N}_{P}pts", "n": n, "m": m, "N": N,
                   "rule": "fixed step t_max/N (one table)" if fixed else "Eq. 17 (N nodes on [0, T])",
                   "t_max": args.t_max, "tol_gap": TOL, "tol_T": 1e-5, "points": P,
                   "variables": "paper's p" if variables == H.VARS_INITIAL else "terminal-time q",
                   "search": "newton hybrid" if args.newton else "certified bisection", "rounds": steps,
                   "status_counts": {str(k): int(v) for k, v in zip(*np.unique(r["status"].cpu().numpy(),
                                                                            return_counts=True))},
                   "T_mean": float(Tv.mean()), "T_max": float(Tv.max()), "accel": bool(fixed),
                   "max_iter": max_iter,
                   "final_gap_median": float(np.median(r["gap"].cpu().numpy())),
                   "final_gap_max": float(np.nanmax(r["gap"].cpu().numpy())),
                   "tables": "one float64 table on [0, t_max] for every point and candidate" if fixed else
                             "one float64 table per point and candidate horizon"},
        "roofline": None if fixed else
                    {"bound": "hbm", "kernel": "pdhg_generic_kernel<float> (per-point tables)", "achieved": None,
                     "peak": measured_peaks()[0]["hbm_gbs"], "unit": "GB/s", "frac": None, "traffic": None,
                     "note": "each point reads its own 4 MB float32 table twice per iteration; the step also "
                             "builds one float64 table per point and candidate"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def measured_peaks():
    """Measured peaks of this GPU pool (copy bandwidth, cuBLAS bf16), or
    the fallback figures when the file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def run_c4(args):
    """The learned warm start on the 100-mass spring chain: 65,536 fresh
    points, value solves at T = 10 (gap <= 1e-5) started from the network's
    prediction of p* in terminal-time variables on the tensor-core kernel, cold
    fallback; compared with the cold solve (same kernel) and with the paper's
    plain iteration (Eq. 15 in its own variable, CUDA-core tiled kernel) on the
    same GB300."""
    rank, world, local = rank_env()
    points = args.points if args.points != POINTS else C4["points"]
    n, m, N, T = 200, 10, C4["N"], C4["T"]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(fn=_oracle_chain_slice)
        per_proc = 2
        wall, ok_all, it_all = pool.step(per_proc)
        pool.close()
        cpu = {"value": ok_all / wall, "unit": "solves/s", "cores": pool.procs, "kind": "oracle",
               "sample": f"FP64 numpy oracle (Eq. 15 in terminal-time variables, tau {C4['tau']}): {pool.procs} "
                         f"processes x 1 thread, {per_proc} points each (the first {pool.procs * per_proc} of the "
                         f"{points} points), gap<=1e-5, {wall:.1f} s wall, mean {it_all:.0f} iterations",
               "single_core": {"ms_per_solve": 1e3 * wall / per_proc, "unit": "ms"}}
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://", device_id=torch.device("cuda", local))
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    from paper_1712_08226_gb300.warmstart import WarmStartNet, value_warm
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    H._lib.load()
    sysd = wl.spring_chain()
    S = H.System.from_dict(sysd)
    x = wl.normal_points(5 + 1000 * rank, points, n, 1.0)
    x_dev = torch.tensor(x, dtype=torch.float32, device="cuda")
    base = dict(N=N, tol_gap=TOL, gap_every=8, precision=H.FP32, profile=True)
    opts_warm = H.Options(tau=C4["tau"], max_iter=100000, variables=H.VARS_TERMINAL, **base)
    opts_cold = H.Options(tau=C4["tau"], max_iter=100000, variables=H.VARS_TERMINAL, **base)
    opts_plain = H.Options(tau=C4["tau_paper"], max_iter=400000, **base)
    # untimed set-up: labels from the GPU solver (cold, terminal-time
    # variables, gap 1e-5) on fresh seeded points; the network is trained by
    # the library's own forward/backward/Adam kernels
    t0 = time.perf_counter()
    tp = args.train_points if args.train_points != 8192 else C4["train_points"]
    xtr = torch.tensor(wl.normal_points(4 + 1000 * rank, tp, n, 1.0), dtype=torch.float32, device="cuda")
    lab = H.value(S, xtr, T, H.Options(tau=C4["tau"], max_iter=100000, variables=H.VARS_TERMINAL,
                                       **dict(base, profile=False)))
    okm = lab["status"] == 0
    xtr, ptr = xtr[okm].contiguous(), lab["p"][okm].contiguous()
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    epochs = args.train_epochs if args.train_epochs != 60 else C4["train_epochs"]
    net = WarmStartNet(n, n, hidden=256, seed=0)
    net.set_normalisation(xtr, ptr)
    t0 = time.perf_counter()
    hist = net.fit(xtr, ptr, epochs=epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    train_info = {"train_points": int(xtr.shape[0]), "label_s": round(t_label, 1), "epochs": epochs,
                  "train_s": round(time.perf_counter() - t0, 1), "loss_first_epoch": hist[0],
                  "loss_last_epoch": hist[-1], "network": "200-256-256-200 GELU, bf16 weights, fp32 accumulation"}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(f, xx, steps):
        ms, sv, un, ok, its, fb = [], [], 0, 0, None, 0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = f(xx)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            sv.append(H.last_profile()[1])
            it = r["iters"].to(torch.int64)
            un += int((it + 1).sum().item())
            ok += int((r["status"] == 0).sum().item())
            its = it.cpu().numpy()
            if "n_fallback" in r:
                fb = int(r["n_fallback"].item())
        return dict(ms=ms, solve_ms=sv, units=un, ok=ok, iters=its, fallback=fb)

    warm = lambda xx: value_warm(S, xx, T, net, opts_warm)          # noqa: E731
    cold = lambda xx: H.value(S, xx, T, opts_cold)                  # noqa: E731
    plain = lambda xx: H.value(S, xx, T, opts_plain)                # noqa: E731
    for _ in range(args.warmup):
        warm(x_dev)
    torch.cuda.synchronize()
    compare = {}
    if not args.no_compare:
        rc = timed(cold, x_dev, 1)
        compare["cold_terminal_tensor"] = {"solves_per_s": rc["ok"] / (rc["ms"][0] * 1e-3), "ms_per_step": rc["ms"][0],
                                           "mean_iters": float(rc["iters"].mean()), "max_iters": int(rc["iters"].max()),
                                           "points": points}
        xp = x_dev[:C4["plain_points"]].contiguous()
        rp = timed(plain, xp, 1)
        compare["plain_cold_paper_eq15"] = {"solves_per_s": rp["ok"] / (rp["ms"][0] * 1e-3), "ms_per_step": rp["ms"][0],
                                            "mean_iters": float(rp["iters"].mean()), "max_iters": int(rp["iters"].max()),
                                            "points": int(xp.shape[0]), "kernel": "pdhg_tile_kernel (CUDA cores)"}
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    res = timed(warm, x_dev, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    # end to end through the C ABI with host buffers (pinned), copies inside the call
    x_host = torch.tensor(x, dtype=torch.float32).pin_memory().numpy()
    e2e_s, ok_e2e = [], 0
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        t0 = time.perf_counter()
        rh = value_warm(S, x_host, T, net, opts_warm)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_s.append(dt)
            ok_e2e = int((rh["status"] == 0).sum())
    if not e2e_s:
        e2e_s = [float("nan")]
    from paper_1712_08226_gb300 import shard
    t_local = shard.reduce_max([statistics.mean(res["ms"]), statistics.mean(e2e_s) * 1e3], dist,
                               device="cuda" if dist else None)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    value = shard.job_throughput(res["ok"] / args.steps, world, t_local[0] * 1e-3)
    fpi = 4 * N * m * n + 2 * n                   # two table products + the diagonal prox
    solve_s = statistics.mean(res["solve_ms"]) * 1e-3
    achieved = res["units"] / args.steps * fpi / solve_s / 1e12
    pk, src = measured_peaks()
    peak = pk["bf16_tflops_sustained"] * 1.1 / 2.25
    iters = res["iters"]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(t_local[0]), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; 100-mass chain, x~N(0,I))",
        "config": {"workload": f"c4_warm_start_spring_chain_n200_m10_box_N512_T10_value_{points}pts",
                   "n": n, "m": m, "N": N, "t": T, "points_per_gpu": points, "tol_gap": TOL, "tau": C4["tau"],
                   "solve": "value at a shared horizon (a time-to-reach search per point at this size needs ~20 rounds of 1e4-iteration solves)",
                   "start": "warm (network prediction of p*), cold fallback",
                   "iteration": "Eq. 15 in terminal-time variables p = e^{TA^T} q, tensor-core kernel (3 x tf32)",
                   "l2": "flushed between timed steps (512 MB write)",
                   "mean_iters": float(iters.mean()), "p99_iters": float(np.percentile(iters, 99)),
                   "max_iters": int(iters.max()), "fallback_points": res["fallback"],
                   "certified_per_step": res["ok"] / args.steps, "ms_solve": statistics.mean(res["solve_ms"]),
                   "warm_start_training": train_info, "cold_start_comparison": compare},
        "roofline": {"bound": "tensor", "kernel": "pdhg_tc_kernel<10>", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"tf32 = {src} bf16 sustained {pk['bf16_tflops_sustained']} x 1.1/2.25 "
                                    f"(nominal tf32/bf16 ratio)",
                     "flops_per_point_iter": fpi, "flops_note": "algorithmic; the kernel runs 3 tf32 passes per product",
                     "point_iters_per_s": res["units"] / args.steps / solve_s},
        "cpu_baseline": cpu,
        "e2e": {"value": shard.job_throughput(ok_e2e, world, t_local[1] * 1e-3), "unit": "solves/s",
                "h2d_bytes_per_step": points * n * 4 + 4, "d2h_bytes_per_step": points * (4 * n + 16) + 4},
        # per warm step: horizons, table, standardise + 3 tensor-core GEMMs of the
        # network, 3 ordering kernels, map in, operand prep + tensor-core solve,
        # fallback list, fallback prep + solve, map back
        "gpu_launches": 16 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_trajectory(args):
    """Secondary line: optimal control and state samples (Eq. 27, 33) for the
    100-mass chain, 4,096 points, T = 10, S = 1,000 samples, from the
    certified p* of value solves at gap 1e-5 (terminal-time variables, tiled
    kernel; not timed).  Metric: trajectories per second."""
    rank, world, local = rank_env()
    import torch
    torch.cuda.set_device(local)
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    H._lib.load()
    P = args.points if args.points != POINTS else 4096
    n, m, N, T, S = 200, 10, 512, 10.0, 1000
    sysd = H.System.from_dict(wl.spring_chain())
    x = torch.tensor(wl.normal_points(3 + 1000 * rank, P, n, 1.0), dtype=torch.float32, device="cuda")
    r = H.value(sysd, x, T, H.Options(N=N, tau=0.1, tol_gap=TOL, max_iter=400000, variables=H.VARS_TERMINAL))
    certified = int((r["status"] == 0).sum().item())
    p = r["p"].contiguous()
    Tv = torch.full((P,), T, dtype=torch.float32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    o = H.Options()
    for _ in range(args.warmup):
        H.trajectory(sysd, x, Tv, p, S, o)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = H.trajectory(sysd, x, Tv, p, S, o)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    t = statistics.mean(ms) * 1e-3
    out_bytes = P * (S + 1) * (n + m) * 4
    fma64 = P * S * (2.0 * n * n + 2.0 * n * m)          # lambda and x recurrences, control product
    line = {
        "metric": "optimal trajectories/sec (chain workload, 1,001 samples each)", "value": P / t,
        "unit": "trajectories/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (recurrences), f32 (output)", "data": "synthetic (seeded)",
        "config": {"workload": f"spring_chain_n200_m10_T10_S1000_{P}pts", "n": n, "m": m, "S": S, "T": T,
                   "points": P, "output_bytes": out_bytes, "output_GBps": out_bytes / t / 1e9,
                   "l2": "flushed between timed steps (512 MB write)",
                   "p_source": f"certified value solves at gap {TOL:g} ({certified} of {P} certified)"},
        "roofline": {"bound": "alu", "kernel": "trajectory_kernel<float> (float64 recurrences)",
                     "achieved": 2 * fma64 / t / 1e12, "peak": 1.25, "unit": "TFLOP/s",
                     "frac": 2 * fma64 / t / 1e12 / 1.25, "traffic": None,
                     "peak_source": "nominal GB300 FP64 rate (not measured on this pool)",
                     "hbm_write_frac": out_bytes / t / 1e9 / 6795.8},   # measured copy bandwidth
        "cpu_baseline": None, "e2e": None, "gpu_launches": 3 * args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


w0_tau = wl.workload_random10(1)["tau"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--points", type=int, default=POINTS, help="points per GPU (smaller cases for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the cold-start comparison runs")
    ap.add_argument("--cold", action="store_true", help="time the cold accelerated solve instead of the warm one")
    ap.add_argument("--systems", type=int, default=8, help="ragged workload: how many of the 64 systems")
    ap.add_argument("--streams", type=int, default=8, help="ragged workload: systems in flight at once")
    ap.add_argument("--workload", default="c4",
                    choices=["c4", "random10", "chain", "dimension", "ragged", "trajectory", "chain_ttr"],
                    help="c4 (default): learned warm start on the 100-mass chain; random10: the n = 10 batch; "
                         "the others: secondary workloads")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tensor", "tile"],
                    help="chain workload: solve kernel for the large state")
    ap.add_argument("--accel", action="store_true", help="secondary chain workload: accelerated steps")
    ap.add_argument("--paper-variables", action="store_true",
                    help="chain workload: iterate in the paper's variable p instead of terminal-time variables")
    ap.add_argument("--warm", action="store_true", help="secondary chain workload: learned warm start")
    ap.add_argument("--newton", action="store_true", help="chain_ttr workload: Newton hybrid instead of bisection")
    ap.add_argument("--t-max", type=float, default=40.0, help="chain_ttr workload: upper end of the bracket")
    ap.add_argument("--ttr-rule", choices=["fixed", "paper"], default="fixed",
                    help="chain_ttr workload: fixed-step rule with one shared table, or Eq. 17 per point")
    ap.add_argument("--train-points", type=int, default=8192, help="chain warm start: labelled training points")
    ap.add_argument("--train-epochs", type=int, default=60, help="chain warm start: training epochs")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER_DEFAULT,
                    help="secondary workloads: iteration cap (small values only for profiler captures)")
    args = ap.parse_args()
    if args.workload == "trajectory" and args.impl == "ours":
        run_trajectory(args)
        return
    if args.workload == "chain_ttr" and args.impl == "ours":
        run_chain_ttr(args)
        return
    if args.workload == "c4" and args.impl == "ours":
        run_c4(args)
        return
    if args.workload not in ("random10", "c4") and args.impl == "ours":
        run_secondary(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = rank_env()

    # CPU baseline first (before any CUDA work): the FP64 oracle on one core
    # (fresh single-threaded process) and on every host core (one spawned
    # single-threaded process per core, each on its own slice of the points)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = 512
        v1, d = cpu_oracle_sample(sample)
        pool = OraclePool()
        per_proc = 96
        wall, ok_all, it_all = pool.step(per_proc)
        pool.close()
        cpu = {"value": ok_all / wall, "unit": "solves/s", "cores": pool.procs, "kind": "oracle",
               "sample": f"FP64 numpy oracle (the paper's iteration, Eq. 15, tau {w0_tau}): {pool.procs} processes x "
                         f"1 thread, {per_proc} points each ({pool.procs * per_proc} of the {POINTS} points), "
                         f"gap<=1e-5, {wall:.1f} s wall, mean {it_all:.0f} iterations",
               "single_core": {"value": v1, "unit": "solves/s", "cores": 1,
                               "ms_per_solve": 1e3 * d["dt"] / max(1, d["ok"]),
                               "sample": f"first {sample} points, {d['dt']:.1f} s"}}

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://", device_id=torch.device("cuda", local))
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    from paper_1712_08226_gb300.warmstart import value_warm
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    H._lib.load()

    points = args.points
    w = workload(rank, points)
    sysd = H.System.from_dict(w["system"])
    n, m, N = 10, 2, w["N"]
    x_dev = torch.tensor(w["x"], dtype=torch.float32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    # the paper's iteration (Eq. 15, theta = 1) from its cold start, in the
    # paper's variable: the plain cold baseline of the comparison
    opts_plain = H.Options(N=N, tau=w["tau"], tol_gap=TOL, max_iter=100000, gap_every=8, precision=H.FP32,
                           profile=True, accel=False, park_iters=512)
    # the accelerated iteration (strongly convex G), paper's variable, cold
    opts_accel = H.Options(N=N, tau=TAU_ACCEL, tol_gap=TOL, max_iter=100000, gap_every=8, precision=H.FP32,
                           profile=True, accel=True, park_iters=1024)
    # Eq. 15 in terminal-time variables, cold
    opts_cold = H.Options(N=N, tau=TAU_TERM, tol_gap=TOL, max_iter=100000, gap_every=8, precision=H.FP32,
                          profile=True, accel=False, park_iters=PARK_TERM, variables=H.VARS_TERMINAL)
    # warm start from the network, Eq. 15 in terminal-time variables, cold fallback
    opts_warm = H.Options(N=N, tau=TAU_TERM, tol_gap=TOL, max_iter=100000, gap_every=8, precision=H.FP32,
                          profile=True, accel=False, park_iters=PARK_TERM, variables=H.VARS_TERMINAL)

    net, train_info = (None, None) if args.cold else train_warm_start(H, sysd, w, rank)

    def call(kind):
        if kind == "warm":
            return value_warm(sysd, x_dev, w["t"], net, opts_warm)
        return H.value(sysd, x_dev, w["t"], {"cold": opts_cold, "plain": opts_plain, "accel": opts_accel}[kind])

    def timed(kind, steps):
        """Device time per step (CUDA events on the launching stream), L2 flushed before each."""
        ms, sv, tb, un, okc, iters_all, fb = [], [], [], 0, 0, None, 0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = call(kind)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            a, b_ = H.last_profile()
            tb.append(a)
            sv.append(b_)
            it = r["iters"].to(torch.int64)
            un += int((it + 1).sum().item())
            okc += int((r["status"] == 0).sum().item())
            iters_all = it.cpu().numpy()
            if "n_fallback" in r:
                fb = int(r["n_fallback"].item())
        return dict(ms=ms, solve_ms=sv, pre_ms=tb, units=un, ok=okc, iters=iters_all, fallback=fb)

    main_kind = "cold" if args.cold else "warm"
    for _ in range(args.warmup):
        call(main_kind)
    torch.cuda.synchronize()

    compare = {}
    if not args.no_compare:
        for kind in ("plain", "accel", "cold") if main_kind == "warm" else ("plain", "accel"):
            call(kind)
            rr = timed(kind, max(1, min(3, args.steps)))
            compare[kind] = {"solves_per_s": rr["ok"] / len(rr["ms"]) / (statistics.mean(rr["ms"]) * 1e-3),
                             "ms_per_step": statistics.mean(rr["ms"]), "mean_iters": float(rr["iters"].mean()),
                             "max_iters": int(rr["iters"].max()), "steps": len(rr["ms"])}

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    res = timed(main_kind, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    step_ms, solve_ms, pre_ms, units, ok, iters_last = (res["ms"], res["solve_ms"], res["pre_ms"], res["units"],
                                                        res["ok"], res["iters"])

    # end to end through the C ABI with host buffers (pinned), copies inside the call
    x_pin = torch.tensor(w["x"], dtype=torch.float32).pin_memory()
    x_host = x_pin.numpy()
    e2e_s, ok_e2e = [], 0
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        t0 = time.perf_counter()
        if main_kind == "warm":
            rh = value_warm(sysd, x_host, w["t"], net, opts_warm)
        else:
            rh = H.value(sysd, x_host, w["t"], opts_cold)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_s.append(dt)
            ok_e2e = int((rh["status"] == 0).sum())
    if not e2e_s:
        e2e_s = [float("nan")]

    from paper_1712_08226_gb300 import shard
    mean_ms = statistics.mean(step_ms)
    t_local = shard.reduce_max([mean_ms, statistics.mean(e2e_s) * 1e3], dist, device="cuda" if dist else None)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    solves_per_step = ok / args.steps
    value = shard.job_throughput(solves_per_step, world, t_local[0] * 1e-3)
    e2e_value = shard.job_throughput(ok_e2e, world, t_local[1] * 1e-3)

    fpi = flops_per_point_iter(n, m, N)
    achieved = units / args.steps * fpi / (statistics.mean(solve_ms) * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak = sms * 128 * 2 * max_mhz * 1e6 / 1e12          # FP32 FMA lanes x 2 FLOP x max SM clock
    h2d = points * n * 4 + 4
    d2h = points * (4 + 4 * n + 4 + 4 + 4) + (4 if main_kind == "warm" else 0)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(t_local[0]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; random n=10 system, x~N(0,4I))",
        "config": {"workload": f"random_n10_m2_t2_N256_{points}pts", "n": n, "m": m, "N": N, "t": w["t"],
                   "points_per_gpu": points, "tol_gap": TOL, "tau": TAU_TERM,
                   "start": "warm (network prediction), cold fallback" if main_kind == "warm" else "cold",
                   "iteration": "Eq. 15 in terminal-time variables p = e^{TA^T} q, three phases",
                   "l2": "flushed between timed steps (512 MB write)",
                   "mean_iters": float(iters_last.mean()), "p99_iters": float(np.percentile(iters_last, 99)),
                   "max_iters": int(iters_last.max()), "fallback_points": res["fallback"],
                   "certified_per_step": solves_per_step,
                   "ms_tables_and_prediction": statistics.mean(pre_ms), "ms_solve": statistics.mean(solve_ms),
                   "warm_start_training": train_info,
                   "cold_start_comparison": compare},
        "roofline": {"bound": "alu", "kernel": "pdhg_small_kernel<10,2,4> + <10,2,32>", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {max_mhz:.0f} MHz (max SM clock)",
                     "flops_per_point_iter": fpi,
                     "point_iters_per_s": units / args.steps / (statistics.mean(solve_ms) * 1e-3)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": (9 if main_kind == "warm" else 5) * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
