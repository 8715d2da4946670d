"""Benchmark: NFFT-accelerated tree Sinkhorn (Algorithm 2) on the 10-node d=2 path workload.

One step = one complete solve to marginal violation <= 1e-6 through the C ABI
(normalisation, binning, kernel Fourier coefficients, the Sinkhorn sweeps with NFFT
fast summation, stop tests and outputs), inputs already resident in device memory.
The metric is Sinkhorn iterations per second at that violation; the dense direct
path is measured beside it on the same workload, and the per-step latency is
reported as p50 / p99.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own copy of the workload (replicas:
the tree path has no exchange step) and rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Sinkhorn iters/s, NFFT vs dense BF16-split at marginal err≤1e-6; p50/p99 latency"
WORKLOAD = "path10_d2"
TOL = 1e-6
ROOT_CENTRE = -1             # Algorithm 2 rooted at a centre of the tree (fewest backward levels)
FLUSH_BYTES = 256 << 20      # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense comparison (profiling runs)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["path10_d2", "star9_d3", "path3_d1", "circle5_d1"],
                    help="profiling runs only: the reported line is defined on path10_d2")
    ap.add_argument("--path", default="nfft", choices=["nfft", "dense", "tc"],
                    help="profiling runs only: kernel path of the timed solves")
    ap.add_argument("--n", type=int, default=0, help="profiling runs only: points per marginal")
    ap.add_argument("--max-iter", type=int, default=5000, help="profiling runs only: iteration cap")
    ap.add_argument("--serving-requests", type=int, default=32,
                    help="requests of the Poisson-arrival serving replay (0: skip)")
    return ap.parse_args()


def reduce_over_ranks(total_s, iters, world, device=None):
    """Whole-job figures of `world` replicas: the slowest rank's timed seconds and the sum of the
    ranks' iterations (each rank solves its own copy; there is no exchange step)."""
    if world <= 1:
        return total_s, float(iters)
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_s], dtype=torch.float64, device=device)
    n = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t[0]), float(n[0])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: $MOT_CLOCKS_DIR if set, else the system temporary directory; the JSON
        # line carries their summary
        out_dir = os.environ.get("MOT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001 - clocks are reported as unavailable
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# algorithmic bytes of the fast-summation kernels (per launch, for the roofline)
# ----------------------------------------------------------------------------------------
def algorithmic_bytes(prob, n_grid):
    """Bytes the method must move per kernel product, by kernel class (FP32 values, FP64
    weights; window tables excluded), averaged over the forward (gamma, scaling update) and
    backward (beta) products of a sweep:

    spread : source coordinates (4 d N) + source factors (4 N each, 2 on average) + grid write (4 n^d)
    fftconv: grid read + grid write (8 n^d)
    gather : grid read (4 n^d) + target coordinates (4 d N) + target factors / message (8 N on
             average) + on forward products the scaling write and mu (16 N)
    fused  : spread + gather without the grid round trips (the grid stays in shared memory)
    """
    d, N = prob.d, prob.n[0]
    G = 4 * n_grid ** d
    spread = 4 * d * N + 8 * N + G
    gather = G + 4 * d * N + 8 * N + 8 * N          # forward products add 16 N, backward none
    return {"spread": spread, "gather": gather, "fftconv": 2 * G, "fused": spread + gather - 2 * G}


def circle1d_launch_bytes(prob, n_grid):
    """Bytes per launch of the batched 1-D circle kernels (one launch = the n_1 column products
    of a batch; equal point counts; window tables excluded):

    spread : the messages X (4 n_1 N) + phi (4 N) + the grid accumulation (4 n_1 n)
    gather : the grids (4 n_1 n) + the messages Y written (4 n_1 N)
    circle : the row dot of a scaling update reads beta_k and gamma_k (8 n_1 N) + phi^1 (4 n_1)
    """
    N = prob.n[0]
    G = 4 * N * n_grid
    return {"spread": 4 * N * N + 4 * N + G, "gather": G + 4 * N * N, "circle": 8 * N * N + 4 * N}


def products_per_solve(prob, iters, check_every):
    """Kernel products executed by one solve: the initial backward pass, 2(K-1) per sweep and
    the K-1 forward products of each check pass."""
    checks = -(-iters // check_every)
    return (1 + 2 * iters + checks) * (prob.K - 1)


def kernel_source_hash(cls):
    files = {"spread": ["nfft.cu", "common.cuh", "epilogue.cuh"], "gather": ["nfft.cu", "common.cuh", "epilogue.cuh"],
             "fused": ["nfft.cu", "common.cuh", "epilogue.cuh", "window.cuh"],
             "fftconv": ["nfft.cu", "fft_smem.cuh"], "dense": ["dense.cu", "common.cuh", "epilogue.cuh"]}.get(cls, [])
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2208_03120_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(cls, workload=WORKLOAD):
    """DRAM traffic per launch of the kernel class on a workload (default sizes) from the
    committed ncu summary, or None if there is none or the kernel source changed since the
    counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
        e = t.get(workload, {}).get(cls)
        if e and e.get("source_hash") == kernel_source_hash(cls):
            return e.get("dram_bytes_per_launch")
    except Exception:  # noqa: BLE001
        pass
    return None


# ----------------------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# ----------------------------------------------------------------------------------------
def oracle_rate(prob, budget_s=20.0, max_products=36):
    """Sweeps per second of the oracle's Algorithm 2 on the full workload, from a bounded
    sample: the sweep's kernel products (one beta and one gamma product per edge, the oracle's
    FP64 direct summation) run edge by edge, alternating matvec / rmatvec, until the budget is
    spent (at least one product); the O(N) scaling updates between them are not timed.
    Returns (sweeps/s, products timed, wall seconds, cores used)."""
    import numpy as np
    from oracle import sinkhorn as OS
    ts = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta)
    per_sweep = 2 * (ts.K - 1)
    t_cpu0 = time.process_time()
    t0 = time.perf_counter()
    done = 0
    while done < max_products and (done == 0 or time.perf_counter() - t0 < budget_s):
        k = 1 + (done // 2) % (ts.K - 1)
        ker = ts.Kpk[k]
        if done % 2 == 0:
            ker.matvec(np.ones(ker.shape[1]))
        else:
            ker.rmatvec(np.ones(ker.shape[0]))
        done += 1
    wall = time.perf_counter() - t0
    cpu = time.process_time() - t_cpu0
    return done / (wall * per_sweep), done, wall, max(1, round(cpu / wall))


def oracle_sample_text(prob, n_products, wall):
    return (f"{n_products} of the {2 * (prob.K - 1)} kernel products of one Algorithm-2 sweep (oracle FP64 "
            f"direct summation, {prob.n[0]}x{prob.n[0]} each) in {wall:.1f} s, scaled to one sweep; the "
            f"O(N) scaling updates are not timed")


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2208_03120_gb300 import workloads as W
    prob = W.path10_d2()
    rates = []
    for _ in range(max(1, args.steps)):
        r, nprod, wall, cores = oracle_rate(prob, budget_s=15.0 / max(1, args.steps) + 3.0)
        rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value if value else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": prob.K, "d": prob.d, "N": prob.n[0], "eta": prob.eta,
                   "topology": "path", "l2": "inputs in host memory (CPU run)"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: " + oracle_sample_text(prob, nprod, wall)},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tc_roofline(M, wp, wx, wm, topo, wo, wws, stream, flush):
    """Tensor-core roofline of the split-BF16 circle path: per GEMM launch the three BF16
    products of the batched column product, 3 x 2 n0 n_t n_s flops, over the launch's
    CUDA-event duration, against the measured dense BF16 peak (burst: each launch is short)."""
    import torch
    topt = M.options(path=M.MOT_PATH_DENSE_BF16X3, tol_viol=TOL, max_iter=3000, timing=1)
    with torch.cuda.stream(stream):
        flush.random_(0, 255)
    o = M.mot_solve(wx, wm, wp.eta, topo, edges=wp.edges, opt=topt, workspace=wws, stream=stream)
    torch.cuda.synchronize()
    n = wp.n
    # batches: Gam_k (k = 2..K-1) from Gam_{k-1}, beta_k (k = 1..K-2) from beta_{k+1}
    flops = [6.0 * n[0] * n[k] * n[k - 1] for k in range(2, wp.K)] + \
            [6.0 * n[0] * n[k] * n[k + 1] for k in range(1, wp.K - 1)]
    per_launch = sum(flops) / len(flops)
    launches = o.kernel_launches["tcgemm"]
    avg_s = o.kernel_ms["tcgemm"] / 1e3 / max(1, launches)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = per_launch / avg_s / 1e12
    total = sum(o.kernel_ms.values())
    return {"bound": "tensor", "kernel": "tcgemm", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "measured burst" if "bf16_tflops" in peaks else "fallback",
            "avg_launch_us": avg_s * 1e6, "alg_flops_per_launch": per_launch,
            "share": {k: round(v / total, 4) for k, v in o.kernel_ms.items() if v > 0}}


def scaleup_tree(M, W, dev, stream, flush, n=1_000_000):
    """The 10-node d=2 path workload scaled to N = 10^6 points per marginal (same
    distributions): there the products are large enough for the HBM roofline to mean
    something.  NFFT path to violation 1e-6; roofline of its dominant kernel class."""
    import torch
    prob = W.path10_d2(n=n)
    prob.root = ROOT_CENTRE
    x = [torch.from_numpy(a).to(dev) for a in prob.x]
    mu = [torch.from_numpy(m).to(dev) for m in prob.mu]
    opt = M.options(path=M.MOT_PATH_NFFT, tol_viol=TOL, max_iter=3000)
    ws = torch.empty(M.mot_workspace_bytes(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, root=prob.root, opt=opt),
                     dtype=torch.uint8, device=dev)

    def solve(o):
        with torch.cuda.stream(stream):
            flush.random_(0, 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, root=prob.root, opt=o, workspace=ws,
                              stream=stream)
            e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    solve(opt)
    tt, ti = 0.0, 0
    for _ in range(2):
        out, t = solve(opt)
        tt += t
        ti += out.iters
    ot, _ = solve(M.options(path=M.MOT_PATH_NFFT, tol_viol=TOL, max_iter=3000, timing=1))
    share = {k: v / sum(ot.kernel_ms.values()) for k, v in ot.kernel_ms.items() if v > 0}
    dom = max(share, key=share.get)
    alg = algorithmic_bytes(prob, ot.n_grid)
    prods = products_per_solve(prob, ot.iters, 10)
    avg_s = ot.kernel_ms[dom] / 1e3 / ot.kernel_launches[dom]
    per_launch = alg.get(dom, 0.0) * prods / ot.kernel_launches[dom]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = per_launch / avg_s / 1e9
    return {"value": ti / tt, "unit": "iters/s", "N": n, "iters_per_solve": out.iters, "violation": out.violation,
            "status": out.status, "n_grid": ot.n_grid,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "avg_launch_us": avg_s * 1e6, "alg_bytes_per_launch": per_launch,
                         "share": {k: round(v, 4) for k, v in share.items()}}}


def serving_replay(M, W, dev, n_requests, flush):
    """Poisson-arrival replay through the continuous-batching server (mot_server_*).

    Requests: topology uniform over {path, star, circle}, K ~ U{3..20}, d ~ U{1,2,3},
    N log-uniform on [500, 20000] (circles capped at N = 2000: their messages are K N^2),
    eta in {0.01, 0.05, 0.1}; each solved to violation 1e-6 with at most 500 sweeps.
    Inputs are uploaded before the replay.  The arrival rate is 75% of the capacity measured
    by solving the first requests one after another; latency = completion - arrival.
    Path per request: NFFT for trees and d = 1 circles; circles in d >= 2 take the tensor-core
    dense path (their N right-hand sides make the batched NFFT launch-bound)."""
    import torch
    reqs = W.serving_stream(n_requests=n_requests, rate_hz=1.0, seed=None, circle_n_max=2000)
    opt_nfft = M.options(path=M.MOT_PATH_NFFT, tol_viol=TOL, max_iter=500)
    opt_tc = M.options(path=M.MOT_PATH_DENSE_BF16X3, tol_viol=TOL, max_iter=500)

    def opt_of(p):
        return opt_tc if (p.topology == W.CIRCLE and p.d >= 2) else opt_nfft
    dev_in = []
    for r in reqs:
        p = r.problem
        dev_in.append(([torch.from_numpy(a).to(dev) for a in p.x], [torch.from_numpy(m).to(dev) for m in p.mu]))
    torch.cuda.synchronize()
    # single-stream capacity from the first requests, solved one after another
    n_cal = min(8, n_requests)
    t0 = time.perf_counter()
    for i in range(n_cal):
        p = reqs[i].problem
        M.mot_solve(*dev_in[i], p.eta, p.topology, edges=p.edges, opt=opt_of(p))
    torch.cuda.synchronize()
    service = (time.perf_counter() - t0) / n_cal
    rate = 0.75 / service
    gaps = [reqs[0].arrival_s] + [reqs[i].arrival_s - reqs[i - 1].arrival_s for i in range(1, n_requests)]
    arrivals, t = [], 0.0
    for g in gaps:                      # the stream's exponential gaps rescaled to the chosen rate
        t += g / rate
        arrivals.append(t)
    srv = M.Server(pool_bytes=16 << 30, max_active=8, device=dev)
    done, nxt = {}, 0
    start = time.perf_counter()
    while len(done) < n_requests:
        now = time.perf_counter() - start
        while nxt < n_requests and arrivals[nxt] <= now:
            p = reqs[nxt].problem
            srv.submit(*dev_in[nxt], p.eta, p.topology, edges=p.edges, opt=opt_of(p), tag=nxt)
            nxt += 1
        active, pending = srv.progress()
        for res in srv.poll():
            done[res["tag"]] = (time.perf_counter() - start, res)
        if nxt < n_requests and active == 0 and pending == 0:
            time.sleep(max(0.0, min(0.002, arrivals[nxt] - (time.perf_counter() - start))))
    wall = time.perf_counter() - start
    srv.close()
    lat = sorted(done[i][0] - arrivals[i] for i in range(n_requests))
    iters = sum(done[i][1]["iters"] for i in range(n_requests))
    status = {}
    for i in range(n_requests):
        s_ = M.strerror(done[i][1]["status"])
        status[s_] = status.get(s_, 0) + 1
    pct = lambda q: 1e3 * lat[min(len(lat) - 1, int(q * len(lat)))]   # noqa: E731
    return {"requests": n_requests, "arrival_rate_hz": rate, "single_stream_service_ms": 1e3 * service,
            "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": 1e3 * lat[-1]},
            "throughput_req_s": n_requests / wall, "iters_per_s": iters / wall, "status": status,
            "max_active": 8, "pool_gb": 16, "max_iter": 500,
            "mix": "path/star/circle, K 3-20, d 1-3, N 500-20000 (circle <= 2000)",
            "path_policy": "NFFT for trees and d=1 circles, tensor-core dense for d>=2 circles",
            "n_tensor_core": sum(1 for r in reqs if r.problem.topology == W.CIRCLE and r.problem.d >= 2)}


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    from paper_2208_03120_gb300 import build, motfft as M, workloads as W

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    prob = W.WORKLOADS[args.workload](n=args.n) if args.n else W.WORKLOADS[args.workload]()
    prob.root = ROOT_CENTRE
    topo = M.MOT_CIRCLE if prob.topology == W.CIRCLE else M.MOT_TREE
    path = {"nfft": M.MOT_PATH_NFFT, "dense": M.MOT_PATH_DENSE, "tc": M.MOT_PATH_DENSE_BF16X3}[args.path]
    x = [torch.from_numpy(a).to(dev) for a in prob.x]
    mu = [torch.from_numpy(m).to(dev) for m in prob.mu]
    stream = torch.cuda.Stream(device=dev)
    tol = TOL if args.max_iter >= 5000 else -1.0
    opt = M.options(path=path, tol_viol=tol, max_iter=args.max_iter)
    ws = torch.empty(M.mot_workspace_bytes(x, mu, prob.eta, topo, edges=prob.edges, root=prob.root, opt=opt),
                     dtype=torch.uint8, device=dev)
    u = [torch.empty(n, dtype=torch.float64, device=dev) for n in prob.n]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def solve(o=opt):
        with torch.cuda.stream(stream):
            return M.mot_solve(x, mu, prob.eta, topo, edges=prob.edges, root=prob.root, opt=o, workspace=ws,
                               stream=stream, u_out=u)

    for _ in range(args.warmup):
        out = solve()
    torch.cuda.synchronize()

    # ---- timed region: K solves, L2 flushed between them ------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    times, iters, launches = [], 0, 0
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.random_(0, 255)                      # evict L2 (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        out = solve()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        iters += out.iters
        launches += out.launches
        if out.status != 0 and tol > 0:
            raise SystemExit(f"solve did not converge: status {out.status}, violation {out.violation}")
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total = sum(times)
    total, iters_all = reduce_over_ranks(total, iters, world, dev)
    value = iters_all / total
    last = out

    # ---- per-kernel durations (events around each launch on the launching stream) -------
    topt = M.options(path=path, tol_viol=tol, max_iter=args.max_iter, timing=1)
    kms = {k: 0.0 for k in M.KERNEL_CLASSES}
    kls = {k: 0 for k in M.KERNEL_CLASSES}
    for _ in range(max(1, min(args.steps, 3))):
        with torch.cuda.stream(stream):
            flush.random_(0, 255)
        o2 = solve(topt)
        for k in kms:
            kms[k] += o2.kernel_ms[k]
            kls[k] += o2.kernel_launches[k]
    share = {k: kms[k] / sum(kms.values()) for k in kms if kms[k] > 0}
    dom = max(share, key=share.get)
    alg = algorithmic_bytes(prob, last.n_grid)
    nsolve = max(1, min(args.steps, 3))
    prods = nsolve * products_per_solve(prob, o2.iters, 10)
    avg_s = kms[dom] / 1e3 / kls[dom]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    per_launch = alg.get(dom, 0.0) * prods / kls[dom]
    if prob.topology == W.CIRCLE and prob.d == 1 and path == M.MOT_PATH_NFFT:
        per_launch = circle1d_launch_bytes(prob, last.n_grid).get(dom, 0.0)
        prods = kls[dom] * prob.n[0]
    achieved = per_launch / avg_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": load_traffic(dom, args.workload) if not args.n else None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "avg_launch_us": avg_s * 1e6, "alg_bytes_per_launch": per_launch,
                "alg_bytes_per_product": per_launch * kls[dom] / max(1, prods), "products_per_launch": prods / kls[dom],
                "share": {k: round(v, 4) for k, v in share.items()}}

    # ---- dense comparison on the same workload -------------------------------------------
    dense = None
    if not args.no_dense:
        dopt = M.options(path=M.MOT_PATH_DENSE, tol_viol=tol, max_iter=args.max_iter)
        dws = torch.empty(M.mot_workspace_bytes(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=dopt),
                          dtype=torch.uint8, device=dev)
        dt, di = 0.0, 0
        for r in range(3):
            with torch.cuda.stream(stream):
                flush.random_(0, 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                o3 = M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, root=prob.root, opt=dopt,
                                 workspace=dws, stream=stream)
                e1.record(stream)
            e1.synchronize()
            if r > 0:
                dt += e0.elapsed_time(e1) / 1e3
                di += o3.iters
        dense = {"path": "dense FP32 SIMT direct summation (one right-hand side: the tensor-core "
                         "BF16-split path needs several right-hand sides)",
                 "value": di / dt, "unit": "iters/s", "iters_per_solve": o3.iters, "violation": o3.violation}

    # ---- the other workloads (same metric, reported beside the headline) -------------------
    others = {}
    if not args.no_dense and args.workload == WORKLOAD:
        for wname, wtopo in (("star9_d3", M.MOT_TREE), ("circle5_d1", M.MOT_CIRCLE)):
            wp = W.WORKLOADS[wname]()
            wx = [torch.from_numpy(a).to(dev) for a in wp.x]
            wm = [torch.from_numpy(m).to(dev) for m in wp.mu]
            entry = {}
            paths = [("nfft", M.MOT_PATH_NFFT, 3), ("dense", M.MOT_PATH_DENSE, 2)]
            if wtopo == M.MOT_CIRCLE:
                paths.append(("dense_bf16x3", M.MOT_PATH_DENSE_BF16X3, 3))
            for pname, path, reps in paths:
                wo = M.options(path=path, tol_viol=TOL, max_iter=3000)
                wws = torch.empty(M.mot_workspace_bytes(wx, wm, wp.eta, wtopo, edges=wp.edges, opt=wo),
                                  dtype=torch.uint8, device=dev)
                tt, ti = 0.0, 0
                for r in range(reps + 1):
                    with torch.cuda.stream(stream):
                        flush.random_(0, 255)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        ow = M.mot_solve(wx, wm, wp.eta, wtopo, edges=wp.edges, opt=wo, workspace=wws, stream=stream)
                        e1.record(stream)
                    e1.synchronize()
                    if r > 0:
                        tt += e0.elapsed_time(e1) / 1e3
                        ti += ow.iters
                entry[pname] = {"value": ti / tt, "unit": "iters/s", "iters_per_solve": ow.iters,
                                "violation": ow.violation, "status": ow.status}
                if path == M.MOT_PATH_DENSE_BF16X3:
                    entry[pname]["roofline"] = tc_roofline(M, wp, wx, wm, wtopo, wo, wws, stream, flush)
                del wws
            others[wname] = entry

    # ---- the circle at N = 10^4: NFFT against the dense tensor-core path --------------------
    if not args.no_dense and args.workload == WORKLOAD:
        wp = W.circle5_d1(n=10_000)
        wx = [torch.from_numpy(a).to(dev) for a in wp.x]
        wm = [torch.from_numpy(m).to(dev) for m in wp.mu]
        entry = {}
        for pname, path_ in (("nfft", M.MOT_PATH_NFFT), ("dense_bf16x3", M.MOT_PATH_DENSE_BF16X3)):
            wo = M.options(path=path_, tol_viol=TOL, max_iter=200)
            wws = torch.empty(M.mot_workspace_bytes(wx, wm, wp.eta, M.MOT_CIRCLE, opt=wo), dtype=torch.uint8,
                              device=dev)
            tt, ti = 0.0, 0
            for r in range(2):
                with torch.cuda.stream(stream):
                    flush.random_(0, 255)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ow = M.mot_solve(wx, wm, wp.eta, M.MOT_CIRCLE, opt=wo, workspace=wws, stream=stream)
                    e1.record(stream)
                e1.synchronize()
                if r > 0:
                    tt += e0.elapsed_time(e1) / 1e3
                    ti += ow.iters
            entry[pname] = {"value": ti / tt, "unit": "iters/s", "iters_per_solve": ow.iters,
                            "violation": ow.violation, "status": ow.status, "ms_per_solve": 1e3 * tt}
            if path_ == M.MOT_PATH_DENSE_BF16X3:
                entry[pname]["roofline"] = tc_roofline(M, wp, wx, wm, M.MOT_CIRCLE, wo, wws, stream, flush)
            del wws
        others["circle5_d1_N1e4"] = entry

    # ---- generalised Euler flow (Section 6.3): sigma-closing circle + pair marginals ----------
    if not args.no_dense and args.workload == WORKLOAD:
        entry = {}
        for sigma in ("reflect", "fold"):
            wp = W.euler5_d1(sigma=sigma)
            wx = [torch.from_numpy(a).to(dev) for a in wp.x]
            wm = [torch.from_numpy(m).to(dev) for m in wp.mu]
            wc = torch.from_numpy(wp.x_close).to(dev)
            sub = {}
            for pname, path_ in (("nfft", M.MOT_PATH_NFFT), ("dense", M.MOT_PATH_DENSE),
                                 ("dense_bf16x3", M.MOT_PATH_DENSE_BF16X3)):
                wo = M.options(path=path_, tol_viol=TOL, max_iter=2000)
                wws = torch.empty(M.mot_workspace_bytes(wx, wm, wp.eta, M.MOT_CIRCLE, opt=wo, x_close=wc),
                                  dtype=torch.uint8, device=dev)
                tt, ti = 0.0, 0
                for r in range(4):
                    with torch.cuda.stream(stream):
                        flush.random_(0, 255)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        ow = M.mot_solve(wx, wm, wp.eta, M.MOT_CIRCLE, opt=wo, workspace=wws, stream=stream,
                                         x_close=wc, pair=True)
                        e1.record(stream)
                    e1.synchronize()
                    if r > 0:
                        tt += e0.elapsed_time(e1) / 1e3
                        ti += ow.iters
                sub[pname] = {"value": ti / tt, "unit": "iters/s", "iters_per_solve": ow.iters,
                              "violation": ow.violation, "status": ow.status, "ms_per_solve": 1e3 * tt / 3}
                del wws
            entry[sigma] = sub
        entry["note"] = ("K=5, N=400 uniform on [0,1], eta=0.05; whole solves to violation 1e-6 including "
                         "set-up and the K-1 pair marginals Pi_{1,k} written as FP64 400x400 matrices")
        others["euler5_d1"] = entry

    # ---- scale-up of the headline workload (N = 10^6) ---------------------------------------
    if not args.no_dense and args.workload == WORKLOAD:
        others["path10_d2_N1e6"] = scaleup_tree(M, W, dev, stream, flush)

    # ---- serving: Poisson arrivals through the continuous-batching server -------------------
    serving = None
    if rank == 0 and args.serving_requests > 0 and args.workload == WORKLOAD:
        serving = serving_replay(M, W, dev, args.serving_requests, flush)

    # ---- end to end through the C ABI with host buffers ---------------------------------
    xh = [torch.from_numpy(a).pin_memory() for a in prob.x]
    muh = [torch.from_numpy(m).pin_memory() for m in prob.mu]
    uh = [torch.empty(n, dtype=torch.float64).pin_memory() for n in prob.n]
    xd = [torch.empty_like(a, device=dev) for a in xh]
    mud = [torch.empty_like(m, device=dev) for m in muh]
    h2d = sum(a.numel() * a.element_size() for a in xh) + sum(m.numel() * m.element_size() for m in muh)
    d2h = sum(a.numel() * a.element_size() for a in uh)
    et, ei = 0.0, 0
    for r in range(max(1, min(args.steps, 5)) + 1):
        with torch.cuda.stream(stream):
            flush.random_(0, 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for a, b in zip(xd, xh):
                a.copy_(b, non_blocking=True)
            for a, b in zip(mud, muh):
                a.copy_(b, non_blocking=True)
            o4 = M.mot_solve(xd, mud, prob.eta, topo, edges=prob.edges, root=prob.root, opt=opt, workspace=ws,
                             stream=stream, u_out=u)
            for a, b in zip(uh, u):
                a.copy_(b, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        if r > 0:
            et += e0.elapsed_time(e1) / 1e3
            ei += o4.iters
    e2e = {"value": ei / et, "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- CPU baseline: the oracle on this machine's host cores ---------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, nprod, wall, cores = oracle_rate(prob, budget_s=20.0)
        cpu = {"value": r, "unit": "iters/s", "cores": cores, "kind": "oracle",
               "sample": oracle_sample_text(prob, nprod, wall)}

    lat = sorted(times)
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "topology": "path", "K": prob.K, "d": prob.d, "N": prob.n[0],
                   "eta": prob.eta, "tol_viol": TOL, "n_grid": last.n_grid, "M": last.M,
                   "iters_per_solve": last.iters, "parallelism": f"replicas{world}",
                   "root": "centre of the path (library choice, MOT_ROOT_CENTRE)",
                   "schedule": "wavefront across sweeps (library default, options.wavefront)",
                   "l2": "flushed between steps (256 MB write)"},
        "latency_ms": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "dense": dense,
        "other_workloads": others,
        "serving": serving,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches,
        "violation": last.violation,
        "cost": last.cost_dual,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
