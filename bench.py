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
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Sinkhorn iters/s, NFFT vs dense BF16-split at marginal err≤1e-6; p50/p99 latency"
WORKLOAD = "path10_d2"
TOL = 1e-6
FLUSH_BYTES = 256 << 20      # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense comparison (profiling runs)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["path10_d2", "star9_d3", "path3_d1"],
                    help="profiling runs only: the reported line is defined on path10_d2")
    ap.add_argument("--n", type=int, default=0, help="profiling runs only: points per marginal")
    ap.add_argument("--max-iter", type=int, default=5000, help="profiling runs only: iteration cap")
    return ap.parse_args()


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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

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
    """Bytes the method must move per launch of each kernel class, averaged over one
    iteration's launches (FP32 values, FP64 weights; window tables excluded).

    spread : source coordinates (4 d N) + source factors (4 N each) + grid write (4 n^d)
    fftconv: grid read + grid write (8 n^d)
    gather : grid read (4 n^d) + target coordinates (4 d N) + target factors (4 N each)
             + message / scaling write (4 N) [+ mu (12 N) on scaling updates]
    """
    K, d = prob.K, prob.d
    N = prob.n[0]
    G = 4 * n_grid ** d
    # path tree: forward level = K-1 tasks (2 source factors; targets: <=1 child factor, mu,
    # phi write), backward = K-1 levels of 1 task (phi + <=1 child factor; message write)
    fwd_spread = (K - 1) * (4 * d * N + 8 * N + G)
    fwd_gather = (K - 1) * (G + 4 * d * N + 4 * N + 12 * N + 4 * N + 4 * N) + (4 * N + 12 * N + 4 * N)
    bwd_spread = 4 * d * N + 8 * N + G
    bwd_gather = G + 4 * d * N + 4 * N
    launches = K   # one forward launch + (K-1) backward launches per class
    out = {
        "spread": (fwd_spread + (K - 1) * bwd_spread) / launches,
        "gather": (fwd_gather + (K - 1) * bwd_gather) / launches,
        "fftconv": ((K - 1) * 2 * G + (K - 1) * 2 * G) / launches,
    }
    # the fused 2-D kernel does all three with the grid in shared memory: its algorithmic
    # bytes are the point data and the vectors only (no grid round trips)
    out["fused"] = out["spread"] + out["gather"] - 2 * G * (2 * (K - 1)) / launches
    return out


def kernel_source_hash(cls):
    files = {"spread": ["nfft.cu", "common.cuh", "epilogue.cuh"], "gather": ["nfft.cu", "common.cuh", "epilogue.cuh"],
             "fused": ["nfft.cu", "common.cuh", "epilogue.cuh", "window.cuh"],
             "fftconv": ["nfft.cu", "fft_smem.cuh"], "dense": ["dense.cu", "common.cuh", "epilogue.cuh"]}.get(cls, [])
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2208_03120_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(cls):
    """DRAM traffic per launch of the kernel class from the committed ncu summary, or None
    if the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
        e = t.get(WORKLOAD, {}).get(cls)
        if e and e.get("source_hash") == kernel_source_hash(cls):
            return e.get("dram_bytes_per_launch")
    except Exception:  # noqa: BLE001
        pass
    return None


# ----------------------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# ----------------------------------------------------------------------------------------
def oracle_rate(prob, budget_s=20.0, max_iters=50):
    """Algorithm 2 with dense FP64 kernel products on the host cores, on the full workload,
    for as many sweeps as fit in the budget (at least one)."""
    from oracle import sinkhorn as OS
    ts = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta)
    t_cpu0 = time.process_time()
    t0 = time.perf_counter()
    done = [0]

    def cb(r, phi):
        done[0] = r
        if time.perf_counter() - t0 > budget_s:
            raise StopIteration

    try:
        ts.run(max_iters, callback=cb)
    except StopIteration:
        pass
    wall = time.perf_counter() - t0
    cpu = time.process_time() - t_cpu0
    return done[0] / wall, done[0], wall, max(1, round(cpu / wall))


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2208_03120_gb300 import workloads as W
    prob = W.path10_d2()
    rates = []
    for _ in range(max(1, args.steps)):
        r, iters, wall, cores = oracle_rate(prob, budget_s=15.0 / max(1, args.steps) + 5.0, max_iters=3)
        rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value if value else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": prob.K, "d": prob.d, "N": prob.n[0], "eta": prob.eta,
                   "topology": "path", "l2": "inputs in host memory (CPU run)"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                         "sample": "Algorithm 2 sweeps of the full workload with dense FP64 kernel products, "
                                   "bounded per step (>= 1 sweep)"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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
    x = [torch.from_numpy(a).to(dev) for a in prob.x]
    mu = [torch.from_numpy(m).to(dev) for m in prob.mu]
    stream = torch.cuda.Stream(device=dev)
    tol = TOL if args.max_iter >= 5000 else -1.0
    opt = M.options(path=M.MOT_PATH_NFFT, tol_viol=tol, max_iter=args.max_iter)
    ws = torch.empty(M.mot_workspace_bytes(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=opt),
                     dtype=torch.uint8, device=dev)
    u = [torch.empty(n, dtype=torch.float64, device=dev) for n in prob.n]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def solve(o=opt):
        with torch.cuda.stream(stream):
            return M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=o, workspace=ws, stream=stream,
                               u_out=u)

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
    if world > 1:
        t = torch.tensor([total, float(iters)], dtype=torch.float64, device=dev)
        tmax = t[:1].clone()
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(t[1:], op=torch.distributed.ReduceOp.SUM)
        total, iters_all = float(tmax[0]), float(t[1])
    else:
        iters_all = float(iters)
    value = iters_all / total
    last = out

    # ---- per-kernel durations (events around each launch on the launching stream) -------
    topt = M.options(path=M.MOT_PATH_NFFT, tol_viol=tol, max_iter=args.max_iter, timing=1)
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
    avg_s = kms[dom] / 1e3 / kls[dom]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = alg.get(dom, 0.0) / avg_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": load_traffic(dom),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "avg_launch_us": avg_s * 1e6, "alg_bytes_per_launch": alg.get(dom),
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
                o3 = M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=dopt, workspace=dws,
                                 stream=stream)
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
        for wname, topo in (("star9_d3", M.MOT_TREE), ("circle5_d1", M.MOT_CIRCLE)):
            wp = W.WORKLOADS[wname]()
            wx = [torch.from_numpy(a).to(dev) for a in wp.x]
            wm = [torch.from_numpy(m).to(dev) for m in wp.mu]
            entry = {}
            for pname, path, reps in (("nfft", M.MOT_PATH_NFFT, 3), ("dense", M.MOT_PATH_DENSE, 2)):
                wo = M.options(path=path, tol_viol=TOL, max_iter=3000)
                wws = torch.empty(M.mot_workspace_bytes(wx, wm, wp.eta, topo, edges=wp.edges, opt=wo),
                                  dtype=torch.uint8, device=dev)
                tt, ti = 0.0, 0
                for r in range(reps + 1):
                    with torch.cuda.stream(stream):
                        flush.random_(0, 255)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        ow = M.mot_solve(wx, wm, wp.eta, topo, edges=wp.edges, opt=wo, workspace=wws, stream=stream)
                        e1.record(stream)
                    e1.synchronize()
                    if r > 0:
                        tt += e0.elapsed_time(e1) / 1e3
                        ti += ow.iters
                entry[pname] = {"value": ti / tt, "unit": "iters/s", "iters_per_solve": ow.iters,
                                "violation": ow.violation, "status": ow.status}
                del wws
            others[wname] = entry

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
            o4 = M.mot_solve(xd, mud, prob.eta, M.MOT_TREE, edges=prob.edges, opt=opt, workspace=ws, stream=stream,
                             u_out=u)
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
        r, n_it, wall, cores = oracle_rate(prob, budget_s=20.0, max_iters=3)
        cpu = {"value": r, "unit": "iters/s", "cores": cores, "kind": "oracle",
               "sample": f"{n_it} Algorithm-2 sweep(s) of the full workload with dense FP64 kernel products "
                         f"({2 * (prob.K - 1)} products of {prob.n[0]}x{prob.n[0]} per sweep), {wall:.1f} s"}

    lat = sorted(times)
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "topology": "path", "K": prob.K, "d": prob.d, "N": prob.n[0],
                   "eta": prob.eta, "tol_viol": TOL, "n_grid": last.n_grid, "M": last.M,
                   "iters_per_solve": last.iters, "parallelism": f"replicas{world}",
                   "l2": "flushed between steps (256 MB write)"},
        "latency_ms": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "dense": dense,
        "other_workloads": others,
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
