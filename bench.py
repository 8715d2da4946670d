"""Benchmark: NFFT-accelerated tree Sinkhorn (Algorithm 2) on the 10-node d=2 path workload.

One step = one complete solve to marginal violation <= 1e-6 through the C ABI
(normalisation, binning, kernel Fourier coefficients, the Sinkhorn sweeps with the fast
summation -- on this workload its trigonometric sums evaluated exactly in one thread-block
cluster per product -- stop tests and outputs), inputs already resident in device memory.
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
    ap.add_argument("--serving-requests", type=int, default=200,
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
def bytes_per_product(prob, n_grid, nfac=1):
    """Algorithmic bytes of one fast-summation product, the byte count of the hot-path scope:

        B = 4 [(d+1) N_src + (d+1) N_tgt + N |C|] + 16 n^d

    source coordinates and value, target coordinates and output, |C| further factor vectors (the
    children's messages; one on average on a path), and four passes over the n^d FP32 grid (spread
    write, transform in and out, gather read).  Window tables excluded.  Split by kernel class:
    spread = source side + grid write, fftconv = grid read + write, gather = target side + grid
    read; the fused and persistent kernels carry all of it."""
    d, N = prob.d, prob.n[0]
    G = 4 * n_grid ** d
    src = 4 * (d + 1) * N
    tgt = 4 * (d + 1) * N + 4 * N * nfac
    total = src + tgt + 4 * G
    return {"product": total, "spread": src + G, "fftconv": 2 * G, "gather": tgt + G, "fused": total,
            "wave": total}


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


def hbm_roofline(prob, n_grid, dom, kms, kls, nsolve, iters, peaks, traffic=None, check_every=10):
    """HBM roofline of the dominant kernel class over `nsolve` timed solves (timing mode: CUDA
    events around every launch): algorithmic bytes per launch (bytes_per_product x products per
    launch) over the class's average launch duration, against the measured copy bandwidth.
    Products per launch: for the persistent wavefront kernel 2 (K-1) S + (K-1) (S sweeps of a chunk
    and its check pass; S = sweeps / launches); otherwise the solve's products (initial backward
    pass, 2 (K-1) per sweep, K-1 per check) over the class's launches."""
    alg = bytes_per_product(prob, n_grid)
    if dom == "wave":
        S = nsolve * iters / kls[dom]
        prods = 2 * (prob.K - 1) * S + (prob.K - 1)
    else:
        prods = nsolve * products_per_solve(prob, iters, check_every) / kls[dom]
    avg_s = kms[dom] / 1e3 / kls[dom]
    per_launch = alg.get(dom, 0.0) * prods
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = per_launch / avg_s / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "avg_launch_us": avg_s * 1e6, "alg_bytes_per_launch": per_launch,
            "alg_bytes_per_product": alg["product"], "products_per_launch": prods,
            "share": {k: round(v / sum(kms.values()), 4) for k, v in kms.items() if v > 0}}


# FP32 fused multiply-add peak of the GPU: 152 SMs x 128 FP32 lanes x 2 flops x the maximum SM clock
# (2070 MHz); the packed fma.rn.f32x2 form issues two lanes' worth per instruction but runs on the
# same 128 lanes per SM.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def flops_per_exact_product(prob):
    """Multiply-add flops of one product on the exact-sum path (d = 2, 33 trigonometric values per
    coordinate): the adjoint contraction A = sum_j e(y_j) (v_j e(x_j))^T (33 x 33 per source) and
    the targets' bilinear forms e(y_i)^T B e(x_i) (33 x 33 per target), 2 flops per multiply-add."""
    N = prob.n[0]
    return 2.0 * 33 * 33 * (N + N)


def alu_roofline(prob, n_grid, dom, kms, kls, nsolve, iters, peaks, traffic=None):
    """FP32 roofline of the persistent kernel on the exact-sum path: algorithmic flops per launch
    (flops_per_exact_product x products per launch) over the class's average launch duration,
    against FP32_PEAK_TFLOPS.  The HBM byte model of the same launch is kept beside it."""
    hb = hbm_roofline(prob, n_grid, dom, kms, kls, nsolve, iters, peaks, traffic=traffic)
    prods = hb["products_per_launch"]
    avg_s = hb["avg_launch_us"] / 1e6
    flops = flops_per_exact_product(prob) * prods
    achieved = flops / avg_s / 1e12
    return {"bound": "alu", "kernel": dom + " (k_wave_nd, exact trigonometric sums)", "achieved": achieved,
            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
            "avg_launch_us": hb["avg_launch_us"], "alg_flops_per_launch": flops,
            "alg_flops_per_product": flops_per_exact_product(prob), "products_per_launch": prods,
            "hbm_model": {"achieved_gbs": hb["achieved"], "peak_gbs": hb["peak"], "frac": hb["frac"],
                          "alg_bytes_per_launch": hb["alg_bytes_per_launch"]},
            "share": hb["share"]}


def products_per_solve(prob, iters, check_every):
    """Kernel products executed by one solve: the initial backward pass, 2(K-1) per sweep and
    the K-1 forward products of each check pass."""
    checks = -(-iters // check_every)
    return (1 + 2 * iters + checks) * (prob.K - 1)


def kernel_source_hash(cls):
    # the persistent kernel's traffic also depends on the host's schedule (solver.cu)
    files = {"spread": ["nfft.cu", "common.cuh", "epilogue.cuh"], "gather": ["nfft.cu", "common.cuh", "epilogue.cuh"],
             "fused": ["nfft.cu", "common.cuh", "epilogue.cuh", "window.cuh"],
             "wave": ["ndft2d.cu", "wave.cuh", "common.cuh", "epilogue.cuh", "solver.cu", "kernels.h"],
             "fftconv": ["nfft.cu", "fft_smem.cuh"], "dense": ["dense.cu", "common.cuh", "epilogue.cuh"],
             "local": ["local.cu", "kernels.h", "solver.cu"]}.get(cls, [])
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
def oracle_sweeps(prob, warmup, steps):
    """The oracle's Algorithm 2 (``oracle.sinkhorn.TreeSinkhorn``, FP64) on the full workload, timed
    sweep by sweep on this machine's host cores.  Its edge kernels run in their dense mode: the
    K-1 kernel matrices (10^4 x 10^4 at N = 10^4) are formed once, untimed, and every product is a
    dense FP64 matrix-vector product.  The run starts from phi = 1 with the initial backward pass
    (untimed) and times sweeps warmup .. warmup + steps - 1, each with its 2 (K-1) products and the
    O(N) scaling updates.  Returns (sweeps/s, per-sweep seconds, matrix set-up seconds, cores)."""
    from oracle import sinkhorn as OS
    OS.EdgeKernel.DENSE_LIMIT = max(OS.EdgeKernel.DENSE_LIMIT, max(prob.n) ** 2)
    t0 = time.perf_counter()
    ts = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta)
    setup = time.perf_counter() - t0
    stamps = []
    c0 = time.process_time()
    w0 = time.perf_counter()
    stamps.append(w0)
    ts.run(warmup + steps, callback=lambda r, phi: stamps.append(time.perf_counter()))
    cores = max(1, round((time.process_time() - c0) / (time.perf_counter() - w0)))
    per = [b - a for a, b in zip(stamps[:-1], stamps[1:])][warmup:]
    return len(per) / sum(per), per, setup, cores


def oracle_sample_text(prob, nsweeps, setup):
    return (f"{nsweeps} full sweeps of Algorithm 2 (oracle, FP64, dense {prob.n[0]}x{prob.n[0]} kernel "
            f"matrices formed once in {setup:.1f} s, not timed), each with its {2 * (prob.K - 1)} products and "
            f"the O(N) scaling updates, after the initial backward pass")


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2208_03120_gb300 import workloads as W
    prob = W.path10_d2()
    value, per, setup, cores = oracle_sweeps(prob, max(0, args.warmup), max(1, args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value if value else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": prob.K, "d": prob.d, "N": prob.n[0], "eta": prob.eta,
                   "topology": "path", "l2": "inputs in host memory (CPU run)",
                   "step": "one full sweep of Algorithm 2"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                         "sample": oracle_sample_text(prob, len(per), setup)},
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
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    roof = hbm_roofline(prob, ot.n_grid, dom, ot.kernel_ms, ot.kernel_launches, 1, ot.iters, peaks)
    # spread and gather each move their side of every product: report both
    for side in ("spread", "gather"):
        if side != dom and ot.kernel_launches[side]:
            r2 = hbm_roofline(prob, ot.n_grid, side, ot.kernel_ms, ot.kernel_launches, 1, ot.iters, peaks)
            roof[side + "_frac"] = r2["frac"]
    return {"value": ti / tt, "unit": "iters/s", "N": n, "iters_per_solve": out.iters, "violation": out.violation,
            "status": out.status, "n_grid": ot.n_grid, "roofline": roof}


def star_roofline(M, wp, wx, wm, wo, wws, stream, flush):
    """HBM roofline of the dominant class of the d = 3 star (3-kernel NFFT path), one timed solve."""
    import torch
    topt = M.options(path=M.MOT_PATH_NFFT, tol_viol=TOL, max_iter=3000, timing=1)
    with torch.cuda.stream(stream):
        flush.random_(0, 255)
    o = M.mot_solve(wx, wm, wp.eta, M.MOT_TREE, edges=wp.edges, opt=topt, workspace=wws, stream=stream)
    torch.cuda.synchronize()
    share = {k: v / sum(o.kernel_ms.values()) for k, v in o.kernel_ms.items() if v > 0}
    dom = max(share, key=share.get)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    return hbm_roofline(wp, o.n_grid, dom, o.kernel_ms, o.kernel_launches, 1, o.iters, peaks)


SERVING_CAPS = {2: 2000, 3: 2000}   # circle N caps by dimension (d = 1 circles run at full N)


def serving_replay(M, W, dev, n_requests, flush, runs=2):
    """Poisson-arrival replay through the continuous-batching server (mot_server_*).

    Requests: the first `n_requests` of the seeded stream -- topology uniform over {path, star,
    circle}, K ~ U{3..20}, d ~ U{1,2,3}, N log-uniform on [500, 20000], eta in {0.01, 0.05, 0.1};
    each solved to violation 1e-6 with at most 500 sweeps.  Circles in d >= 2 are capped at
    N = 2000: they take the tensor-core dense path, whose products cost O(N^3) (at N = 20000 one
    sweep of K = 20 takes about a second, hundreds of sweeps per request); d = 1 circles (batched
    NFFT) and all trees run at their drawn N.  Inputs are uploaded before the replay.  The arrival
    rate is 75% of the capacity measured by solving the first 8 requests one after another;
    latency = completion - arrival.  The replay runs `runs` times; p50 / p99 of each run and their
    spread are reported."""
    import torch
    reqs = W.serving_stream(n_requests=n_requests, rate_hz=1.0, seed=None, circle_n_max=SERVING_CAPS)
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
    pool_gb = 120
    out = []
    for run in range(runs):
        srv = M.Server(pool_bytes=pool_gb << 30, max_active=8, device=dev)
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
        del srv                         # release the pool before the next replay allocates its own
        torch.cuda.empty_cache()
        lat = sorted(done[i][0] - arrivals[i] for i in range(n_requests))
        iters = sum(done[i][1]["iters"] for i in range(n_requests))
        status = {}
        for i in range(n_requests):
            s_ = M.strerror(done[i][1]["status"])
            status[s_] = status.get(s_, 0) + 1
        pct = lambda q: 1e3 * lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]   # noqa: E731
        out.append({"latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": 1e3 * lat[-1]},
                    "throughput_req_s": n_requests / wall, "iters_per_s": iters / wall, "status": status})
    p99 = [r["latency_ms"]["p99"] for r in out]
    p50 = [r["latency_ms"]["p50"] for r in out]
    return {"requests": n_requests, "arrival_rate_hz": rate, "single_stream_service_ms": 1e3 * service,
            "latency_ms": {"p50": statistics.median(p50), "p99": statistics.median(p99),
                           "p50_runs": p50, "p99_runs": p99},
            "throughput_req_s": statistics.median([r["throughput_req_s"] for r in out]),
            "runs": out, "max_active": 8, "pool_gb": pool_gb, "max_iter": 500,
            "mix": "path/star/circle, K 3-20, d 1-3, N 500-20000 (circles in d >= 2 capped at 2000)",
            "path_policy": "NFFT for trees and d=1 circles, tensor-core dense for d>=2 circles",
            "n_tensor_core": sum(1 for r in reqs if r.problem.topology == W.CIRCLE and r.problem.d >= 2),
            "n_circle_d1": sum(1 for r in reqs if r.problem.topology == W.CIRCLE and r.problem.d == 1),
            "max_n_circle_d1": max([r.problem.n[0] for r in reqs if r.problem.topology == W.CIRCLE
                                    and r.problem.d == 1] or [0])}


def local_bench(M, W, dev, stream, flush, eta=2e-4, sweeps=40):
    """The small-eta local path (Section 6.1, closing remark) on the 10-node d = 2 path shape at
    eta = 2e-4, where the FP32 scaling form is out of range: `sweeps` sweeps of Algorithm 2 in the
    log domain (violation reported, not a stop test: convergence at this eta takes thousands of
    sweeps), r_cut = sqrt(40 eta).  Roofline of the log-sum-exp kernel: one exponential per pair
    within r_cut (counted exactly on the host with a k-d tree), against the nominal MUFU exp2 rate
    (16 per SM per cycle x 152 SMs x the median SM clock under load)."""
    import numpy as np
    import torch
    from scipy.spatial import cKDTree
    prob = W.path10_d2()
    prob.eta = eta
    prob.root = ROOT_CENTRE
    r_cut = math.sqrt(40.0 * eta)
    x = [torch.from_numpy(a).to(dev) for a in prob.x]
    mu = [torch.from_numpy(m).to(dev) for m in prob.mu]
    opt = M.options(path=M.MOT_PATH_LOCAL, r_cut=r_cut, tol_viol=-1.0, max_iter=sweeps)
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
    ot, _ = solve(M.options(path=M.MOT_PATH_LOCAL, r_cut=r_cut, tol_viol=-1.0, max_iter=sweeps, timing=1))
    # exponentials per solve: every product of edge e evaluates one per pair within r_cut
    xs = [a.astype(np.float64) for a in prob.x]
    pairs = [cKDTree(xs[k]).count_neighbors(cKDTree(xs[k + 1]), r_cut) for k in range(prob.K - 1)]
    checks = -(-sweeps // 10)
    exps = (1 + 2 * sweeps + checks) * float(sum(pairs))
    launches = ot.kernel_launches["local"]
    t_local = ot.kernel_ms["local"] / 1e3
    clk = 2070.0
    peak = 16 * 152 * clk * 1e6 / 1e12          # T exp/s
    achieved = exps / t_local / 1e12
    return {"value": ti / tt, "unit": "iters/s", "eta": eta, "r_cut": r_cut, "sweeps": sweeps,
            "violation": out.violation, "status": out.status, "pairs_per_product": float(sum(pairs)) / (prob.K - 1),
            "roofline": {"bound": "alu", "kernel": "local (k_lse)", "achieved": achieved, "peak": peak,
                         "unit": "Texp/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": "nominal MUFU: 16 ex2 per SM per cycle x 152 SMs x 2070 MHz",
                         "avg_launch_us": 1e6 * t_local / max(1, launches), "exps_per_launch": exps / max(1, launches),
                         "share": {k: round(v / sum(ot.kernel_ms.values()), 4)
                                   for k, v in ot.kernel_ms.items() if v > 0}}}


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
    nsolve = max(1, min(args.steps, 3))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    # d = 2 on grids up to 64 with sets of up to 32768 points: the fused products evaluate the
    # trigonometric sums exactly (FP32 contractions), so their roofline is the FP32 one
    exact = (path == M.MOT_PATH_NFFT and prob.d == 2 and last.n_grid <= 64 and max(prob.n) <= 32768
             and dom == "wave")
    rf = alu_roofline if exact else hbm_roofline
    roofline = rf(prob, last.n_grid, dom, kms, kls, nsolve, o2.iters, peaks,
                  traffic=load_traffic(dom, args.workload) if not args.n else None)
    if prob.topology == W.CIRCLE and prob.d == 1 and path == M.MOT_PATH_NFFT:
        per_launch = circle1d_launch_bytes(prob, last.n_grid).get(dom, 0.0)
        avg_s = kms[dom] / 1e3 / kls[dom]
        roofline.update(achieved=per_launch / avg_s / 1e9, alg_bytes_per_launch=per_launch,
                        frac=per_launch / avg_s / 1e9 / roofline["peak"])
    # the dominant kernel's launches take no longer than the timed step they belong to
    roofline["launch_time_per_step_ms"] = kms[dom] / nsolve
    roofline["within_step"] = bool(kms[dom] / nsolve <= 1.05 * 1e3 * total / args.steps)

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
                if wname == "star9_d3" and path == M.MOT_PATH_NFFT:
                    entry[pname]["roofline"] = star_roofline(M, wp, wx, wm, wo, wws, stream, flush)
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

    # ---- the small-eta local path (log domain, truncated sums) ---------------------------------
    if not args.no_dense and args.workload == WORKLOAD:
        others["path10_d2_eta2e-4_local"] = local_bench(M, W, dev, stream, flush)

    # ---- serving: Poisson arrivals through the continuous-batching server -------------------
    serving = None
    if rank == 0 and args.serving_requests > 0 and args.workload == WORKLOAD:
        serving = serving_replay(M, W, dev, args.serving_requests, flush)

    # ---- end to end through the C ABI with host buffers ---------------------------------
    # the step's inputs (every set's points and weights) and results (every set's potentials) each
    # live in one contiguous pinned host buffer per type, copied in one transfer each way; the
    # per-set arguments of mot_solve are views of the matching device buffers
    def offsets(sizes):                     # each array starts on a 256-byte boundary
        offs, o = [], 0
        for n in sizes:
            offs.append(o)
            o += (int(n) + 63) // 64 * 64
        return offs, o
    xo, xt = offsets(a.size for a in prob.x)
    mo, mt = offsets(m.size for m in prob.mu)
    uo, ut = offsets(prob.n)
    xh_all = torch.zeros(xt, dtype=torch.float32).pin_memory()
    muh_all = torch.zeros(mt, dtype=torch.float64).pin_memory()
    for o, a in zip(xo, prob.x):
        xh_all[o:o + a.size] = torch.from_numpy(a.reshape(-1))
    for o, m in zip(mo, prob.mu):
        muh_all[o:o + m.size] = torch.from_numpy(m.reshape(-1))
    uh_all = torch.empty(ut, dtype=torch.float64).pin_memory()
    xd_all = torch.empty_like(xh_all, device=dev)
    mud_all = torch.empty_like(muh_all, device=dev)
    ud_all = torch.empty(ut, dtype=torch.float64, device=dev)
    xd = [xd_all[o:o + a.size].view(a.shape) for o, a in zip(xo, prob.x)]
    mud = [mud_all[o:o + m.size] for o, m in zip(mo, prob.mu)]
    ud = [ud_all[o:o + n] for o, n in zip(uo, prob.n)]
    # bytes of the inputs and results themselves (the copies also move the alignment padding)
    h2d = sum(a.nbytes for a in prob.x) + sum(m.nbytes for m in prob.mu)
    d2h = 8 * sum(int(n) for n in prob.n)
    et, ei = 0.0, 0
    for r in range(max(1, args.steps) + 1):      # as many steps as the device-timed figure
        with torch.cuda.stream(stream):
            flush.random_(0, 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xd_all.copy_(xh_all, non_blocking=True)
            mud_all.copy_(muh_all, non_blocking=True)
            o4 = M.mot_solve(xd, mud, prob.eta, topo, edges=prob.edges, root=prob.root, opt=opt, workspace=ws,
                             stream=stream, u_out=ud)
            uh_all.copy_(ud_all, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        if r > 0:
            et += e0.elapsed_time(e1) / 1e3
            ei += o4.iters
    e2e = {"value": ei / et, "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- CPU baseline: the oracle on this machine's host cores ---------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, per, setup, cores = oracle_sweeps(prob, 1, 4)
        cpu = {"value": r, "unit": "iters/s", "cores": cores, "kind": "oracle",
               "sample": oracle_sample_text(prob, len(per), setup)}

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
                   "fast_summation": ("exact trigonometric sums, Eqs. ndft*/ndft as FP32 contractions "
                                      "(library default for d = 2 on grids up to 64, options.ndft)"
                                      if exact else "NFFT through the oversampled grid"),
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
