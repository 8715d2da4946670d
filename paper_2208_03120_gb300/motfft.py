"""Thin ctypes binding of libmotfft (include/motfft.h): argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors into
the pointers and sizes of the C ABI, allocates the caller-owned workspace and
outputs with torch, and raises :class:`MotError` for a non-zero status.  There is
no fallback: if ``libmotfft.so`` is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmotfft.so")

MOT_OK, MOT_EINVAL, MOT_ENOTTREE, MOT_ENOMEM, MOT_ENUMERIC, MOT_ENOCONV, MOT_ETIMEOUT, MOT_ECUDA, MOT_EUNSUPPORTED = range(9)
MOT_TREE, MOT_CIRCLE = 0, 1
MOT_PATH_NFFT, MOT_PATH_DENSE, MOT_PATH_DENSE_BF16X3, MOT_PATH_LOCAL = 0, 1, 2, 3
MOT_NKCLASS = 12
KERNEL_CLASSES = ["spread", "fftconv", "gather", "dense", "node", "setup", "circle", "fused", "tcgemm", "split",
                  "wave", "local"]


class MotError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({strerror(status)}){' ' + detail if detail else ''}")


class Problem(C.Structure):
    _fields_ = [
        ("K", C.c_int), ("d", C.c_int),
        ("n", C.POINTER(C.c_int64)),
        ("x", C.POINTER(C.c_void_p)),
        ("mu", C.POINTER(C.c_void_p)),
        ("topology", C.c_int),
        ("edges", C.POINTER(C.c_int)),
        ("edge_w", C.POINTER(C.c_double)),
        ("free_nodes", C.POINTER(C.c_ubyte)),
        ("eta", C.c_double),
        ("root", C.c_int),
        ("x_close", C.c_void_p),
    ]


class ServerResult(C.Structure):
    _fields_ = [
        ("tag", C.c_longlong), ("status", C.c_int), ("iters", C.c_int),
        ("violation", C.c_double), ("cost_dual", C.c_double), ("cost_primal", C.c_double),
        ("submit_ms", C.c_double), ("admit_ms", C.c_double), ("done_ms", C.c_double),
    ]


class Options(C.Structure):
    _fields_ = [
        ("path", C.c_int), ("max_iter", C.c_int),
        ("tol_viol", C.c_double), ("delta_S", C.c_double),
        ("check_every", C.c_int), ("min_iter", C.c_int),
        ("n_grid", C.c_int), ("m", C.c_int), ("p", C.c_int),
        ("eps_B", C.c_double),
        ("use_graphs", C.c_int), ("timing", C.c_int), ("wavefront", C.c_int),
        ("r_cut", C.c_double), ("ndft", C.c_int),
    ]


class Result(C.Structure):
    _fields_ = [
        ("u", C.POINTER(C.c_void_p)),
        ("violation", C.c_double), ("cost_dual", C.c_double), ("cost_primal", C.c_double),
        ("mass", C.c_double), ("S_last", C.c_double), ("S_prev", C.c_double),
        ("iters", C.c_int), ("status", C.c_int),
        ("clamped", C.c_longlong), ("launches", C.c_longlong),
        ("scale", C.c_double), ("eta_norm", C.c_double),
        ("n_grid", C.c_int), ("M", C.c_int),
        ("kernel_ms", C.c_double * MOT_NKCLASS),
        ("kernel_launches", C.c_longlong * MOT_NKCLASS),
        ("pair", C.POINTER(C.c_void_p)),
    ]


_lib_handle = None


def lib() -> C.CDLL:
    """Load libmotfft.so (raises if it is missing: there is no CPU fallback)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built; run __graft_entry__.build() first")
        h = C.CDLL(LIB_PATH)
        h.mot_strerror.restype = C.c_char_p
        h.mot_strerror.argtypes = [C.c_int]
        h.mot_last_cuda_error.restype = C.c_char_p
        h.mot_abi_version.restype = C.c_int
        h.mot_options_default.argtypes = [C.POINTER(Options)]
        h.mot_workspace_bytes.argtypes = [C.POINTER(Problem), C.POINTER(Options), C.POINTER(C.c_size_t)]
        h.mot_solve.argtypes = [C.POINTER(Problem), C.POINTER(Options), C.c_void_p, C.c_size_t,
                                C.POINTER(C.c_void_p), C.POINTER(Result), C.c_void_p]
        h.mot_fastsum_workspace_bytes.argtypes = [C.c_int, C.c_int64, C.c_int64, C.c_int, C.POINTER(Options),
                                                  C.POINTER(C.c_size_t)]
        h.mot_fastsum.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.c_int, C.c_void_p, C.POINTER(Options), C.c_void_p, C.c_size_t,
                                  C.POINTER(C.c_double), C.c_void_p]
        h.mot_fastsum_static.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                         C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Options),
                                         C.POINTER(C.c_double), C.c_void_p]
        h.mot_server_create.argtypes = [C.c_void_p, C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]
        h.mot_server_submit.argtypes = [C.c_void_p, C.POINTER(Problem), C.POINTER(Options), C.POINTER(C.c_void_p),
                                        C.c_longlong]
        h.mot_server_progress.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        h.mot_server_poll.argtypes = [C.c_void_p, C.POINTER(ServerResult), C.c_int, C.POINTER(C.c_int)]
        h.mot_server_destroy.argtypes = [C.c_void_p]
        h.mot_test_tc_wait.argtypes = [C.c_longlong, C.c_int]
        h.mot_test_wave_clusters.argtypes = [C.c_int]
        h.mot_struct_sizes.argtypes = [C.POINTER(C.c_size_t)]
        h.mot_struct_sizes.restype = None
        h.mot_boundary_poly.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double)]
        h.mot_plan_grid.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        h.mot_wave_schedule.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int)]
        _lib_handle = h
    return _lib_handle


def strerror(status: int) -> str:
    try:
        return lib().mot_strerror(status).decode()
    except Exception:  # noqa: BLE001 - message only
        return "?"


def _check(status: int, where: str, allow=(MOT_OK,)):
    if status not in allow:
        detail = lib().mot_last_cuda_error().decode() if status == MOT_ECUDA else ""
        raise MotError(status, where, detail)
    return status


def options(**kw) -> Options:
    o = Options()
    lib().mot_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream_ptr(stream) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check_tensor(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


# ----------------------------------------------------------------------------------------
# kernel matrix-vector product
# ----------------------------------------------------------------------------------------

def mot_fastsum_workspace_bytes(d: int, n_src: int, n_tgt: int, nrhs: int = 1, opt: Optional[Options] = None) -> int:
    nb = C.c_size_t(0)
    _check(lib().mot_fastsum_workspace_bytes(d, n_src, n_tgt, nrhs, C.byref(opt or options()), C.byref(nb)),
           "mot_fastsum_workspace_bytes")
    return nb.value


def mot_fastsum(x_src, x_tgt, alpha, eta: float, opt: Optional[Options] = None, workspace=None, stream=None,
                out=None):
    """beta = K alpha with K_ij = exp(-||x_tgt[i] - x_src[j]||^2 / eta) (Eq. fastsum-sum).

    x_src: (n_src, d) float32 CUDA; x_tgt: (n_tgt, d); alpha: (n_src,) or (nrhs, n_src) float32.
    Returns (beta, scale) with beta shaped like alpha over the targets.
    """
    import torch
    opt = opt or options()
    _check_tensor(x_src, torch.float32, "x_src")
    _check_tensor(x_tgt, torch.float32, "x_tgt")
    _check_tensor(alpha, torch.float32, "alpha")
    d = x_src.shape[1]
    if x_tgt.shape[1] != d:
        raise ValueError("dimension mismatch")
    a2 = alpha.reshape(-1, x_src.shape[0])
    nrhs = a2.shape[0]
    n_src, n_tgt = x_src.shape[0], x_tgt.shape[0]
    if workspace is None:
        nb = mot_fastsum_workspace_bytes(d, n_src, n_tgt, nrhs, opt)
        workspace = torch.empty(nb, dtype=torch.uint8, device=x_src.device)
    beta = out if out is not None else torch.empty((nrhs, n_tgt), dtype=torch.float32, device=x_src.device)
    scale = C.c_double(0.0)
    _check(lib().mot_fastsum(d, float(eta), x_src.data_ptr(), n_src, x_tgt.data_ptr(), n_tgt, a2.data_ptr(), nrhs,
                             beta.data_ptr(), C.byref(opt), workspace.data_ptr(), workspace.numel(),
                             C.byref(scale), _stream_ptr(stream)), "mot_fastsum")
    if alpha.dim() == 1:
        beta = beta.reshape(n_tgt)
    return beta, scale.value


MOT_STATIC_SCRATCH_BYTES = 32 << 20


def hook_tc_wait(wait_ns: int = 1_000_000_000, stall_loads: bool = False) -> None:
    """Test hook of the tensor-core kernel's bounded waits (mot_test_tc_wait): the wait limit in
    ns and a switch that makes the kernel issue no operand loads, so that its first wait runs
    out.  ``hook_tc_wait()`` restores the defaults."""
    _check(lib().mot_test_tc_wait(int(wait_ns), 1 if stall_loads else 0), "mot_test_tc_wait")


def hook_wave_clusters(nclusters: int = 0) -> None:
    """Test hook (mot_test_wave_clusters): clusters of the persistent wavefront kernel for solves
    set up afterwards; 0 restores the default (as many as are co-resident)."""
    _check(lib().mot_test_wave_clusters(int(nclusters)), "mot_test_wave_clusters")


def mot_fastsum_static(x_src, x_tgt, alpha, eta: float, opt: Optional[Options] = None, stream=None, out=None):
    """mot_fastsum without a workspace: for callers that cannot allocate GPU memory (the
    library uses its own static device scratch of MOT_STATIC_SCRATCH_BYTES; calls that
    overlap on the GPU must be serialised).  Only ``out`` (optional) is allocated here."""
    import torch
    opt = opt or options()
    _check_tensor(x_src, torch.float32, "x_src")
    _check_tensor(x_tgt, torch.float32, "x_tgt")
    _check_tensor(alpha, torch.float32, "alpha")
    d = x_src.shape[1]
    a2 = alpha.reshape(-1, x_src.shape[0])
    nrhs = a2.shape[0]
    beta = out if out is not None else torch.empty((nrhs, x_tgt.shape[0]), dtype=torch.float32,
                                                   device=x_src.device)
    scale = C.c_double(0.0)
    _check(lib().mot_fastsum_static(d, float(eta), x_src.data_ptr(), x_src.shape[0], x_tgt.data_ptr(),
                                    x_tgt.shape[0], a2.data_ptr(), nrhs, beta.data_ptr(), C.byref(opt),
                                    C.byref(scale), _stream_ptr(stream)), "mot_fastsum_static")
    if alpha.dim() == 1:
        beta = beta.reshape(x_tgt.shape[0])
    return beta, scale.value


# ----------------------------------------------------------------------------------------
# Sinkhorn
# ----------------------------------------------------------------------------------------

class _ProblemHolder:
    """Keeps the ctypes arrays referenced by a Problem alive."""

    def __init__(self, x: Sequence, mu: Sequence, eta: float, topology: int, edges=None, edge_w=None,
                 free_nodes=None, root: int = 0, x_close=None):
        import torch
        K = len(x)
        if len(mu) != K:
            raise ValueError("x and mu lengths differ")
        for k in range(K):
            _check_tensor(x[k], torch.float32, f"x[{k}]")
            _check_tensor(mu[k], torch.float64, f"mu[{k}]")
        self.x = list(x)
        self.mu = list(mu)
        self.n_arr = (C.c_int64 * K)(*[int(t.shape[0]) for t in x])
        self.x_arr = (C.c_void_p * K)(*[t.data_ptr() for t in x])
        self.mu_arr = (C.c_void_p * K)(*[t.data_ptr() for t in mu])
        p = Problem()
        p.K = K
        p.d = int(x[0].shape[1])
        p.n = self.n_arr
        p.x = self.x_arr
        p.mu = self.mu_arr
        p.topology = topology
        if edges is not None:
            flat = [int(v) for e in edges for v in e]
            self.e_arr = (C.c_int * len(flat))(*flat)
            p.edges = self.e_arr
        if edge_w is not None:
            self.w_arr = (C.c_double * len(edge_w))(*[float(v) for v in edge_w])
            p.edge_w = self.w_arr
        if free_nodes is not None:
            self.f_arr = (C.c_ubyte * K)(*[1 if v else 0 for v in free_nodes])
            p.free_nodes = self.f_arr
        p.eta = float(eta)
        p.root = int(root)
        if x_close is not None:
            _check_tensor(x_close, torch.float32, "x_close")
            if tuple(x_close.shape) != tuple(x[0].shape):
                raise ValueError("x_close must have the shape of x[0]")
            self.x_close = x_close
            p.x_close = x_close.data_ptr()
        self.p = p


def mot_workspace_bytes(x, mu, eta, topology=MOT_TREE, edges=None, edge_w=None, free_nodes=None, root=0,
                        opt: Optional[Options] = None, x_close=None) -> int:
    h = _ProblemHolder(x, mu, eta, topology, edges, edge_w, free_nodes, root, x_close)
    nb = C.c_size_t(0)
    _check(lib().mot_workspace_bytes(C.byref(h.p), C.byref(opt or options()), C.byref(nb)), "mot_workspace_bytes")
    return nb.value


class SolveOutput:
    def __init__(self, u: List, res: Result, pair: Optional[List] = None):
        self.u = u
        self.pair = pair
        self.violation = res.violation
        self.cost_dual = res.cost_dual
        self.cost_primal = res.cost_primal
        self.mass = res.mass
        self.S_last = res.S_last
        self.S_prev = res.S_prev
        self.iters = res.iters
        self.status = res.status
        self.clamped = res.clamped
        self.launches = res.launches
        self.scale = res.scale
        self.eta_norm = res.eta_norm
        self.n_grid = res.n_grid
        self.M = res.M
        self.kernel_ms = {KERNEL_CLASSES[i]: res.kernel_ms[i] for i in range(MOT_NKCLASS)}
        self.kernel_launches = {KERNEL_CLASSES[i]: res.kernel_launches[i] for i in range(MOT_NKCLASS)}


def mot_solve(x, mu, eta, topology=MOT_TREE, edges=None, edge_w=None, free_nodes=None, root=0,
              opt: Optional[Options] = None, u_warm=None, workspace=None, stream=None, u_out=None,
              allow_noconv: bool = True, x_close=None, pair: bool = False) -> SolveOutput:
    """Sinkhorn for a tree (Algorithm 2) or circle (Algorithm 3); returns u^k = eta log phi^k (FP64).

    Circle only: ``x_close`` = sigma(x^1) for the closing edge of a generalised Euler flow, and
    ``pair=True`` also returns the pair marginals Pi_{1,k} (Section 6.3) as ``out.pair[k]``,
    FP64 (n_1, n_k) tensors for k = 1..K-1 (``out.pair[0]`` is None)."""
    import torch
    opt = opt or options()
    h = _ProblemHolder(x, mu, eta, topology, edges, edge_w, free_nodes, root, x_close)
    dev = x[0].device
    if workspace is None:
        nb = C.c_size_t(0)
        _check(lib().mot_workspace_bytes(C.byref(h.p), C.byref(opt), C.byref(nb)), "mot_workspace_bytes")
        workspace = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    K = len(x)
    u = u_out if u_out is not None else [torch.empty(int(t.shape[0]), dtype=torch.float64, device=dev) for t in x]
    u_arr = (C.c_void_p * K)(*[t.data_ptr() for t in u])
    res = Result()
    res.u = u_arr
    pairs = None
    if pair:
        n0 = int(x[0].shape[0])
        pairs = [None] + [torch.empty((n0, int(t.shape[0])), dtype=torch.float64, device=dev) for t in x[1:]]
        pair_arr = (C.c_void_p * K)(None, *[t.data_ptr() for t in pairs[1:]])
        res.pair = pair_arr
    warm = None
    if u_warm is not None:
        warm = (C.c_void_p * K)(*[t.data_ptr() for t in u_warm])
    allow = (MOT_OK, MOT_ENOCONV) if allow_noconv else (MOT_OK,)
    _check(lib().mot_solve(C.byref(h.p), C.byref(opt), workspace.data_ptr(), workspace.numel(), warm, C.byref(res),
                           _stream_ptr(stream)), "mot_solve", allow)
    return SolveOutput(u, res, pairs)


# ----------------------------------------------------------------------------------------
# serving
# ----------------------------------------------------------------------------------------

class Server:
    """Continuous batching of solves (mot_server_*): requests get their own stream, graph and
    a region of the device pool; ``progress()`` advances them without blocking."""

    def __init__(self, pool_bytes: int, max_active: int = 8, device=None):
        import torch
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=device or "cuda")
        h = C.c_void_p()
        _check(lib().mot_server_create(self.pool.data_ptr(), self.pool.numel(), max_active, C.byref(h)),
               "mot_server_create")
        self.h = h
        self._keep = {}

    def submit(self, x, mu, eta, topology=MOT_TREE, edges=None, edge_w=None, free_nodes=None, root=0,
               opt: Optional[Options] = None, u_out=None, tag: int = 0, x_close=None):
        import torch
        holder = _ProblemHolder(x, mu, eta, topology, edges, edge_w, free_nodes, root, x_close)
        u = u_out if u_out is not None else [torch.empty(int(t.shape[0]), dtype=torch.float64, device=t.device)
                                             for t in x]
        u_arr = (C.c_void_p * len(u))(*[t.data_ptr() for t in u])
        _check(lib().mot_server_submit(self.h, C.byref(holder.p), C.byref(opt or options()), u_arr, int(tag)),
               "mot_server_submit")
        self._keep[int(tag)] = (holder, u, u_arr)
        return u

    def progress(self):
        a, p = C.c_int(0), C.c_int(0)
        _check(lib().mot_server_progress(self.h, C.byref(a), C.byref(p)), "mot_server_progress")
        return a.value, p.value

    def poll(self, max_results: int = 256):
        buf = (ServerResult * max_results)()
        n = C.c_int(0)
        _check(lib().mot_server_poll(self.h, buf, max_results, C.byref(n)), "mot_server_poll")
        out = []
        for i in range(n.value):
            r = buf[i]
            out.append({"tag": r.tag, "status": r.status, "iters": r.iters, "violation": r.violation,
                        "cost_dual": r.cost_dual, "cost_primal": r.cost_primal, "submit_ms": r.submit_ms,
                        "admit_ms": r.admit_ms, "done_ms": r.done_ms,
                        "u": self._keep.pop(int(r.tag), (None, None, None))[1]})
        return out

    def close(self):
        if self.h:
            lib().mot_server_destroy(self.h)
            self.h = None


# C-ABI entry points declared in include/motfft.h (checked by the test-suite).
EXPORTED = ["mot_options_default", "mot_strerror", "mot_last_cuda_error", "mot_abi_version",
            "mot_workspace_bytes", "mot_solve", "mot_fastsum_workspace_bytes", "mot_fastsum",
            "mot_fastsum_static", "mot_server_create", "mot_server_submit", "mot_server_progress",
            "mot_server_poll", "mot_server_destroy", "mot_wave_schedule", "mot_boundary_poly",
            "mot_plan_grid", "mot_struct_sizes", "mot_test_tc_wait",
            "mot_test_wave_clusters"]


def wave_schedule(parent: Sequence[int], S: int, cap: int):
    """mot_wave_schedule (host only): launches of the forward / backward products and root updates
    of an S-sweep wavefront chunk on a tree in breadth-first labels.  Returns
    (tF [S][K], tB [S][K], tR [S], carrier [S], nlaunch)."""
    K = len(parent)
    par = (C.c_int * K)(*[int(v) for v in parent])
    tF = (C.c_int * (S * K))()
    tB = (C.c_int * (S * K))()
    tR = (C.c_int * S)()
    car = (C.c_int * S)()
    n = C.c_int(0)
    _check(lib().mot_wave_schedule(K, par, S, cap, tF, tB, tR, car, C.byref(n)), "mot_wave_schedule")
    F = [[tF[s * K + k] for k in range(K)] for s in range(S)]
    B = [[tB[s * K + k] for k in range(K)] for s in range(S)]
    return F, B, list(tR), list(car), n.value


def boundary_poly(eta: float, tau: float, eps_B: float, p: int):
    """mot_boundary_poly (host only): coefficients of kappa_B(tau - eps_B + t) in powers of t."""
    c = (C.c_double * (2 * p + 1))()
    _check(lib().mot_boundary_poly(float(eta), float(tau), float(eps_B), int(p), c), "mot_boundary_poly")
    return list(c)


def plan_grid(d: int, radius: float, eta_min: float, eta_max: float, n_grid: int = 0, eps_B: float = 1.0 / 16):
    """mot_plan_grid (host only): (n, scale, err_exp) of the normalisation and grid choice."""
    n, s, e = C.c_int(0), C.c_double(0.0), C.c_double(0.0)
    _check(lib().mot_plan_grid(int(d), float(radius), float(eta_min), float(eta_max), int(n_grid), float(eps_B),
                               C.byref(n), C.byref(s), C.byref(e)), "mot_plan_grid")
    return n.value, s.value, e.value
