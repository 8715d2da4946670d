"""The C-ABI library builds, loads and exports every entry point of include/motfft.h;
host-side validation and workspace queries work without a GPU (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "motfft.h")


@pytest.fixture(scope="module")
def M():
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mot_\w+)\s*\(", src)))


def test_header_declarations_exported(M):
    names = _declared()
    assert len(names) >= 8
    lib = M.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(M.EXPORTED) == names


def test_abi_version_and_strerror(M):
    lib = M.lib()
    assert lib.mot_abi_version() == 5
    assert M.strerror(0) == "ok"
    assert "tree" in M.strerror(M.MOT_ENOTTREE)
    assert M.strerror(12345) == "unknown status"


def test_struct_layouts_match_the_library(M):
    """The ctypes mirrors of mot_problem / mot_options / mot_result / mot_server_result have the
    sizes the library was compiled with (a field added on one side only shows here)."""
    out = (C.c_size_t * 4)()
    M.lib().mot_struct_sizes(out)
    assert list(out) == [C.sizeof(M.Problem), C.sizeof(M.Options), C.sizeof(M.Result), C.sizeof(M.ServerResult)]


def test_options_defaults(M):
    o = M.options()
    assert o.max_iter == 1000 and o.check_every == 10 and o.m == 4 and o.p == 3
    assert abs(o.tol_viol - 1e-6) < 1e-18 and abs(o.eps_B - 1 / 16) < 1e-15
    assert o.n_grid == 0 and o.path == M.MOT_PATH_NFFT
    assert o.wavefront == 1 and o.use_graphs == 1 and o.ndft == 1


def _fake_problem(M, K, d, n, edges, topology=0, edge_w=None):
    """Problem with non-null fake device pointers: the workspace query never dereferences them."""
    p = M.Problem()
    p.K, p.d = K, d
    keep = []
    n_arr = (C.c_int64 * K)(*n)
    x_arr = (C.c_void_p * K)(*[0x1000 + 256 * k for k in range(K)])
    mu_arr = (C.c_void_p * K)(*[0x9000 + 256 * k for k in range(K)])
    keep += [n_arr, x_arr, mu_arr]
    p.n, p.x, p.mu = n_arr, x_arr, mu_arr
    p.topology = topology
    if edges is not None:
        flat = [v for e in edges for v in e]
        e_arr = (C.c_int * len(flat))(*flat)
        keep.append(e_arr)
        p.edges = e_arr
    if edge_w is not None:
        w_arr = (C.c_double * len(edge_w))(*edge_w)
        keep.append(w_arr)
        p.edge_w = w_arr
    p.eta = 0.05
    return p, keep


def _ws(M, p, **kw):
    nb = C.c_size_t(0)
    st = M.lib().mot_workspace_bytes(C.byref(p), C.byref(M.options(**kw)), C.byref(nb))
    return st, nb.value


def test_workspace_query_and_validation(M):
    p, keep = _fake_problem(M, 4, 2, [100, 200, 300, 150], [(0, 1), (1, 2), (1, 3)])
    st, nb = _ws(M, p)
    assert st == M.MOT_OK and nb > 0
    st2, nb2 = _ws(M, p, path=M.MOT_PATH_DENSE)
    assert st2 == M.MOT_OK and 0 < nb2
    # larger problems need more workspace
    p3, keep3 = _fake_problem(M, 4, 2, [1000, 2000, 3000, 1500], [(0, 1), (1, 2), (1, 3)])
    assert _ws(M, p3)[1] > nb
    # cycle / disconnected / out-of-range edges are not trees
    pc, kc = _fake_problem(M, 4, 1, [5] * 4, [(0, 1), (1, 2), (2, 0)])
    assert _ws(M, pc)[0] == M.MOT_ENOTTREE
    pd, kd = _fake_problem(M, 4, 1, [5] * 4, [(0, 1), (0, 1), (2, 3)])
    assert _ws(M, pd)[0] == M.MOT_ENOTTREE
    po, ko = _fake_problem(M, 3, 1, [5] * 3, [(0, 1), (1, 7)])
    assert _ws(M, po)[0] == M.MOT_ENOTTREE
    # bad sizes / parameters
    pb, kb = _fake_problem(M, 3, 4, [5] * 3, [(0, 1), (1, 2)])
    assert _ws(M, pb)[0] == M.MOT_EINVAL
    pz, kz = _fake_problem(M, 3, 1, [5, 0, 5], [(0, 1), (1, 2)])
    assert _ws(M, pz)[0] == M.MOT_EINVAL
    pw, kw = _fake_problem(M, 3, 1, [5] * 3, [(0, 1), (1, 2)], edge_w=[1.0, -2.0])
    assert _ws(M, pw)[0] == M.MOT_EINVAL
    assert _ws(M, p, n_grid=48)[0] == M.MOT_EINVAL      # not a power of two
    assert _ws(M, p, n_grid=256)[0] == M.MOT_EINVAL     # beyond the 2-D limit
    assert _ws(M, p, m=6)[0] == M.MOT_EUNSUPPORTED


def test_fastsum_workspace_query(M):
    a = M.mot_fastsum_workspace_bytes(2, 1000, 2000, 1)
    b = M.mot_fastsum_workspace_bytes(2, 1000, 2000, 4)
    c = M.mot_fastsum_workspace_bytes(3, 1000, 2000, 1, M.options(n_grid=32))
    assert 0 < a < b and c > 0
    with pytest.raises(M.MotError):
        M.mot_fastsum_workspace_bytes(4, 10, 10, 1)
    with pytest.raises(M.MotError):
        M.mot_fastsum_workspace_bytes(2, 0, 10, 1)


def test_solve_rejects_without_touching_gpu(M):
    """Argument errors are reported before any CUDA call (misaligned or missing workspace)."""
    p, keep = _fake_problem(M, 3, 1, [5] * 3, [(0, 1), (1, 2)])
    res = M.Result()
    lib = M.lib()
    assert lib.mot_solve(C.byref(p), None, None, 0, None, C.byref(res), None) == M.MOT_EINVAL
    assert lib.mot_solve(C.byref(p), None, C.c_void_p(0x1001), 1 << 20, None, C.byref(res), None) == M.MOT_EINVAL


def test_circle_workspace_query(M):
    p, keep = _fake_problem(M, 5, 1, [200, 210, 220, 230, 240], None, topology=1)
    st, nb = _ws(M, p)
    assert st == M.MOT_OK and nb > 4 * 200 * 210 * 2        # beta and gamma matrices
    p2, k2 = _fake_problem(M, 2, 1, [20, 20], None, topology=1)
    assert _ws(M, p2)[0] == M.MOT_EUNSUPPORTED              # a circle needs K >= 3


def test_euler_closing_points_validation(M):
    """Section 6.3 closing points: accepted for a circle (the workspace grows by the sorted
    copy, d x n_1 floats), rejected for a tree; pair-marginal outputs are circle-only and a
    tree asking for them is rejected before any CUDA call."""
    p, keep = _fake_problem(M, 5, 2, [200, 210, 220, 230, 240], None, topology=1)
    st0, nb0 = _ws(M, p)
    p.x_close = 0x7000
    st1, nb1 = _ws(M, p)
    assert st0 == st1 == M.MOT_OK and nb1 >= nb0 + 2 * 200 * 4
    t, k2 = _fake_problem(M, 3, 1, [5] * 3, [(0, 1), (1, 2)])
    t.x_close = 0x7000
    assert _ws(M, t)[0] == M.MOT_EINVAL
    t.x_close = None
    res = M.Result()
    pairs = (C.c_void_p * 3)(None, 0x8000, 0x8100)
    res.pair = pairs
    assert M.lib().mot_solve(C.byref(t), None, C.c_void_p(0x10000), 1 << 20, None, C.byref(res), None) == M.MOT_EINVAL


def test_server_argument_validation(M):
    """Invalid server arguments are rejected before any CUDA call."""
    lib = M.lib()
    h = C.c_void_p()
    assert lib.mot_server_create(None, 1 << 20, 4, C.byref(h)) == M.MOT_EINVAL
    assert lib.mot_server_create(C.c_void_p(0x1001), 1 << 20, 4, C.byref(h)) == M.MOT_EINVAL
    assert lib.mot_server_create(C.c_void_p(0x1000), 1 << 20, 0, C.byref(h)) == M.MOT_EINVAL
    assert lib.mot_server_progress(None, None, None) == M.MOT_EINVAL
    assert lib.mot_server_destroy(None) == M.MOT_EINVAL


def test_root_validation(M):
    """root = -1 (MOT_ROOT_CENTRE) is accepted; other negative labels are not; a free root is
    unsupported (its sibling updates do not converge)."""
    p, keep = _fake_problem(M, 4, 2, [100, 200, 300, 150], [(0, 1), (1, 2), (1, 3)])
    p.root = -1
    assert _ws(M, p)[0] == M.MOT_OK
    p.root = -2
    assert _ws(M, p)[0] == M.MOT_EINVAL
    p.root = 0
    f = (C.c_ubyte * 4)(1, 0, 0, 0)
    p.free_nodes = f
    assert _ws(M, p)[0] == M.MOT_EUNSUPPORTED
    p.root = -1                     # the centre among constrained nodes: node 1
    assert _ws(M, p)[0] == M.MOT_OK
