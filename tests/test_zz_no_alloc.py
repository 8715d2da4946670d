"""mot_fastsum_static: the allocation-free kernel matrix-vector product, through the C ABI.

Some callers cannot allocate GPU memory or lend the library a workspace: plug-ins whose host
application owns all device memory through its own pool, or real-time loops where an allocation
could block.  For them the library keeps the scratch of this entry point in a static device
array.  The test compares it with mot_fastsum (the workspace entry point) on two calls in a row
with different inputs, within the matvec tolerance of the other GPU tests, checks both against
the oracle's FP64 direct summation (Eq. fastsum-sum), and checks that a request larger than the
static scratch is refused before any GPU work.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import kernel as OK
from paper_2208_03120_gb300 import workloads as W
from tests.gpu_helpers import inf_rel_err, to_dev_points

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def test_static_scratch_matches_workspace_entry_point(M):
    import torch
    rng = np.random.default_rng(2024)
    for call, (d, ns, nt, eta) in enumerate([(2, 4000, 3001, 0.02), (3, 2500, 1999, 0.05)]):
        ps = W.uniform_ball(rng, ns, d, 0.24).astype(np.float32)
        pt = W.uniform_ball(rng, nt, d, 0.24).astype(np.float32)
        an = rng.uniform(0, 1, size=ns).astype(np.float32)
        xs, xt = to_dev_points(ps), to_dev_points(pt)
        a = torch.from_numpy(an).cuda()
        b_ref, s_ref = M.mot_fastsum(xs, xt, a, eta)
        b_st, s_st = M.mot_fastsum_static(xs, xt, a, eta)
        torch.cuda.synchronize()
        assert s_st == s_ref
        err = inf_rel_err(b_st.cpu().numpy(), b_ref.cpu().numpy())
        assert err <= TOL, (call, err)
        exact = OK.direct_sum(pt.astype(np.float64), ps.astype(np.float64), an.astype(np.float64), eta)
        assert inf_rel_err(b_st.cpu().numpy(), exact) <= TOL, call


def test_static_scratch_rejects_oversized_request(M):
    """A request whose workspace exceeds MOT_STATIC_SCRATCH_BYTES is refused with MOT_ENOMEM
    before any GPU work (the pointers are never dereferenced)."""
    need = M.mot_fastsum_workspace_bytes(2, 10**6, 10**6, 1)
    assert need > M.MOT_STATIC_SCRATCH_BYTES
    st = M.lib().mot_fastsum_static(2, 0.01, C.c_void_p(256), 10**6, C.c_void_p(512), 10**6, C.c_void_p(768), 1,
                                    C.c_void_p(1024), C.byref(M.options()), None, None)
    assert st == M.MOT_ENOMEM
