"""thermo_dot_noalloc: the context-free FP64 dot product whose scratch is a
static device array (the call allocates nothing).  Compared with the existing
entry point that computes the same reduction, thermo_compliance (c = f^T u,
Sec. 2.3), on two calls in a row; the size limit of the static scratch is
rejected on the host before any launch.  The file name sorts last so that it
also runs after every other GPU test in one session."""
import ctypes as C

import numpy as np
import pytest
import torch

from helpers import gpu_solver, small_problem
from paper_2410_06850_gb300 import thermo
import workloads as W

pytestmark = pytest.mark.gpu

MAX_N = 8192 * 16384


def test_dot_noalloc_matches_compliance_twice():
    pr = small_problem(32, kind="smooth")
    s = gpu_solver(pr, prec=1)
    s.setup_precond()
    u, _ = s.solve(tol=1e-10)
    f = s.load_vector()
    c_ref = s.compliance(u)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    vals = []
    for _ in range(2):
        thermo.dot_noalloc(f, u, out)
        torch.cuda.synchronize()
        vals.append(out.item())
    for v in vals:
        assert abs(v - c_ref) <= 1e-13 * abs(c_ref), (v, c_ref)
    assert vals[0] == vals[1]  # fixed reduction order
    s.close()


def test_dot_noalloc_ragged_chunks_and_empty():
    n = 3 * 8192 + 17  # several chunks and a ragged tail
    x = torch.as_tensor(W.uniform01(21, n) - 0.5).cuda()
    y = torch.as_tensor(W.uniform01(22, n) - 0.5).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    thermo.dot_noalloc(x, y, out)
    ref = float(np.dot(x.cpu().numpy(), y.cpu().numpy()))
    assert abs(out.item() - ref) <= 1e-13 * float(np.dot(np.abs(x.cpu().numpy()), np.abs(y.cpu().numpy())))
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    out.fill_(7.0)
    thermo.dot_noalloc(e, e, out)
    assert out.item() == 0.0


def test_dot_noalloc_rejects_sizes_over_the_static_limit():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    msg = C.create_string_buffer(256)
    # rejected by the host-side size check before any launch
    rc = thermo.lib().thermo_dot_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), MAX_N + 1,
                                         C.c_void_p(out.data_ptr()), None, msg, 256)
    assert rc == thermo.EINVAL
    assert b"static scratch limit" in msg.value
    rc = thermo.lib().thermo_dot_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), -1,
                                         C.c_void_p(out.data_ptr()), None, None, 0)
    assert rc == thermo.EINVAL
